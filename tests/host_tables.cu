// Host harness of the HMVM work-table checks (csrc/hbi_tables.h) with the library's own table
// structures: a small valid set of V^T batches / items and UY tasks / gather indices must pass;
// each corruption listed below, applied alone, must be reported.  Prints one line per case:
// "<name> <violations>".
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "../paper_2110_12165_gb300/csrc/hbi_internal.h"

using namespace hbi;

struct Set {
    std::vector<VtBatch> batches;
    std::vector<VtItem> items;
    std::vector<GemvTask> tasks;
    std::vector<int> gidx;
    TableLimits L;
};

// FP16 factors (8 per 16 bytes), FP32 dense (4 per 16 bytes), FP32 accumulation (4 per 16 bytes)
static Set valid() {
    Set s;
    TableLimits &L = s.L;
    L.es_vt = 2; L.es_u = 2; L.es_d = 4; L.acc_bytes = 4;
    L.n_x = 64; L.n_xt = 64 + 40; L.n_y = 96;
    L.vt_panel_bytes = 40 << 10; L.vt_x_bytes = 8 << 10; L.vt_max_sub = 8; L.vt_split_rows = 32;
    // two items in one batch: 24 rows x 16 columns and 16 rows x 32 columns (t rows 64..103)
    VtItem a{}, b{};
    a.data_off = 0; a.x_off = 0; a.out_off = 64; a.scale_off = -1; a.rows = 24; a.cpad = 16; a.lo = 0; a.hi = 16;
    a.flags = 3; a.poff = 0; a.zoff = 0;
    b.data_off = 24 * 16; b.x_off = 16; b.out_off = 88; b.scale_off = -1; b.rows = 16; b.cpad = 32; b.lo = 0;
    b.hi = 30; b.flags = 3; b.poff = 24 * 16; b.zoff = 16;
    s.items = {a, b};
    VtBatch bt{};
    bt.data_off = 0; bt.pbytes = (24 * 16 + 16 * 32) * 2; bt.xbytes = (16 + 32) * 4; bt.item0 = 0; bt.nitems = 2;
    s.batches = {bt};
    L.n_data1 = 24 * 16 + 16 * 32;
    // two UY tasks of 48 rows: dense 8 + factor 16 columns, and dense 4 + factor 8 columns
    GemvTask t0{}, t1{};
    t0.data_off = 0; t0.data_off_d = 0; t0.out_off = 0; t0.gather_off = 0; t0.rows = 48; t0.cpad = 16; t0.cpad_d = 8;
    t1.data_off = 48 * 16; t1.data_off_d = 48 * 8; t1.out_off = 48; t1.gather_off = 24; t1.rows = 48; t1.cpad = 8;
    t1.cpad_d = 4;
    s.tasks = {t0, t1};
    L.n_data2 = 48 * 16 + 48 * 8;
    L.n_data3 = 48 * 8 + 48 * 4;
    for (int j = 0; j < 8; ++j) s.gidx.push_back(j);           // dense columns: x
    for (int j = 0; j < 15; ++j) s.gidx.push_back(64 + j);     // factor columns: t
    s.gidx.push_back(-1);                                      // padding
    for (int j = 0; j < 4; ++j) s.gidx.push_back(8 + j);
    s.gidx.push_back(-2 - 70);                                 // the pair t 70, 71
    for (int j = 0; j < 7; ++j) s.gidx.push_back(80 + j);
    L.n_gather = (int64_t)s.gidx.size();
    L.smem_uy = 24 * 4;
    return s;
}

static int64_t check(const Set &s) {
    std::string first;
    return check_vt_tables(s.batches, s.items, s.L, &first) + check_uy_tables(s.tasks, s.gidx, s.L, &first);
}

int main() {
    std::vector<std::pair<std::string, std::function<void(Set &)>>> cases = {
        {"valid", [](Set &) {}},
        {"vt_batch_past_stream", [](Set &s) { s.batches[0].data_off = 8; s.items[0].data_off = 8; s.items[1].data_off += 8; }},
        {"vt_batch_item_range", [](Set &s) { s.batches[0].nitems = 3; }},
        {"vt_item_x_slice", [](Set &s) { s.items[1].x_off = 96; }},
        {"vt_item_x_unaligned", [](Set &s) { s.items[1].x_off = 17; }},
        {"vt_item_t_rows", [](Set &s) { s.items[1].out_off = 90; }},
        {"vt_item_hi_past_cpad", [](Set &s) { s.items[0].hi = 17; }},
        {"vt_item_poff", [](Set &s) { s.items[1].poff += 8; }},
        {"vt_split_rows", [](Set &s) { s.items[0].flags = 1; s.items[0].rows = 40; }},
        {"uy_u_segment", [](Set &s) { s.tasks[1].data_off += 16; }},
        {"uy_dense_segment", [](Set &s) { s.tasks[1].rows = 64; }},
        {"uy_output_rows", [](Set &s) { s.tasks[1].out_off = 60; }},
        {"uy_gather_range", [](Set &s) { s.tasks[1].gather_off = 30; }},
        {"uy_gather_index_high", [](Set &s) { s.gidx[3] = 104; }},
        {"uy_gather_index_neg", [](Set &s) { s.gidx[3] = -5000; }},
        {"uy_pair_past_end", [](Set &s) { s.gidx[28] = -2 - 103; }},
        {"uy_smem", [](Set &s) { s.L.smem_uy = 16; }},
        {"uy_cpad_unaligned", [](Set &s) { s.tasks[0].cpad = 12; }},
    };
    for (auto &c : cases) {
        Set s = valid();
        c.second(s);
        printf("%s %lld\n", c.first.c_str(), (long long)check(s));
    }
    return 0;
}
