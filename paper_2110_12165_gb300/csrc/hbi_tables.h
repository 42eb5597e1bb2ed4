// Bounds checks of the HMVM work tables (the V^T batches and items, the UY tasks and their
// gather indices) against the buffers they index.  Host code without CUDA dependencies: the
// packer runs it on every operator it builds, and the CPU tests compile it into a host harness
// and feed it corrupted tables.  The bounds-checked build of the product kernels
// (HBI_BOUNDS_CHECK) checks the same conditions on the device, launch by launch.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace hbi {

// Sizes the tables must stay inside (elements unless stated otherwise).
struct TableLimits {
    int64_t n_data1 = 0, n_data2 = 0, n_data3 = 0;   // V^T, U and dense streams
    int64_t n_x = 0;        // x entries (n_in N) at the head of [x | t]
    int64_t n_xt = 0;       // entries of [x | t] (without the 16 zero guard entries)
    int64_t n_y = 0;        // outputs (n_out N)
    int64_t n_gather = 0;   // gather indices
    int es_vt = 2, es_u = 2, es_d = 4, acc_bytes = 4;   // element sizes (bytes)
    int smem_uy = 0;        // dynamic shared memory of a UY CTA (bytes)
    int vt_panel_bytes = 0, vt_x_bytes = 0, vt_max_sub = 0, vt_split_rows = 0;
};

namespace tables_detail {
inline void note(int64_t &bad, std::string *first, const std::string &what) {
    if (bad++ == 0 && first) *first = what;
}
}  // namespace tables_detail

// The V^T stage batches (in CTA order) and their items: every bulk copy and shared-memory
// access of the V^T kernel inside its buffers.  Returns the number of violations; *first
// describes the first.
template <typename Batch, typename Item>
int64_t check_vt_tables(const std::vector<Batch> &batches, const std::vector<Item> &items, const TableLimits &L,
                        std::string *first) {
    using tables_detail::note;
    int64_t bad = 0;
    const int64_t vec = 16 / L.es_vt, za = 16 / L.acc_bytes;
    for (size_t bi = 0; bi < batches.size(); ++bi) {
        const Batch &b = batches[bi];
        const std::string where = "V^T batch " + std::to_string(bi) + ": ";
        if (b.nitems < 1 || b.nitems > L.vt_max_sub || b.item0 < 0 || (int64_t)b.item0 + b.nitems > (int64_t)items.size()) {
            note(bad, first, where + "item range");
            continue;
        }
        if (b.pbytes < 0 || b.pbytes > L.vt_panel_bytes || b.xbytes < 0 || b.xbytes > L.vt_x_bytes || b.pbytes % 16 ||
            b.xbytes % 16 || b.data_off < 0 || (b.data_off * L.es_vt) % 16 || b.data_off * L.es_vt + b.pbytes > L.n_data1 * L.es_vt)
            note(bad, first, where + "panel or x bytes");
        int64_t pacc = 0, xacc = 0;
        for (int k = 0; k < b.nitems; ++k) {
            const Item &it = items[b.item0 + k];
            const std::string wi = where + "item " + std::to_string(k) + ": ";
            const bool whole = (it.flags & 3) == 3;
            if (it.rows < 1 || it.cpad <= 0 || it.cpad % vec || it.lo < 0 || it.lo >= it.hi || it.hi > it.cpad)
                note(bad, first, wi + "shape");
            if (it.x_off < 0 || it.x_off % za || it.x_off + it.cpad > L.n_xt + 16) note(bad, first, wi + "x slice");
            if (it.out_off < L.n_x || it.out_off + it.rows > L.n_xt) note(bad, first, wi + "t rows");
            if (it.data_off != b.data_off + pacc || (int64_t)it.poff != pacc ||
                (int64_t)it.zoff * L.acc_bytes != xacc)
                note(bad, first, wi + "offsets inside the batch");
            if (!whole && it.rows > L.vt_split_rows) note(bad, first, wi + "rows of a split row block");
            pacc += (int64_t)it.rows * it.cpad;
            xacc += (int64_t)it.cpad * L.acc_bytes;
        }
        if (pacc * L.es_vt != b.pbytes || xacc != b.xbytes) note(bad, first, where + "bytes of its items");
    }
    return bad;
}

// The UY tasks and their gather indices: stream segments, gather range, output rows and
// shared memory; a gather index is -1 (padding), an entry of [x | t], or -2 - t for the pair
// t, t + 1 of an FP32-accurate leading factor column.
template <typename Task>
int64_t check_uy_tables(const std::vector<Task> &tasks, const std::vector<int> &gidx, const TableLimits &L,
                        std::string *first) {
    using tables_detail::note;
    int64_t bad = 0;
    for (size_t ti = 0; ti < tasks.size(); ++ti) {
        const Task &t = tasks[ti];
        const std::string where = "UY task " + std::to_string(ti) + ": ";
        if (t.rows < 1 || t.cpad < 0 || t.cpad_d < 0 || t.cpad % (16 / L.es_u) || t.cpad_d % (16 / L.es_d)) {
            note(bad, first, where + "shape");
            continue;
        }
        if (t.data_off < 0 || t.data_off + (int64_t)t.rows * t.cpad > L.n_data2) note(bad, first, where + "U segment");
        if (t.data_off_d < 0 || t.data_off_d + (int64_t)t.rows * t.cpad_d > L.n_data3) note(bad, first, where + "dense segment");
        if (t.out_off < 0 || t.out_off + t.rows > L.n_y) note(bad, first, where + "output rows");
        if ((int64_t)(t.cpad + t.cpad_d) * L.acc_bytes > L.smem_uy) note(bad, first, where + "gathered input size");
        const int64_t c = (int64_t)t.cpad + t.cpad_d;
        if (t.gather_off < 0 || t.gather_off + c > L.n_gather || t.gather_off + c > (int64_t)gidx.size()) {
            note(bad, first, where + "gather range");
            continue;
        }
        for (int64_t j = 0; j < c; ++j) {
            const int64_t g = gidx[t.gather_off + j];
            const bool ok = g == -1 || (g >= 0 && g < L.n_xt) || (g <= -2 && -2 - g >= 0 && -2 - g + 1 < L.n_xt);
            if (!ok) note(bad, first, where + "gather index " + std::to_string(g) + " at " + std::to_string(j));
        }
    }
    return bad;
}

}  // namespace hbi
