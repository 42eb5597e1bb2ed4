// Test infrastructure: the library's entry functions (hbi_entry_math.cuh, __host__
// __device__) and element frames (hbi_host.cpp) run on the host, so that the CPU tests can
// compare the CUDA path's entries with the oracle's without a GPU.
//
// usage: host_entries <in.bin> <out.bin>
//   in:  int32 n, nv, op, half, npairs; float64 mu, nu; float64 verts[n][nv][3];
//        float64 rake[n]; int32 pairs[npairs][2] (receiver, source)
//   out: float64 E[npairs][n_out][n_in]; exit status 2 if a receiver lies on a source edge
#include <cstdio>
#include <vector>

#include "../paper_2110_12165_gb300/csrc/hbi_entry_math.cuh"
#include "../paper_2110_12165_gb300/csrc/hbi_internal.h"

template <typename T>
static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int hdr[5];
    double par[2];
    if (!rd(f, hdr, 5) || !rd(f, par, 2)) return 1;
    const int n = hdr[0], nv = hdr[1], op = hdr[2], half = hdr[3], np = hdr[4];
    std::vector<double> verts((size_t)n * nv * 3), rake(n);
    std::vector<int> pr(2 * (size_t)np);
    if (!rd(f, verts.data(), verts.size()) || !rd(f, rake.data(), rake.size()) || !rd(f, pr.data(), pr.size()))
        return 1;
    fclose(f);
    const hbi::Frames F = hbi::element_frames(n, nv, verts.data());
    std::vector<double> geom(12 * (size_t)n);
    for (int e = 0; e < n; ++e)
        for (int k = 0; k < 3; ++k) {
            geom[12 * (size_t)e + k] = F.c[3 * (size_t)e + k];
            geom[12 * (size_t)e + 3 + k] = F.n[3 * (size_t)e + k];
            geom[12 * (size_t)e + 6 + k] = F.s[3 * (size_t)e + k];
            geom[12 * (size_t)e + 9 + k] = F.d[3 * (size_t)e + k];
        }
    const int nin = (op == HBI_OP_VEC_SHEAR || op == HBI_OP_VEC_FULL) ? 2 : 1;
    const int nout = op == HBI_OP_RAKE_SHEAR ? 1 : (op == HBI_OP_VEC_FULL ? 3 : 2);
    const hbi::EntryGeo g{geom.data(), verts.data(), rake.data(), nv, op, nin, nout, par[0], par[1]};
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 1;
    bool ok = true;
    for (int p = 0; p < np; ++p) {
        double E[3][2];
        ok &= half ? hbi::pair_op<true>(g, pr[2 * p], pr[2 * p + 1], E)
                   : hbi::pair_op<false>(g, pr[2 * p], pr[2 * p + 1], E);
        for (int a = 0; a < nout; ++a) fwrite(E[a], sizeof(double), nin, o);
    }
    fclose(o);
    return ok ? 0 : 2;
}
