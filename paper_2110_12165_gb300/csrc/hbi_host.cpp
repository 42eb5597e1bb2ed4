// Host-side set-up of the H-matrix: element frames (Sec. 2.1), the binary cluster tree on
// element centres (Sec. 3.1.1), the lattice truncation (Sec. 3.2) and the block partition
// by the admissibility condition of Eq. 17.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "hbi_internal.h"

namespace hbi {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error() { return g_last_error.c_str(); }

// Normal by the right-hand rule of the vertex order; centre = vertex mean (collocation
// point); strike = normalise(z x n), or x for a horizontal element; dip = n x strike.
Frames element_frames(int n, int nv, const double *verts) {
    Frames F;
    F.c.resize(3 * (size_t)n);
    F.n.resize(3 * (size_t)n);
    F.s.resize(3 * (size_t)n);
    F.d.resize(3 * (size_t)n);
    for (int e = 0; e < n; ++e) {
        const double *v = verts + (size_t)e * nv * 3;
        double c[3] = {0, 0, 0};
        for (int a = 0; a < nv; ++a)
            for (int k = 0; k < 3; ++k) c[k] += v[3 * a + k];
        for (int k = 0; k < 3; ++k) c[k] /= nv;
        double p[3], q[3];
        if (nv == 3) {
            for (int k = 0; k < 3; ++k) { p[k] = v[3 + k] - v[k]; q[k] = v[6 + k] - v[k]; }
        } else {  // diagonals of the quadrilateral
            for (int k = 0; k < 3; ++k) { p[k] = v[6 + k] - v[k]; q[k] = v[9 + k] - v[3 + k]; }
        }
        double nn[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
        double ln = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int k = 0; k < 3; ++k) nn[k] /= ln;
        double st[3] = {-nn[1], nn[0], 0.0};  // z x n
        double ls = std::sqrt(st[0] * st[0] + st[1] * st[1]);
        if (ls < 1e-12) { st[0] = 1; st[1] = 0; st[2] = 0; }
        else { st[0] /= ls; st[1] /= ls; }
        double dp[3] = {nn[1] * st[2] - nn[2] * st[1], nn[2] * st[0] - nn[0] * st[2], nn[0] * st[1] - nn[1] * st[0]};
        for (int k = 0; k < 3; ++k) {
            F.c[3 * e + k] = c[k];
            F.n[3 * e + k] = nn[k];
            F.s[3 * e + k] = st[k];
            F.d[3 * e + k] = dp[k];
        }
    }
    return F;
}

namespace {
struct TreeBuilder {
    const std::vector<double> &c;
    int leaf;
    Tree &T;
    std::vector<int> tmp;

    int build(int start, int size, int depth) {
        int id = (int)T.cl.size();
        T.cl.push_back(Cluster{start, size, depth, -1, -1, {0, 0, 0}, {0, 0, 0}});
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = start; i < start + size; ++i)
            for (int k = 0; k < 3; ++k) {
                double v = c[3 * (size_t)T.perm[i] + k];
                lo[k] = std::min(lo[k], v);
                hi[k] = std::max(hi[k], v);
            }
        for (int k = 0; k < 3; ++k) { T.cl[id].lo[k] = lo[k]; T.cl[id].hi[k] = hi[k]; }
        if (size <= leaf) return id;
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
        const double mid = 0.5 * (lo[ax] + hi[ax]);
        // stable split at the midpoint of the longest box side (ties to the upper half)
        auto first = T.perm.begin() + start, last = first + size;
        auto below = [&](int e) { return c[3 * (size_t)e + ax] < mid; };
        tmp.assign(first, last);
        auto it = std::stable_partition(tmp.begin(), tmp.end(), below);
        int nl = (int)(it - tmp.begin());
        if (nl == 0 || nl == size) {  // degenerate: median split, ties by element index
            std::stable_sort(tmp.begin(), tmp.end(), [&](int a, int b) {
                double ca = c[3 * (size_t)a + ax], cb = c[3 * (size_t)b + ax];
                return ca < cb || (ca == cb && a < b);
            });
            nl = size / 2;
        }
        std::copy(tmp.begin(), tmp.end(), first);
        int c0 = build(start, nl, depth + 1);
        int c1 = build(start + nl, size - nl, depth + 1);
        T.cl[id].child0 = c0;
        T.cl[id].child1 = c1;
        return id;
    }
};

void collect_leaves(const Tree &T, int c, std::vector<int> &out) {
    const Cluster &C = T.cl[c];
    if (C.child0 < 0) { out.push_back(c); return; }
    collect_leaves(T, C.child0, out);
    collect_leaves(T, C.child1, out);
}
void collect_lattice(const Tree &T, int c, int L, std::vector<int> &out) {
    const Cluster &C = T.cl[c];
    if (C.depth == L || C.child0 < 0) { out.push_back(c); return; }
    collect_lattice(T, C.child0, L, out);
    collect_lattice(T, C.child1, L, out);
}

double diam(const Cluster &A) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s += (A.hi[k] - A.lo[k]) * (A.hi[k] - A.lo[k]);
    return std::sqrt(s);
}
double dist(const Cluster &A, const Cluster &B) {
    double s = 0;
    for (int k = 0; k < 3; ++k) {
        double g = std::max(0.0, std::max(B.lo[k] - A.hi[k], A.lo[k] - B.hi[k]));
        s += g * g;
    }
    return std::sqrt(s);
}

struct Partitioner {
    const Tree &T;
    int nin, nout;
    double eta;
    std::vector<Block> &out;
    void push(int t, int s, int lr) {
        const Cluster &A = T.cl[t], &S = T.cl[s];
        out.push_back(Block{t, s, (int64_t)nout * A.start, (int64_t)nout * A.size, (int64_t)nin * S.start,
                            (int64_t)nin * S.size, lr, 0, nullptr, nullptr});
    }
    void run(int t, int s) {
        const Cluster &A = T.cl[t], &S = T.cl[s];
        if (std::min(diam(A), diam(S)) < eta * dist(A, S)) { push(t, s, 1); return; }  // Eq. 17
        bool la = A.child0 < 0, ls = S.child0 < 0;
        if (la && ls) { push(t, s, 0); return; }
        if (la) { run(t, S.child0); run(t, S.child1); return; }
        if (ls) { run(A.child0, s); run(A.child1, s); return; }
        run(A.child0, S.child0); run(A.child0, S.child1);
        run(A.child1, S.child0); run(A.child1, S.child1);
    }
};
}  // namespace

Tree build_tree(const std::vector<double> &centres, int n, int leaf_size, int lattice_depth) {
    Tree T;
    T.perm.resize(n);
    std::iota(T.perm.begin(), T.perm.end(), 0);
    T.cl.reserve(4 * (size_t)n / std::max(1, leaf_size) + 8);
    TreeBuilder B{centres, leaf_size, T, {}};
    B.build(0, n, 0);
    collect_leaves(T, 0, T.leaves);
    collect_lattice(T, 0, lattice_depth, T.lattice);
    return T;
}

// Sec. 3.2: an H-matrix partition inside every lattice block (lattice row-major order).
// lattice_ij (optional): for every block, the row and column index of its lattice block.
std::vector<Block> build_partition(const Tree &T, int nin, int nout, double eta, std::vector<int> *lattice_ij) {
    std::vector<Block> out;
    Partitioner P{T, nin, nout, eta, out};
    for (size_t I = 0; I < T.lattice.size(); ++I)
        for (size_t J = 0; J < T.lattice.size(); ++J) {
            const size_t before = out.size();
            P.run(T.lattice[I], T.lattice[J]);
            if (lattice_ij)
                for (size_t b = before; b < out.size(); ++b) {
                    lattice_ij->push_back((int)I);
                    lattice_ij->push_back((int)J);
                }
        }
    return out;
}

}  // namespace hbi
