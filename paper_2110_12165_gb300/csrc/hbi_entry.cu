// Device-side entry generation and ACA (the build of the H-matrix, Sec. 3.1.2).
//
// Entries (Sec. 2.1, Eqs. 3-6): traction at receiver centre x_i from uniform slip b on
// source element j in a homogeneous isotropic full space.  The element is a dislocation
// loop; its elastic distortion is the loop integral
//     beta_nm(x) = sum_edges int c_ijpq b_i eps_hjm t_h  dG_np/dr_q (x - xi(s)) ds
// of the Kelvin Green's function G_np = [(3-4nu) delta_np / r + r_n r_p / r^3] / (16 pi mu (1-nu)).
// For a straight edge it reduces to the scalar integrals
//     J_k = int u^k / r^3 du (k = 0, 1),   K_k = int u^k / r^5 du (k = 0..3),
// with r = dperp + u t (dperp perpendicular to the edge), which are integrated here in
// closed form.  The even integrands are evaluated through their tails int_u^inf (stable
// when the receiver lies on or near the edge's extension), the odd ones directly.
#include <cuda_runtime.h>

#include <cmath>

#include "hbi_internal.h"

namespace hbi {

struct EntryGeo {
    const double *geom;   // permuted: c, n, s, d (12 doubles per element)
    const double *verts;  // permuted: nv x 3 per element
    const double *rake;   // permuted rake angle (single-component operators)
    int nv, op, nin, nout;
    double mu, nu;
};

__host__ __device__ __forceinline__ double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__host__ __device__ __forceinline__ void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// tails int_u^inf g(v) dv for u >= 0, r = sqrt(d2 + u^2)
__host__ __device__ __forceinline__ double tail_j0(double u, double r) { return 1.0 / (r * (r + u)); }
__host__ __device__ __forceinline__ double tail_k0(double u, double r) {
    double rp = r + u;
    return (2.0 * r + u) / (3.0 * r * r * r * rp * rp);
}
__host__ __device__ __forceinline__ double tail_k2(double u, double r) {
    return (r * r + r * u + u * u) / (3.0 * r * r * r * (r + u));
}

// Adds one edge's contribution to beta for the two Burgers vectors b[0], b[1].
// Returns false if the receiver lies on the edge itself.
__host__ __device__ bool edge_beta(const double *x, const double *A, const double *B, const double (*b)[3],
                          double nu, double (*beta)[9]) {
    double t[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double L = sqrt(dot3(t, t));
    t[0] /= L; t[1] /= L; t[2] /= L;
    const double R0[3] = {x[0] - A[0], x[1] - A[1], x[2] - A[2]};
    const double RB[3] = {x[0] - B[0], x[1] - B[1], x[2] - B[2]};
    const double s0 = dot3(R0, t);
    const double dv[3] = {R0[0] - s0 * t[0], R0[1] - s0 * t[1], R0[2] - s0 * t[2]};
    const double d2 = dot3(dv, dv);
    const double uA = s0, uB = s0 - L;
    const double rA = sqrt(dot3(R0, R0)), rB = sqrt(dot3(RB, RB));
    double J0, K0, K2;
    bool ok = true;
    if (uB >= 0.0) {
        J0 = tail_j0(uB, rB) - tail_j0(uA, rA);
        K0 = tail_k0(uB, rB) - tail_k0(uA, rA);
        K2 = tail_k2(uB, rB) - tail_k2(uA, rA);
    } else if (uA <= 0.0) {
        J0 = tail_j0(-uA, rA) - tail_j0(-uB, rB);
        K0 = tail_k0(-uA, rA) - tail_k0(-uB, rB);
        K2 = tail_k2(-uA, rA) - tail_k2(-uB, rB);
    } else {
        // receiver projects inside the edge: antiderivatives are odd, no cancellation
        if (!(d2 > 1e-20 * L * L)) ok = false;
        const double rA3 = rA * rA * rA, rB3 = rB * rB * rB;
        J0 = uA / (d2 * rA) - uB / (d2 * rB);
        K0 = uA * (3.0 * d2 + 2.0 * uA * uA) / (3.0 * d2 * d2 * rA3) -
             uB * (3.0 * d2 + 2.0 * uB * uB) / (3.0 * d2 * d2 * rB3);
        K2 = uA * uA * uA / (3.0 * d2 * rA3) - uB * uB * uB / (3.0 * d2 * rB3);
    }
    const double rA3 = rA * rA * rA, rB3 = rB * rB * rB;
    const double J1 = 1.0 / rB - 1.0 / rA;
    const double K1 = (1.0 / rB3 - 1.0 / rA3) / 3.0;
    const double K3 = (-1.0 / rA + d2 / (3.0 * rA3)) - (-1.0 / rB + d2 / (3.0 * rB3));
    const double I1[3] = {dv[0] * J0 + t[0] * J1, dv[1] * J0 + t[1] * J1, dv[2] * J0 + t[2] * J1};
    const double Cmu = 1.0 / (16.0 * M_PI * (1.0 - nu));
#pragma unroll
    for (int ib = 0; ib < 2; ++ib) {
        const double *bb = b[ib];
        const double bd = dot3(bb, dv), bt = dot3(bb, t), bI = dot3(bb, I1);
        double txb[3];
        cross3(t, bb, txb);
        // Q = sum_p b_p int r_n r_p r_q / r^5  (symmetric)
        const double cdd = K0 * bd + K1 * bt, cdt = K1 * bd + K2 * bt, ctt = K2 * bd + K3 * bt;
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            double Qn[3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                Qn[q] = cdd * dv[n] * dv[q] + cdt * (dv[n] * t[q] + t[n] * dv[q]) + ctt * t[n] * t[q];
            double z[3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                z[q] = -(1.0 - 2.0 * nu) * (bb[n] * I1[q] + (q == n ? bI : 0.0)) + I1[n] * bb[q] - 3.0 * Qn[q];
            double tz[3];
            cross3(t, z, tz);
#pragma unroll
            for (int m = 0; m < 3; ++m) beta[ib][3 * n + m] += Cmu * (-4.0 * nu * I1[n] * txb[m] + 2.0 * tz[m]);
        }
    }
    return ok;
}

// ------------------------------------------------------------------ half space
// Sec. 2.1 places the elements in an elastic half space with a traction-free surface
// z = 0 (z up, material z < 0).  A half-space entry is the full-space entry above plus a
// correction: Mindlin's (1936) point-force solution minus Kelvin's, carried over the source
// element by the Volterra representation
//     u_k(x) = int_S b_i c_ijpq n_j  dG_kp(x, xi) / dxi_q  dS(xi)
// (b = u(+) - u(-), n the source normal, the + side).  The correction is singular only at
// the source's mirror image above the surface, so inside the half space it is smooth: it is
// integrated with Radon's seven-point (degree 5) triangle rule on a uniform subdivision of
// the source, fine enough against the vertical distance from the receiver to the image.
// Its derivatives d2 G_kp / dx_m dxi_q are exact: the formulas are evaluated on jets that
// carry one x-direction, two xi-directions and the two mixed second derivatives.

// f with df along a (x-direction), b0 and b1 (xi-directions) and d2f along (a, b0), (a, b1)
struct Jet {
    double v, a, b0, b1, ab0, ab1;
};
__host__ __device__ __forceinline__ Jet operator+(const Jet &x, const Jet &y) {
    return {x.v + y.v, x.a + y.a, x.b0 + y.b0, x.b1 + y.b1, x.ab0 + y.ab0, x.ab1 + y.ab1};
}
__host__ __device__ __forceinline__ Jet operator-(const Jet &x, const Jet &y) {
    return {x.v - y.v, x.a - y.a, x.b0 - y.b0, x.b1 - y.b1, x.ab0 - y.ab0, x.ab1 - y.ab1};
}
__host__ __device__ __forceinline__ Jet operator*(const Jet &x, const Jet &y) {
    return {x.v * y.v, x.a * y.v + x.v * y.a, x.b0 * y.v + x.v * y.b0, x.b1 * y.v + x.v * y.b1,
            x.ab0 * y.v + x.a * y.b0 + x.b0 * y.a + x.v * y.ab0, x.ab1 * y.v + x.a * y.b1 + x.b1 * y.a + x.v * y.ab1};
}
__host__ __device__ __forceinline__ Jet operator*(double c, const Jet &x) {
    return {c * x.v, c * x.a, c * x.b0, c * x.b1, c * x.ab0, c * x.ab1};
}
__host__ __device__ __forceinline__ Jet operator+(double c, const Jet &x) { return {c + x.v, x.a, x.b0, x.b1, x.ab0, x.ab1}; }
__host__ __device__ __forceinline__ Jet operator-(double c, const Jet &x) {
    return {c - x.v, -x.a, -x.b0, -x.b1, -x.ab0, -x.ab1};
}
// g(x) from g, g', g'' at x.v (chain rule to second order)
__host__ __device__ __forceinline__ Jet chain(const Jet &x, double g0, double g1, double g2) {
    return {g0, g1 * x.a, g1 * x.b0, g1 * x.b1, g1 * x.ab0 + g2 * x.a * x.b0, g1 * x.ab1 + g2 * x.a * x.b1};
}
__host__ __device__ __forceinline__ Jet jrecip(const Jet &x) {
    const double r = 1.0 / x.v;
    return chain(x, r, -r * r, 2.0 * r * r * r);
}
__host__ __device__ __forceinline__ Jet jsqrt(const Jet &x) {
    const double r = sqrt(x.v);
    return chain(x, r, 0.5 / r, -0.25 / (r * x.v));
}

// Mindlin's correction, column p (unit force along his x, y or downward axis) in his frame
// (depth axis down), times 16 pi mu (1 - nu): (x, y) the horizontal offset receiver -
// source, Z and c the receiver and source depths, R2 the distance to the image point.
__host__ __device__ void mindlin_corr(int p, const Jet &x, const Jet &y, const Jet &Z, const Jet &c, double nu,
                                      Jet out[3]) {
    const Jet zc = Z + c;
    const Jet R2 = jsqrt(x * x + y * y + zc * zc);
    const Jet iR = jrecip(R2), iR2 = iR * iR, iR3 = iR2 * iR, iR5 = iR3 * iR2;
    const Jet iq = jrecip(R2 + zc), cZ = c * Z;
    const double k34 = 3.0 - 4.0 * nu, A = 4.0 * (1.0 - nu) * (1.0 - 2.0 * nu);
    if (p < 2) {
        const Jet &h = p == 0 ? x : y, &o = p == 0 ? y : x;   // along the force, across it
        const Jet hh = h * h;
        out[p] = iR + k34 * (hh * iR3) + 2.0 * (cZ * iR3) * (1.0 - 3.0 * (hh * iR2)) + A * iq * (1.0 - hh * iR * iq);
        out[1 - p] = h * o * (k34 * iR3 - 6.0 * (cZ * iR5) - A * (iR * iq * iq));
        out[2] = h * (k34 * ((Z - c) * iR3) - 6.0 * (cZ * zc * iR5) + A * (iR * iq));
    } else {
        const Jet w = k34 * ((Z - c) * iR3) + 6.0 * (cZ * zc * iR5) - A * (iR * iq);
        out[0] = x * w;
        out[1] = y * w;
        out[2] = (8.0 * (1.0 - nu) * (1.0 - nu) - k34) * iR + (k34 * (zc * zc) - 2.0 * cZ) * iR3 +
                 6.0 * (cZ * zc * zc * iR5);
    }
}

// beta[ib][3k+m] += w * sum_pq M[ib][p][q] d2 G^corr_kp / dx_m dxi_q at receiver x, source
// point xi (this library's frame: vertical components change sign against Mindlin's).
__host__ __device__ void hs_point(const double *x, const double *xi, const double (*M)[3][3], double w, double K,
                                  double nu, double (*beta)[9]) {
    for (int m = 0; m < 3; ++m)
        for (int p = 0; p < 3; ++p) {
            const double *d0 = M[0][p], *d1 = M[1][p];
            const Jet X{x[0] - xi[0], m == 0 ? 1.0 : 0.0, -d0[0], -d1[0], 0.0, 0.0};
            const Jet Y{x[1] - xi[1], m == 1 ? 1.0 : 0.0, -d0[1], -d1[1], 0.0, 0.0};
            const Jet Z{-x[2], m == 2 ? -1.0 : 0.0, 0.0, 0.0, 0.0, 0.0};
            const Jet C{-xi[2], 0.0, -d0[2], -d1[2], 0.0, 0.0};
            Jet col[3];
            mindlin_corr(p, X, Y, Z, C, nu, col);
            const double sp = (p == 2 ? -w : w) * K;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double sk = k == 2 ? -sp : sp;
                beta[0][3 * k + m] += sk * col[k].ab0;
                beta[1][3 * k + m] += sk * col[k].ab1;
            }
        }
}

// Radon's seven-point rule: barycentric points and weights (sum 1), exact to degree 5.
struct RadonRule {
    double l[7][3], w[7];
};
__host__ __device__ __forceinline__ RadonRule radon7() {
    const double r15 = sqrt(15.0);
    const double a1 = (6.0 - r15) / 21.0, b1 = 1.0 - 2.0 * a1, w1 = (155.0 - r15) / 1200.0;
    const double a2 = (6.0 + r15) / 21.0, b2 = 1.0 - 2.0 * a2, w2 = (155.0 + r15) / 1200.0;
    RadonRule R = {{{1.0 / 3, 1.0 / 3, 1.0 / 3}, {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                    {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}},
                   {9.0 / 40.0, w1, w1, w1, w2, w2, w2}};
    return R;
}

// Largest sub-triangle diameter over vertical image distance of the half-space quadrature,
// and the subdivision cap (4^7 sub-triangles).  A source triangle whose diameter is at most
// HS_FAR of its distance to the receiver's image (less its diameter) takes the degree-2
// three-point rule instead (error about rho^3 / 3 of the correction, rho that ratio).
constexpr double HS_RATIO = 0.25;
constexpr int HS_MAX_LEVEL = 7;
constexpr double HS_FAR = 0.02;

// Correction of the distortion beta at receiver x from unit slips b[2] on source element j.
__host__ __device__ void hs_correction(const EntryGeo &g, const double *x, int j, const double (*b)[3],
                                       double (*beta)[9]) {
    const double *gj = g.geom + 12 * (size_t)j, *n = gj + 3;
    const double lam = 2.0 * g.mu * g.nu / (1.0 - 2.0 * g.nu);
    double M[2][3][3];
    for (int ib = 0; ib < 2; ++ib) {
        const double bn = dot3(b[ib], n);
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
                M[ib][p][q] = (p == q ? lam * bn : 0.0) + g.mu * (b[ib][p] * n[q] + b[ib][q] * n[p]);
    }
    const double K = 1.0 / (16.0 * M_PI * g.mu * (1.0 - g.nu));
    const RadonRule R = radon7();
    const double *vj = g.verts + (size_t)j * g.nv * 3;
    for (int t = 1; t + 1 < g.nv; ++t) {   // fan (v0, v_t, v_t+1)
        const double *A = vj, *B = vj + 3 * t, *C = vj + 3 * (t + 1);
        double e1[3], e2[3], e3[3], cr[3];
        for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; e3[k] = C[k] - B[k]; }
        const double diam = sqrt(fmax(dot3(e1, e1), fmax(dot3(e2, e2), dot3(e3, e3))));
        cross3(e1, e2, cr);
        const double area = 0.5 * sqrt(dot3(cr, cr));
        // distance from the receiver to the image of the triangle's centroid
        const double dI[3] = {x[0] - (A[0] + B[0] + C[0]) / 3.0, x[1] - (A[1] + B[1] + C[1]) / 3.0,
                              x[2] + (A[2] + B[2] + C[2]) / 3.0};
        const double Rimg = sqrt(dot3(dI, dI));
        if (Rimg > diam && diam <= HS_FAR * (Rimg - diam)) {
            for (int q = 0; q < 3; ++q) {
                const double la = q == 0 ? 2.0 / 3.0 : 1.0 / 6.0, lb = q == 1 ? 2.0 / 3.0 : 1.0 / 6.0,
                             lc = q == 2 ? 2.0 / 3.0 : 1.0 / 6.0;
                const double xi[3] = {la * A[0] + lb * B[0] + lc * C[0], la * A[1] + lb * B[1] + lc * C[1],
                                      la * A[2] + lb * B[2] + lc * C[2]};
                hs_point(x, xi, M, area / 3.0, K, g.nu, beta);
            }
            continue;
        }
        const double D = -x[2] - fmax(A[2], fmax(B[2], C[2]));
        int L = 0;
        while (L < HS_MAX_LEVEL && diam > HS_RATIO * D * (double)(1 << L)) ++L;
        const int ns = 1 << L;
        const double wa = area / ((double)ns * ns);   // sub-triangle area
        const double h = 1.0 / ns;
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < ns - i; ++k)
                for (int up = 0; up < 2; ++up) {
                    if (up == 1 && k == ns - i - 1) continue;
                    // sub-triangle in (s, t) parameters of A + s e1 + t e2
                    double s0[3], t0[3];
                    if (up == 0) { s0[0] = i; t0[0] = k; s0[1] = i + 1; t0[1] = k; s0[2] = i; t0[2] = k + 1; }
                    else { s0[0] = i + 1; t0[0] = k; s0[1] = i + 1; t0[1] = k + 1; s0[2] = i; t0[2] = k + 1; }
                    for (int q = 0; q < 7; ++q) {
                        const double ss = h * (R.l[q][0] * s0[0] + R.l[q][1] * s0[1] + R.l[q][2] * s0[2]);
                        const double tt = h * (R.l[q][0] * t0[0] + R.l[q][1] * t0[1] + R.l[q][2] * t0[2]);
                        const double xi[3] = {A[0] + ss * e1[0] + tt * e2[0], A[1] + ss * e1[1] + tt * e2[1],
                                              A[2] + ss * e1[2] + tt * e2[2]};
                        hs_point(x, xi, M, wa * R.w[q], K, g.nu, beta);
                    }
                }
    }
}

// Full 3x2 traction response T[c_out][c_in]: rows = strike shear, dip shear, normal stress
// change (compression positive); columns = unit slip along source strike, source dip.
// HALF: in the half space (full-space part + the correction above).
template <bool HALF>
__host__ __device__ bool pair_full(const EntryGeo &g, int i, int j, double T[3][2]) {
    const double *gi = g.geom + 12 * (size_t)i, *gj = g.geom + 12 * (size_t)j;
    const double b[2][3] = {{gj[6], gj[7], gj[8]}, {gj[9], gj[10], gj[11]}};
    double beta[2][9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { beta[0][k] = 0.0; beta[1][k] = 0.0; }
    const double *vj = g.verts + (size_t)j * g.nv * 3;
    bool ok = true;
    for (int a = 0; a < g.nv; ++a) {
        int a1 = (a + 1 == g.nv) ? 0 : a + 1;
        ok &= edge_beta(gi, vj + 3 * a, vj + 3 * a1, b, g.nu, beta);
    }
    if (HALF) hs_correction(g, gi, j, b, beta);
    const double lam = 2.0 * g.mu * g.nu / (1.0 - 2.0 * g.nu);
    const double *n = gi + 3, *s = gi + 6, *d = gi + 9;
#pragma unroll
    for (int ib = 0; ib < 2; ++ib) {
        const double *B = beta[ib];
        const double tr = B[0] + B[4] + B[8];
        double tv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                double sig = (k == l ? lam * tr : 0.0) + g.mu * (B[3 * k + l] + B[3 * l + k]);
                acc += sig * n[l];
            }
            tv[k] = acc;
        }
        T[0][ib] = dot3(s, tv);
        T[1][ib] = dot3(d, tv);
        T[2][ib] = -dot3(n, tv);
    }
    return ok;
}

// Operator entries E[c_out][c_in] (n_out x n_in of the operator form).
template <bool HALF>
__host__ __device__ bool pair_op(const EntryGeo &g, int i, int j, double E[3][2]) {
    double T[3][2];
    bool ok = pair_full<HALF>(g, i, j, T);
    if (g.op == HBI_OP_VEC_FULL || g.op == HBI_OP_VEC_SHEAR) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { E[a][0] = T[a][0]; E[a][1] = T[a][1]; }
        return ok;
    }
    double sj, cj, si, ci;
    sincos(g.rake[j], &sj, &cj);
    sincos(g.rake[i], &si, &ci);
    const double c0 = T[0][0] * cj + T[0][1] * sj, c1 = T[1][0] * cj + T[1][1] * sj,
                 c2 = T[2][0] * cj + T[2][1] * sj;
    E[0][0] = ci * c0 + si * c1;
    E[1][0] = c2;
    return ok;
}

// ---------------------------------------------------------------- dense fill
struct DenseJob {
    int tau_start, tau_size, sig_start, sig_size;
    double *dst;          // row-major (nout*tau_size) x (nin*sig_size)
};

template <bool HALF>
__global__ void dense_fill_kernel(EntryGeo g, const DenseJob *jobs, int *bad) {
    const DenseJob jb = jobs[blockIdx.x];
    const int np = jb.tau_size * jb.sig_size;
    const int nc = g.nin * jb.sig_size;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int ii = p / jb.sig_size, jj = p - ii * jb.sig_size;
        double E[3][2];
        if (!pair_op<HALF>(g, jb.tau_start + ii, jb.sig_start + jj, E)) atomicOr(bad, 1);
        for (int a = 0; a < g.nout; ++a)
            for (int c = 0; c < g.nin; ++c)
                jb.dst[(size_t)(ii * g.nout + a) * nc + jj * g.nin + c] = E[a][c];
    }
}

// ---------------------------------------------------------------------- ACA
struct AcaJob {
    int tau_start, tau_size, sig_start, sig_size;
    int m, nc, rmax, rcap;
    double *U, *V;        // m x rmax and nc x rmax, column-major
    unsigned char *flags; // m + nc bytes (used rows, used columns)
};
struct AcaOut { int rank, status; };  // status: 0 converged, 1 rank budget exhausted, 2 capped, 3 singular

constexpr int ACA_THREADS = 256;
constexpr int ACA_WARPS = ACA_THREADS / 32;

// block-wide argmax of (value, index) with ties to the smaller index; -1 if all excluded
__device__ void block_argmax(double v, int idx, double *sv, int *si, double &best, int &bidx) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, v, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
    }
    if (lane == 0) { sv[w] = v; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        int bi = si[0];
        for (int k = 1; k < ACA_WARPS; ++k)
            if (si[k] >= 0 && (bi < 0 || sv[k] > bv || (sv[k] == bv && si[k] < bi))) { bv = sv[k]; bi = si[k]; }
        sv[0] = bv; si[0] = bi;
    }
    __syncthreads();
    best = sv[0];
    bidx = si[0];
    __syncthreads();
}

__device__ double block_sum(double v, double *sv) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sv[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < ACA_WARPS; ++k) s += sv[k];
        sv[0] = s;
    }
    __syncthreads();
    double r = sv[0];
    __syncthreads();
    return r;
}

// Adaptive cross approximation with partial pivoting (Sec. 3.1.2; Bebendorf 2000), one
// CTA per block: start at row 0; pivot column = argmax of the residual row over unused
// columns; next row = argmax |u_k| over unused rows (ties to the smaller index); a zero
// residual row moves on to the first unused row; stop once |u_k||v_k| <= eps ||S_k||_F
// (Frobenius norm of the approximant updated recursively).  Reaching the rank cap
// floor(m n / (m + n)) marks the block for dense storage.
template <bool HALF>
__global__ void __launch_bounds__(ACA_THREADS) aca_kernel(EntryGeo g, const AcaJob *jobs, AcaOut *outs,
                                                          double eps) {
    __shared__ double sv[ACA_WARPS];
    __shared__ int si[ACA_WARPS];
    __shared__ double s_cross[ACA_WARPS];
    const AcaJob jb = jobs[blockIdx.x];
    const int m = jb.m, nc = jb.nc;
    unsigned char *urow = jb.flags, *ucol = jb.flags + m;
    for (int k = threadIdx.x; k < m + nc; k += blockDim.x) jb.flags[k] = 0;
    __syncthreads();
    int k = 0, i = 0, status = 0;
    double normS2 = 0.0;
    bool singular = false;
    for (int guard = 0; guard < m + nc + 2; ++guard) {
        if (k >= jb.rcap) { status = 2; break; }
        if (k >= jb.rmax) { status = 1; break; }
        // residual row i -> V[:, k]
        double *vk = jb.V + (size_t)k * nc;
        {
            const int ie = jb.tau_start + i / g.nout, co = i % g.nout;
            for (int jj = threadIdx.x; jj < jb.sig_size; jj += blockDim.x) {
                double E[3][2];
                if (!pair_op<HALF>(g, ie, jb.sig_start + jj, E)) singular = true;
                for (int c = 0; c < g.nin; ++c) {
                    const int J = jj * g.nin + c;
                    double val = E[co][c];
                    for (int l = 0; l < k; ++l) val -= jb.U[(size_t)l * m + i] * jb.V[(size_t)l * nc + J];
                    vk[J] = val;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) urow[i] = 1;
        double best;
        int j;
        {
            double v = -1.0;
            int idx = -1;
            for (int J = threadIdx.x; J < nc; J += blockDim.x) {
                if (ucol[J]) continue;
                double a = fabs(vk[J]);
                if (idx < 0 || a > v) { v = a; idx = J; }
            }
            block_argmax(v, idx, sv, si, best, j);
        }
        if (j < 0 || !(best > 0.0)) {
            // zero residual row: move to the first unused row
            int nxt = -1;
            {
                int idx = -1;
                for (int I = threadIdx.x; I < m; I += blockDim.x)
                    if (!urow[I]) { idx = I; break; }
                double dummy;
                block_argmax(idx >= 0 ? -(double)idx : -1e300, idx, sv, si, dummy, nxt);
            }
            if (nxt < 0) break;
            i = nxt;
            continue;
        }
        const double piv = vk[j];
        for (int J = threadIdx.x; J < nc; J += blockDim.x) vk[J] /= piv;
        // residual column j -> U[:, k]
        double *uk = jb.U + (size_t)k * m;
        {
            const int je = jb.sig_start + j / g.nin, ci = j % g.nin;
            for (int ii = threadIdx.x; ii < jb.tau_size; ii += blockDim.x) {
                double E[3][2];
                if (!pair_op<HALF>(g, jb.tau_start + ii, je, E)) singular = true;
                for (int a = 0; a < g.nout; ++a) {
                    const int I = ii * g.nout + a;
                    double val = E[a][ci];
                    for (int l = 0; l < k; ++l) val -= jb.V[(size_t)l * nc + j] * jb.U[(size_t)l * m + I];
                    uk[I] = val;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) ucol[j] = 1;
        // norms: ||u||^2, ||v||^2 and sum_l (u_l . u)(v_l . v)
        double pu = 0.0, pv = 0.0;
        for (int I = threadIdx.x; I < m; I += blockDim.x) pu += uk[I] * uk[I];
        for (int J = threadIdx.x; J < nc; J += blockDim.x) pv += vk[J] * vk[J];
        const double uu = block_sum(pu, sv), vv = block_sum(pv, sv);
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            double cw = 0.0;
            for (int l = w; l < k; l += ACA_WARPS) {
                double a = 0.0, b = 0.0;
                const double *ul = jb.U + (size_t)l * m, *vl = jb.V + (size_t)l * nc;
                for (int I = lane; I < m; I += 32) a += ul[I] * uk[I];
                for (int J = lane; J < nc; J += 32) b += vl[J] * vk[J];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                }
                cw += a * b;
            }
            if (lane == 0) s_cross[w] = cw;
            __syncthreads();
            double cross = 0.0;
            for (int q = 0; q < ACA_WARPS; ++q) cross += s_cross[q];
            __syncthreads();
            normS2 += 2.0 * cross + uu * vv;
        }
        ++k;
        if (sqrt(uu * vv) <= eps * sqrt(normS2 > 0.0 ? normS2 : 0.0)) break;
        // next row: argmax |u_k| over unused rows
        int nxt;
        {
            double v = -1.0;
            int idx = -1;
            for (int I = threadIdx.x; I < m; I += blockDim.x) {
                if (urow[I]) continue;
                double a = fabs(uk[I]);
                if (idx < 0 || a > v) { v = a; idx = I; }
            }
            block_argmax(v, idx, sv, si, best, nxt);
        }
        if (nxt < 0) break;
        i = nxt;
    }
    // reduce the singular flag
    __shared__ int s_sing;
    if (threadIdx.x == 0) s_sing = 0;
    __syncthreads();
    if (singular) atomicOr(&s_sing, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        outs[blockIdx.x].rank = k;
        outs[blockIdx.x].status = s_sing ? 3 : status;
    }
}

// ------------------------------------------------------------- host driver
namespace {
template <typename T>
hbi_status dev_alloc(T **p, size_t count, std::vector<void *> &owned) {
    void *q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return HBI_ERR_OOM;
    }
    owned.push_back(q);
    *p = (T *)q;
    return HBI_OK;
}
}  // namespace

hbi_status device_build_factors(hbi_handle *h, const Tree &T, std::vector<Block> &blocks, double eps,
                                std::vector<void *> &owned) {
    EntryGeo g{h->d_geom, h->d_verts, h->d_rake, h->nv, h->op, h->nin, h->nout, h->mu, h->nu};
    int *d_bad = nullptr;
    hbi_status st = dev_alloc(&d_bad, 1, owned);
    if (st) return st;
    HBI_CUDA_TRY(cudaMemset(d_bad, 0, sizeof(int)));

    // ---- low-rank candidates: ACA with growing rank budgets
    std::vector<int> pending;
    for (int b = 0; b < (int)blocks.size(); ++b)
        if (blocks[b].lowrank) pending.push_back(b);
    const int budgets[] = {48, 256, 2048};
    for (int pass = 0; pass < 3 && !pending.empty(); ++pass) {
        // batches bounded by a workspace budget
        size_t free_b = 0, total_b = 0;
        HBI_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const size_t cap_bytes = std::max<size_t>((size_t)(0.45 * (double)free_b), (size_t)1 << 28);
        std::vector<int> next;
        size_t pos = 0;
        while (pos < pending.size()) {
            std::vector<AcaJob> jobs;
            std::vector<int> ids;
            size_t bytes = 0;
            while (pos < pending.size()) {
                const Block &B = blocks[pending[pos]];
                const int rcap = (int)((B.m * B.nc) / (B.m + B.nc));
                const int rmax = std::max(1, std::min(rcap, budgets[pass]));
                size_t need = (size_t)(B.m + B.nc) * rmax * sizeof(double) + (size_t)(B.m + B.nc) + 64;
                if (!jobs.empty() && bytes + need > cap_bytes) break;
                const Cluster &A = T.cl[B.tau], &S = T.cl[B.sig];
                jobs.push_back(AcaJob{A.start, A.size, S.start, S.size, (int)B.m, (int)B.nc, rmax, rcap,
                                      nullptr, nullptr, nullptr});
                ids.push_back(pending[pos]);
                bytes += need;
                ++pos;
            }
            // one allocation for the batch's factors (kept until packing), one for flags
            size_t nd = 0, nf = 0;
            for (auto &J : jobs) { nd += (size_t)(J.m + J.nc) * J.rmax; nf += (size_t)(J.m + J.nc); }
            double *d_fac = nullptr;
            unsigned char *d_flags = nullptr;
            if ((st = dev_alloc(&d_fac, nd, owned))) return st;
            HBI_CUDA_TRY(cudaMalloc(&d_flags, nf ? nf : 1));
            size_t od = 0, of = 0;
            for (auto &J : jobs) {
                J.U = d_fac + od;
                J.V = d_fac + od + (size_t)J.m * J.rmax;
                J.flags = d_flags + of;
                od += (size_t)(J.m + J.nc) * J.rmax;
                of += (size_t)(J.m + J.nc);
            }
            AcaJob *d_jobs = nullptr;
            AcaOut *d_outs = nullptr;
            HBI_CUDA_TRY(cudaMalloc(&d_jobs, jobs.size() * sizeof(AcaJob)));
            HBI_CUDA_TRY(cudaMalloc(&d_outs, jobs.size() * sizeof(AcaOut)));
            HBI_CUDA_TRY(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(AcaJob), cudaMemcpyHostToDevice));
            if (h->half_space)
                aca_kernel<true><<<(unsigned)jobs.size(), ACA_THREADS>>>(g, d_jobs, d_outs, eps);
            else
                aca_kernel<false><<<(unsigned)jobs.size(), ACA_THREADS>>>(g, d_jobs, d_outs, eps);
            HBI_CUDA_TRY(cudaGetLastError());
            std::vector<AcaOut> outs(jobs.size());
            HBI_CUDA_TRY(cudaMemcpy(outs.data(), d_outs, outs.size() * sizeof(AcaOut), cudaMemcpyDeviceToHost));
            cudaFree(d_jobs);
            cudaFree(d_outs);
            cudaFree(d_flags);
            for (size_t q = 0; q < jobs.size(); ++q) {
                Block &B = blocks[ids[q]];
                if (outs[q].status == 3) {
                    set_error("receiver on an element edge (singular stress)");
                    return HBI_ERR_SINGULAR;
                }
                if (outs[q].status == 0) {
                    B.rank = outs[q].rank;
                    B.d_src = jobs[q].U;       // U column-major, leading dimension m
                    B.d_src2 = jobs[q].V;      // V column-major, leading dimension nc
                } else if (outs[q].status == 2) {
                    B.lowrank = 0;             // rank cap: dense storage
                } else {
                    if (pass == 2) {
                        set_error("ACA did not converge within rank 2048");
                        return HBI_ERR_ACA_FAIL;
                    }
                    next.push_back(ids[q]);
                }
            }
        }
        pending.swap(next);
    }

    // ---- dense blocks (near field and rank-capped)
    std::vector<DenseJob> djobs;
    size_t nd = 0;
    for (auto &B : blocks)
        if (!B.lowrank) nd += (size_t)B.m * B.nc;
    double *d_dense = nullptr;
    if ((st = dev_alloc(&d_dense, nd, owned))) return st;
    size_t od = 0;
    for (auto &B : blocks) {
        if (B.lowrank) continue;
        const Cluster &A = T.cl[B.tau], &S = T.cl[B.sig];
        djobs.push_back(DenseJob{A.start, A.size, S.start, S.size, d_dense + od});
        B.d_src = d_dense + od;
        B.d_src2 = nullptr;
        B.rank = 0;
        od += (size_t)B.m * B.nc;
    }
    if (!djobs.empty()) {
        DenseJob *d_dj = nullptr;
        HBI_CUDA_TRY(cudaMalloc(&d_dj, djobs.size() * sizeof(DenseJob)));
        HBI_CUDA_TRY(cudaMemcpy(d_dj, djobs.data(), djobs.size() * sizeof(DenseJob), cudaMemcpyHostToDevice));
        if (h->half_space)
            dense_fill_kernel<true><<<(unsigned)djobs.size(), 256>>>(g, d_dj, d_bad);
        else
            dense_fill_kernel<false><<<(unsigned)djobs.size(), 256>>>(g, d_dj, d_bad);
        HBI_CUDA_TRY(cudaGetLastError());
        HBI_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(d_dj);
    }
    int bad = 0;
    HBI_CUDA_TRY(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) {
        set_error("receiver on an element edge (singular stress)");
        return HBI_ERR_SINGULAR;
    }
    return HBI_OK;
}

}  // namespace hbi
