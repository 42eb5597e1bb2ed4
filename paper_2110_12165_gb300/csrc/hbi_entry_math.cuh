// Entries of the operator (Sec. 2.1, Eqs. 3-6), host and device: the traction at the centre
// x_i of receiver element i from uniform slip b on source element j.
//
// Full space (homogeneous, isotropic): the element is a dislocation loop; its elastic
// distortion is the loop integral
//     beta_nm(x) = sum_edges int c_ijpq b_i eps_hjm t_h  dG_np/dr_q (x - xi(s)) ds
// of the Kelvin Green's function G_np = [(3-4nu) delta_np / r + r_n r_p / r^3] / (16 pi mu (1-nu)).
// For a straight edge it reduces to the scalar integrals
//     J_k = int u^k / r^3 du (k = 0, 1),   K_k = int u^k / r^5 du (k = 0..3),
// with r = dperp + u t (dperp perpendicular to the edge), which are integrated here in
// closed form.  The even integrands are evaluated through their tails int_u^inf (stable
// when the receiver lies on or near the edge's extension), the odd ones directly.
//
// Half space: the full-space entry plus the correction in the half-space section below.
//
// The functions are __host__ __device__: the entry kernels use them on the device, and the
// CPU tests compile them for the host to check them against the oracle without a GPU.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/hbi.h"

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

}  // namespace hbi
