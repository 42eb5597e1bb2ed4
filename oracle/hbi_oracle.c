/*
 * hbi_oracle.c -- plain, slow, FP64 CPU oracle for the BEM / lattice-H-matrix
 * earthquake-sequence hot path of Ozawa, Ida, Hoshino & Ando (arXiv 2110.12165).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only tests/, the smoke check and the CPU-baseline leg of the benchmark use
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Contents, each following the passage cited beside it:
 *   - element frames and collocation at element centres           (Sec. 2.1, Eqs. 5-6)
 *   - full-space stress of a uniform-slip polygonal element        (Sec. 2.1, Eqs. 3-4).
 *     The element is a dislocation loop along its boundary; its elastic distortion is
 *     the line integral  beta_nm(x) = sum_edges int c_ijpq b_i eps_hjm t_h
 *     dG_np/dr_q (x - xi) ds  (Volterra representation + Stokes' theorem), with the
 *     Kelvin full-space Green's function G.  The integral is evaluated here by adaptive
 *     Gauss-Legendre quadrature (the CUDA library integrates it in closed form).
 *   - half-space stress of the same element (Sec. 2.1: free surface z = 0): the full-space
 *     stress plus Mindlin's (1936) point-force correction carried over the element by the
 *     Volterra representation; xi-derivatives by the complex step, x-derivatives by
 *     fourth-order central differences, the element integral by subdivided Gauss-Legendre
 *     product rules (the CUDA library differentiates with forward-mode jets and integrates
 *     with Radon's seven-point rule)
 *   - dense BEM matvec                                               (Eqs. 5-6)
 *   - binary cluster tree on element centres                        (Sec. 3.1.1)
 *   - admissibility min(diam) < eta dist                             (Eq. 17)
 *   - lattice truncation at depth L + per-lattice-block partition    (Sec. 3.2)
 *   - ACA with partial pivoting, Frobenius stopping rule, rank cap   (Sec. 3.1.2, Eqs. 18-19)
 *   - H-matrix x vector, fixed block order                           (Sec. 3.1.3, Eq. 20)
 *   - rate-state right-hand side                                     (Eqs. 7-13, 21-22)
 *   - Cash-Karp Runge-Kutta 4(5), step control, slip update          (Eqs. 14-16)
 *   - sensitivities of a fixed-step run by the complex step (Squire & Trapp 1998): the
 *     whole fixed-step Cash-Karp map of Eqs. 7-13 evaluated in complex arithmetic with a
 *     parameter moved by i h gives dL/dp = Im L / h to rounding (no differencing error);
 *     it checks the library's hand-written discrete adjoint by an independent route
 *
 * Readings of garbled / silent passages:
 *   Eq. 7 and 13a-c: the state enters as exp(phi/a) (exp(-phi/a) in 13a-c).
 *   Eqs. 14-15: the error ratio (err/eps_RK) carries the exponents -0.25 / -0.2.
 *   Eq. 12: S_ij is A_ij.  RK tableau: Cash & Karp (1990).
 *   Eqs. 21-22: loading computed with the H-matrix (one H-matvec of -V_pl * rake).
 */
#include <complex.h>
#undef I   /* I is a row index below; the imaginary unit is written _Complex_I */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HO_PI 3.14159265358979323846

/* operator kinds: inputs -> outputs (component order inside one element) */
enum { HO_OP_RAKE_SHEAR = 0,        /* tau_r            <- V_r           */
       HO_OP_RAKE_SHEAR_NORMAL = 1, /* (tau_r, sigma)   <- V_r           */
       HO_OP_VEC_SHEAR = 2,         /* (tau_s, tau_d)   <- (V_s, V_d)    */
       HO_OP_VEC_FULL = 3 };        /* (tau_s, tau_d, sigma) <- (V_s, V_d) */

static int op_nin(int op) { return (op == HO_OP_VEC_SHEAR || op == HO_OP_VEC_FULL) ? 2 : 1; }
static int op_nout(int op) { return op == HO_OP_RAKE_SHEAR ? 1 : (op == HO_OP_VEC_FULL ? 3 : 2); }

/* ------------------------------------------------------------------ vectors */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------ Gauss-Legendre (Newton) */
#define GL_N 8
static double gl_tab_x[GL_N + 1][GL_N], gl_tab_w[GL_N + 1][GL_N];   /* rules of 1..GL_N points */
static double *gl_x = gl_tab_x[GL_N], *gl_w = gl_tab_w[GL_N];
static int gl_ready = 0;

/* Nodes are the roots of the Legendre polynomial P_n, found by Newton's method from
 * the Chebyshev-like starting guesses; weights 2 / ((1 - x^2) P_n'(x)^2). */
static void gl_rule(int n, double *xs, double *ws) {
    for (int i = 0; i < n; i++) {
        double x = cos(HO_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static void gl_init(void) {
    if (gl_ready) return;
    for (int n = 1; n <= GL_N; n++) gl_rule(n, gl_tab_x[n], gl_tab_w[n]);
    gl_ready = 1;
}

int ho_gauss_legendre(double *x, double *w) {
    gl_init();
    for (int i = 0; i < GL_N; i++) { x[i] = gl_x[i]; w[i] = gl_w[i]; }
    return GL_N;
}

/* --------------------------------------------------------- element frames */
/* Normal from the vertex order (right-hand rule), centre = vertex mean (Sec. 2.1:
 * stress is evaluated at the element centre).  Strike = normalised z x n (x if the
 * element is horizontal); dip = n x strike (up-dip when n points up). */
static void elem_frame(int nv, const double *v, double *c, double *n, double *s, double *d, double *area) {
    double e1[3], e2[3], nn[3];
    for (int k = 0; k < 3; k++) {
        c[k] = 0.0;
        for (int a = 0; a < nv; a++) c[k] += v[3 * a + k];
        c[k] /= nv;
    }
    if (nv == 3) {
        for (int k = 0; k < 3; k++) { e1[k] = v[3 + k] - v[k]; e2[k] = v[6 + k] - v[k]; }
    } else {
        for (int k = 0; k < 3; k++) { e1[k] = v[6 + k] - v[k]; e2[k] = v[9 + k] - v[3 + k]; }
    }
    cross3(e1, e2, nn);
    double ln = norm3(nn);
    *area = 0.5 * ln;
    for (int k = 0; k < 3; k++) n[k] = nn[k] / ln;
    double z[3] = {0, 0, 1}, t[3];
    cross3(z, n, t);
    double lt = norm3(t);
    if (lt < 1e-12) { s[0] = 1; s[1] = 0; s[2] = 0; }
    else for (int k = 0; k < 3; k++) s[k] = t[k] / lt;
    cross3(n, s, d);
}

int ho_elem_frames(int n_elem, int nv, const double *verts, double *cent, double *nrm,
                   double *strike, double *dip, double *area) {
    for (int e = 0; e < n_elem; e++)
        elem_frame(nv, verts + (size_t)e * nv * 3, cent + 3 * e, nrm + 3 * e, strike + 3 * e,
                   dip + 3 * e, area + e);
    return 0;
}

/* ------------------------------------------------ Kelvin Green's function */
/* G_np(r) = [(3-4nu) delta_np / r + r_n r_p / r^3] / (16 pi mu (1-nu))  (full space);
 * dG[n][p][q] = dG_np / dr_q. */
static void kelvin_dG(const double *r, double mu, double nu, double dG[3][3][3]) {
    double R2 = dot3(r, r), R = sqrt(R2), R3 = R2 * R, R5 = R3 * R2;
    double C = 1.0 / (16.0 * HO_PI * mu * (1.0 - nu));
    for (int n = 0; n < 3; n++)
        for (int p = 0; p < 3; p++)
            for (int q = 0; q < 3; q++) {
                double v = -(3.0 - 4.0 * nu) * (n == p) * r[q] / R3
                           + ((n == q) * r[p] + (p == q) * r[n]) / R3
                           - 3.0 * r[n] * r[p] * r[q] / R5;
                dG[n][p][q] = C * v;
            }
}

int ho_kelvin_G(const double *r, double mu, double nu, double *G) {
    double R = norm3(r), C = 1.0 / (16.0 * HO_PI * mu * (1.0 - nu));
    for (int n = 0; n < 3; n++)
        for (int p = 0; p < 3; p++)
            G[3 * n + p] = C * ((3.0 - 4.0 * nu) * (n == p) / R + r[n] * r[p] / (R * R * R));
    return 0;
}

int ho_kelvin_dG(const double *r, double mu, double nu, double *out27) {
    double dG[3][3][3];
    kelvin_dG(r, mu, nu, dG);
    memcpy(out27, dG, sizeof dG);
    return 0;
}

static double cijkl(int i, int j, int k, int l, double lam, double mu) {
    return lam * (i == j) * (k == l) + mu * ((i == k) * (j == l) + (i == l) * (j == k));
}
static double levi(int i, int j, int k) {
    if (i == j || j == k || i == k) return 0.0;
    return ((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1.0 : -1.0;
}

/* ------------------------------------------------ loop-integral quadrature */
typedef struct {
    const double *x;   /* receiver */
    const double *A;   /* edge start */
    const double *t;   /* unit edge direction */
    double mu, nu;
    int nb;
    double F[3][3][3][3];  /* F[ib][p][q][m] = sum_ijh c_ijpq b_i eps_hjm t_h */
    double beta[3][3][3];
    int bad;
} edge_ctx;

static void edge_integrate(edge_ctx *E, double s0, double s1, int depth) {
    double len = s1 - s0, R0[3], pc[3];
    for (int k = 0; k < 3; k++) R0[k] = E->x[k] - E->A[k];
    double proj = dot3(R0, E->t);
    if (proj < s0) proj = s0;
    if (proj > s1) proj = s1;
    for (int k = 0; k < 3; k++) pc[k] = R0[k] - proj * E->t[k];
    double dist = norm3(pc);
    if (dist <= 1e-12 * (len > 0 ? len : 1.0)) { E->bad = 1; return; }
    if (len > 0.5 * dist && depth < 60) {
        double mid = 0.5 * (s0 + s1);
        edge_integrate(E, s0, mid, depth + 1);
        edge_integrate(E, mid, s1, depth + 1);
        return;
    }
    for (int g = 0; g < GL_N; g++) {
        double s = 0.5 * (s0 + s1) + 0.5 * len * gl_x[g], w = 0.5 * len * gl_w[g];
        double r[3], dG[3][3][3];
        for (int k = 0; k < 3; k++) r[k] = R0[k] - s * E->t[k];
        kelvin_dG(r, E->mu, E->nu, dG);
        for (int ib = 0; ib < E->nb; ib++)
            for (int n = 0; n < 3; n++)
                for (int m = 0; m < 3; m++) {
                    double acc = 0.0;
                    for (int p = 0; p < 3; p++)
                        for (int q = 0; q < 3; q++) acc += E->F[ib][p][q][m] * dG[n][p][q];
                    E->beta[ib][n][m] += w * acc;
                }
    }
}

/* Stress tensor sig[ib][3][3] at x from uniform displacement discontinuity b[ib]
 * (b = u(+) - u(-), the + side being the one the right-hand normal of the vertex
 * order points to) over the planar polygon P (nv vertices). Returns 0, or -1 if x lies
 * on the boundary of the polygon (stress singular there), -2 if nb is not 1..3. */
static int polygon_stress(int nv, const double *P, int nb, const double *b, double mu, double nu,
                          const double *x, double *sig) {
    gl_init();
    if (nb < 1 || nb > 3) return -2;
    double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    double beta[3][3][3];
    memset(beta, 0, sizeof beta);
    int bad = 0;
    for (int a = 0; a < nv; a++) {
        const double *A = P + 3 * a, *B = P + 3 * ((a + 1) % nv);
        double t[3], L;
        for (int k = 0; k < 3; k++) t[k] = B[k] - A[k];
        L = norm3(t);
        for (int k = 0; k < 3; k++) t[k] /= L;
        edge_ctx E;
        memset(&E, 0, sizeof E);
        E.x = x; E.A = A; E.t = t; E.mu = mu; E.nu = nu; E.nb = nb;
        for (int ib = 0; ib < nb; ib++)
            for (int p = 0; p < 3; p++)
                for (int q = 0; q < 3; q++)
                    for (int m = 0; m < 3; m++) {
                        double acc = 0.0;
                        for (int i = 0; i < 3; i++)
                            for (int j = 0; j < 3; j++)
                                for (int h = 0; h < 3; h++)
                                    acc += cijkl(i, j, p, q, lam, mu) * b[3 * ib + i] * levi(h, j, m) * t[h];
                        E.F[ib][p][q][m] = acc;
                    }
        edge_integrate(&E, 0.0, L, 0);
        bad |= E.bad;
        for (int ib = 0; ib < nb; ib++)
            for (int n = 0; n < 3; n++)
                for (int m = 0; m < 3; m++) beta[ib][n][m] += E.beta[ib][n][m];
    }
    for (int ib = 0; ib < nb; ib++) {
        double tr = beta[ib][0][0] + beta[ib][1][1] + beta[ib][2][2];
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++)
                sig[9 * ib + 3 * k + l] = lam * (k == l) * tr + mu * (beta[ib][k][l] + beta[ib][l][k]);
    }
    return bad ? -1 : 0;
}

int ho_stress_polygon(int nv, const double *P, int nb, const double *b, double mu, double nu,
                      const double *x, double *sig) {
    return polygon_stress(nv, P, nb, b, mu, nu, x, sig);
}

/* ------------------------------------------------------------ half space */
/* Sec. 2.1 evaluates the elements in an elastic half space with a traction-free surface.
 * Here the half-space stress of an element is the full-space stress above plus a
 * correction: the difference between Mindlin's (1936) point-force solution for the half
 * space and Kelvin's, carried over the source element by the Volterra representation
 *     u_k(x) = int_S b_i c_ijpq n_j  dG_kp(x, xi) / dxi_q  dS(xi)
 * (b = u(+) - u(-), n the source normal pointing to the + side).  Coordinates: z up, free
 * surface z = 0, material z < 0.  Mindlin's formulas use a downward depth axis: Z = -x_z
 * for the receiver, c = -xi_z for the source, and the horizontal offsets x - xi.  The
 * correction is the part of his solution in R2, the distance from the receiver to the
 * source's mirror image; it is regular wherever Z + c > 0, so inside the half space it is
 * integrated over the element by ordinary quadrature. */
typedef double complex cplx;

/* Mindlin correction, column p (unit force along his x, y or downward axis), Mindlin frame,
 * times 16 pi mu (1 - nu).  (x, y): horizontal offset receiver - source; Z, c: depths. */
static void mindlin_corr_col(int p, cplx x, cplx y, cplx Z, cplx c, double nu, cplx out[3]) {
    const cplx zc = Z + c, R2 = csqrt(x * x + y * y + zc * zc), q = R2 + zc;
    const cplx R3 = R2 * R2 * R2, R5 = R3 * R2 * R2, cZ = c * Z;
    const double k34 = 3.0 - 4.0 * nu, A = 4.0 * (1.0 - nu) * (1.0 - 2.0 * nu);
    if (p < 2) {
        const cplx h = p == 0 ? x : y, o = p == 0 ? y : x;   /* along the force, across it */
        out[p] = 1.0 / R2 + k34 * h * h / R3 + 2.0 * cZ / R3 * (1.0 - 3.0 * h * h / (R2 * R2)) +
                 A / q * (1.0 - h * h / (R2 * q));
        out[1 - p] = h * o * (k34 / R3 - 6.0 * cZ / R5 - A / (R2 * q * q));
        out[2] = h * (k34 * (Z - c) / R3 - 6.0 * cZ * zc / R5 + A / (R2 * q));
    } else {
        const cplx w = k34 * (Z - c) / R3 + 6.0 * cZ * zc / R5 - A / (R2 * q);
        out[0] = x * w;
        out[1] = y * w;
        out[2] = (8.0 * (1.0 - nu) * (1.0 - nu) - k34) / R2 + (k34 * zc * zc - 2.0 * cZ) / R3 +
                 6.0 * cZ * zc * zc / R5;
    }
}

/* Correction column p in this library's frame: displacement at x from a unit force along
 * axis p at xi (vertical components change sign between the frames). */
static void hs_corr_col(int p, const cplx *x, const cplx *xi, double mu, double nu, cplx g[3]) {
    cplx m[3];
    mindlin_corr_col(p, x[0] - xi[0], x[1] - xi[1], -x[2], -xi[2], nu, m);
    const double K = 1.0 / (16.0 * HO_PI * mu * (1.0 - nu)), sp = p == 2 ? -K : K;
    g[0] = sp * m[0];
    g[1] = sp * m[1];
    g[2] = -sp * m[2];
}

/* G[k][p] of the half space (Kelvin + correction), or the correction alone. */
static void hs_green(const double *x, const double *xi, double mu, double nu, int with_kelvin, double *G) {
    cplx xc[3] = {x[0], x[1], x[2]}, sc[3] = {xi[0], xi[1], xi[2]}, g[3];
    double K[9];
    if (with_kelvin) {
        double r[3] = {x[0] - xi[0], x[1] - xi[1], x[2] - xi[2]};
        ho_kelvin_G(r, mu, nu, K);
    }
    for (int p = 0; p < 3; p++) {
        hs_corr_col(p, xc, sc, mu, nu, g);
        for (int k = 0; k < 3; k++) G[3 * k + p] = creal(g[k]) + (with_kelvin ? K[3 * k + p] : 0.0);
    }
}

int ho_halfspace_G(const double *x, const double *xi, double mu, double nu, int with_kelvin, double *G) {
    if (!(x[2] <= 0.0 && xi[2] <= 0.0) || x[2] + xi[2] >= 0.0) return -1;
    hs_green(x, xi, mu, nu, with_kelvin, G);
    return 0;
}

/* du[k][m] = d u_k / d x_m at x of the correction field of a point source of unit area at
 * xi with moment density M[p][q] = c_ijpq b_i n_j: sum_pq M_pq d2 G_kp / dx_m dxi_q.  The
 * xi-derivative along row p of M is a complex step (exact to rounding); the x-derivative a
 * fourth-order central difference with a step of 1e-3 of the vertical image distance. */
static void hs_point_grad(const double *x, const double *xi, const double M[3][3], double mu, double nu,
                          double du[3][3]) {
    const double D = -x[2] - xi[2], hx = 1e-3 * D;
    static const double st[4] = {-2.0, -1.0, 1.0, 2.0}, wt[4] = {1.0, -8.0, 8.0, -1.0};
    for (int k = 0; k < 3; k++)
        for (int m = 0; m < 3; m++) du[k][m] = 0.0;
    for (int m = 0; m < 3; m++)
        for (int s = 0; s < 4; s++) {
            cplx xs[3] = {x[0], x[1], x[2]};
            xs[m] += st[s] * hx;
            for (int p = 0; p < 3; p++) {
                const double nrm = sqrt(M[p][0] * M[p][0] + M[p][1] * M[p][1] + M[p][2] * M[p][2]);
                if (nrm == 0.0) continue;
                const double t = 1e-20 * D / nrm;
                cplx xi_c[3], g[3];
                for (int q = 0; q < 3; q++) xi_c[q] = xi[q] + _Complex_I * (t * M[p][q]);
                hs_corr_col(p, xs, xi_c, mu, nu, g);
                for (int k = 0; k < 3; k++) du[k][m] += wt[s] * cimag(g[k]) / t / (12.0 * hx);
            }
        }
}

/* Subdivision rule of the element quadrature: a triangle is integrated directly once its
 * diameter is at most hs_ratio times its vertical distance to the receiver's image. */
static double hs_ratio = 0.5;
void ho_set_halfspace_ratio(double r) { hs_ratio = r; }
/* 1: the product rule's order follows the distance to the image (below); 0: GL_N always. */
static int hs_adaptive = 1;
void ho_set_halfspace_adaptive(int on) { hs_adaptive = on; }

typedef struct {
    const double *x;
    int nb;
    double M[3][3][3];
    double mu, nu;
    double du[3][3][3];
} hs_ctx;

/* Triangle ABC: 4-way midpoint subdivision until small against its image distance, then the
 * GL_N x GL_N collapsed (Duffy) product rule: P(u, v) = A + u (B - A) + u v (C - B),
 * dS = u |(B - A) x (C - B)| du dv. */
static void hs_triangle(hs_ctx *H, const double *A, const double *B, const double *C, int depth) {
    double e[3], diam = 0.0;
    const double *V[3] = {A, B, C};
    for (int a = 0; a < 3; a++) {
        const double *P = V[a], *Q = V[(a + 1) % 3];
        for (int k = 0; k < 3; k++) e[k] = Q[k] - P[k];
        if (norm3(e) > diam) diam = norm3(e);
    }
    double zmax = A[2];
    if (B[2] > zmax) zmax = B[2];
    if (C[2] > zmax) zmax = C[2];
    const double D = -H->x[2] - zmax;
    if (diam > hs_ratio * D && depth < 14) {
        double ab[3], bc[3], ca[3];
        for (int k = 0; k < 3; k++) {
            ab[k] = 0.5 * (A[k] + B[k]);
            bc[k] = 0.5 * (B[k] + C[k]);
            ca[k] = 0.5 * (C[k] + A[k]);
        }
        hs_triangle(H, A, ab, ca, depth + 1);
        hs_triangle(H, ab, B, bc, depth + 1);
        hs_triangle(H, ca, bc, C, depth + 1);
        hs_triangle(H, ab, bc, ca, depth + 1);
        return;
    }
    double BA[3], CB[3], cr[3];
    for (int k = 0; k < 3; k++) { BA[k] = B[k] - A[k]; CB[k] = C[k] - B[k]; }
    cross3(BA, CB, cr);
    const double J = norm3(cr);
    /* Rule order: the integrand is analytic away from the image of the triangle, at least
     * R = |x - image of the centroid| - diam from it, and an n x n rule errs by about
     * (diam / (2 R))^(2n); the smallest n reaching 1e-13 (all GL_N with hs_adaptive off). */
    int nq = GL_N;
    if (hs_adaptive) {
        const double ci[3] = {(A[0] + B[0] + C[0]) / 3.0, (A[1] + B[1] + C[1]) / 3.0, -(A[2] + B[2] + C[2]) / 3.0};
        const double d[3] = {H->x[0] - ci[0], H->x[1] - ci[1], H->x[2] - ci[2]};
        const double R = norm3(d) - diam;
        if (R > 0.0) {
            const double q = diam / (2.0 * R);
            for (int n = 2; n < GL_N; n++)
                if (pow(q, 2.0 * n) <= 1e-13) { nq = n; break; }
        }
    }
    const double *gx = gl_tab_x[nq], *gw = gl_tab_w[nq];
    for (int gu = 0; gu < nq; gu++)
        for (int gv = 0; gv < nq; gv++) {
            const double u = 0.5 * (1.0 + gx[gu]), v = 0.5 * (1.0 + gx[gv]);
            const double w = 0.25 * gw[gu] * gw[gv] * u * J;
            double xi[3], du[3][3];
            for (int k = 0; k < 3; k++) xi[k] = A[k] + u * BA[k] + u * v * CB[k];
            for (int ib = 0; ib < H->nb; ib++) {
                hs_point_grad(H->x, xi, H->M[ib], H->mu, H->nu, du);
                for (int k = 0; k < 3; k++)
                    for (int m = 0; m < 3; m++) H->du[ib][k][m] += w * du[k][m];
            }
        }
}

/* Correction stress sig[ib][3][3] at x (x_z <= 0) from uniform slip b[ib] over the planar
 * polygon P (normal from the vertex order), the polygon split into the triangles
 * (P0, Pa, Pa+1).  Returns -1 unless every vertex has z <= 0, x is on or below the surface
 * and the two are not both on it (the correction is singular where they meet). */
static int polygon_stress_hs_corr(int nv, const double *P, int nb, const double *b, double mu, double nu,
                                  const double *x, double *sig) {
    gl_init();
    double zmax = -INFINITY;
    for (int a = 0; a < nv; a++)
        if (P[3 * a + 2] > zmax) zmax = P[3 * a + 2];
    if (!(zmax <= 0.0) || !(x[2] <= 0.0) || !(-x[2] - zmax > 0.0) || nb < 1 || nb > 3) return -1;
    double c[3], n[3], s[3], d[3], area;
    elem_frame(nv, P, c, n, s, d, &area);
    hs_ctx H;
    memset(&H, 0, sizeof H);
    H.x = x; H.nb = nb; H.mu = mu; H.nu = nu;
    const double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    for (int ib = 0; ib < nb; ib++) {
        const double *bb = b + 3 * ib, bn = dot3(bb, n);
        for (int p = 0; p < 3; p++)
            for (int q = 0; q < 3; q++) H.M[ib][p][q] = lam * bn * (p == q) + mu * (bb[p] * n[q] + bb[q] * n[p]);
    }
    for (int a = 1; a + 1 < nv; a++) hs_triangle(&H, P, P + 3 * a, P + 3 * (a + 1), 0);
    for (int ib = 0; ib < nb; ib++) {
        const double tr = H.du[ib][0][0] + H.du[ib][1][1] + H.du[ib][2][2];
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++)
                sig[9 * ib + 3 * k + l] = lam * (k == l) * tr + mu * (H.du[ib][k][l] + H.du[ib][l][k]);
    }
    return 0;
}

/* Half-space stress (full space + correction) of a uniform-slip polygon at x; with
 * corr_only, the correction alone. */
int ho_stress_polygon_hs(int nv, const double *P, int nb, const double *b, double mu, double nu,
                         const double *x, int corr_only, double *sig) {
    double sc[27];
    int rc = polygon_stress_hs_corr(nv, P, nb, b, mu, nu, x, sc);
    if (rc) return rc;
    if (corr_only) {
        memcpy(sig, sc, sizeof(double) * 9 * nb);
        return 0;
    }
    rc = polygon_stress(nv, P, nb, b, mu, nu, x, sig);
    for (int k = 0; k < 9 * nb; k++) sig[k] += sc[k];
    return rc;
}

/* ------------------------------------------------------- mesh + entries */
typedef struct {
    int n, nv;
    const double *verts;
    double *cent, *nrm, *str, *dip, *area;
    double mu, nu;
    int half;   /* 1: half space z < 0 with a free surface z = 0 */
} mesh_t;

/* Operator kinds may carry HO_HALF_SPACE: the half-space form of the same operator. */
#define HO_HALF_SPACE 16

static void mesh_init(mesh_t *M, int n, int nv, const double *verts, double mu, double nu) {
    gl_init(); /* before any parallel region */
    M->n = n; M->nv = nv; M->verts = verts; M->mu = mu; M->nu = nu; M->half = 0;
    M->cent = malloc(sizeof(double) * 3 * n);
    M->nrm = malloc(sizeof(double) * 3 * n);
    M->str = malloc(sizeof(double) * 3 * n);
    M->dip = malloc(sizeof(double) * 3 * n);
    M->area = malloc(sizeof(double) * n);
    ho_elem_frames(n, nv, verts, M->cent, M->nrm, M->str, M->dip, M->area);
}
static void mesh_free(mesh_t *M) {
    free(M->cent); free(M->nrm); free(M->str); free(M->dip); free(M->area);
}

/* Full 3x2 traction response T[c_out][c_in] at the centre of receiver i to unit slip
 * of source j along its strike (c_in = 0) and dip (c_in = 1) directions.
 * c_out: 0 = strike shear s.sig.n, 1 = dip shear d.sig.n, 2 = normal stress change,
 * compression positive (-n.sig.n). */
static int pair_full(const mesh_t *M, int i, int j, double T[3][2]) {
    double b[6], sig[18];
    for (int k = 0; k < 3; k++) { b[k] = M->str[3 * j + k]; b[3 + k] = M->dip[3 * j + k]; }
    int rc = M->half ? ho_stress_polygon_hs(M->nv, M->verts + (size_t)j * M->nv * 3, 2, b, M->mu, M->nu,
                                            M->cent + 3 * i, 0, sig)
                     : polygon_stress(M->nv, M->verts + (size_t)j * M->nv * 3, 2, b, M->mu, M->nu,
                                      M->cent + 3 * i, sig);
    const double *n = M->nrm + 3 * i, *s = M->str + 3 * i, *d = M->dip + 3 * i;
    for (int ib = 0; ib < 2; ib++) {
        double tr[3];
        for (int k = 0; k < 3; k++)
            tr[k] = sig[9 * ib + 3 * k] * n[0] + sig[9 * ib + 3 * k + 1] * n[1] + sig[9 * ib + 3 * k + 2] * n[2];
        T[0][ib] = dot3(s, tr);
        T[1][ib] = dot3(d, tr);
        T[2][ib] = -dot3(n, tr);
    }
    return rc;
}

/* Operator entries E[c_out][c_in] for operator kind op; rake angles (strike->dip) enter
 * the single-component forms. */
static int pair_op(const mesh_t *M, int op, const double *rake, int i, int j, double E[3][2]) {
    double T[3][2];
    int rc = pair_full(M, i, j, T);
    if (op == HO_OP_VEC_FULL || op == HO_OP_VEC_SHEAR) {
        for (int a = 0; a < 3; a++)
            for (int c = 0; c < 2; c++) E[a][c] = T[a][c];
        return rc;
    }
    double cj = cos(rake[j]), sj = sin(rake[j]), ci = cos(rake[i]), si = sin(rake[i]);
    double col[3];
    for (int a = 0; a < 3; a++) col[a] = T[a][0] * cj + T[a][1] * sj;
    E[0][0] = ci * col[0] + si * col[1];
    E[1][0] = col[2];
    return rc;
}

/* Entries of the operator for a list of (receiver, source) element pairs:
 * out[p][c_out][c_in] with the op's n_out x n_in shape. */
int ho_pair_entries(int n, int nv, const double *verts, double mu, double nu, int op,
                    const double *rake, int npairs, const int *recv, const int *src, double *out) {
    mesh_t M;
    mesh_init(&M, n, nv, verts, mu, nu);
    M.half = (op & HO_HALF_SPACE) != 0;
    op &= ~HO_HALF_SPACE;
    int no = op_nout(op), ni = op_nin(op), bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int p = 0; p < npairs; p++) {
        double E[3][2];
        bad |= pair_op(&M, op, rake, recv[p], src[p], E) != 0;
        for (int a = 0; a < no; a++)
            for (int c = 0; c < ni; c++) out[(size_t)p * no * ni + a * ni + c] = E[a][c];
    }
    mesh_free(&M);
    return bad ? -1 : 0;
}

/* Dense operator rows (Eqs. 5-6): for each receiver element in `rows`, y_row[c_out] =
 * sum_j E_ij x_j, x in original order, component-major (x[c*n + j]). Output
 * y[r * n_out + c_out]. */
int ho_dense_rows(int n, int nv, const double *verts, double mu, double nu, int op,
                  const double *rake, int nrows, const int *rows, const double *x, double *y) {
    mesh_t M;
    mesh_init(&M, n, nv, verts, mu, nu);
    M.half = (op & HO_HALF_SPACE) != 0;
    op &= ~HO_HALF_SPACE;
    int no = op_nout(op), ni = op_nin(op), bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int r = 0; r < nrows; r++) {
        double acc[3] = {0, 0, 0};
        for (int j = 0; j < n; j++) {
            double E[3][2];
            bad |= pair_op(&M, op, rake, rows[r], j, E) != 0;
            for (int a = 0; a < no; a++)
                for (int c = 0; c < ni; c++) acc[a] += E[a][c] * x[(size_t)c * n + j];
        }
        for (int a = 0; a < no; a++) y[(size_t)r * no + a] = acc[a];
    }
    mesh_free(&M);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------ cluster tree */
typedef struct {
    int start, size, depth, child[2];
    double lo[3], hi[3];
} cluster_t;

typedef struct {
    int n, leaf;
    int *perm;            /* tree position -> original element */
    cluster_t *cl;
    int ncl, cap;
    const double *cent;
} tree_t;

static int cmp_axis;
static const double *cmp_cent;
static int cmp_idx(const void *a, const void *b) {
    int ia = *(const int *)a, ib = *(const int *)b;
    double ca = cmp_cent[3 * ia + cmp_axis], cb = cmp_cent[3 * ib + cmp_axis];
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (ia > ib) - (ia < ib);
}

/* Sec. 3.1.1: binary cluster tree on element centres.  Split the bounding box of the
 * centres at the midpoint of its longest side (stable partition, ties to the right);
 * if one side would be empty, split at the median.  Leaves hold <= leaf elements. */
static int tree_build(tree_t *T, int start, int size, int depth) {
    if (T->ncl == T->cap) {
        T->cap *= 2;
        T->cl = realloc(T->cl, sizeof(cluster_t) * T->cap);
    }
    int id = T->ncl++;
    cluster_t *C = &T->cl[id];
    C->start = start; C->size = size; C->depth = depth; C->child[0] = C->child[1] = -1;
    for (int k = 0; k < 3; k++) { C->lo[k] = 1e300; C->hi[k] = -1e300; }
    for (int i = start; i < start + size; i++)
        for (int k = 0; k < 3; k++) {
            double v = T->cent[3 * T->perm[i] + k];
            if (v < C->lo[k]) C->lo[k] = v;
            if (v > C->hi[k]) C->hi[k] = v;
        }
    if (size <= T->leaf) return id;
    int axis = 0;
    for (int k = 1; k < 3; k++)
        if (C->hi[k] - C->lo[k] > C->hi[axis] - C->lo[axis]) axis = k;
    double mid = 0.5 * (C->lo[axis] + C->hi[axis]);
    int *tmp = malloc(sizeof(int) * size), nl = 0;
    for (int i = start; i < start + size; i++)
        if (T->cent[3 * T->perm[i] + axis] < mid) tmp[nl++] = T->perm[i];
    int nr = 0;
    for (int i = start; i < start + size; i++)
        if (!(T->cent[3 * T->perm[i] + axis] < mid)) tmp[nl + nr++] = T->perm[i];
    if (nl == 0 || nr == 0) {
        memcpy(tmp, T->perm + start, sizeof(int) * size);
        cmp_axis = axis; cmp_cent = T->cent;
        qsort(tmp, size, sizeof(int), cmp_idx);
        nl = size / 2;
    }
    memcpy(T->perm + start, tmp, sizeof(int) * size);
    free(tmp);
    int c0 = tree_build(T, start, nl, depth + 1);
    int c1 = tree_build(T, start + nl, size - nl, depth + 1);
    T->cl[id].child[0] = c0;
    T->cl[id].child[1] = c1;
    return id;
}

static double cl_diam(const cluster_t *C) {
    double d2 = 0;
    for (int k = 0; k < 3; k++) d2 += (C->hi[k] - C->lo[k]) * (C->hi[k] - C->lo[k]);
    return sqrt(d2);
}
static double cl_dist(const cluster_t *A, const cluster_t *B) {
    double d2 = 0;
    for (int k = 0; k < 3; k++) {
        double g = 0;
        if (B->lo[k] > A->hi[k]) g = B->lo[k] - A->hi[k];
        else if (A->lo[k] > B->hi[k]) g = A->lo[k] - B->hi[k];
        d2 += g * g;
    }
    return sqrt(d2);
}
/* Eq. 17 */
static int admissible(const cluster_t *A, const cluster_t *B, double eta) {
    double da = cl_diam(A), db = cl_diam(B);
    return (da < db ? da : db) < eta * cl_dist(A, B);
}

/* ---------------------------------------------------------- block partition */
typedef struct {
    int tau, sig;        /* cluster ids */
    int row0, m, col0, nc; /* DOF offsets / sizes (interleaved components) */
    int lowrank, rank;
    size_t off;          /* offset into data */
} block_t;

typedef struct {
    mesh_t M;
    tree_t T;
    int op, nin, nout;
    const double *rake;
    double *rake_copy;
    double eps, eta;
    int lattice_depth;
    block_t *blk;
    int nblk, cap;
    double *data;
    size_t ndata;
    int *lattice;        /* lattice cluster ids */
    int nlat;
    int status;
} hmat_t;

static void push_block(hmat_t *H, int tau, int sig, int lr) {
    if (H->nblk == H->cap) {
        H->cap = H->cap ? 2 * H->cap : 1024;
        H->blk = realloc(H->blk, sizeof(block_t) * H->cap);
    }
    block_t *B = &H->blk[H->nblk++];
    const cluster_t *A = &H->T.cl[tau], *S = &H->T.cl[sig];
    B->tau = tau; B->sig = sig;
    B->row0 = H->nout * A->start; B->m = H->nout * A->size;
    B->col0 = H->nin * S->start; B->nc = H->nin * S->size;
    B->lowrank = lr; B->rank = 0; B->off = 0;
}

static int is_leaf(const cluster_t *C) { return C->child[0] < 0; }

static void partition(hmat_t *H, int tau, int sig) {
    const cluster_t *A = &H->T.cl[tau], *S = &H->T.cl[sig];
    if (admissible(A, S, H->eta)) { push_block(H, tau, sig, 1); return; }
    if (is_leaf(A) && is_leaf(S)) { push_block(H, tau, sig, 0); return; }
    if (is_leaf(A)) { partition(H, tau, S->child[0]); partition(H, tau, S->child[1]); return; }
    if (is_leaf(S)) { partition(H, A->child[0], sig); partition(H, A->child[1], sig); return; }
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) partition(H, A->child[a], S->child[b]);
}

static void collect_lattice(hmat_t *H, int c, int L) {
    const cluster_t *C = &H->T.cl[c];
    if (C->depth == L || is_leaf(C)) { H->lattice[H->nlat++] = c; return; }
    collect_lattice(H, C->child[0], L);
    collect_lattice(H, C->child[1], L);
}

/* --------------------------------------------------------------------- ACA */
/* scalar entry of block B: row I (receiver comp I % nout of element tau.start + I/nout),
 * column J (source comp J % nin of element sig.start + J/nin). */
static void block_row(const hmat_t *H, const block_t *B, int I, double *row) {
    const cluster_t *A = &H->T.cl[B->tau], *S = &H->T.cl[B->sig];
    int i = H->T.perm[A->start + I / H->nout], co = I % H->nout;
    for (int jj = 0; jj < S->size; jj++) {
        double E[3][2];
        pair_op(&H->M, H->op, H->rake, i, H->T.perm[S->start + jj], E);
        for (int c = 0; c < H->nin; c++) row[jj * H->nin + c] = E[co][c];
    }
}
static void block_col(const hmat_t *H, const block_t *B, int J, double *col) {
    const cluster_t *A = &H->T.cl[B->tau], *S = &H->T.cl[B->sig];
    int j = H->T.perm[S->start + J / H->nin], ci = J % H->nin;
    for (int ii = 0; ii < A->size; ii++) {
        double E[3][2];
        pair_op(&H->M, H->op, H->rake, H->T.perm[A->start + ii], j, E);
        for (int a = 0; a < H->nout; a++) col[ii * H->nout + a] = E[a][ci];
    }
}

/* Dense block, row-major m x nc. */
static double *block_dense(const hmat_t *H, const block_t *B) {
    double *D = malloc(sizeof(double) * (size_t)B->m * B->nc);
    const cluster_t *A = &H->T.cl[B->tau], *S = &H->T.cl[B->sig];
    for (int ii = 0; ii < A->size; ii++)
        for (int jj = 0; jj < S->size; jj++) {
            double E[3][2];
            pair_op(&H->M, H->op, H->rake, H->T.perm[A->start + ii], H->T.perm[S->start + jj], E);
            for (int a = 0; a < H->nout; a++)
                for (int c = 0; c < H->nin; c++)
                    D[(size_t)(ii * H->nout + a) * B->nc + jj * H->nin + c] = E[a][c];
        }
    return D;
}

/* Sec. 3.1.2: adaptive cross approximation with partial pivoting (Bebendorf 2000).
 * A ~ sum_k u_k v_k^T (u_k: m, v_k: nc; the paper's g_ki = u_k[i], h_kj = v_k[j]).
 * Start at row 0; pivot column = argmax |residual row| over unused columns; next row =
 * argmax |u_k| over unused rows (ties -> smallest index); a zero residual row moves to
 * the next unused row.  Stop once |u_k||v_k| <= eps ||S_k||_F (recursive Frobenius
 * norm of the approximant).  If the rank reaches floor(m nc / (m + nc)) the block is
 * stored dense instead (rank cap).  Returns rank, or -1 for "store dense";
 * U, V are column-major (m x r, nc x r). */
typedef void (*aca_row_fn)(const void *ctx, int I, double *row);
typedef void (*aca_col_fn)(const void *ctx, int J, double *col);

static int aca_generic(int m, int nc, double eps, aca_row_fn rowf, aca_col_fn colf, const void *ctx,
                       double **Uo, double **Vo) {
    int rcap = (int)(((long)m * nc) / (m + nc));
    int cap = 8;
    double *U = malloc(sizeof(double) * (size_t)m * cap), *V = malloc(sizeof(double) * (size_t)nc * cap);
    char *urow = calloc(m, 1), *ucol = calloc(nc, 1);
    double *row = malloc(sizeof(double) * nc), *col = malloc(sizeof(double) * m);
    double normS2 = 0.0;
    int k = 0, i = 0;
    for (;;) {
        if (k >= rcap) { k = -1; break; }
        rowf(ctx, i, row);
        for (int l = 0; l < k; l++) {
            double ui = U[(size_t)l * m + i];
            for (int J = 0; J < nc; J++) row[J] -= ui * V[(size_t)l * nc + J];
        }
        urow[i] = 1;
        int j = -1;
        double best = 0.0;
        for (int J = 0; J < nc; J++)
            if (!ucol[J] && fabs(row[J]) > best) { best = fabs(row[J]); j = J; }
        if (j < 0) {
            int nxt = -1;
            for (int I = 0; I < m; I++) if (!urow[I]) { nxt = I; break; }
            if (nxt < 0) break;
            i = nxt;
            continue;
        }
        if (k == cap) {
            cap *= 2;
            U = realloc(U, sizeof(double) * (size_t)m * cap);
            V = realloc(V, sizeof(double) * (size_t)nc * cap);
        }
        double piv = row[j];
        double *v = V + (size_t)k * nc, *u = U + (size_t)k * m;
        for (int J = 0; J < nc; J++) v[J] = row[J] / piv;
        colf(ctx, j, col);
        for (int l = 0; l < k; l++) {
            double vj = V[(size_t)l * nc + j];
            for (int I = 0; I < m; I++) col[I] -= vj * U[(size_t)l * m + I];
        }
        for (int I = 0; I < m; I++) u[I] = col[I];
        ucol[j] = 1;
        double uu = 0, vv = 0, cross = 0;
        for (int I = 0; I < m; I++) uu += u[I] * u[I];
        for (int J = 0; J < nc; J++) vv += v[J] * v[J];
        for (int l = 0; l < k; l++) {
            double a = 0, b = 0;
            for (int I = 0; I < m; I++) a += U[(size_t)l * m + I] * u[I];
            for (int J = 0; J < nc; J++) b += V[(size_t)l * nc + J] * v[J];
            cross += a * b;
        }
        normS2 += 2.0 * cross + uu * vv;
        k++;
        if (sqrt(uu * vv) <= eps * sqrt(normS2 > 0 ? normS2 : 0)) break;
        int nxt = -1;
        double bu = -1.0;
        for (int I = 0; I < m; I++)
            if (!urow[I] && fabs(u[I]) > bu) { bu = fabs(u[I]); nxt = I; }
        if (nxt < 0) break;
        i = nxt;
    }
    free(urow); free(ucol); free(row); free(col);
    if (k < 0) { free(U); free(V); *Uo = *Vo = NULL; return -1; }
    *Uo = U; *Vo = V;
    return k;
}

typedef struct { const hmat_t *H; const block_t *B; } blk_ctx;
static void blk_row(const void *c, int I, double *row) { const blk_ctx *b = c; block_row(b->H, b->B, I, row); }
static void blk_col(const void *c, int J, double *col) { const blk_ctx *b = c; block_col(b->H, b->B, J, col); }
static int aca(const hmat_t *H, const block_t *B, double **Uo, double **Vo) {
    blk_ctx c = {H, B};
    return aca_generic(B->m, B->nc, H->eps, blk_row, blk_col, &c, Uo, Vo);
}

/* ACA on an explicit row-major m x nc matrix (for tests of the approximation itself). */
typedef struct { const double *A; int m, nc; } mat_ctx;
static void mat_row(const void *c, int I, double *row) { const mat_ctx *a = c; memcpy(row, a->A + (size_t)I * a->nc, sizeof(double) * a->nc); }
static void mat_col(const void *c, int J, double *col) { const mat_ctx *a = c; for (int I = 0; I < a->m; I++) col[I] = a->A[(size_t)I * a->nc + J]; }
/* returns rank (U: m x r, V: nc x r column-major written to U, V with room for rmax), -1 if capped */
int ho_aca_matrix(int m, int nc, const double *A, double eps, int rmax, double *U, double *V) {
    mat_ctx c = {A, m, nc};
    double *Uo, *Vo;
    int r = aca_generic(m, nc, eps, mat_row, mat_col, &c, &Uo, &Vo);
    if (r < 0) return -1;
    if (r > rmax) { free(Uo); free(Vo); return -2; }
    memcpy(U, Uo, sizeof(double) * (size_t)m * r);
    memcpy(V, Vo, sizeof(double) * (size_t)nc * r);
    free(Uo); free(Vo);
    return r;
}

/* ------------------------------------------------------------- H build */
/* A bounded sample of the operator (for timing the oracle on meshes it cannot build whole in
 * reasonable time): when set to a lattice row a >= 0, the build computes the factors of the
 * blocks whose rows lie in lattice cluster a only, exactly as the whole build computes them
 * (every block's ACA is independent of the others); the other blocks are not built,
 * so the product gives the rows of lattice row a of the whole product and zeros elsewhere.
 * The other blocks keep their place and kind in the partition, with rank -1 and no data.
 * -1 (the default) builds every block. */
static int sample_lattice_row = -1;
void ho_set_sample_lattice_row(int a) { sample_lattice_row = a; }

void *ho_build(int n, int nv, const double *verts, double mu, double nu, int op, const double *rake,
               double eps, int leaf, int lattice_depth, double eta) {
    hmat_t *H = calloc(1, sizeof(hmat_t));
    mesh_init(&H->M, n, nv, verts, mu, nu);
    H->M.half = (op & HO_HALF_SPACE) != 0;
    op &= ~HO_HALF_SPACE;
    H->op = op; H->nin = op_nin(op); H->nout = op_nout(op);
    H->rake_copy = malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) H->rake_copy[i] = rake ? rake[i] : 0.0;
    H->rake = H->rake_copy;
    H->eps = eps; H->eta = eta; H->lattice_depth = lattice_depth;
    tree_t *T = &H->T;
    T->n = n; T->leaf = leaf; T->cent = H->M.cent;
    T->perm = malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) T->perm[i] = i;
    T->cap = 64; T->ncl = 0;
    T->cl = malloc(sizeof(cluster_t) * T->cap);
    tree_build(T, 0, n, 0);
    H->lattice = malloc(sizeof(int) * T->ncl);
    H->nlat = 0;
    collect_lattice(H, 0, lattice_depth);
    /* Sec. 3.2: an H-matrix partition inside each lattice block, lattice row-major. */
    for (int a = 0; a < H->nlat; a++)
        for (int b = 0; b < H->nlat; b++) partition(H, H->lattice[a], H->lattice[b]);
    /* rows of the sampled lattice row, if any (DOF range [s_lo, s_hi)) */
    int s_lo = 0, s_hi = H->nout * n;
    if (sample_lattice_row >= 0 && sample_lattice_row < H->nlat) {
        const cluster_t *Ls = &T->cl[H->lattice[sample_lattice_row]];
        s_lo = H->nout * Ls->start;
        s_hi = H->nout * (Ls->start + Ls->size);
    }
    /* factors per block (independent -> parallel; each block computed sequentially) */
    double **DU = calloc(H->nblk, sizeof(double *)), **DV = calloc(H->nblk, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 1)
    for (int ib = 0; ib < H->nblk; ib++) {
        block_t *B = &H->blk[ib];
        if (B->row0 < s_lo || B->row0 >= s_hi) {   /* outside the sample: rank -1, no data */
            B->rank = -1;
            continue;
        }
        if (B->lowrank) {
            double *U, *V;
            int r = aca(H, B, &U, &V);
            if (r < 0) { B->lowrank = 0; DU[ib] = block_dense(H, B); }
            else { B->rank = r; DU[ib] = U; DV[ib] = V; }
        } else {
            DU[ib] = block_dense(H, B);
        }
    }
    size_t tot = 0;
    for (int ib = 0; ib < H->nblk; ib++) {
        block_t *B = &H->blk[ib];
        B->off = tot;
        if (B->rank < 0) continue;   /* outside the sample */
        tot += B->lowrank ? (size_t)(B->m + B->nc) * B->rank : (size_t)B->m * B->nc;
    }
    H->data = malloc(sizeof(double) * (tot ? tot : 1));
    H->ndata = tot;
    for (int ib = 0; ib < H->nblk; ib++) {
        block_t *B = &H->blk[ib];
        if (B->rank < 0) continue;   /* outside the sample */
        if (B->lowrank) {
            if (B->rank) memcpy(H->data + B->off, DU[ib], sizeof(double) * (size_t)B->m * B->rank);
            if (B->rank) memcpy(H->data + B->off + (size_t)B->m * B->rank, DV[ib], sizeof(double) * (size_t)B->nc * B->rank);
            free(DV[ib]);
        } else {
            memcpy(H->data + B->off, DU[ib], sizeof(double) * (size_t)B->m * B->nc);
        }
        free(DU[ib]);
    }
    free(DU); free(DV);
    return H;
}

void ho_free(void *h) {
    hmat_t *H = h;
    if (!H) return;
    mesh_free(&H->M);
    free(H->rake_copy); free(H->T.perm); free(H->T.cl); free(H->lattice); free(H->blk); free(H->data);
    free(H);
}

/* sizes: [n, nclusters, nblocks, ndata, nlattice, nin, nout, n_lowrank] */
int ho_info(void *h, long *out) {
    hmat_t *H = h;
    long nlr = 0;
    for (int i = 0; i < H->nblk; i++) nlr += H->blk[i].lowrank;
    out[0] = H->M.n; out[1] = H->T.ncl; out[2] = H->nblk; out[3] = (long)H->ndata;
    out[4] = H->nlat; out[5] = H->nin; out[6] = H->nout; out[7] = nlr;
    return 0;
}

/* perm[n]; clusters[ncl][6] = start,size,depth,child0,child1,0; cl_box[ncl][6];
 * blocks[nblk][8] = row0,m,col0,nc,lowrank,rank,off,tau; data[ndata];
 * lattice[nlat] */
int ho_export(void *h, int *perm, long *clusters, double *cl_box, long *blocks, double *data, long *lattice) {
    hmat_t *H = h;
    if (perm) memcpy(perm, H->T.perm, sizeof(int) * H->M.n);
    if (clusters)
        for (int c = 0; c < H->T.ncl; c++) {
            const cluster_t *C = &H->T.cl[c];
            long *o = clusters + 6 * c;
            o[0] = C->start; o[1] = C->size; o[2] = C->depth; o[3] = C->child[0]; o[4] = C->child[1]; o[5] = 0;
            for (int k = 0; k < 3; k++) { cl_box[6 * c + k] = C->lo[k]; cl_box[6 * c + 3 + k] = C->hi[k]; }
        }
    if (blocks)
        for (int b = 0; b < H->nblk; b++) {
            const block_t *B = &H->blk[b];
            long *o = blocks + 8 * b;
            o[0] = B->row0; o[1] = B->m; o[2] = B->col0; o[3] = B->nc;
            o[4] = B->lowrank; o[5] = B->rank; o[6] = (long)B->off; o[7] = B->tau;
        }
    if (data) memcpy(data, H->data, sizeof(double) * H->ndata);
    if (lattice)
        for (int i = 0; i < H->nlat; i++) lattice[i] = H->lattice[i];
    return 0;
}

/* ------------------------------------------------------------------ HMVM */
/* Eq. 20 in the permuted, component-interleaved index space: y = sum_blocks. */
static void hmv_perm(const hmat_t *H, const double *xp, double *yp) {
    int ndof_out = H->nout * H->M.n;
    memset(yp, 0, sizeof(double) * ndof_out);
    double *t = NULL;
    int tcap = 0;
    for (int ib = 0; ib < H->nblk; ib++) {
        const block_t *B = &H->blk[ib];
        if (B->rank < 0) continue;   /* outside a sampled build's lattice row */
        const double *D = H->data + B->off;
        if (!B->lowrank) {
            for (int I = 0; I < B->m; I++) {
                double acc = 0.0;
                for (int J = 0; J < B->nc; J++) acc += D[(size_t)I * B->nc + J] * xp[B->col0 + J];
                yp[B->row0 + I] += acc;
            }
        } else {
            int r = B->rank;
            if (r > tcap) { tcap = r; t = realloc(t, sizeof(double) * tcap); }
            const double *U = D, *V = D + (size_t)B->m * r;
            for (int l = 0; l < r; l++) {
                double acc = 0.0;
                for (int J = 0; J < B->nc; J++) acc += V[(size_t)l * B->nc + J] * xp[B->col0 + J];
                t[l] = acc;
            }
            for (int I = 0; I < B->m; I++) {
                double acc = 0.0;
                for (int l = 0; l < r; l++) acc += U[(size_t)l * B->m + I] * t[l];
                yp[B->row0 + I] += acc;
            }
        }
    }
    free(t);
}

/* x original order component-major (x[c*n + j]) -> y original order (y[c*n + i]). */
int ho_hmatvec(void *h, const double *x, double *y) {
    hmat_t *H = h;
    int n = H->M.n, ni = H->nin, no = H->nout;
    double *xp = malloc(sizeof(double) * ni * n), *yp = malloc(sizeof(double) * no * n);
    for (int p = 0; p < n; p++)
        for (int c = 0; c < ni; c++) xp[ni * p + c] = x[(size_t)c * n + H->T.perm[p]];
    hmv_perm(H, xp, yp);
    for (int p = 0; p < n; p++)
        for (int c = 0; c < no; c++) y[(size_t)c * n + H->T.perm[p]] = yp[no * p + c];
    free(xp); free(yp);
    return 0;
}

/* in the permuted interleaved space directly (for factor-level parity) */
int ho_hmatvec_perm(void *h, const double *xp, double *yp) {
    hmv_perm((hmat_t *)h, xp, yp);
    return 0;
}

/* ------------------------------------------------------ rate-state ODE */
typedef struct {
    const double *a, *b, *dc, *rake;   /* per element */
    const double *tau_dot, *sig_dot;   /* loading rates (Eqs. 21-22) */
    double f0, V0, Vpl, mu, cs;
} ho_fric;

/* Eq. 7, read as tau/sigma = a asinh(V/(2 V0) exp(phi/a)), solved for V. */
static double slip_rate(double phi, double tau, double sig, double a, double V0) {
    return 2.0 * V0 * exp(-phi / a) * sinh(tau / (a * sig));
}

/* Eqs. 13a-c (with the Eq. 7 reading exp(-phi/a)): out = dV/dtau, dV/dsigma, dV/dphi. */
static void dV_partials(double phi, double tau, double sig, double a, double V0, double *out) {
    double e = exp(-phi / a), arg = tau / (a * sig);
    out[0] = 2.0 * V0 / (a * sig) * e * cosh(arg);
    out[1] = -2.0 * V0 * tau / (a * sig * sig) * e * cosh(arg);
    out[2] = -2.0 * V0 / a * e * sinh(arg);
}

int ho_slip_rate(int n, const double *phi, const double *tau, const double *sig, const double *a,
                 double V0, double *V, double *partials) {
    for (int i = 0; i < n; i++) {
        V[i] = slip_rate(phi[i], tau[i], sig[i], a[i], V0);
        if (partials) dV_partials(phi[i], tau[i], sig[i], a[i], V0, partials + 3 * i);
    }
    return 0;
}

int ho_steady_state(int n, const double *V, const double *a, const double *b, const double *sig,
                    double f0, double V0, double *phi, double *tau) {
    for (int i = 0; i < n; i++) {
        phi[i] = f0 - b[i] * log(V[i] / V0);                         /* Eq. 8 = 0 */
        tau[i] = a[i] * sig[i] * asinh(V[i] / (2.0 * V0) * exp(phi[i] / a[i]));  /* Eq. 7 */
    }
    return 0;
}

/* Eqs. 21-22: loading rates from one H-matvec of the backslip -V_pl along the rake. */
int ho_loading(void *h, const double *rake, double Vpl, double *tau_dot, double *sig_dot) {
    hmat_t *H = h;
    int n = H->M.n, ni = H->nin, no = H->nout;
    double *x = malloc(sizeof(double) * ni * n), *y = malloc(sizeof(double) * no * n);
    for (int j = 0; j < n; j++) {
        if (ni == 1) x[j] = -Vpl;
        else { x[j] = -Vpl * cos(rake[j]); x[n + j] = -Vpl * sin(rake[j]); }
    }
    ho_hmatvec(h, x, y);
    for (int i = 0; i < n; i++) {
        if (H->op == HO_OP_RAKE_SHEAR) { tau_dot[i] = y[i]; sig_dot[i] = 0.0; }
        else if (H->op == HO_OP_RAKE_SHEAR_NORMAL) { tau_dot[i] = y[i]; sig_dot[i] = y[n + i]; }
        else {
            tau_dot[i] = cos(rake[i]) * y[i] + sin(rake[i]) * y[n + i];
            sig_dot[i] = (H->op == HO_OP_VEC_FULL) ? y[2 * n + i] : 0.0;
        }
    }
    free(x); free(y);
    return 0;
}

/* dy/dt for y = (phi[n], tau[n], sigma[n])  (Eqs. 7-13), V returned in Vout. */
/* Eqs. 8, 10, 12 and 13a-c at element i, given the element's stress rates s_i (its n_out
 * operator outputs: tau | tau, sigma | tau_s, tau_d[, sigma]) and slip rate V. */
static void rhs_element(int op, const ho_fric *F, int i, double phi, double tau, double sig, double V,
                        const double *s_i, double *dphi_out, double *dtau_out, double *dsig_out) {
    double AV, BV;
    if (op == HO_OP_RAKE_SHEAR) { AV = s_i[0]; BV = 0.0; }
    else if (op == HO_OP_RAKE_SHEAR_NORMAL) { AV = s_i[0]; BV = s_i[1]; }
    else {
        AV = cos(F->rake[i]) * s_i[0] + sin(F->rake[i]) * s_i[1];
        BV = (op == HO_OP_VEC_FULL) ? s_i[2] : 0.0;
    }
    double eta_rad = F->mu / (2.0 * F->cs);
    double a = F->a[i], b = F->b[i], V0 = F->V0;
    double dphi = (b / F->dc[i]) * (V0 * exp((F->f0 - phi) / b) - V);                 /* Eq. 8 */
    double dsig = BV + F->sig_dot[i];                                                  /* Eq. 10 */
    double dV[3];
    dV_partials(phi, tau, sig, a, V0, dV);                                             /* Eqs. 13a-c */
    double dtau = (AV + F->tau_dot[i] - eta_rad * (dV[1] * dsig + dV[2] * dphi))
                  / (1.0 + eta_rad * dV[0]);                                           /* Eq. 12 */
    *dphi_out = dphi;
    *dtau_out = dtau;
    *dsig_out = dsig;
}

int ho_rhs(void *h, const ho_fric *F, const double *y, double *dydt, double *Vout) {
    hmat_t *H = h;
    int n = H->M.n, ni = H->nin, no = H->nout;
    const double *phi = y, *tau = y + n, *sig = y + 2 * n;
    double *V = malloc(sizeof(double) * n), *x = malloc(sizeof(double) * ni * n),
           *s = malloc(sizeof(double) * no * n);
    for (int i = 0; i < n; i++) V[i] = slip_rate(phi[i], tau[i], sig[i], F->a[i], F->V0);
    for (int j = 0; j < n; j++) {
        if (ni == 1) x[j] = V[j];
        else { x[j] = V[j] * cos(F->rake[j]); x[n + j] = V[j] * sin(F->rake[j]); }
    }
    ho_hmatvec(h, x, s);
    for (int i = 0; i < n; i++) {
        double s_i[3];
        for (int c = 0; c < no; c++) s_i[c] = s[(size_t)c * n + i];
        rhs_element(H->op, F, i, phi[i], tau[i], sig[i], V[i], s_i, &dydt[i], &dydt[n + i], &dydt[2 * n + i]);
    }
    if (Vout) memcpy(Vout, V, sizeof(double) * n);
    free(V); free(x); free(s);
    return 0;
}

/* The element-wise right-hand side at selected elements rows[k] of the state y (3n), given
 * their stress rates s_rows[k][n_out] (for example rows of the dense operator applied to the
 * slip-rate deficit, which then carry the loading: tau_dot = sig_dot = 0).  Out: dydt_rows
 * [k][3] = (dphi, dtau, dsigma). */
int ho_rhs_rows(int op, const ho_fric *F, int n, const double *y, int nrows, const int *rows,
                const double *s_rows, double *dydt_rows) {
    int no = op == HO_OP_RAKE_SHEAR ? 1 : (op == HO_OP_VEC_FULL ? 3 : 2);
    for (int k = 0; k < nrows; k++) {
        int i = rows[k];
        if (i < 0 || i >= n) return -1;
        double V = slip_rate(y[i], y[n + i], y[2 * n + i], F->a[i], F->V0);
        rhs_element(op, F, i, y[i], y[n + i], y[2 * n + i], V, s_rows + (size_t)k * no, &dydt_rows[3 * k],
                    &dydt_rows[3 * k + 1], &dydt_rows[3 * k + 2]);
    }
    return 0;
}

/* Cash & Karp (1990) embedded Runge-Kutta 4(5) tableau. */
static const double CK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double CK_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

int ho_cash_karp_tableau(double *c, double *a, double *b5, double *b4) {
    memcpy(c, CK_C, sizeof CK_C);
    memcpy(a, CK_A, sizeof CK_A);
    memcpy(b5, CK_B5, sizeof CK_B5);
    memcpy(b4, CK_B4, sizeof CK_B4);
    return 0;
}

/* Generic embedded step for dy/dt = f(y) of size m (used with the rate-state RHS and
 * with test problems).  err = max_i |y5 - y4| / max(|y5|, 1e-30). */
typedef void (*rhs_fn)(void *ctx, const double *y, double *dy);

static double ck_step(rhs_fn f, void *ctx, int m, const double *y, double dt, double *y5, double *work) {
    double *k[6], *ys = work + 6 * (size_t)m;
    for (int s = 0; s < 6; s++) k[s] = work + (size_t)s * m;
    for (int s = 0; s < 6; s++) {
        for (int i = 0; i < m; i++) {
            double acc = 0.0;
            for (int l = 0; l < s; l++) acc += CK_A[s][l] * k[l][i];
            ys[i] = y[i] + dt * acc;
        }
        f(ctx, ys, k[s]);
    }
    double err = 0.0;
    for (int i = 0; i < m; i++) {
        double s5 = 0.0, s4 = 0.0;
        for (int l = 0; l < 6; l++) { s5 += CK_B5[l] * k[l][i]; s4 += CK_B4[l] * k[l][i]; }
        y5[i] = y[i] + dt * s5;
        double y4 = y[i] + dt * s4;
        double den = fabs(y5[i]) > 1e-30 ? fabs(y5[i]) : 1e-30;
        double e = fabs(y5[i] - y4) / den;
        if (!isfinite(e)) e = INFINITY;   /* a non-finite trial is rejected (Eq. 14, err -> inf) */
        if (e > err) err = e;
    }
    return err;
}

/* Eqs. 14-15 (reading: exponents on err/eps). Returns 1 on accept. */
static int controller(double err, double eps, double dt, double *dt_new) {
    if (!(err <= eps)) {   /* a NaN error (non-finite trial) is rejected, dt halves */
        double d = 0.9 * dt * pow(err / eps, -0.25);
        *dt_new = d > 0.5 * dt ? d : 0.5 * dt;
        return 0;
    }
    double d = err > 0 ? 0.9 * dt * pow(err / eps, -0.2) : 2.0 * dt;
    *dt_new = d < 2.0 * dt ? d : 2.0 * dt;
    return 1;
}

int ho_controller(double err, double eps, double dt, double *dt_new) { return controller(err, eps, dt, dt_new); }

typedef struct { void *H; const ho_fric *F; } rs_ctx;
static void rs_rhs(void *c, const double *y, double *dy) {
    rs_ctx *C = c;
    ho_rhs(C->H, C->F, y, dy, NULL);
}

/* Test ODE y' = -lambda y (componentwise rate in ctx). */
static void lin_rhs(void *c, const double *y, double *dy) {
    const double *lam = c;
    dy[0] = -lam[0] * y[0];
}
int ho_ck_linear_step(double lam, double y0, double dt, double *y5, double *err) {
    double work[7], out;
    *err = ck_step(lin_rhs, &lam, 1, &y0, dt, &out, work);
    *y5 = out;
    return 0;
}

/* One attempted step of the rate-state system; returns err, y5 in y_new. */
int ho_rk_attempt(void *h, const ho_fric *F, const double *y, double dt, double *y_new, double *err) {
    hmat_t *H = h;
    int m = 3 * H->M.n;
    double *work = malloc(sizeof(double) * 7 * (size_t)m);
    rs_ctx C = {h, F};
    *err = ck_step(rs_rhs, &C, m, y, dt, y_new, work);
    free(work);
    return 0;
}

/* Advance n_steps accepted steps (Eqs. 14-16).  y (3n) and D (n) updated in place;
 * t, dt in/out.  rec[s][4] = t, dt_used, max V, rejects before acceptance.
 * Returns number of accepted steps, or -1 if the step size underflows (< 1e-12 s). */
int ho_run(void *h, const ho_fric *F, double *y, double *D, double *t, double *dt, double eps,
           int n_steps, double *rec) {
    hmat_t *H = h;
    int n = H->M.n, m = 3 * n;
    double *work = malloc(sizeof(double) * 7 * (size_t)m), *y5 = malloc(sizeof(double) * m),
           *V0v = malloc(sizeof(double) * n), *V1v = malloc(sizeof(double) * n), *dy = malloc(sizeof(double) * m);
    rs_ctx C = {h, F};
    int acc = 0, rej = 0;
    while (acc < n_steps) {
        double err = ck_step(rs_rhs, &C, m, y, *dt, y5, work);
        if (!(*dt > 1e-12)) { acc = -1; break; }   /* step-size underflow */
        double dt_new;
        if (controller(err, eps, *dt, &dt_new)) {
            for (int i = 0; i < n; i++) V0v[i] = slip_rate(y[i], y[n + i], y[2 * n + i], F->a[i], F->V0);
            for (int i = 0; i < n; i++) V1v[i] = slip_rate(y5[i], y5[n + i], y5[2 * n + i], F->a[i], F->V0);
            double vmax = 0;
            for (int i = 0; i < n; i++) {
                D[i] += 0.5 * (*dt) * (V0v[i] + V1v[i]);                 /* Eq. 16 */
                if (V1v[i] > vmax) vmax = V1v[i];
            }
            memcpy(y, y5, sizeof(double) * m);
            *t += *dt;
            if (rec) {
                rec[4 * acc + 0] = *t; rec[4 * acc + 1] = *dt; rec[4 * acc + 2] = vmax; rec[4 * acc + 3] = rej;
            }
            acc++;
            rej = 0;
        } else {
            rej++;
        }
        *dt = dt_new;
    }
    (void)dy;
    free(work); free(y5); free(V0v); free(V1v); free(dy);
    return acc;
}

/* ------------------------------------------------ rake-free (vector) friction
 * The paper's friction is scalar along a fixed rake (Eqs. 5-13).  Without a fixed rake the
 * shear traction is a vector tau = (tau_s, tau_d) in the (strike, dip) frame and the slip
 * rate is parallel to it: V = g(|tau|, phi, sigma) tau/|tau| with g the Eq. 7 slip rate at
 * the traction magnitude.  The quasi-dynamic balance tau = tau_el - eta V (eta = mu/(2 c_s))
 * gives (I + eta dV/dtau) dtau/dt = dtau_el/dt - eta (dV/dphi dphi/dt + dV/dsigma dsigma/dt),
 * with dV/dtau = g' t t^T + (g/|tau|)(I - t t^T) (t = tau/|tau|, g' = dg/d|tau|) and the
 * other partials along t; dtau_el/dt and dsigma/dt come from the product of the slip-rate
 * deficit V - V_pl r (plate motion along the loading direction r).  Aging law unchanged. */

/* y = (phi[n], tau_s[n], tau_d[n], sigma[n]); V out as (V_s[n], V_d[n]). */
int ho_rhs_vec(void *h, const ho_fric *F, const double *y, double *dydt, double *Vout) {
    hmat_t *H = h;
    int n = H->M.n;
    if (H->op != HO_OP_VEC_FULL && H->op != HO_OP_VEC_SHEAR) return -1;
    const double *phi = y, *ts = y + n, *td = y + 2 * n, *sig = y + 3 * n;
    double *x = malloc(sizeof(double) * 2 * n), *s = malloc(sizeof(double) * H->nout * n);
    double *g = malloc(sizeof(double) * n), *ux = malloc(sizeof(double) * n), *uy = malloc(sizeof(double) * n),
           *tn = malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) {
        tn[i] = sqrt(ts[i] * ts[i] + td[i] * td[i]);
        if (tn[i] > 0.0) { ux[i] = ts[i] / tn[i]; uy[i] = td[i] / tn[i]; }
        else { ux[i] = cos(F->rake[i]); uy[i] = sin(F->rake[i]); }   /* no traction: the loading direction */
        g[i] = slip_rate(phi[i], tn[i], sig[i], F->a[i], F->V0);
        x[i] = g[i] * ux[i] - F->Vpl * cos(F->rake[i]);             /* slip-rate deficit */
        x[n + i] = g[i] * uy[i] - F->Vpl * sin(F->rake[i]);
    }
    ho_hmatvec(h, x, s);
    double eta = F->mu / (2.0 * F->cs);
    for (int i = 0; i < n; i++) {
        double a = F->a[i], b = F->b[i], V0 = F->V0;
        double dphi = (b / F->dc[i]) * (V0 * exp((F->f0 - phi[i]) / b) - g[i]);     /* Eq. 8 */
        double dsig = (H->op == HO_OP_VEC_FULL) ? s[2 * n + i] : 0.0;              /* Eq. 10 */
        double dV[3];
        dV_partials(phi[i], tn[i], sig[i], a, V0, dV);       /* dg/d|tau|, dg/dsigma, dg/dphi */
        double gt = tn[i] > 0.0 ? g[i] / tn[i] : dV[0];       /* g/|tau| -> g' as |tau| -> 0 */
        double rs = s[i] - eta * (dV[2] * dphi + dV[1] * dsig) * ux[i];
        double rd = s[n + i] - eta * (dV[2] * dphi + dV[1] * dsig) * uy[i];
        double par = rs * ux[i] + rd * uy[i];
        double ps = rs - par * ux[i], pd = rd - par * uy[i];
        double kpar = par / (1.0 + eta * dV[0]), kper = 1.0 / (1.0 + eta * gt);
        dydt[i] = dphi;
        dydt[n + i] = kpar * ux[i] + kper * ps;
        dydt[2 * n + i] = kpar * uy[i] + kper * pd;
        dydt[3 * n + i] = dsig;
        if (Vout) { Vout[i] = g[i] * ux[i]; Vout[n + i] = g[i] * uy[i]; }
    }
    free(x); free(s); free(g); free(ux); free(uy); free(tn);
    return 0;
}

/* Embedded step of the vector system: the error of an element is its largest relative
 * change among phi, the traction vector (relative to |tau5|) and sigma. */
static double ck_step_vec(void *h, const ho_fric *F, int n, const double *y, double dt, double *y5,
                          double *work) {
    int m = 4 * n;
    double *k[6], *ys = work + 6 * (size_t)m;
    for (int s = 0; s < 6; s++) k[s] = work + (size_t)s * m;
    for (int s = 0; s < 6; s++) {
        for (int i = 0; i < m; i++) {
            double acc = 0.0;
            for (int l = 0; l < s; l++) acc += CK_A[s][l] * k[l][i];
            ys[i] = y[i] + dt * acc;
        }
        ho_rhs_vec(h, F, ys, k[s], NULL);
    }
    double err = 0.0, y4[4];
    for (int i = 0; i < n; i++) {
        for (int c = 0; c < 4; c++) {
            int j = c * n + i;
            double s5 = 0.0, s4 = 0.0;
            for (int l = 0; l < 6; l++) { s5 += CK_B5[l] * k[l][j]; s4 += CK_B4[l] * k[l][j]; }
            y5[j] = y[j] + dt * s5;
            y4[c] = y[j] + dt * s4;
        }
        double tn5 = sqrt(y5[n + i] * y5[n + i] + y5[2 * n + i] * y5[2 * n + i]);
        double dts = y5[n + i] - y4[1], dtd = y5[2 * n + i] - y4[2];
        double e0 = fabs(y5[i] - y4[0]) / fmax(fabs(y5[i]), 1e-30);
        double e1 = sqrt(dts * dts + dtd * dtd) / fmax(tn5, 1e-30);
        double e2 = fabs(y5[3 * n + i] - y4[3]) / fmax(fabs(y5[3 * n + i]), 1e-30);
        double e = fmax(e0, fmax(e1, e2));   /* fmax drops NaN: the three are tested below */
        if (!isfinite(e0) || !isfinite(e1) || !isfinite(e2) || !(y5[3 * n + i] > 0.0)) e = INFINITY;   /* rejected */
        if (e > err) err = e;
    }
    return err;
}

int ho_rk_attempt_vec(void *h, const ho_fric *F, const double *y, double dt, double *y_new, double *err) {
    int n = ((hmat_t *)h)->M.n;
    double *work = malloc(sizeof(double) * 7 * 4 * (size_t)n);
    *err = ck_step_vec(h, F, n, y, dt, y_new, work);
    free(work);
    return 0;
}

/* As ho_run for y = (phi, tau_s, tau_d, sigma) (4n) and slip D = (D_s, D_d) (2n). */
int ho_run_vec(void *h, const ho_fric *F, double *y, double *D, double *t, double *dt, double eps,
               int n_steps, double *rec) {
    int n = ((hmat_t *)h)->M.n, m = 4 * n;
    double *work = malloc(sizeof(double) * 7 * (size_t)m), *y5 = malloc(sizeof(double) * m),
           *dy = malloc(sizeof(double) * m), *V0v = malloc(sizeof(double) * 2 * n), *V1v = malloc(sizeof(double) * 2 * n);
    int acc = 0, rej = 0;
    while (acc < n_steps) {
        double err = ck_step_vec(h, F, n, y, *dt, y5, work);
        if (!(*dt > 1e-12)) { acc = -1; break; }
        double dt_new;
        if (controller(err, eps, *dt, &dt_new)) {
            ho_rhs_vec(h, F, y, dy, V0v);
            ho_rhs_vec(h, F, y5, dy, V1v);
            double vmax = 0.0;
            for (int i = 0; i < n; i++) {
                D[i] += 0.5 * (*dt) * (V0v[i] + V1v[i]);             /* Eq. 16, per component */
                D[n + i] += 0.5 * (*dt) * (V0v[n + i] + V1v[n + i]);
                double vm = sqrt(V1v[i] * V1v[i] + V1v[n + i] * V1v[n + i]);
                if (vm > vmax) vmax = vm;
            }
            memcpy(y, y5, sizeof(double) * m);
            *t += *dt;
            if (rec) {
                rec[4 * acc + 0] = *t; rec[4 * acc + 1] = *dt; rec[4 * acc + 2] = vmax; rec[4 * acc + 3] = rej;
            }
            acc++;
            rej = 0;
        } else {
            rej++;
        }
        *dt = dt_new;
    }
    free(work); free(y5); free(dy); free(V0v); free(V1v);
    return acc;
}

/* ------------------------------------------------------ complex-step sensitivities */
typedef double complex cplx;

/* Eq. 7 (reading exp(-phi/a)) and Eqs. 13a-c in complex arithmetic */
static cplx slip_rate_c(cplx phi, cplx tau, cplx sig, cplx a, double V0) {
    return 2.0 * V0 * cexp(-phi / a) * csinh(tau / (a * sig));
}
static void dV_partials_c(cplx phi, cplx tau, cplx sig, cplx a, double V0, cplx *out) {
    cplx e = cexp(-phi / a), arg = tau / (a * sig);
    out[0] = 2.0 * V0 / (a * sig) * e * ccosh(arg);
    out[1] = -2.0 * V0 * tau / (a * sig * sig) * e * ccosh(arg);
    out[2] = -2.0 * V0 / a * e * csinh(arg);
}

/* dy/dt of Eqs. 8, 10, 12 for a complex state y (3n) and complex a, d_c; the product is
 * linear and real, so H (x_re + i x_im) = H x_re + i H x_im. */
static void rhs_c(hmat_t *H, const ho_fric *F, const cplx *a, const cplx *dc, const cplx *y, cplx *dydt,
                  cplx *V, double *xr, double *xi, double *sr, double *si) {
    int n = H->M.n, ni = H->nin, no = H->nout;
    const cplx *phi = y, *tau = y + n, *sig = y + 2 * n;
    for (int i = 0; i < n; i++) {
        V[i] = slip_rate_c(phi[i], tau[i], sig[i], a[i], F->V0);
        if (ni == 1) { xr[i] = creal(V[i]); xi[i] = cimag(V[i]); }
        else {
            cplx xs = V[i] * cos(F->rake[i]), xd = V[i] * sin(F->rake[i]);
            xr[i] = creal(xs); xi[i] = cimag(xs); xr[n + i] = creal(xd); xi[n + i] = cimag(xd);
        }
    }
    ho_hmatvec(H, xr, sr);
    ho_hmatvec(H, xi, si);
    double eta_rad = F->mu / (2.0 * F->cs);
    for (int i = 0; i < n; i++) {
        cplx s_i[3];
        for (int c = 0; c < no; c++) s_i[c] = sr[(size_t)c * n + i] + _Complex_I * si[(size_t)c * n + i];
        cplx AV, BV;
        if (H->op == HO_OP_RAKE_SHEAR) { AV = s_i[0]; BV = 0.0; }
        else if (H->op == HO_OP_RAKE_SHEAR_NORMAL) { AV = s_i[0]; BV = s_i[1]; }
        else {
            AV = cos(F->rake[i]) * s_i[0] + sin(F->rake[i]) * s_i[1];
            BV = (H->op == HO_OP_VEC_FULL) ? s_i[2] : 0.0;
        }
        double b = F->b[i];
        cplx dphi = (b / dc[i]) * (F->V0 * cexp((F->f0 - phi[i]) / b) - V[i]);      /* Eq. 8 */
        cplx dsig = BV + F->sig_dot[i];                                              /* Eq. 10 */
        cplx dV[3];
        dV_partials_c(phi[i], tau[i], sig[i], a[i], F->V0, dV);                      /* Eqs. 13a-c */
        cplx dtau = (AV + F->tau_dot[i] - eta_rad * (dV[1] * dsig + dV[2] * dphi))
                    / (1.0 + eta_rad * dV[0]);                                       /* Eq. 12 */
        dydt[i] = dphi;
        dydt[n + i] = dtau;
        dydt[2 * n + i] = dsig;
    }
}

/* n_steps Cash-Karp steps of the given sizes from y0 (3n, real) with a + i h a_dir and
 * d_c + i h dc_dir, each step accepted as it is (the 5th-order solution), then the loss
 * L = 1/2 sum_i (ln V_i(y_N) - target_i)^2.  out = (Re L, Im L / h): the loss and its
 * derivative along (a_dir, dc_dir) at fixed b. */
int ho_fixed_loss_cs(void *h, const ho_fric *F, const double *a_dir, const double *dc_dir, double step,
                     const double *y0, const double *dts, int n_steps, const double *target, double *out) {
    hmat_t *H = h;
    int n = H->M.n, m = 3 * n;
    cplx *a = malloc(sizeof(cplx) * n), *dc = malloc(sizeof(cplx) * n), *y = malloc(sizeof(cplx) * m),
         *ys = malloc(sizeof(cplx) * m), *k = malloc(sizeof(cplx) * 6 * (size_t)m), *V = malloc(sizeof(cplx) * n);
    double *xr = malloc(sizeof(double) * 2 * n), *xi = malloc(sizeof(double) * 2 * n),
           *sr = malloc(sizeof(double) * 3 * n), *si = malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < n; i++) {
        a[i] = F->a[i] + _Complex_I * step * (a_dir ? a_dir[i] : 0.0);
        dc[i] = F->dc[i] + _Complex_I * step * (dc_dir ? dc_dir[i] : 0.0);
    }
    for (int j = 0; j < m; j++) y[j] = y0[j];
    for (int st = 0; st < n_steps; st++) {
        double dt = dts[st];
        for (int s = 0; s < 6; s++) {
            for (int j = 0; j < m; j++) {
                cplx acc = 0.0;
                for (int l = 0; l < s; l++) acc += CK_A[s][l] * k[(size_t)l * m + j];
                ys[j] = y[j] + dt * acc;
            }
            rhs_c(H, F, a, dc, ys, k + (size_t)s * m, V, xr, xi, sr, si);
        }
        for (int j = 0; j < m; j++) {
            cplx acc = 0.0;
            for (int l = 0; l < 6; l++) acc += CK_B5[l] * k[(size_t)l * m + j];
            y[j] += dt * acc;
        }
    }
    cplx L = 0.0;
    for (int i = 0; i < n; i++) {
        cplx r = clog(slip_rate_c(y[i], y[n + i], y[2 * n + i], a[i], F->V0)) - target[i];
        L += 0.5 * r * r;
    }
    out[0] = creal(L);
    out[1] = step != 0.0 ? cimag(L) / step : 0.0;
    free(a); free(dc); free(y); free(ys); free(k); free(V); free(xr); free(xi); free(sr); free(si);
    return 0;
}

int ho_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the OpenMP loops from now on (k >= 1); returns the previous count */
int ho_set_num_threads(int k) {
    int prev = ho_num_threads();
#ifdef _OPENMP
    if (k >= 1) omp_set_num_threads(k);
#else
    (void)k;
#endif
    return prev;
}
