/*
 * CPU FP64 oracle for the constant-displacement-discontinuity (DD) influence
 * coefficients of rectangular elements in a 3D full space.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  It shares no code with the CUDA path.
 *
 * What it computes (Sec. 3.1, eq. TractionBIE-general reduced to the fracture
 * integral for an unbounded medium, eq. ElasSystem):  E_ij[alpha][m] is the traction
 * component alpha (receiver frame s1, s2, n) at the centroid of element i produced by
 * a unit DD component m (source frame s1, s2, n) that is constant over the rectangle
 * of element j.  Sign convention: delta = u+ - u- with the normal pointing from the
 * minus to the plus face (Sec. 2.2), T - T0 = E delta (eq. ElasSystem).
 *
 * Derivation (the paper integrates triangles analytically and prints no formula; the
 * rectangle version is written out here from the textbook point source):
 *   A DD b on dA with normal nu acts as a moment density M_pq = lambda (b.nu) d_pq
 *   + mu (b_p nu_q + b_q nu_p); its displacement is u_k = -M_pq d_q G_kp with Kelvin's
 *   tensor G_kp = [(3-4v) d_kp / r + r_k r_p / r^3] / (16 pi mu (1-v)).
 *   In source-local coordinates (plane x3 = 0) the integral over the rectangle
 *   reduces to derivatives of phi(x) = int int 1/R dxi deta, and the displacement
 *   gradient for b = e_m is
 *     u_{k,j} = -1/(8 pi (1-v)) [ 2(1-v) d_km phi_{3j} - (1-2v)(d_m3 phi_{kj}
 *               - d_k3 phi_{mj}) - d_j3 phi_{mk} - x3 phi_{mkj} ].
 *   Stress follows from Hooke's law, traction from the receiver normal.
 *   phi's second and third derivatives are corner sums of elementary antiderivatives
 *   (no logarithm or arctangent is needed at this order).
 * parity pinned by: the coplanar closed forms and self terms, brute-force quadrature
 * of the point source, far-field asymptotics, Sneddon's penny crack (tests).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_OK 0
#define ORC_SINGULAR (-4)

/* d2[i][j] = phi_ij, d3[i][j][k] = phi_ijk at the source-local point (x1,x2,x3) for the
 * rectangle |xi| <= a, |eta| <= b.  Returns ORC_SINGULAR when the point lies on the
 * rectangle's boundary (in-plane, within tol). */
static int phi_derivatives(const double x[3], double a, double b, double tol,
                           double d2[3][3], double d3[3][3][3])
{
    /* phi is even in each coordinate: evaluate at |x| and restore the signs below. */
    double sg[3], y[3];
    for (int i = 0; i < 3; ++i) {
        sg[i] = x[i] < 0.0 ? -1.0 : 1.0;
        y[i] = fabs(x[i]);
    }
    if (y[2] <= tol) {
        int on_edge_1 = fabs(y[0] - a) <= tol && y[1] <= b + tol;
        int on_edge_2 = fabs(y[1] - b) <= tol && y[0] <= a + tol;
        if (on_edge_1 || on_edge_2) return ORC_SINGULAR;
    }
    double z = y[2];
    double s11 = 0, s22 = 0, s12 = 0, s13 = 0, s23 = 0;
    double t111 = 0, t112 = 0, t122 = 0, t222 = 0, t113 = 0, t123 = 0, t223 = 0;
    for (int cu = 0; cu < 2; ++cu) {
        for (int cv = 0; cv < 2; ++cv) {
            double su = cu == 0 ? 1.0 : -1.0;
            double sv = cv == 0 ? 1.0 : -1.0;
            double s = su * sv;              /* corner sign of the double integral */
            double u = y[0] + su * a;        /* u = x1 - xi at xi = -su a */
            double v = y[1] + sv * b;
            double R = sqrt(u * u + v * v + z * z);
            double p = 1.0 / R;
            /* Av = 1/(v+R), Au = 1/(u+R), rationalised when the sum cancels */
            double Av = v >= 0.0 ? 1.0 / (v + R) : (R - v) / (u * u + z * z);
            double Au = u >= 0.0 ? 1.0 / (u + R) : (R - u) / (v * v + z * z);
            /* phi_1 = sum s ln(v+R), phi_2 = sum s ln(u+R); differentiate those */
            s11 += s * u * p * Av;
            s22 += s * v * p * Au;
            s12 += s * p;
            s13 += s * z * p * Av;
            s23 += s * z * p * Au;
            t111 += s * (p * Av - u * u * p * p * Av * (p + Av));
            t222 += s * (p * Au - v * v * p * p * Au * (p + Au));
            t112 += s * (-u * p * p * p);
            t122 += s * (-v * p * p * p);
            t123 += s * (-z * p * p * p);
            t113 += s * (-u * z * p * p * Av * (p + Av));
            t223 += s * (-v * z * p * p * Au * (p + Au));
        }
    }
    /* phi is harmonic off the element: the x3-x3 derivatives follow */
    double s33 = -s11 - s22;
    double t133 = -t111 - t122;
    double t233 = -t112 - t222;
    double t333 = -t113 - t223;

    double D2[3][3] = {{s11, s12, s13}, {s12, s22, s23}, {s13, s23, s33}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            d2[i][j] = D2[i][j] * sg[i] * sg[j];
    /* fill the symmetric third-derivative tensor from its 10 distinct entries */
    double T[3][3][3];
    int idx[10][3] = {{0,0,0},{0,0,1},{0,1,1},{1,1,1},{0,0,2},{0,1,2},{1,1,2},{0,2,2},{1,2,2},{2,2,2}};
    double val[10] = {t111, t112, t122, t222, t113, t123, t223, t133, t233, t333};
    for (int q = 0; q < 10; ++q) {
        int i = idx[q][0], j = idx[q][1], k = idx[q][2];
        double w = val[q];
        T[i][j][k] = T[i][k][j] = T[j][i][k] = T[j][k][i] = T[k][i][j] = T[k][j][i] = w;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                d3[i][j][k] = T[i][j][k] * sg[i] * sg[j] * sg[k];
    return ORC_OK;
}

/* Frames are given as three unit vectors s1, s2, n (global components). */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

/*
 * One 3x3 influence block: out[alpha*3 + m] = traction component alpha (receiver frame)
 * at xr from a unit DD component m (source frame) on the source rectangle.
 */
int orc_influence(const double xr[3], const double r1[3], const double r2[3], const double rn[3],
                  const double cs[3], const double q1[3], const double q2[3], const double qn[3],
                  double a, double b, double mu, double nu, double out[9])
{
    const double* rf[3] = {r1, r2, rn};  /* receiver frame */
    const double* sf[3] = {q1, q2, qn};  /* source frame */
    double d[3] = {xr[0] - cs[0], xr[1] - cs[1], xr[2] - cs[2]};
    double x[3], nloc[3], eloc[3][3];
    for (int i = 0; i < 3; ++i) {
        x[i] = dot3(sf[i], d);
        nloc[i] = dot3(sf[i], rn);
        for (int al = 0; al < 3; ++al) eloc[al][i] = dot3(sf[i], rf[al]);
    }
    double d2[3][3], d3[3][3][3];
    double tol = 1e-9 * (a < b ? a : b);
    int st = phi_derivatives(x, a, b, tol, d2, d3);
    if (st != ORC_OK) {
        for (int q = 0; q < 9; ++q) out[q] = NAN;
        return st;
    }
    double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    double K = 1.0 / (8.0 * M_PI * (1.0 - nu));
    for (int m = 0; m < 3; ++m) {
        double G[3][3];  /* G[k][j] = u_{k,j} for b = e_m */
        for (int k = 0; k < 3; ++k) {
            for (int j = 0; j < 3; ++j) {
                double term = 0.0;
                if (k == m) term += 2.0 * (1.0 - nu) * d2[2][j];
                term -= (1.0 - 2.0 * nu) * ((m == 2 ? d2[k][j] : 0.0) - (k == 2 ? d2[m][j] : 0.0));
                if (j == 2) term -= d2[m][k];
                term -= x[2] * d3[m][k][j];
                G[k][j] = -K * term;
            }
        }
        double th = G[0][0] + G[1][1] + G[2][2];
        double sig[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                sig[i][j] = (i == j ? lam * th : 0.0) + mu * (G[i][j] + G[j][i]);
        double t[3];
        for (int i = 0; i < 3; ++i) t[i] = sig[i][0] * nloc[0] + sig[i][1] * nloc[1] + sig[i][2] * nloc[2];
        for (int al = 0; al < 3; ++al) out[al * 3 + m] = dot3(eloc[al], t);
    }
    return ORC_OK;
}

/* Geometry arrays: c, s1, s2, n are N x 3 row-major; a, b are N. */
typedef struct {
    int64_t N;
    const double *c, *s1, *s2, *n, *a, *b;
} orc_geom;

static int orc_block_ij(const orc_geom* g, int64_t i, int64_t j, double mu, double nu, double out[9])
{
    return orc_influence(g->c + 3 * i, g->s1 + 3 * i, g->s2 + 3 * i, g->n + 3 * i,
                         g->c + 3 * j, g->s1 + 3 * j, g->s2 + 3 * j, g->n + 3 * j,
                         g->a[j], g->b[j], mu, nu, out);
}

/* Blocks for a list of (receiver, source) element pairs: out is npairs x 9.
 * Returns the number of singular pairs (their blocks are NaN). */
int64_t orc_blocks(int64_t N, const double* c, const double* s1, const double* s2, const double* n,
                   const double* a, const double* b, double E, double nu,
                   int64_t npairs, const int64_t* ri, const int64_t* sj, double* out)
{
    orc_geom g = {N, c, s1, s2, n, a, b};
    double mu = E / (2.0 * (1.0 + nu));
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+:bad)
    for (int64_t p = 0; p < npairs; ++p)
        if (orc_block_ij(&g, ri[p], sj[p], mu, nu, out + 9 * p) != ORC_OK) bad++;
    return bad;
}

/* Rows of the dense matrix for the receiver elements rows[0..nr): out is (3 nr) x (3N)
 * row-major, DOF order (s1, s2, n) per element (Sec. 3.1). */
int64_t orc_dense_rows(int64_t N, const double* c, const double* s1, const double* s2, const double* n,
                       const double* a, const double* b, double E, double nu,
                       int64_t nr, const int64_t* rows, double* out)
{
    orc_geom g = {N, c, s1, s2, n, a, b};
    double mu = E / (2.0 * (1.0 + nu));
    int64_t bad = 0;
    int64_t ld = 3 * N;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:bad)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows[r];
        for (int64_t j = 0; j < N; ++j) {
            double blk[9];
            if (orc_block_ij(&g, i, j, mu, nu, blk) != ORC_OK) bad++;
            for (int al = 0; al < 3; ++al)
                for (int m = 0; m < 3; ++m)
                    out[(3 * r + al) * ld + 3 * j + m] = blk[al * 3 + m];
        }
    }
    return bad;
}

/* Matrix-free dense product restricted to receiver rows: y[3r + al] = sum_j E_{rows[r], j} x_j
 * for nrhs right-hand sides stored as x[k * 3N + dof], y[k * 3 nr + dof]. */
int64_t orc_dense_matvec_rows(int64_t N, const double* c, const double* s1, const double* s2,
                              const double* n, const double* a, const double* b, double E, double nu,
                              int64_t nr, const int64_t* rows, int64_t nrhs, const double* x, double* y)
{
    orc_geom g = {N, c, s1, s2, n, a, b};
    double mu = E / (2.0 * (1.0 + nu));
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+:bad)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows[r];
        for (int64_t k = 0; k < nrhs; ++k)
            for (int al = 0; al < 3; ++al) y[k * 3 * nr + 3 * r + al] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double blk[9];
            if (orc_block_ij(&g, i, j, mu, nu, blk) != ORC_OK) { bad++; continue; }
            for (int64_t k = 0; k < nrhs; ++k) {
                const double* xj = x + k * 3 * N + 3 * j;
                for (int al = 0; al < 3; ++al)
                    y[k * 3 * nr + 3 * r + al] += blk[al * 3 + 0] * xj[0] + blk[al * 3 + 1] * xj[1]
                                                 + blk[al * 3 + 2] * xj[2];
            }
        }
    }
    return bad;
}

/* phi derivatives exposed for the pins (source-local point, rectangle half sides). */
int orc_phi_derivatives(const double x[3], double a, double b, double d2[9], double d3[27])
{
    double D2[3][3], D3[3][3][3];
    int st = phi_derivatives(x, a, b, 1e-9 * (a < b ? a : b), D2, D3);
    memcpy(d2, D2, sizeof(D2));
    memcpy(d3, D3, sizeof(D3));
    return st;
}
