/*
 * CPU FP64 oracle for the constant-displacement-discontinuity (DD) influence
 * coefficients of rectangular and triangular elements in a 3D full space.
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
 *   phi's second and third derivatives are integrals over the element's edges (Stokes'
 *   theorem, below), each edge integrated numerically by adaptive Gauss-Legendre
 *   quadrature: the oracle shares no closed-form antiderivative with the device kernel,
 *   whose rectangle derivatives are corner sums and whose triangle ones are closed-form
 *   edge sums.
 * parity pinned by: the coplanar closed forms and self terms, brute-force quadrature
 * of the point source, far-field asymptotics, Sneddon's penny crack (tests).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_OK 0
#define ORC_SINGULAR (-4)

/* ---------------------------------------------------------------- triangles
 * The paper's element (Sec. 3.1) is a triangle.  phi = int int_T 1/R over the triangle;
 * every derivative of phi with an in-plane index alpha is a boundary integral by
 * Stokes' theorem (d/dx_alpha of 1/R = -d/dxi_alpha of 1/R):
 *   phi_{,alpha beta}       =  sum_edges n_alpha int_edge d_beta / R^3 ds,
 *   phi_{,alpha beta gamma} = -sum_edges n_alpha int_edge (3 d_beta d_gamma / R^5
 *                                                         - delta_beta gamma / R^3) ds,
 * d = x - xi(s), n the outward in-plane normal of the edge.  The x3-x3 derivatives
 * follow from Laplace's equation, as for the rectangle.  At a point inside the triangle
 * in its plane these are the values the derivatives take in the limit x3 -> 0 (the
 * finite parts of the hypersingular integrals).  The oracle integrates every edge
 * numerically -- adaptive Gauss-Legendre (16 nodes from Newton's method on P_16),
 * bisection until the two levels agree to 1e-15 of the integral's scale -- and uses no
 * closed-form antiderivative. */
#define GL_N 16
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    for (int i = 0; i < GL_N; ++i) {
        double x = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* the 8 edge integrands at xi = A + s tau: d_beta / R^3 (beta = 1..3), then
 * 3 d_b d_g / R^5 - delta_bg / R^3 for (b, g) = (1,1), (1,2), (2,2), (1,3), (2,3) */
#define EDGE_NF 8
static void edge_integrand(const double x[3], const double A[2], const double tau[2], double s, double f[EDGE_NF])
{
    double d0 = x[0] - (A[0] + s * tau[0]), d1 = x[1] - (A[1] + s * tau[1]), d2 = x[2];
    double R2 = d0 * d0 + d1 * d1 + d2 * d2, R = sqrt(R2);
    double r3 = 1.0 / (R2 * R), r5 = r3 / R2;
    f[0] = d0 * r3;
    f[1] = d1 * r3;
    f[2] = d2 * r3;
    f[3] = 3.0 * d0 * d0 * r5 - r3;
    f[4] = 3.0 * d0 * d1 * r5;
    f[5] = 3.0 * d1 * d1 * r5 - r3;
    f[6] = 3.0 * d0 * d2 * r5;
    f[7] = 3.0 * d1 * d2 * r5;
}

static void edge_gl(const double x[3], const double A[2], const double tau[2], double s0, double s1,
                    double out[EDGE_NF])
{
    double h = 0.5 * (s1 - s0), m = 0.5 * (s1 + s0), f[EDGE_NF];
    for (int c = 0; c < EDGE_NF; ++c) out[c] = 0.0;
    for (int i = 0; i < GL_N; ++i) {
        edge_integrand(x, A, tau, m + h * gl_x[i], f);
        for (int c = 0; c < EDGE_NF; ++c) out[c] += gl_w[i] * h * f[c];
    }
}

static void edge_adapt(const double x[3], const double A[2], const double tau[2], double s0, double s1,
                       const double whole[EDGE_NF], double scale, int depth, double acc[EDGE_NF])
{
    double m = 0.5 * (s0 + s1), l[EDGE_NF], r[EDGE_NF], err = 0.0;
    edge_gl(x, A, tau, s0, m, l);
    edge_gl(x, A, tau, m, s1, r);
    for (int c = 0; c < EDGE_NF; ++c) err = fmax(err, fabs(l[c] + r[c] - whole[c]));
    if (err <= 1e-15 * scale || depth >= 60) {
        for (int c = 0; c < EDGE_NF; ++c) acc[c] += l[c] + r[c];
        return;
    }
    edge_adapt(x, A, tau, s0, m, l, scale, depth + 1, acc);
    edge_adapt(x, A, tau, m, s1, r, scale, depth + 1, acc);
}

/* d2, d3 of phi at the point x (coordinates in the element's plane frame, element in
 * x3 = 0: the convex polygon with the nv vertices (pv[0], pv[1]), (pv[2], pv[3]), ... in
 * either orientation).  Returns ORC_SINGULAR when the point lies on the polygon's
 * boundary (in-plane, within tol). */
static int poly_phi_derivatives(const double x[3], const double* pv, int nv, double tol, double d2[3][3],
                                double d3[3][3][3])
{
    gl_init();
    double area2 = 0.0;  /* shoelace */
    for (int k = 0; k < nv; ++k) {
        const double* P = pv + 2 * k;
        const double* Q = pv + 2 * ((k + 1) % nv);
        area2 += P[0] * Q[1] - Q[0] * P[1];
    }
    const int rev = area2 < 0.0;  /* traverse counter-clockwise */
    double s[3][3] = {{0}}, t[2][EDGE_NF] = {{0}};
    /* s[alpha][beta] for alpha in-plane; t[alpha][c] the sums of n_alpha * integrand c */
    for (int e = 0; e < nv; ++e) {
        const int ia = rev ? (nv - e) % nv : e, ib = rev ? (nv - e - 1 + nv) % nv : (e + 1) % nv;
        const double* P = pv + 2 * ia;
        const double* Q = pv + 2 * ib;
        double L = hypot(Q[0] - P[0], Q[1] - P[1]);
        double tau[2] = {(Q[0] - P[0]) / L, (Q[1] - P[1]) / L};
        double nrm[2] = {tau[1], -tau[0]};
        /* the point on the edge (in-plane, within tol of the segment) is singular */
        if (fabs(x[2]) <= tol) {
            double w = (x[0] - P[0]) * tau[0] + (x[1] - P[1]) * tau[1];
            double dist = fabs((x[0] - P[0]) * nrm[0] + (x[1] - P[1]) * nrm[1]);
            if (dist <= tol && w >= -tol && w <= L + tol) return ORC_SINGULAR;
        }
        double whole[EDGE_NF], acc[EDGE_NF] = {0}, scale = 0.0;
        edge_gl(x, P, tau, 0.0, L, whole);
        /* the scale of the integrals: the integrands' size at the closest point */
        double w = fmin(fmax((x[0] - P[0]) * tau[0] + (x[1] - P[1]) * tau[1], 0.0), L);
        double dc[3] = {x[0] - P[0] - w * tau[0], x[1] - P[1] - w * tau[1], x[2]};
        double dmin = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
        scale = fmin(L, dmin) / (dmin * dmin * dmin);
        for (int c = 0; c < EDGE_NF; ++c) scale = fmax(scale, fabs(whole[c]));
        edge_adapt(x, P, tau, 0.0, L, whole, scale, 0, acc);
        for (int al = 0; al < 2; ++al) {
            for (int b = 0; b < 3; ++b) s[al][b] += nrm[al] * acc[b];
            for (int c = 0; c < EDGE_NF; ++c) t[al][c] += nrm[al] * acc[c];
        }
    }
    double s11 = s[0][0], s22 = s[1][1], s12 = s[0][1], s13 = s[0][2], s23 = s[1][2];
    /* t_{alpha beta gamma} = -sum n_alpha int (3 d_b d_g / R^5 - delta / R^3) */
    double t111 = -t[0][3], t112 = -t[0][4], t122 = -t[0][5], t222 = -t[1][5];
    double t113 = -t[0][6], t123 = -t[0][7], t223 = -t[1][7];
    double s33 = -s11 - s22, t133 = -t111 - t122, t233 = -t112 - t222, t333 = -t113 - t223;
    double D2[3][3] = {{s11, s12, s13}, {s12, s22, s23}, {s13, s23, s33}};
    memcpy(d2, D2, sizeof(D2));
    int idx[10][3] = {{0,0,0},{0,0,1},{0,1,1},{1,1,1},{0,0,2},{0,1,2},{1,1,2},{0,2,2},{1,2,2},{2,2,2}};
    double val[10] = {t111, t112, t122, t222, t113, t123, t223, t133, t233, t333};
    for (int q = 0; q < 10; ++q) {
        int i = idx[q][0], j = idx[q][1], k = idx[q][2];
        double v = val[q];
        d3[i][j][k] = d3[i][k][j] = d3[j][i][k] = d3[j][k][i] = d3[k][i][j] = d3[k][j][i] = v;
    }
    return ORC_OK;
}

/* The rectangle |x1| <= a, |x2| <= b and the triangle tv as polygons. */
static int phi_derivatives(const double x[3], double a, double b, double tol, double d2[3][3],
                           double d3[3][3][3])
{
    const double pv[8] = {-a, -b, a, -b, a, b, -a, b};
    return poly_phi_derivatives(x, pv, 4, tol, d2, d3);
}

static int tri_phi_derivatives(const double x[3], const double tv[6], double tol, double d2[3][3],
                               double d3[3][3][3])
{
    return poly_phi_derivatives(x, tv, 3, tol, d2, d3);
}

/* Frames are given as three unit vectors s1, s2, n (global components). */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

/* Traction block from phi's derivatives at the source-local point x: out[alpha*3 + m] is
 * traction component alpha (receiver frame, eloc[alpha] its axes on the source frame,
 * nloc the receiver normal there) from a unit DD component m of the source. */
static void traction_block(const double x[3], const double nloc[3], double eloc[3][3], double d2[3][3],
                           double d3[3][3][3], double mu, double nu, double out[9])
{
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
}

/* receiver point and frame on the source frame (origin at the source's collocation point) */
static void local_frame(const double xr[3], const double r1[3], const double r2[3], const double rn[3],
                        const double cs[3], const double q1[3], const double q2[3], const double qn[3],
                        double x[3], double nloc[3], double eloc[3][3])
{
    const double* rf[3] = {r1, r2, rn};
    const double* sf[3] = {q1, q2, qn};
    double d[3] = {xr[0] - cs[0], xr[1] - cs[1], xr[2] - cs[2]};
    for (int i = 0; i < 3; ++i) {
        x[i] = dot3(sf[i], d);
        nloc[i] = dot3(sf[i], rn);
        for (int al = 0; al < 3; ++al) eloc[al][i] = dot3(sf[i], rf[al]);
    }
}

/*
 * One 3x3 influence block: out[alpha*3 + m] = traction component alpha (receiver frame)
 * at xr from a unit DD component m (source frame) on the source rectangle.
 */
int orc_influence(const double xr[3], const double r1[3], const double r2[3], const double rn[3],
                  const double cs[3], const double q1[3], const double q2[3], const double qn[3],
                  double a, double b, double mu, double nu, double out[9])
{
    double x[3], nloc[3], eloc[3][3], d2[3][3], d3[3][3][3];
    local_frame(xr, r1, r2, rn, cs, q1, q2, qn, x, nloc, eloc);
    int st = phi_derivatives(x, a, b, 1e-9 * (a < b ? a : b), d2, d3);
    if (st != ORC_OK) {
        for (int q = 0; q < 9; ++q) out[q] = NAN;
        return st;
    }
    traction_block(x, nloc, eloc, d2, d3, mu, nu, out);
    return ORC_OK;
}

/* The same block from a source triangle given by its three vertices v (global, 9
 * numbers), collocated at cs with frame q1, q2, qn (qn normal to the triangle). */
int orc_influence_tri(const double xr[3], const double r1[3], const double r2[3], const double rn[3],
                      const double cs[3], const double q1[3], const double q2[3], const double qn[3],
                      const double v[9], double mu, double nu, double out[9])
{
    double x[3], nloc[3], eloc[3][3], d2[3][3], d3[3][3][3], tv[6];
    local_frame(xr, r1, r2, rn, cs, q1, q2, qn, x, nloc, eloc);
    for (int k = 0; k < 3; ++k) {
        double dv[3] = {v[3 * k] - cs[0], v[3 * k + 1] - cs[1], v[3 * k + 2] - cs[2]};
        tv[2 * k] = dot3(q1, dv);
        tv[2 * k + 1] = dot3(q2, dv);
    }
    double area = 0.5 * fabs((tv[2] - tv[0]) * (tv[5] - tv[1]) - (tv[3] - tv[1]) * (tv[4] - tv[0]));
    int st = tri_phi_derivatives(x, tv, 1e-9 * sqrt(area), d2, d3);
    if (st != ORC_OK) {
        for (int q = 0; q < 9; ++q) out[q] = NAN;
        return st;
    }
    traction_block(x, nloc, eloc, d2, d3, mu, nu, out);
    return ORC_OK;
}

/* Geometry arrays: c, s1, s2, n are N x 3 row-major; a, b are N (half sides of the
 * rectangles); shape is N (0 rectangle, 1 triangle) or NULL (all rectangles); tri is
 * N x 9 (the three vertices of each triangle, global; rows of rectangles unused). */
typedef struct {
    int64_t N;
    const double *c, *s1, *s2, *n, *a, *b;
    const int32_t* shape;
    const double* tri;
} orc_geom;

static int orc_block_ij(const orc_geom* g, int64_t i, int64_t j, double mu, double nu, double out[9])
{
    if (g->shape && g->shape[j] == 1)
        return orc_influence_tri(g->c + 3 * i, g->s1 + 3 * i, g->s2 + 3 * i, g->n + 3 * i,
                                 g->c + 3 * j, g->s1 + 3 * j, g->s2 + 3 * j, g->n + 3 * j,
                                 g->tri + 9 * j, mu, nu, out);
    return orc_influence(g->c + 3 * i, g->s1 + 3 * i, g->s2 + 3 * i, g->n + 3 * i,
                         g->c + 3 * j, g->s1 + 3 * j, g->s2 + 3 * j, g->n + 3 * j,
                         g->a[j], g->b[j], mu, nu, out);
}

/* Blocks for a list of (receiver, source) element pairs: out is npairs x 9.
 * Returns the number of singular pairs (their blocks are NaN). */
int64_t orc_blocks(int64_t N, const double* c, const double* s1, const double* s2, const double* n,
                   const double* a, const double* b, const int32_t* shape, const double* tri, double E,
                   double nu, int64_t npairs, const int64_t* ri, const int64_t* sj, double* out)
{
    orc_geom g = {N, c, s1, s2, n, a, b, shape, tri};
    gl_init();
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
                       const double* a, const double* b, const int32_t* shape, const double* tri, double E,
                       double nu, int64_t nr, const int64_t* rows, double* out)
{
    orc_geom g = {N, c, s1, s2, n, a, b, shape, tri};
    gl_init();
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
                              const double* n, const double* a, const double* b, const int32_t* shape,
                              const double* tri, double E, double nu, int64_t nr, const int64_t* rows,
                              int64_t nrhs, const double* x, double* y)
{
    orc_geom g = {N, c, s1, s2, n, a, b, shape, tri};
    gl_init();
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

/* phi derivatives of a triangle (source-local point, vertices in the source plane
 * frame, tv = x0, y0, x1, y1, x2, y2), exposed for the pins. */
int orc_tri_phi_derivatives(const double x[3], const double tv[6], double d2[9], double d3[27])
{
    double D2[3][3], D3[3][3][3];
    gl_init();
    double area = 0.5 * fabs((tv[2] - tv[0]) * (tv[5] - tv[1]) - (tv[3] - tv[1]) * (tv[4] - tv[0]));
    int st = tri_phi_derivatives(x, tv, 1e-9 * sqrt(area), D2, D3);
    memcpy(d2, D2, sizeof(D2));
    memcpy(d3, D3, sizeof(D3));
    return st;
}
