/*
 * hmat.h -- C ABI of the GB300 H-matrix displacement-discontinuity BEM hot path.
 *
 * The library evaluates the 3D full-space influence coefficients of constant-DD
 * rectangles (Sec. 3.1, eq. TractionBIE-general reduced to the fracture integral,
 * eq. ElasSystem), compresses the far field of the collocation matrix E into an
 * H-matrix (Sec. 3.1: near-field blocks kept dense, far-field blocks low rank), applies
 * it (the O(n log n) product of Sec. 3.1) and solves the elastic tangent system
 * A = E - diag(k) - shift I (eq. jac_mech with C^ep = diag(k) and eta/dt = shift) by
 * restarted GMRES with a leaf block-Jacobi preconditioner (Sec. 3.3.1).
 *
 * Conventions shared by every entry point:
 *   - DOF order is element-major with (s1, s2, n) per element, in the user's element
 *     order (Sec. 3.1); tractions are ordered the same way.
 *   - Sign: delta = u+ - u- (Sec. 2.2) and T - T0 = E delta (eq. ElasSystem); the
 *     diagonal of E is negative.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller and not
 *     retained after the call returns; every other pointer is host memory, also
 *     caller-owned and copied if needed.  Handles (hm_tree, hm_hmat, hm_lp) are
 *     owned by the library and freed by their destroy function.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - Every function returns an hm_status; 0 is success, a negative value an error
 *     whose text hm_last_error() returns (per calling thread).  Nothing throws.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hm_status;
#define HM_OK 0
#define HM_EINVAL (-1)          /* bad argument */
#define HM_ENOMEM (-2)          /* device or host allocation failed */
#define HM_ECUDA (-3)           /* a CUDA call failed */
#define HM_ESINGULAR_GEOM (-4)  /* a collocation point lies on a source element's edge */
#define HM_ENOCONV (-5)         /* iteration limit reached before the tolerance */
#define HM_EBREAKDOWN (-6)      /* breakdown of an iteration */
#define HM_ENAN (-7)            /* NaN or Inf met in the data */
#define HM_ETIMEOUT (-8)        /* a bounded device wait gave up */

/* Precision / dtype codes. */
#define HM_F32 1
#define HM_F64 2
#define HM_BF16 3
#define HM_F32_BF16 4  /* storage: keep both FP32 and BF16 copies of the factors */

/* Text of the last error raised on the calling thread ("" if none). */
const char* hm_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int hm_version(void);

/* Element shapes. */
#define HM_SHAPE_RECT 0 /* rectangle c +- a s1 +- b s2 */
#define HM_SHAPE_TRI 1  /* triangle (Sec. 3.1: the paper's element) given by its vertices */

/* Element geometry, host SoA (Sec. 2.2 frame, Sec. 3.1 collocation at centroids):
 * c, s1, s2, n are N x 3 row-major (collocation point and the orthonormal frame; the
 * DD components of an element are along s1, s2, n).  a and b are the half sides along
 * s1 and s2 of a rectangle (> 0; the entries of triangles are not read).
 * shape: N codes HM_SHAPE_RECT / HM_SHAPE_TRI, or NULL (every element a rectangle).
 * tri: N x 9 row-major, the three vertices (global) of every triangle (rows of
 * rectangles unused; may be NULL when no element is a triangle).  A triangle must be
 * non-degenerate, lie in the plane through c normal to n (within 1e-6 of its size),
 * and contain c (the collocation point; the centroid in the paper).  Invalid geometry
 * returns HM_EINVAL, non-finite values HM_ENAN.  The caller keeps ownership; the
 * library copies. */
typedef struct {
    int64_t N;
    const double* c;
    const double* s1;
    const double* s2;
    const double* n;
    const double* a;
    const double* b;
    const int32_t* shape;
    const double* tri;
} hm_elements;

/* ---------------------------------------------------------------- influence blocks
 * 3x3 influence blocks for a list of (receiver i, source j) element pairs (Sec. 3.1,
 * eq. ElasSystem): out_dev[9p + 3 alpha + m] is the traction component alpha (frame of
 * receiver ri_dev[p]) at its centroid due to a unit DD component m (frame of source
 * sj_dev[p]) constant over the source element.  Evaluated in FP64 on the device.
 * ri_dev, sj_dev: npairs int64 element indices; out_dev: 9 npairs doubles.
 * Returns HM_ESINGULAR_GEOM (after writing every other block) if a receiver lies on a
 * source edge; those blocks are NaN.  Synchronises the stream. */
hm_status hm_influence_blocks(const hm_elements* el, double E, double nu, int64_t npairs,
                              const int64_t* ri_dev, const int64_t* sj_dev, double* out_dev,
                              void* stream);

/* The same blocks without any device allocation, for callers that may not call
 * cudaMalloc where they evaluate coefficients (a pooled or caching allocator that owns
 * all device memory, a latency-critical path where cudaMalloc/cudaFree would
 * synchronise the device, an embedding with a fixed memory budget).  The paper has no
 * counterpart: it is an interface convenience of this library.
 * The geometry is copied into one fixed scratch array in the library's device globals
 * (8 MiB, held by every GPU that loads the library until the process exits), so N is
 * limited to 65,536 elements; a larger N returns HM_EINVAL without touching the GPU.
 * The first call on a device looks up that array's address (set-up once per device):
 * make that first call before any stream capture.  Every call shares the array and
 * leaves its contents behind; the error word is cleared at the start of each call.
 * Calls that overlap on the GPU (from several threads or streams) race on the array.
 * Rectangles only: a triangle among the elements returns HM_EINVAL.
 * Arguments, outputs and errors are those of hm_influence_blocks; synchronises the
 * stream. */
hm_status hm_influence_blocks_noalloc(const hm_elements* el, double E, double nu, int64_t npairs,
                                      const int64_t* ri_dev, const int64_t* sj_dev, double* out_dev,
                                      void* stream);

/* ---------------------------------------------------------------- cluster tree
 * Binary cluster tree over element centroids and the block partition (Sec. 3.1 relies
 * on an H-matrix; the rules are: split a cluster of more than leaf_size elements at the
 * median of its longest centroid-box axis (the first n/2 in (coordinate, index) order go
 * left); a pair (s, t) is admissible (low rank) iff min(diam B_s, diam B_t) <= eta
 * dist(B_s, B_t) > 0 on element-vertex boxes; non-admissible leaf pairs are dense).
 * Built on the host; the handle is independent of the element arrays afterwards. */
typedef struct hm_tree hm_tree;

typedef struct {
    int64_t n_elements;
    int64_t n_nodes;
    int64_t n_leaves;
    int64_t n_near;  /* dense (near-field) leaf x leaf blocks */
    int64_t n_far;   /* admissible (low-rank) blocks */
    int32_t leaf_size;
    int32_t depth;
    double eta;
} hm_tree_info;

hm_status hm_build_cluster_tree(const hm_elements* el, int leaf_size, double eta, hm_tree** out);
hm_status hm_tree_get_info(const hm_tree* t, hm_tree_info* info);
/* Copy the tree to host arrays (any may be NULL): perm[n_elements] (user index of the
 * element at cluster position k), node begin/end/left/right [n_nodes] (left = -1 for a
 * leaf), near[2 n_near] and far[2 n_far] as (row node, column node) pairs. */
hm_status hm_tree_export(const hm_tree* t, int64_t* perm, int64_t* begin, int64_t* end,
                         int64_t* left, int64_t* right, int64_t* near, int64_t* far);
void hm_tree_destroy(hm_tree* t);

/* ---------------------------------------------------------------- H-matrix assembly
 * Assemble the H-matrix of E on the device: dense near-field tiles in FP32 (FP64
 * evaluation), admissible blocks compressed by adaptive cross approximation with
 * element (3-row) pivots and recompressed in FP64 to relative Frobenius accuracy
 * trunc_factor * aca_eps per block (0.1 of that for the cross approximation itself),
 * factors stored in `storage` (HM_F32, HM_BF16 or both).  aca_eps is the accuracy the
 * product is meant to meet; trunc_factor (0 = HM_TRUNC_DEFAULT) spends that budget per
 * block: an admissible block carries a small share of any row's sum, so its own
 * relative error reaches the product attenuated.  max_rank caps the ACA rank (0 = 160,
 * at most 256): a block whose approximation does not converge below the cap is refined
 * into the blocks of its children clusters (a pair of leaves is stored dense instead).
 * Synchronises the stream (the packed layout depends on the ranks). */
#define HM_TRUNC_DEFAULT 30.0
typedef struct {
    double E;
    double nu;
    double aca_eps;
    int storage;
    int max_rank;
    double trunc_factor;
} hm_assemble_opts;

typedef struct hm_hmat hm_hmat;

typedef struct {
    int64_t n_dof;            /* 3 N */
    int64_t near_entries;     /* stored dense entries (unpadded) */
    int64_t far_entries;      /* stored factor entries sum 3 r (|s| + |t|) (unpadded) */
    int64_t stored_bytes;     /* bytes of all stored coefficients, padding included */
    int64_t algorithmic_bytes;/* 4 near_entries + factor bytes + x/y traffic, one RHS */
    int32_t rank_min, rank_max;
    double rank_mean;
    double assemble_seconds;
    int32_t storage;
    int32_t pad_;
    int64_t n_far_lowrank;    /* admissible blocks stored as factors */
    int64_t n_far_dense;      /* admissible blocks whose factors would exceed the dense block */
    int64_t u_entries;        /* sum over low-rank blocks of 3 |s| r (row factors) */
    int64_t v_entries;        /* sum over low-rank blocks of 3 |t| r (column factors) */
    int64_t tb_len;           /* sum of the ranks (length of the V^T x vector) */
    int64_t p_len;            /* per-leaf partials of V^T x */
    int64_t n_far_refined;    /* admissible blocks whose cross approximation did not converge
                                 below the rank cap, replaced by their children's blocks */
    int64_t n_leaves;         /* leaf clusters (block-Jacobi blocks) */
    int64_t coeff_blocks;     /* 3x3 influence blocks the assembly evaluated (near tiles and
                                 the rows and columns of the cross approximation) */
} hm_hmat_info;

hm_status hm_assemble_hmat(const hm_tree* t, const hm_elements* el, const hm_assemble_opts* opt,
                           void* stream, hm_hmat** out);
hm_status hm_hmat_get_info(const hm_hmat* h, hm_hmat_info* info);
/* Low-rank factors of far block b to host, FP64, column-major: U[3|s| x r],
 * V[3|t| x r] with block = U V^T in cluster order of the two clusters.  Blocks
 * 0 .. n-1 are those of the partition (hm_tree_export order); a block refined during
 * assembly (see n_far_refined) is followed by its children's blocks, numbered from n on
 * in order of refinement.  rank_out receives r, -1 for a block stored dense or -2 for a
 * refined block (U, V untouched); pass U = V = NULL to query the rank only. */
hm_status hm_hmat_far_factors(const hm_hmat* h, int64_t b, int32_t* rank_out, double* U, double* V);
void hm_hmat_destroy(hm_hmat* h);

/* ---------------------------------------------------------------- H-matrix product
 * y = E x for nrhs right-hand sides (the product of Sec. 3.1 on the stored H-matrix).
 * x_dev, y_dev: nrhs x 3N, RHS-major (x_dev[k * 3N + dof]), user element order.
 * dtype HM_F32: float vectors, FP32 accumulation.  dtype HM_F64: double vectors; the
 * FP32/BF16 stored coefficients are applied with compensated float-float accumulation,
 * so the result is the product of the stored operator to about 1e-13 relative.
 * x_dev and y_dev must not overlap.  Asynchronous. */
hm_status hm_matvec(const hm_hmat* h, const void* x_dev, void* y_dev, int nrhs, int dtype,
                    void* stream);

/* hm_matvec with the factor precision chosen: factors HM_F32 or HM_BF16 (it must be
 * stored: storage HM_F32_BF16 keeps both), or 0 for the default of hm_matvec (FP32 when
 * stored).  With BF16 factors and FP32 vectors, the V^T x contraction of 16 right-hand
 * sides and the U t contraction of one right-hand side run on the tensor cores
 * (BF16 x BF16 -> FP32, the vector split into BF16 hi + lo: about 16 bits of it kept). */
hm_status hm_matvec_factors(const hm_hmat* h, const void* x_dev, void* y_dev, int nrhs, int dtype, int factors,
                            void* stream);

/* The same product for vectors in host memory (pinned memory is fastest): x_host is
 * copied to library-owned device scratch, the product runs on `stream`, y is copied
 * back to y_host and the stream is synchronised before returning. */
hm_status hm_matvec_host(const hm_hmat* h, const void* x_host, void* y_host, int nrhs, int dtype,
                         void* stream);

/* Per-phase timing of the products that follow, with CUDA events recorded on their
 * stream between the phases.  enable = 1 clears the accumulators and starts recording,
 * enable = 0 stops.  hm_hmat_timing_read synchronises with the last recorded event and
 * returns, in milliseconds summed over the timed products: out[0] gather, out[1] phase 1
 * (V^T x), out[2] reduction of the partials, out[3] phase 2 ([D | U] z), out[4] scatter,
 * and out[5] the number of timed products. */
hm_status hm_hmat_timing(const hm_hmat* h, int enable);
hm_status hm_hmat_timing_read(const hm_hmat* h, double* out6);

/* ---------------------------------------------------------------- tangent solve
 * Solve A x = b with A = E - diag(k) - C^ep - shift I: the elastic block of the Jacobian
 * (eq. jac_mech) with the interface tangent as an isotropic stiffness k per element
 * (K_s = K_n = k, Sec. 2.2) and/or a block-diagonal consistent tangent C^ep (3x3 per
 * element, opts.cep_dev, e.g. from hm_interface_update), and the quasi-dynamic term
 * eta/dt = shift (eq. ElasSystem).  With C^ep the point-Jacobi and leaf block-Jacobi
 * blocks and the ILU pattern hold its whole 3x3 blocks; the learned preconditioner
 * takes k only (HM_EINVAL with C^ep).  The paper solves this A11 system with a Krylov
 * method and a Jacobi preconditioner (Sec. 3.3.1); here: restarted flexible GMRES(m)
 * with right preconditioning, classical Gram-Schmidt applied twice, Givens rotations,
 * all Krylov vectors, dot products and rotations in FP64 on the device, x0 = 0.
 *   precond HM_PRECOND_NONE, HM_PRECOND_JACOBI3 (the paper's Jacobi preconditioner:
 *   the inverse of every element's 3x3 diagonal block of A), HM_PRECOND_BLOCKJ (inverse
 *   of every diagonal leaf block of A, i.e. that Jacobi taken per cluster-tree leaf), or
 *   HM_PRECOND_LEARNED (block-Jacobi corrected by a trained network, see hm_lp_*), or
 *   HM_PRECOND_ILU: the incomplete-LU preconditioner of Sec. 3.3.1 -- ILU(0) of
 *   -diag(k) - shift plus the fraction ilu_p of the near-field entries of E (inadmissible
 *   leaf pairs, FP32 stored values) with the largest magnitude, ties by (row, column) in
 *   cluster order, the diagonal always in the pattern, rows listed leaf-colour by
 *   leaf-colour (see hm_ilu_export); factored in FP64 at every call, the pattern kept on
 *   the H-matrix for later calls with the same ilu_p.
 *   mode HM_SOLVE_F64: every product with FP32 factors in compensated FP64 ("plain").
 *   mode HM_SOLVE_MIXED: iterative refinement -- the residual b - A x in compensated
 *   FP64 with the FP32 factors, corrections from FGMRES on the BF16-factor operator
 *   with FP32 products to inner_tol (needs storage HM_F32_BF16).
 *   mode HM_SOLVE_PLAIN32: the same refinement with the corrections on the FP32-factor
 *   operator (FP32 products): the plain FP32 path, without BF16 factors.
 *   method HM_METHOD_BICGSTAB: right-preconditioned BiCGSTAB (van der Vorst, 1992), the
 *   method the paper uses for its A11 solves, instead of FGMRES (same preconditioners
 *   and modes; restart ignored; maxit counts BiCGSTAB iterations of two products each;
 *   outer counts refinement steps in the mixed modes; the run restarts from the true
 *   residual, at most 8 times, if the recurrence's residual has drifted from it).
 * Converged when ||b - A x||_2 <= tol ||b||_2, recomputed in compensated FP64 with the
 * FP32 factors.  k_dev: N doubles (per element, user order) or NULL; b_dev, x_dev:
 * nrhs x 3N doubles, user order (x is overwritten); info: nrhs entries.  Synchronises
 * the stream.  Returns HM_ENAN (before any iteration) if shift, k or b holds a NaN or
 * an infinity, HM_ENOCONV if a right-hand side did not converge within maxit. */
#define HM_PRECOND_NONE 0
#define HM_PRECOND_BLOCKJ 1
#define HM_PRECOND_LEARNED 2
#define HM_PRECOND_JACOBI3 3
#define HM_PRECOND_ILU 4
#define HM_METHOD_FGMRES 0
#define HM_METHOD_BICGSTAB 1
#define HM_SOLVE_F64 1
#define HM_SOLVE_MIXED 2
#define HM_SOLVE_PLAIN32 3

typedef struct hm_lp hm_lp;  /* learned block-Jacobi correction (below) */

typedef struct {
    double tol;        /* relative residual target (0 = 1e-8) */
    int restart;       /* Krylov dimension m (0 = 50) */
    int maxit;         /* cap on the total Krylov iterations (0 = 2000) */
    int precond;
    int mode;
    double inner_tol;  /* mixed: relative tolerance of each correction solve (0 = 1e-2) */
    int max_outer;     /* mixed: cap on refinement steps (0 = 40) */
    int pad_;
    const hm_lp* lp;   /* model for HM_PRECOND_LEARNED (NULL otherwise) */
    double ilu_p;      /* HM_PRECOND_ILU: fraction of the near-field entries kept (0 = 0.01) */
    const double* cep_dev;  /* block-diagonal C^ep (device, N x 9: per element in user order, row-major
                               3x3 in its frame (s1, s2, n), e.g. from hm_interface_update) or NULL */
    int method;        /* HM_METHOD_FGMRES (0) or HM_METHOD_BICGSTAB */
    int reuse_precond; /* 1: keep the preconditioner of the previous call on this H-matrix when it was
                          built for the same k_dev, cep_dev, shift, precond, ilu_p and lp (the caller
                          promises the arrays behind the pointers are unchanged) */
} hm_solve_opts;

typedef struct {
    int iters;         /* Krylov iterations */
    int outer;         /* restarts (F64) or refinement steps (mixed) */
    int status;        /* HM_OK, HM_ENOCONV or HM_EBREAKDOWN */
    int pad_;
    double relres;     /* final ||b - A x|| / ||b|| (compensated FP64, FP32 factors) */
    double seconds;
} hm_solve_info;

hm_status hm_gmres_solve(const hm_hmat* h, const double* k_dev, double shift, const double* b_dev,
                         double* x_dev, int nrhs, const hm_solve_opts* opt, hm_solve_info* info,
                         void* stream);

/* z = M^-1 r with the preconditioner hm_gmres_solve builds for A = E - diag(k) - C^ep -
 * shift I and these options (precond, ilu_p, lp, cep_dev, reuse_precond; the other
 * fields are ignored), for a caller's own Krylov method -- e.g. the nested solves of
 * Sec. 3.3.1 -- and for checking the preconditioners.  r_dev, z_dev: nrhs x 3N doubles,
 * user order, not overlapping.  Synchronises the stream. */
hm_status hm_precond_apply(const hm_hmat* h, const double* k_dev, double shift, const hm_solve_opts* opt,
                           const double* r_dev, double* z_dev, int nrhs, void* stream);

/* The ILU preconditioner that hm_gmres_solve builds for A = E - diag(k) - C^ep - shift I
 * and the fraction p (Sec. 3.3.1), to host arrays (any may be NULL; pass NULL arrays first to
 * learn n and nnz).  n_out: 3N; nnz_out: entries of the pattern; n_colours_out: leaf
 * colours.  order[n]: factorization position -> cluster DOF position (the cluster order
 * of hm_tree_export: DOF 3 q + c of the element at cluster position q); rowptr[n + 1],
 * col[nnz]: the pattern in factorization order, columns increasing; a_val[nnz]: the
 * selected entries of E (the diagonal holds E's entry if selected, else 0; with C^ep
 * every element's 3x3 block is in the pattern, E's entry or 0), before -k - C^ep - shift
 * is added; lu_val[nnz]: ILU(0) of the matrix with -k - C^ep - shift added (multipliers
 * of the unit lower factor left of the diagonal, the upper factor on and right of it).
 * k_dev as in hm_gmres_solve, cep_dev as opts.cep_dev there (NULL: none).  Synchronises
 * the stream. */
hm_status hm_ilu_export(const hm_hmat* h, const double* k_dev, const double* cep_dev, double shift, double p,
                        int64_t* n_out, int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr,
                        int32_t* col, double* a_val, double* lu_val, void* stream);

/* z = (L U)^-1 r with the factors of the last ILU factorization of this H-matrix (made by
 * hm_gmres_solve with HM_PRECOND_ILU or by hm_ilu_export with lu_val): forward
 * substitution with the unit lower factor, backward substitution with the upper one, in
 * FP64 on the device.  r_dev, z_dev: nrhs x 3N doubles, user order (must not overlap).
 * HM_EINVAL if no factorization exists.  Asynchronous. */
hm_status hm_ilu_apply(const hm_hmat* h, const double* r_dev, double* z_dev, int nrhs, void* stream);

/* ---------------------------------------------------------------- coupled flow
 * Fluid flow in the fractures and the coupled hydro-mechanical Jacobian (Sec. 3.2, eq.
 * flow_discretized and res_flow; Sec. 3.3.1).  The pressure is bilinear on the
 * rectangular elements with nodes at the vertices (the caller's connectivity: elements
 * share a node by index, also across intersecting planes); per element, at the opening
 * w = w0 + delta_n, storage w / M and the cubic-law conductance w^3 / (12 mu):
 *   S = sum (w/M) m^e, L = sum (w^3 / 12 mu) k^e, V^e = int N dS (A/4 per node),
 *   m^e = int N^T N, k^e = int grad N^T grad N (closed forms of the rectangle);
 *   r_f = V Delta delta_n + (S + dt L) Delta p + dt L (p^n - p^o) - dt f_f.
 * The Jacobian of [r_m; r_f] in [Delta delta (3N, user order); Delta p (nodes)]:
 *   A11 = E - diag(k) - C^ep - shift I (shift = eta/dt), A12 = N_p (the mean of an
 *   element's nodal pressures on its normal row: the interpolated value at the
 *   centroid), A21 = d r_f / d Delta delta (only the normal DD: V^e + m^e Delta p^e / M +
 *   dt (3 w^2 / 12 mu) k^e (Delta p^e + p^n,e - p^o,e) per element), A22 = S + dt L.
 * No-flux outer boundary; the flow is the same on every plane (no matrix permeability). */
typedef struct hm_flow hm_flow;

typedef struct {
    double mu;   /* fluid viscosity */
    double M;    /* Biot modulus of the filled interface */
    double w0;   /* initial hydraulic width */
    double dt;   /* time step */
} hm_flow_params;

/* Mesh set-up on the host: conn (host, N x 4 int32) the element's nodes in the order
 * (-a, -b), (+a, -b), (+a, +b), (-a, +b) of its (s1, s2) frame, n_nodes nodes, a and b
 * (host, N) the half sides.  HM_EINVAL for an index out of range, a repeated node in an
 * element or a non-positive half side. */
hm_status hm_flow_create(int64_t N, const int32_t* conn, int64_t n_nodes, const double* a, const double* b,
                         hm_flow** out);
/* The same for a mesh of rectangles (bilinear pressure) and triangles (linear pressure,
 * the paper's elements, Sec. 3.2): shape (host, N; NULL: all rectangles) HM_SHAPE_RECT /
 * HM_SHAPE_TRI; conn (host, N x 4): a rectangle's four nodes as above, a triangle's
 * three nodes in the order of its vertices and -1; a, b the rectangles' half sides (the
 * entries of triangles unread); tri (host, N x 9; NULL if no triangle) the triangles'
 * global vertices, in the order of their nodes.  Element matrices are computed here:
 * closed forms of the bilinear rectangle, and for a triangle of area A the mass
 * A/12 (1 + delta_ij), the load A/3 and the stiffness (e_i . e_j) / (4 A), e_i the edge
 * opposite node i.  HM_EINVAL also for a degenerate triangle or a triangle without -1 in
 * its fourth slot; HM_ENAN for a non-finite vertex. */
hm_status hm_flow_create_mesh(int64_t N, const int32_t* shape, const int32_t* conn, int64_t n_nodes,
                              const double* a, const double* b, const double* tri, hm_flow** out);
void hm_flow_destroy(hm_flow* f);
/* The flow blocks at the current iterate (device arrays): dn_dev (N) delta_n at t^(n+1),
 * dp_dev (n_nodes) Delta p, pn_dev (n_nodes) p^n - p^o (either may be NULL: zero).
 * Gathers every entry in a fixed order (repeatable bit for bit).  Asynchronous. */
hm_status hm_flow_assemble(hm_flow* f, const hm_flow_params* prm, const double* dn_dev, const double* dp_dev,
                           const double* pn_dev, void* stream);
/* To host arrays (any may be NULL): nnz_out; rowptr[n_nodes + 1], col[nnz] the node
 * pattern (columns increasing); a22[nnz] = S + dt L; a21[4N]: A21's column of every
 * element's normal DD, on its nodes in connectivity order (a triangle's fourth entry is
 * 0).  Synchronises. */
hm_status hm_flow_export(const hm_flow* f, int64_t* nnz_out, int64_t* rowptr, int32_t* col, double* a22,
                         double* a21, void* stream);
/* y = J x for x, y of length 3N + n_nodes (device; A11 by the compensated FP64 product
 * with the FP32 factors).  k_dev, cep_dev, shift as in hm_gmres_solve.  Synchronises. */
hm_status hm_coupled_matvec(const hm_hmat* h, const hm_flow* f, const double* k_dev, const double* cep_dev,
                            double shift, const double* x_dev, double* y_dev, void* stream);

typedef struct {
    double tol;          /* relative residual of the coupled system (0 = 1e-8) */
    int restart;         /* outer FGMRES restart (0 = 30) */
    int maxit;           /* outer iterations (0 = 300) */
    int inner_precond;   /* preconditioner of the A11 solves (HM_PRECOND_*, not LEARNED) */
    int inner_method;    /* HM_METHOD_FGMRES or HM_METHOD_BICGSTAB for the A11 solves */
    double inner_tol;    /* relative tolerance of each A11 solve (0 = 1e-6) */
    double schur_tol;    /* relative tolerance of each Schur solve (0 = 1e-6) */
    double ilu_p;        /* inner HM_PRECOND_ILU fraction (0 = 0.01) */
    double flow_scale;   /* factor on the flow rows (Sec. 3.3.2's residual scaling); 0 = the ratio of
                            the RMS diagonal of A11 to that of S~ (both blocks weigh in the test) */
} hm_coupled_opts;

typedef struct {
    int iters;           /* outer iterations */
    int inner_iters;     /* Krylov iterations of all A11 solves */
    int schur_iters;     /* BiCGSTAB iterations of all Schur solves */
    int status;          /* HM_OK or HM_ENOCONV */
    double relres;       /* the scaled relative residual (see hm_coupled_solve) */
    double seconds;
} hm_coupled_info;

/* Solve J x = b (Sec. 3.3.1): restarted FGMRES right-preconditioned by the upper block
 * triangular P_up = [[A11, A12], [0, S~]] with S~ = A22 - A21 diag(A11)^-1 A12 (the
 * paper's first approximation; sparse, the pattern of A22).  Applying P_up^-1: z2 =
 * S~^-1 y2 by Jacobi-preconditioned BiCGSTAB to schur_tol, z1 = A11^-1 (y1 - A12 z2) by
 * hm_gmres_solve's path to inner_tol (the nested solves of the paper).  The flow rows
 * are scaled by flow_scale (the residual scaling of Sec. 3.3.2), and tol and relres refer
 * to ||diag(I, s I)(b - J x)|| / ||diag(I, s I) b||.  FP64 throughout;
 * x0 = 0; b_dev, x_dev of length 3N + n_nodes.  Needs hm_flow_assemble first.  HM_ENOCONV
 * if the tolerance is not met within maxit, HM_EBREAKDOWN for a zero diagonal in A11's
 * normal rows or in S~.  Synchronises the stream. */
hm_status hm_coupled_solve(const hm_hmat* h, const hm_flow* f, const double* k_dev, const double* cep_dev,
                           double shift, const double* b_dev, double* x_dev, const hm_coupled_opts* opt,
                           hm_coupled_info* info, void* stream);

/* ---------------------------------------------------------------- interface law
 * Constitutive update of the fault / fracture interface and its consistent tangent
 * (Sec. 2.2: poroelastoplastic interface with a Coulomb yield surface F_c = |tau| +
 * f T'_n - c, a tensile cut-off F_t = T'_n - sigma_t, non-associated Coulomb flow along
 * s_hat + psi n and associated tensile flow along n; Sec. 3.1.1: elastic predictor -
 * plastic corrector; eq. jac_mech: C^ep = d(Delta T') / d(Delta delta)).  Per point, in
 * its local frame (s1, s2, n):
 *   T' - T'^n = C (Delta delta - Delta delta^p), C = diag(Ks, Ks, Kn) (constant);
 *   f = (fp - fr) W(chi_s / dc) + fr, psi = psip W(chi_s / dc), c = cp W(chi_t / wc),
 *   sigma_t = sigp W(chi_t / wc), W(x) = max(0, 1 - x) (W = 0 when wc = 0);
 *   chi_s = max over time of |delta^p_s|, chi_t = max over time of |delta^p|, taken at
 *   t^(n+1) (backward Euler, like f, psi, c, sigma_t in the return);
 *   mode at the trial state with the strengths of t^n: elastic if F_c <= 0 and F_t <= 0,
 *   else Coulomb if h = |tau| - (c - f sigma_t) - (sqrt(1 + f^2) - f)(T'_n - sigma_t) > 0,
 *   else tensile; a Coulomb return with no root before tau = 0 returns to the cone's apex
 *   (tau = 0, f T'_n = c, shear fully inelastic);
 *   full damage when wc = 0 (pre-existing fracture) or chi_t >= wc: a fully damaged
 *   point with a tensile trial traction is open (T' = 0, C^ep = 0, Delta delta + C^-1 T'^n
 *   inelastic); otherwise it is in contact with its normal inelastic DD at
 *   min(delta^p_n, w_R), w_R = alphaR wc + w_dil, and frictional without cohesion; a
 *   tensile or apex return that reaches full damage ends open;
 *   w_dil (the dilatant part of w_R) grows by psi dl in every Coulomb return.
 * The plastic multiplier solves a scalar equation (Newton safeguarded by bisection);
 * parameters must keep it monotone (interface stiffness above the softening rates).
 * C^ep is exact within the active mode (forward-mode dual numbers and the implicit
 * function theorem at the multiplier's root).
 * Arrays (device, n points, row-major): T_dev, dp_dev (n x 3: T'^n and delta^p_n),
 * chi_dev (n x 3: chi_s, chi_t, w_dil), dd_dev (n x 3: Delta delta) in; T1_dev, dp1_dev,
 * chi1_dev (n x 3) out, each may be the same array as its input; cep_dev (n x 9, row i =
 * traction component i, column j = DD component j) or NULL (no tangent, cheaper);
 * mode_dev (n int32: 0 elastic, 1 Coulomb, 2 tensile, 3 open, 4 apex, plus 256 where the
 * multiplier did not converge) or NULL.
 * counts (host, 6 int64) or NULL: points per mode and, last, points whose multiplier did
 * not converge; with counts the call synchronises the stream and returns HM_ENOCONV if
 * that last count is not 0.  HM_EINVAL for Ks or Kn <= 0, dc <= 0, a negative or
 * non-finite parameter. */
typedef struct {
    double Ks, Kn;   /* shear and normal stiffness of the interface */
    double fp, fr;   /* peak and residual friction coefficients */
    double psip;     /* peak dilatancy coefficient */
    double dc;       /* slip-weakening distance (> 0) */
    double cp;       /* peak cohesion */
    double sigp;     /* peak tensile strength */
    double wc;       /* critical inelastic DD of cohesion and tensile strength (0: pre-existing fracture) */
    double alphaR;   /* residual width after full damage, fraction of wc */
} hm_interface_params;

hm_status hm_interface_update(const hm_interface_params* prm, int64_t n, const double* T_dev,
                              const double* dp_dev, const double* chi_dev, const double* dd_dev, double* T1_dev,
                              double* dp1_dev, double* chi1_dev, double* cep_dev, int32_t* mode_dev,
                              int64_t* counts, void* stream);

/* ---------------------------------------------------------------- batching
 * Independent faults: the operator of several non-interacting fractures is
 * block-diagonal, one block E_f per fault (eq. ElasSystem on each fault alone, each with
 * the E, nu it was assembled with).  hm_batch_create concatenates the assembled
 * H-matrices hs[0..nf-1] into one new H-matrix whose vectors are the faults' vectors
 * back to back (fault 0's 3 N_0 DOFs, then fault 1's, ...): one arena of coefficients
 * and one work list, so a product is one persistent launch per phase over all faults.
 * All parts must use the same factor storage.  The parts are copied (device to device)
 * and stay valid and owned by the caller; destroy them to free their memory.  The result
 * is used with every hm_hmat function (product, solve of the block-diagonal system,
 * info); hm_hmat_far_factors numbers the blocks fault by fault.  Synchronises the
 * stream. */
hm_status hm_batch_create(const hm_hmat* const* hs, int nf, void* stream, hm_hmat** out);

/* The product of hm_matvec replayed from a CUDA graph: the first call for a given
 * (x_dev, y_dev, nrhs, dtype) runs the product once, captures it on a library-owned
 * stream and instantiates it; later calls with the same arguments launch the graph on
 * `stream` (one host call per product).  Graphs are dropped when the product scratch
 * grows (more right-hand sides).  While per-phase timing is enabled it runs the plain
 * product.  Asynchronous after the first call. */
hm_status hm_matvec_graph(const hm_hmat* h, const void* x_dev, void* y_dev, int nrhs, int dtype,
                          void* stream);

/* Tile shape of the product's coefficient streams (an implementation choice of this
 * library; the paper states none).  chunk_bytes (a multiple of 16 in [2048, 32768]) and
 * chunk_cols ([8, 128]) bound one pipeline chunk -- whole columns of one tile or factor
 * slice -- and so the grain of the byte split over the SMs; ring (4 or 6) is the depth of
 * the shared-memory copy ring and warps (16 or 8) the consumer warps of the single-RHS
 * product with FP32 vectors (products with several right-hand sides or FP64 vectors keep
 * 4 stages and their own warp counts, and BF16 factors keep 16 warps in the row phase,
 * whose U slices run on tensor cores).  The default is {32768, 128, 4, 16}. */
typedef struct {
    int32_t chunk_bytes;
    int32_t chunk_cols;
    int32_t ring;
    int32_t warps;
} hm_tile_shape;

/* Set the tile shape of an H-matrix: its product plans are cut again (synchronises the
 * stream; product graphs captured before are dropped).  HM_EINVAL for a shape outside
 * the ranges above. */
hm_status hm_hmat_set_tile_shape(hm_hmat* h, const hm_tile_shape* shape, void* stream);
hm_status hm_hmat_get_tile_shape(const hm_hmat* h, hm_tile_shape* shape);
/* Time `reps` single-RHS FP32-vector products (FP32 factors when stored) under each of
 * shapes[0 .. n_shapes - 1] with CUDA events and keep the fastest on h.  JSON to json_out:
 *   {"candidates": [{"chunk_bytes", "chunk_cols", "ring", "warps", "ms"}, ...],
 *    "best": {... , "ms"}, "tuned": n} */
hm_status hm_tune_tile_shape(hm_hmat* h, const hm_tile_shape* shapes, int n_shapes, int reps, char* json_out,
                             size_t cap, void* stream);

/* Autotuner of leaf size, admissibility and tile shape: for each (leaf_sizes[i], etas[j])
 * in order, build the cluster tree and partition (Sec. 3.1), assemble with `opt` (every
 * candidate meets the same accuracy aca_eps), and for each of shapes[0 .. n_shapes - 1]
 * (the default shape if n_shapes is 0) time 20 single-RHS FP32 products with CUDA events
 * on `stream`; stop once budget_ms of wall time has passed (at least one candidate is
 * timed).  Writes a NUL-terminated JSON object to json_out (capacity cap bytes):
 *   {"n_elements": N, "candidates": [{"leaf", "eta", "ms", "stored_bytes", "assemble_s",
 *    "rank_mean", "chunk_bytes", "chunk_cols", "ring", "warps"}, ...],
 *    "best": {"leaf", "eta", "ms", "chunk_bytes", "chunk_cols", "ring", "warps"}, "tuned": n}
 * HM_EINVAL if the buffer is too small (the message states the size needed). */
hm_status hm_autotune(const hm_elements* el, const hm_assemble_opts* opt, const int* leaf_sizes, int n_leaf,
                      const double* etas, int n_eta, const hm_tile_shape* shapes, int n_shapes, int budget_ms,
                      char* json_out, size_t cap, void* stream);

/* ---------------------------------------------------------------- learned correction
 * The paper preconditions the A11 system with (point) Jacobi (Sec. 3.3.1) and learns
 * nothing; this library adds an optional learned correction of its leaf block-Jacobi
 * preconditioner B of A = E - diag(k) (eq. jac_mech), of one of two kinds:
 *   HM_LP_SCALE:  M^-1 r = D B^-1 r,
 *   HM_LP_NEAR:   M^-1 r = y - gamma D B^-1 N y,  y = B^-1 r, N = the near-field tiles of
 *                 E off the diagonal leaf blocks (the first Neumann term of the near
 *                 coupling, damped per leaf and component by the network),
 *   D = diag(d_(leaf, component)),  d = 1 + 0.5 tanh(o),
 *   o = W3 tanh(W2 tanh(W1 f + b1) + b2) + b3,
 * per leaf and DOF component, from eight leaf features f: mean, standard deviation, min
 * and max of log10(k h / E + 1e-6) over the leaf's elements (h = sqrt(4 a b)), the
 * fraction with k h / E < 0.5, log10(element count), |mean normal|, and
 * log10(1 + d / hbar) with d the distance from the leaf centroid to the nearest leaf
 * centroid of another normal direction (1000 hbar if none).  W3 = 0, b3 = 0 is plain
 * block-Jacobi.  Parameters (param_count(H) values, H = 16, 32 or 64 hidden units per
 * layer) in the order W1 (H x 8, row-major), b1, W2 (H x H), b2, W3 (3 x H), b3.
 * Training (Adam, beta = 0.9 / 0.999, eps = 1e-8, full batch) minimises
 *   loss = (1 / n_groups) sum_samples sum_a  q_xx - 2 d_a q_xy + d_a^2 q_yy,
 * a sample being one leaf of one solved system A x = b with q = S / T: S the leaf and
 * component sums of x y, y y, x x over the system's right-hand sides (y = B^-1 b), T
 * the system's sum of x x -- the fit of D B^-1 b to x = A^-1 b; for HM_LP_NEAR the same
 * sums of x' = y - x and y' = w = B^-1 N y (the fit of D w to y - x).  gamma is the
 * caller's choice on validation systems (GMRES iterations as the judge).
 * The model's parameters live in host memory (device copies made on first GPU use), so
 * create / add_samples / get_params / set_fallback / info / save / load need no GPU.
 * A model flagged `fallback` makes HM_PRECOND_LEARNED apply plain block-Jacobi (set it
 * when validation shows no gain). */
typedef struct {
    int32_t hidden;
    int32_t fallback;
    int64_t n_params;
    int64_t n_samples;
    int64_t n_groups;
    int64_t steps;        /* Adam steps taken */
    double last_loss;     /* loss before the last step of the last hm_lp_train */
    int32_t kind;         /* HM_LP_SCALE or HM_LP_NEAR */
    int32_t pad_;
    double gamma;         /* HM_LP_NEAR: factor on d */
} hm_lp_info;

#define HM_LP_SCALE 0
#define HM_LP_NEAR 1

/* number of parameters for `hidden` units (16, 32 or 64), -1 otherwise */
int64_t hm_lp_param_count(int hidden);
/* new model with initial parameters theta0 (host, param_count(hidden) doubles) */
hm_status hm_lp_create(int hidden, const double* theta0, hm_lp** out);
/* add n samples (host: features n x 8 row-major, targets q n x 9 = [q_xy | q_yy | q_xx]),
 * counted as one group */
hm_status hm_lp_add_samples(hm_lp* lp, const double* features, const double* q, int64_t n);
/* add the leaves of one solved system as one group: k_dev (N doubles, user order, or
 * NULL), b_dev and x_dev (nrhs x 3N doubles, user order) with A x = b; computes
 * B^-1 b, the statistics and the features on the device.  Synchronises the stream. */
hm_status hm_lp_add_system(hm_lp* lp, const hm_hmat* h, const double* k_dev, const double* b_dev,
                           const double* x_dev, int nrhs, void* stream);
hm_status hm_lp_clear_samples(hm_lp* lp);
/* loss and gradient (param_count doubles, host; may be NULL) at the current parameters */
hm_status hm_lp_loss_grad(hm_lp* lp, double* loss_out, double* grad_out, void* stream);
/* `steps` full-batch Adam steps with learning rate lr; loss_out: loss before the last step */
hm_status hm_lp_train(hm_lp* lp, int steps, double lr, double* loss_out, void* stream);
/* features (n_leaves x 8) and scalings d (n_leaves x 3) for this H-matrix and k, to host
 * (either may be NULL); leaves in cluster order */
hm_status hm_lp_predict(hm_lp* lp, const hm_hmat* h, const double* k_dev, double* features_out,
                        double* d_out, void* stream);
hm_status hm_lp_get_params(const hm_lp* lp, double* theta_out);
hm_status hm_lp_set_fallback(hm_lp* lp, int fallback);
/* the kind of correction (HM_LP_SCALE, the default, or HM_LP_NEAR) and gamma > 0; the kind
 * can change only while the model holds no samples (HM_EINVAL otherwise) */
hm_status hm_lp_set_kind(hm_lp* lp, int kind, double gamma);
hm_status hm_lp_get_info(const hm_lp* lp, hm_lp_info* info);
/* binary file: "HMLP0002", hidden and fallback (int32), steps (int64), kind (int32),
 * gamma (double), then the parameters and both Adam moments (float32 each); load also
 * reads the "HMLP0001" files of the scale kind (no kind or gamma fields) */
hm_status hm_lp_save(const hm_lp* lp, const char* path);
hm_status hm_lp_load(const char* path, hm_lp** out);
void hm_lp_destroy(hm_lp* lp);

/* Synchronise `stream` and report whether a device-side wait of an earlier product on
 * this H-matrix gave up (HM_ETIMEOUT; the flags and the product's split-row arrival
 * counts are then cleared).  The product kernels bound every wait on their copy
 * pipeline instead of spinning forever. */
hm_status hm_hmat_check(const hm_hmat* h, void* stream);

/* Limit of the product's bounded waits, limit_s in [1e-6, 10] seconds (default 2), and a
 * switch for testing the failure path: withhold_chunk >= 0 makes the producer of the
 * row phase stop before that chunk of its plan (the copies of that chunk and of the
 * later chunks of its CTA are never issued), so that the consumers' waits run out; the
 * product is then garbage and hm_hmat_check returns HM_ETIMEOUT.  -1 turns it off.
 * Host-side settings of this H-matrix; product graphs captured before are dropped. */
hm_status hm_hmat_set_wait(hm_hmat* h, double limit_s, int64_t withhold_chunk);

/* ---------------------------------------------------------------- ILU building blocks
 * Sec. 3.3.1 preconditions the mechanical block with an incomplete LU factorization of
 * C^ep plus the fraction p of the near-field (full-rank block) entries of E with the
 * largest absolute value.  These host functions are the setup steps of that
 * preconditioner on plain caller-owned host arrays (nothing is retained; no device is
 * used).  Sparse matrices are CSR: rowptr[n + 1] (int64, rowptr[0] = 0, non-decreasing),
 * col[rowptr[n]] (int32), columns strictly increasing within a row, the diagonal present
 * in every row (HM_EINVAL otherwise). */

/* The ceil(p n) entries (i[q], j[q], v[q]) of largest |v|, ties broken by (i, j)
 * ascending (a repeated (i, j) by q): their indices q in that order go to idx_out
 * (capacity ceil(p n)), their count to m_out.  0 < p <= 1 (HM_EINVAL otherwise); a NaN
 * or Inf value is HM_ENAN. */
hm_status hm_ilu_select(int64_t n, const int32_t* i, const int32_t* j, const double* v, double p,
                        int64_t* idx_out, int64_t* m_out);

/* The sparse approximation as CSR: the m selected entries (i[idx[t]], j[idx[t]],
 * v[idx[t]]) of an entry list of length n_entries (positions in [0, n)), minus d[r] on
 * every diagonal (which is always in the pattern), with the rows and columns renumbered
 * by order (new position -> old position; NULL: as they are).  Outputs rowptr_out[n + 1],
 * col_out and val_out (capacity m + n, columns increasing), the entry count to nnz_out.
 * A position selected twice, an index outside [0, n_entries), an out-of-range entry or
 * an order that is not a permutation is HM_EINVAL. */
hm_status hm_ilu_assemble(int32_t n, int64_t n_entries, int64_t m, const int64_t* idx, const int32_t* i,
                          const int32_t* j, const double* v, const double* d, const int32_t* order,
                          int64_t* rowptr_out, int32_t* col_out, double* val_out, int64_t* nnz_out);

/* ILU(0) in place: val holds A on entry and, on return, the multipliers of the unit
 * lower factor below the diagonal and the upper factor on and above it, with
 * (L U)_rc = A_rc at every (r, c) of the pattern; no fill, no pivoting.  A zero pivot is
 * HM_EBREAKDOWN (val then partly factored). */
hm_status hm_ilu0_factor(int32_t n, const int64_t* rowptr, const int32_t* col, double* val);

/* Levels of the two triangular solves with this pattern: lower_out[r] = 0 for a row with
 * no entry left of the diagonal, else 1 + the largest level of the rows it names there;
 * upper_out likewise from the bottom with the entries right of the diagonal.  The level
 * counts go to n_lower_out and n_upper_out.  Any output may be NULL. */
hm_status hm_ilu_levels(int32_t n, const int64_t* rowptr, const int32_t* col, int32_t* lower_out,
                        int32_t* upper_out, int32_t* n_lower_out, int32_t* n_upper_out);

/* Greedy colouring of the leaves that the pattern couples: leaf_of[r] in [0, n_leaves)
 * names the leaf of row r; leaves are taken in order, each gets the smallest colour none
 * of its already coloured neighbours (leaves coupled to it by an entry, in either
 * direction) holds.  Listing the rows colour by colour shortens the dependency chains of
 * the triangular solves.  colour_out[n_leaves]; the colour count to n_colours_out. */
hm_status hm_ilu_leaf_colours(int32_t n, const int64_t* rowptr, const int32_t* col, const int32_t* leaf_of,
                              int32_t n_leaves, int32_t* colour_out, int32_t* n_colours_out);

#ifdef __cplusplus
}
#endif
#endif /* HMAT_H */
