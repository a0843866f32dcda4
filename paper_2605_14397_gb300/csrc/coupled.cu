// Fluid flow in the fractures and the coupled hydro-mechanical Jacobian solve (Sec. 3.2,
// eq. flow_discretized / res_flow; Sec. 3.3.1: the 2 x 2 block Jacobian, the upper block
// triangular preconditioner P_up and its approximate Schur complement).
//
// Flow discretization: bilinear pressure on the rectangular elements, nodes at the
// vertices (the caller's connectivity), cubic-law conductance w^3 / (12 mu) and storage
// w / M per element at the opening w = w0 + delta_n.  The element matrices of a
// rectangle of half sides a, b have closed forms (mass A/36 [4 2 1 2; ...], stiffness
// (b/a)/6 Kx + (a/b)/6 Ky, load A/4 per node), evaluated where they are summed.
//
// Assembly is a gather: every CSR entry of the node-node pattern sums, in a fixed order,
// the element contributions listed for it on the host when the mesh is set up (no
// atomics, so results repeat bit for bit).  A21's columns (only an element's normal DD
// enters the flow residual) are four values per element; A12 = N_p puts the mean of an
// element's nodal pressures on its normal row.
//
// Solve: right-preconditioned restarted FGMRES on [[A11, A12], [A21, A22]] with
// P_up = [[A11, A12], [0, S~]], S~ = A22 - A21 diag(A11)^-1 A12 (the paper's first
// approximation, a sparse matrix with the pattern of A22); P_up^-1 y takes
// z2 = S~^-1 y2 by Jacobi-preconditioned BiCGSTAB on S~ (scalars on the device) and
// z1 = A11^-1 (y1 - A12 z2)
// by the library's tangent solver (nested, to a relative tolerance), so the outer method
// is flexible.  Krylov vectors, dot products and rotations in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <vector>

#include "hmat_impl.h"

struct hm_flow {
    int64_t N = 0, nn = 0, nnz = 0;
    std::vector<int32_t> h_conn;
    std::vector<int64_t> h_rowptr;
    hm::DevBuf<int32_t> conn, col, cel, nel;
    hm::DevBuf<int64_t> rowptr, cptr, nptr;
    hm::DevBuf<uint8_t> cij, nloc;
    hm::DevBuf<double> a, b, a22, a21, ecoef;
    // per element: mass m (4 x 4), stiffness k (4 x 4) and load v (4), row-major; a
    // triangle (conn[4e + 3] = -1) fills the leading 3 x 3 and 3
    hm::DevBuf<double> emat;
    bool assembled = false;
};

namespace hm {
namespace {

constexpr int NT = 256;
inline unsigned gsz(int64_t n) { return (unsigned)std::max<int64_t>(1, ceil_div(n, NT)); }

// nodes of element e: 4 (rectangle) or 3 (triangle: -1 in the fourth slot)
__device__ __forceinline__ int nodes_of(const int32_t* __restrict__ conn, int64_t e) {
    return conn[4 * e + 3] < 0 ? 3 : 4;
}

// per element: storage and conductance coefficients, and A21's column
//   A21[:, e] = v^e + m^e dp^e / M + dt c'(w) k^e (dp^e + pn^e),  c(w) = w^3 / (12 mu)
__global__ void k_flow_elem(int64_t N, const int32_t* __restrict__ conn, const double* __restrict__ emat,
                            const double* __restrict__ dn, const double* __restrict__ dp,
                            const double* __restrict__ pn, double mu, double M, double w0, double dt,
                            double* __restrict__ ecoef, double* __restrict__ a21) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int nv = nodes_of(conn, e);
    const double* m = emat + 36 * e;
    const double* k = m + 16;
    const double* v = m + 32;
    const double w = w0 + dn[e];
    ecoef[2 * e] = w / M;
    ecoef[2 * e + 1] = dt * w * w * w / (12.0 * mu);
    const double dc = dt * 3.0 * w * w / (12.0 * mu);
    double q[4], u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int nd = i < nv ? conn[4 * e + i] : -1;
        q[i] = (nd >= 0 && dp) ? dp[nd] : 0.0;
        u[i] = q[i] + ((nd >= 0 && pn) ? pn[nd] : 0.0);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double s = 0.0;
        if (i < nv) {
            s = v[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) s += m[4 * i + j] * q[j] / M + dc * k[4 * i + j] * u[j];
        }
        a21[4 * e + i] = s;
    }
}

// A22 (or S~ with dsub) entry by entry: the listed element contributions in order;
// S~ subtracts A21[i, e] N_p / d_e for every element pair entry (N_p = 1 / nodes)
__global__ void k_flow_gather(int64_t nnz, const int64_t* __restrict__ cptr, const int32_t* __restrict__ cel,
                              const uint8_t* __restrict__ cij, const int32_t* __restrict__ conn,
                              const double* __restrict__ emat, const double* __restrict__ ecoef,
                              const double* __restrict__ a21, const double* __restrict__ dinv,
                              double* __restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    double s = 0.0;
    for (int64_t t = cptr[q]; t < cptr[q + 1]; ++t) {
        const int64_t e = cel[t];
        const int i = cij[t] >> 2, j = cij[t] & 3;
        s += ecoef[2 * e] * emat[36 * e + 4 * i + j] + ecoef[2 * e + 1] * emat[36 * e + 16 + 4 * i + j];
        if (dinv) s -= a21[4 * e + i] * (1.0 / nodes_of(conn, e)) * dinv[e];
    }
    out[q] = s;
}

// y2 = A21 x1 + A22 x2 (node rows; A21 through the node's element list, in order)
__global__ void k_flow_rows(int64_t nn, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const int64_t* __restrict__ nptr,
                            const int32_t* __restrict__ nel, const uint8_t* __restrict__ nloc,
                            const double* __restrict__ a21, const double* __restrict__ x1,
                            const double* __restrict__ x2, double* __restrict__ y2) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nn) return;
    double s = 0.0;
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) s += val[q] * x2[col[q]];
    if (x1)
        for (int64_t t = nptr[r]; t < nptr[r + 1]; ++t) {
            const int64_t e = nel[t];
            s += a21[4 * e + nloc[t]] * x1[3 * e + 2];
        }
    y2[r] = s;
}

// y1[3e + 2] += sgn * (1 / nodes) sum_i x2[conn[e][i]]  (A12 = N_p)
__global__ void k_np_add(int64_t N, const int32_t* __restrict__ conn, const double* __restrict__ x2, double sgn,
                         double* __restrict__ y1) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int nv = nodes_of(conn, e);
    double s = x2[conn[4 * e]] + x2[conn[4 * e + 1]] + x2[conn[4 * e + 2]];
    if (nv == 4) s += x2[conn[4 * e + 3]];
    y1[3 * e + 2] += sgn * s / nv;
}

__global__ void k_normal_inv(int64_t N, const double* __restrict__ diag, double* __restrict__ dinv,
                             int* __restrict__ bad) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    const double d = diag[3 * e + 2];
    if (!(d != 0.0) || !isfinite(d)) atomicOr(bad, 1);
    dinv[e] = 1.0 / d;
}

__global__ void k_diag_of(int64_t nn, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ dinv, int* __restrict__ bad) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nn) return;
    double d = 0.0;
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q)
        if (col[q] == r) d = val[q];
    if (!(d != 0.0) || !isfinite(d)) atomicOr(bad, 1);
    dinv[r] = 1.0 / d;
}


// per-block partial sums of x . y (fixed order inside and across blocks)
__global__ void k_dot_part(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                           double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) s += x[i] * y[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sm[w];
        part[blockIdx.x] = t;
    }
}

// y = alpha x + beta y
__global__ void k_axpby(int64_t n, double alpha, const double* __restrict__ x, double beta, double* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = alpha * x[i] + beta * y[i];
}

constexpr int DOT_BLOCKS = 304;  // two per SM

struct Dots {
    DevBuf<double> part{(size_t)DOT_BLOCKS};
    double dot(int64_t n, const double* x, const double* y, cudaStream_t st) {
        k_dot_part<<<DOT_BLOCKS, NT, 0, st>>>(n, x, y, part.p);
        HM_LAUNCH_CHECK();
        double h[DOT_BLOCKS];
        HM_CUDA(cudaMemcpyAsync(h, part.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        double s = 0.0;
        for (int b = 0; b < DOT_BLOCKS; ++b) s += h[b];
        return s;
    }
};

void axpby(int64_t n, double alpha, const double* x, double beta, double* y, cudaStream_t st) {
    k_axpby<<<gsz(n), NT, 0, st>>>(n, alpha, x, beta, y);
    HM_LAUNCH_CHECK();
}

}  // namespace

// the flow matrices at the current iterate
void flow_assemble(hm_flow& F, const hm_flow_params& p, const double* dn, const double* dp, const double* pn,
                   cudaStream_t st) {
    if (!(p.mu > 0.0) || !(p.M > 0.0) || !(p.dt > 0.0) || !(p.w0 >= 0.0) || !std::isfinite(p.mu) ||
        !std::isfinite(p.M) || !std::isfinite(p.dt) || !std::isfinite(p.w0))
        fail(HM_EINVAL, "flow_assemble: mu, M, dt must be > 0 and w0 >= 0, all finite");
    if (!dn) fail(HM_EINVAL, "flow_assemble: NULL normal DD");
    if (F.N > 0) {
        k_flow_elem<<<gsz(F.N), NT, 0, st>>>(F.N, F.conn.p, F.emat.p, dn, dp, pn, p.mu, p.M, p.w0, p.dt,
                                             F.ecoef.p, F.a21.p);
        HM_LAUNCH_CHECK();
    }
    if (F.nnz > 0) {
        k_flow_gather<<<gsz(F.nnz), NT, 0, st>>>(F.nnz, F.cptr.p, F.cel.p, F.cij.p, F.conn.p, F.emat.p,
                                                 F.ecoef.p, F.a21.p, nullptr, F.a22.p);
        HM_LAUNCH_CHECK();
    }
    F.assembled = true;
}

// y = J x: y1 = A11 x1 + N_p x2, y2 = A21 x1 + A22 x2 (x, y: [3N | nn], user order)
void coupled_apply(HMat& H, const hm_flow& F, const double* kel, const double* cep, double shift, const double* x,
                   double* y, cudaStream_t st) {
    const int64_t n1 = 3 * F.N;
    tangent_apply_user(H, kel, cep, shift, x, y, st);
    k_np_add<<<gsz(F.N), NT, 0, st>>>(F.N, F.conn.p, x + n1, 1.0, y);
    k_flow_rows<<<gsz(F.nn), NT, 0, st>>>(F.nn, F.rowptr.p, F.col.p, F.a22.p, F.nptr.p, F.nel.p, F.nloc.p, F.a21.p,
                                          x, x + n1, y + n1);
    HM_LAUNCH_CHECK();
}

namespace {

// Scalars of the Schur BiCGSTAB on the device: sc = {rho, alpha, omega, beta, bn, done}
struct SchurScal {
    double rho, alpha, omega, beta, bn2;
    int done, iters, pad;
};

// the sum of DOT_BLOCKS partials, in block order, by one warp (lane-strided, then a
// butterfly: a fixed order)
__device__ __forceinline__ double sum_parts(const double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < DOT_BLOCKS; b += 32) s += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// stage 0: rho_new = (rh, r) -> beta; 1: alpha = rho / (rh, v); 2: omega = (t, s) / (t, t);
// 3: ||r||^2 -> done; -1: ||y||^2 -> bn2.  One warp.
__global__ void k_schur_stage(int stage, const double* __restrict__ p0, const double* __restrict__ p1, double tol,
                              int maxit, SchurScal* __restrict__ sc) {
    const double d0 = sum_parts(p0);
    const double d1 = p1 ? sum_parts(p1) : 0.0;
    if (threadIdx.x != 0) return;
    SchurScal& S = *sc;
    if (stage == -1) {
        S.bn2 = d0;
        S.rho = S.alpha = S.omega = 1.0;
        S.beta = 0.0;
        S.iters = 0;
        S.done = d0 > 0.0 ? 0 : 1;
        return;
    }
    if (S.done) return;
    if (stage == 0) {
        if (!(d0 != 0.0) || !isfinite(d0)) {
            S.done = 1;
            return;
        }
        S.beta = S.iters == 0 ? 0.0 : (d0 / S.rho) * (S.alpha / S.omega);
        S.rho = d0;
    } else if (stage == 1) {
        if (!(d0 != 0.0) || !isfinite(d0)) {
            S.done = 1;
            return;
        }
        S.alpha = S.rho / d0;
    } else if (stage == 2) {
        S.omega = d1 > 0.0 ? d0 / d1 : 0.0;
    } else {
        ++S.iters;
        if (d0 <= tol * tol * S.bn2 || !(S.omega != 0.0) || S.iters >= maxit) S.done = 1;
    }
}

// p = r + beta (p - omega v)
__global__ void k_schur_p(int64_t n, double* __restrict__ p, const double* __restrict__ r,
                          const double* __restrict__ v, const SchurScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || sc->done) return;
    p[i] = r[i] + sc->beta * (p[i] - sc->omega * v[i]);
}
// s = r - alpha v;  z += alpha ph
__global__ void k_schur_s(int64_t n, double* __restrict__ sv, const double* __restrict__ r,
                          const double* __restrict__ v, double* __restrict__ z, const double* __restrict__ ph,
                          const SchurScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || sc->done) return;
    sv[i] = r[i] - sc->alpha * v[i];
    z[i] += sc->alpha * ph[i];
}
// z += omega sh;  r = s - omega t
__global__ void k_schur_zr(int64_t n, double* __restrict__ z, double* __restrict__ r, const double* __restrict__ sh,
                           const double* __restrict__ sv, const double* __restrict__ t,
                           const SchurScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || sc->done) return;
    z[i] += sc->omega * sh[i];
    r[i] = sv[i] - sc->omega * t[i];
}
// x .* y (Jacobi) and the CSR product, skipped once done
__global__ void k_schur_mul(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                            double* __restrict__ z, const SchurScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !sc->done) z[i] = x[i] * y[i];
}
__global__ void k_schur_spmv(int64_t nn, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                             const SchurScal* __restrict__ sc) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nn || sc->done) return;
    double s = 0.0;
    for (int64_t q = rowptr[r]; q < rowptr[r + 1]; ++q) s += val[q] * x[col[q]];
    y[r] = s;
}

// z = S~^-1 y by Jacobi-preconditioned BiCGSTAB to the relative tolerance tol (x0 = 0),
// scalars on the device; the host polls the done flag two iterations behind through
// pinned memory.  Returns the iterations.
struct SchurWS {
    DevBuf<double> v;        // r, rh, p, v, ph, s, sh, t and three partial rows
    DevBuf<SchurScal> sc{(size_t)1};
    SchurScal* h_sc = nullptr;  // pinned
    cudaEvent_t ev[2] = {nullptr, nullptr};
    SchurWS() {
        HM_CUDA(cudaHostAlloc((void**)&h_sc, 2 * sizeof(SchurScal), cudaHostAllocDefault));
        for (cudaEvent_t& e : ev) HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    ~SchurWS() {
        if (h_sc) cudaFreeHost(h_sc);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

int schur_solve(const hm_flow& F, const double* sval, const double* sdinv, const double* y, double* z, double tol,
                int maxit, SchurWS& W, cudaStream_t st) {
    const int64_t n = F.nn;
    if (W.v.n < (size_t)(8 * n + 3 * DOT_BLOCKS)) W.v.alloc((size_t)(8 * n + 3 * DOT_BLOCKS));
    double *r = W.v.p, *rh = r + n, *p = rh + n, *v = p + n, *ph = v + n, *sv = ph + n, *sh = sv + n, *t = sh + n;
    double *pa = t + n, *pb = pa + DOT_BLOCKS, *pc = pb + DOT_BLOCKS;
    SchurScal* sc = W.sc.p;
    const unsigned g = gsz(n);
    auto dot = [&](const double* a, const double* b, double* part) {
        k_dot_part<<<DOT_BLOCKS, NT, 0, st>>>(n, a, b, part);
    };
    HM_CUDA(cudaMemsetAsync(z, 0, n * sizeof(double), st));
    HM_CUDA(cudaMemcpyAsync(r, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaMemcpyAsync(rh, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaMemsetAsync(p, 0, n * sizeof(double), st));
    HM_CUDA(cudaMemsetAsync(v, 0, n * sizeof(double), st));
    dot(y, y, pa);
    k_schur_stage<<<1, 32, 0, st>>>(-1, pa, nullptr, tol, maxit, sc);
    HM_LAUNCH_CHECK();
    for (int it = 0; it < maxit; ++it) {
        if (it >= 2) {
            HM_CUDA(cudaEventSynchronize(W.ev[it % 2]));
            if (W.h_sc[it % 2].done) break;
        }
        dot(rh, r, pa);
        k_schur_stage<<<1, 32, 0, st>>>(0, pa, nullptr, tol, maxit, sc);
        k_schur_p<<<g, NT, 0, st>>>(n, p, r, v, sc);
        k_schur_mul<<<g, NT, 0, st>>>(n, sdinv, p, ph, sc);
        k_schur_spmv<<<g, NT, 0, st>>>(n, F.rowptr.p, F.col.p, sval, ph, v, sc);
        dot(rh, v, pa);
        k_schur_stage<<<1, 32, 0, st>>>(1, pa, nullptr, tol, maxit, sc);
        k_schur_s<<<g, NT, 0, st>>>(n, sv, r, v, z, ph, sc);
        k_schur_mul<<<g, NT, 0, st>>>(n, sdinv, sv, sh, sc);
        k_schur_spmv<<<g, NT, 0, st>>>(n, F.rowptr.p, F.col.p, sval, sh, t, sc);
        dot(t, sv, pb);
        dot(t, t, pc);
        k_schur_stage<<<1, 32, 0, st>>>(2, pb, pc, tol, maxit, sc);
        k_schur_zr<<<g, NT, 0, st>>>(n, z, r, sh, sv, t, sc);
        dot(r, r, pa);
        k_schur_stage<<<1, 32, 0, st>>>(3, pa, nullptr, tol, maxit, sc);
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaMemcpyAsync(W.h_sc + (it % 2), sc, sizeof(SchurScal), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaEventRecord(W.ev[it % 2], st));
    }
    HM_CUDA(cudaMemcpyAsync(W.h_sc, sc, sizeof(SchurScal), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    return W.h_sc[0].iters;
}

}  // namespace

void coupled_solve(HMat& H, const hm_flow& F, const double* kel, const double* cep, double shift, const double* bv,
                   double* x, const hm_coupled_opts& o, hm_coupled_info* info, cudaStream_t st) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (!F.assembled) fail(HM_EINVAL, "coupled_solve: the flow matrices are not assembled (hm_flow_assemble)");
    if (3 * F.N != H.ndof) fail(HM_EINVAL, "coupled_solve: the flow mesh and the H-matrix differ in size");
    if (!bv || !x) fail(HM_EINVAL, "coupled_solve: NULL vector");
    const double tol = o.tol > 0 ? o.tol : 1e-8;
    const int m = o.restart > 0 ? o.restart : 30;
    const int maxit = o.maxit > 0 ? o.maxit : 300;
    const double itol = o.inner_tol > 0 ? o.inner_tol : 1e-6;
    const double stol = o.schur_tol > 0 ? o.schur_tol : 1e-6;
    const int64_t n1 = 3 * F.N, n2 = F.nn, n = n1 + n2;
    Dots D;
    // S~ = A22 - A21 diag(A11)^-1 A12 and its Jacobi inverse
    DevBuf<double> diag(n1), dinv(std::max<int64_t>(F.N, 1)), sval(std::max<int64_t>(F.nnz, 1)),
        sdinv(std::max<int64_t>(n2, 1));
    DevBuf<int> bad(1);
    HM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    tangent_diag_user(H, kel, cep, shift, diag.p, st);
    k_normal_inv<<<gsz(F.N), NT, 0, st>>>(F.N, diag.p, dinv.p, bad.p);
    k_flow_gather<<<gsz(F.nnz), NT, 0, st>>>(F.nnz, F.cptr.p, F.cel.p, F.cij.p, F.conn.p, F.emat.p, F.ecoef.p,
                                             F.a21.p, dinv.p, sval.p);
    k_diag_of<<<gsz(n2), NT, 0, st>>>(n2, F.rowptr.p, F.col.p, sval.p, sdinv.p, bad.p);
    HM_LAUNCH_CHECK();
    {
        int e = 0;
        HM_CUDA(cudaMemcpyAsync(&e, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (e) fail(HM_EBREAKDOWN, "coupled_solve: a zero or non-finite diagonal in A11 or the Schur complement");
    }
    hm_solve_opts io{};
    io.tol = itol;
    io.precond = o.inner_precond;
    io.mode = HM_SOLVE_F64;
    io.method = o.inner_method;
    io.ilu_p = o.ilu_p;
    io.cep_dev = cep;
    io.maxit = 3000;
    io.reuse_precond = 0;  // the first nested solve builds it, the others keep it
    DevBuf<double> V((size_t)(m + 1) * n), Z((size_t)m * n), w(n), r(n), t1(n1), bs(n);
    SchurWS sws;
    std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
    // the flow rows scaled by sr (Sec. 3.3.2 scales residuals to order one): by default
    // the ratio of the RMS diagonal of A11 to that of S~, so that the stopping test
    // weighs both blocks; the solve runs on diag(I, sr I) J, its residual in that norm
    double sr = o.flow_scale;
    if (!(sr > 0.0))
        sr = std::sqrt(D.dot(n1, diag.p, diag.p, st) / (double)n1) *
             std::sqrt(D.dot(n2, sdinv.p, sdinv.p, st) / (double)n2);
    if (!(sr > 0.0) || !std::isfinite(sr)) sr = 1.0;
    HM_CUDA(cudaMemcpyAsync(bs.p, bv, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    axpby(n2, 0.0, bs.p + n1, sr, bs.p + n1, st);
    const double* bsc = bs.p;
    auto apply_scaled = [&](const double* xin, double* yout) {
        coupled_apply(H, F, kel, cep, shift, xin, yout, st);
        axpby(n2, 0.0, yout + n1, sr, yout + n1, st);
    };
    const double bn = std::sqrt(D.dot(n, bsc, bsc, st));
    HM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    int its = 0, inner = 0, schur = 0;
    double rn = bn;
    HM_CUDA(cudaMemcpyAsync(r.p, bsc, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    while (bn > 0.0 && rn > tol * bn && its < maxit) {
        // V0 = r / ||r||
        HM_CUDA(cudaMemsetAsync(V.p, 0, n * sizeof(double), st));
        axpby(n, 1.0 / rn, r.p, 0.0, V.p, st);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = rn;
        int j = 0;
        for (; j < m && its < maxit; ++j) {
            const double* vj = V.p + (size_t)j * n;
            double* zj = Z.p + (size_t)j * n;
            // z = P_up^-1 v of the scaled system: z2 = S~^-1 v2 / sr, z1 = A11^-1 (v1 - N_p z2)
            schur += schur_solve(F, sval.p, sdinv.p, vj + n1, zj + n1, stol, 2000, sws, st);
            axpby(n2, 0.0, zj + n1, 1.0 / sr, zj + n1, st);
            HM_CUDA(cudaMemcpyAsync(t1.p, vj, n1 * sizeof(double), cudaMemcpyDeviceToDevice, st));
            k_np_add<<<gsz(F.N), NT, 0, st>>>(F.N, F.conn.p, zj + n1, -1.0, t1.p);
            HM_LAUNCH_CHECK();
            hm_solve_info ii{};
            try {
                gmres_solve(H, kel, shift, t1.p, zj, 1, io, &ii, st);
            } catch (const Error& e) {
                // an inexact inner solve is still a valid flexible preconditioner step
                if (e.code != HM_ENOCONV) throw;
            }
            io.reuse_precond = 1;
            inner += ii.iters;
            apply_scaled(zj, w.p);
            // modified Gram-Schmidt
            for (int i = 0; i <= j; ++i) {
                const double h = D.dot(n, w.p, V.p + (size_t)i * n, st);
                Hm[(size_t)i * m + j] = h;
                axpby(n, -h, V.p + (size_t)i * n, 1.0, w.p, st);
            }
            const double hn = std::sqrt(D.dot(n, w.p, w.p, st));
            Hm[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) axpby(n, 1.0 / hn, w.p, 0.0, V.p + (size_t)(j + 1) * n, st);
            for (int i = 0; i < j; ++i) {
                const double a = Hm[(size_t)i * m + j], b = Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                Hm[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = Hm[(size_t)j * m + j], b = Hm[(size_t)(j + 1) * m + j];
            const double den = std::hypot(a, b);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? b / den : 0.0;
            Hm[(size_t)j * m + j] = den;
            Hm[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            if (std::fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
                ++j;
                break;
            }
        }
        // x += Z y, y from the triangular system
        std::vector<double> yv(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < j; ++l) s -= Hm[(size_t)i * m + l] * yv[l];
            yv[i] = Hm[(size_t)i * m + i] != 0.0 ? s / Hm[(size_t)i * m + i] : 0.0;
        }
        for (int i = 0; i < j; ++i) axpby(n, yv[i], Z.p + (size_t)i * n, 1.0, x, st);
        // true residual
        apply_scaled(x, w.p);
        HM_CUDA(cudaMemcpyAsync(r.p, bsc, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        axpby(n, -1.0, w.p, 1.0, r.p, st);
        rn = std::sqrt(D.dot(n, r.p, r.p, st));
        if (j == 0) break;
    }
    const double rel = bn > 0 ? rn / bn : 0.0;
    if (info) {
        info->iters = its;
        info->inner_iters = inner;
        info->schur_iters = schur;
        info->status = rel <= tol ? HM_OK : HM_ENOCONV;
        info->relres = rel;
        info->seconds = std::chrono::duration<double>(clk::now() - t0).count();
    }
    if (rel > tol) fail(HM_ENOCONV, "coupled_solve: tolerance not reached within maxit");
}

}  // namespace hm

// ---------------------------------------------------------------- C ABI

namespace hm {
namespace {

// element matrices on the host (row-major m, k, v of 16, 16, 4 entries): the closed
// forms of the bilinear rectangle (nodes (-a,-b), (+a,-b), (+a,+b), (-a,+b)) and of the
// linear triangle (mass A/12 (1 + delta), load A/3, stiffness e_i . e_j / (4 A) with e_i
// the edge opposite node i)
void rect_matrices(double a, double b, double* T) {
    const double xi[4] = {-1.0, 1.0, 1.0, -1.0}, et[4] = {-1.0, -1.0, 1.0, 1.0};
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            const int d = (i - j + 4) & 3;  // 4 on the diagonal, 2 along an edge, 1 across
            T[4 * i + j] = 4.0 * a * b / 36.0 * (d == 0 ? 4.0 : (d == 2 ? 1.0 : 2.0));
            const double xx = xi[i] * xi[j], ee = et[i] * et[j];
            T[16 + 4 * i + j] = (b / a) / 12.0 * xx * (3.0 + ee) + (a / b) / 12.0 * ee * (3.0 + xx);
        }
        T[32 + i] = a * b;
    }
}

double tri_matrices(const double* P, double* T) {
    double e[3][3];
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) e[i][d] = P[3 * ((i + 2) % 3) + d] - P[3 * ((i + 1) % 3) + d];
    // twice the area: |e_2 x e_0| (e_2 = P1 - P0, e_0 = P2 - P1)
    const double cx = e[2][1] * e[0][2] - e[2][2] * e[0][1], cy = e[2][2] * e[0][0] - e[2][0] * e[0][2],
                 cz = e[2][0] * e[0][1] - e[2][1] * e[0][0];
    const double A = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    for (int q = 0; q < 36; ++q) T[q] = 0.0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            T[4 * i + j] = A / 12.0 * (i == j ? 2.0 : 1.0);
            T[16 + 4 * i + j] = (e[i][0] * e[j][0] + e[i][1] * e[j][1] + e[i][2] * e[j][2]) / (4.0 * A);
        }
        T[32 + i] = A / 3.0;
    }
    return A;
}

}  // namespace
}  // namespace hm

extern "C" hm_status hm_flow_create(int64_t N, const int32_t* conn, int64_t n_nodes, const double* a,
                                    const double* b, hm_flow** out) {
    return hm_flow_create_mesh(N, nullptr, conn, n_nodes, a, b, nullptr, out);
}

extern "C" hm_status hm_flow_create_mesh(int64_t N, const int32_t* shape, const int32_t* conn, int64_t n_nodes,
                                         const double* a, const double* b, const double* tri, hm_flow** out) {
    using namespace hm;
    HM_API_BEGIN
    if (!out) fail(HM_EINVAL, "flow_create: NULL output");
    *out = nullptr;
    if (N <= 0 || n_nodes <= 0 || !conn || !a || !b) fail(HM_EINVAL, "flow_create: empty mesh or NULL array");
    if (n_nodes > INT32_MAX || N > INT32_MAX) fail(HM_EINVAL, "flow_create: mesh too large");
    std::vector<double> emat((size_t)36 * N);
    std::vector<int> nv(N);
    for (int64_t e = 0; e < N; ++e) {
        const int sh = shape ? shape[e] : HM_SHAPE_RECT;
        if (sh != HM_SHAPE_RECT && sh != HM_SHAPE_TRI) fail(HM_EINVAL, "flow_create: unknown element shape");
        nv[e] = sh == HM_SHAPE_TRI ? 3 : 4;
        if (sh == HM_SHAPE_TRI && conn[4 * e + 3] != -1)
            fail(HM_EINVAL, "flow_create: a triangle's fourth node slot must be -1");
        for (int i = 0; i < nv[e]; ++i)
            if (conn[4 * e + i] < 0 || conn[4 * e + i] >= n_nodes)
                fail(HM_EINVAL, "flow_create: node index out of range");
        for (int i = 0; i < nv[e]; ++i)
            for (int j = i + 1; j < nv[e]; ++j)
                if (conn[4 * e + i] == conn[4 * e + j]) fail(HM_EINVAL, "flow_create: an element repeats a node");
        if (sh == HM_SHAPE_RECT) {
            if (!(a[e] > 0.0) || !(b[e] > 0.0) || !std::isfinite(a[e]) || !std::isfinite(b[e]))
                fail(HM_EINVAL, "flow_create: half sides must be finite and > 0");
            rect_matrices(a[e], b[e], emat.data() + 36 * e);
        } else {
            if (!tri) fail(HM_EINVAL, "flow_create: triangles need their vertices (tri)");
            for (int q = 0; q < 9; ++q)
                if (!std::isfinite(tri[9 * e + q])) fail(HM_ENAN, "flow_create: non-finite triangle vertex");
            const double A = tri_matrices(tri + 9 * e, emat.data() + 36 * e);
            if (!(A > 0.0)) fail(HM_EINVAL, "flow_create: degenerate triangle");
        }
    }
    auto F = std::make_unique<hm_flow>();
    F->N = N;
    F->nn = n_nodes;
    F->h_conn.assign(conn, conn + 4 * N);
    // node-node pattern (the blocks of the elements), columns increasing
    std::vector<std::vector<int32_t>> adj(n_nodes);
    for (int64_t e = 0; e < N; ++e)
        for (int i = 0; i < nv[e]; ++i)
            for (int j = 0; j < nv[e]; ++j) adj[conn[4 * e + i]].push_back(conn[4 * e + j]);
    std::vector<int64_t> rp(n_nodes + 1, 0);
    std::vector<int32_t> cl;
    for (int64_t r = 0; r < n_nodes; ++r) {
        auto& v = adj[r];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        rp[r + 1] = rp[r] + (int64_t)v.size();
        cl.insert(cl.end(), v.begin(), v.end());
    }
    const int64_t nnz = rp[n_nodes];
    // contributions per entry, in element order
    std::vector<std::vector<std::pair<int32_t, uint8_t>>> con(nnz);
    std::vector<std::vector<std::pair<int32_t, uint8_t>>> nodal(n_nodes);
    for (int64_t e = 0; e < N; ++e)
        for (int i = 0; i < nv[e]; ++i) {
            const int32_t r = conn[4 * e + i];
            nodal[r].push_back({(int32_t)e, (uint8_t)i});
            for (int j = 0; j < nv[e]; ++j) {
                const int32_t c = conn[4 * e + j];
                const int64_t q = std::lower_bound(cl.begin() + rp[r], cl.begin() + rp[r + 1], c) - cl.begin();
                con[q].push_back({(int32_t)e, (uint8_t)(4 * i + j)});
            }
        }
    std::vector<int64_t> cptr(nnz + 1, 0), nptr(n_nodes + 1, 0);
    std::vector<int32_t> cel, nel;
    std::vector<uint8_t> cij, nloc;
    for (int64_t q = 0; q < nnz; ++q) {
        cptr[q + 1] = cptr[q] + (int64_t)con[q].size();
        for (auto& pr : con[q]) {
            cel.push_back(pr.first);
            cij.push_back(pr.second);
        }
    }
    for (int64_t r = 0; r < n_nodes; ++r) {
        nptr[r + 1] = nptr[r] + (int64_t)nodal[r].size();
        for (auto& pr : nodal[r]) {
            nel.push_back(pr.first);
            nloc.push_back(pr.second);
        }
    }
    F->nnz = nnz;
    F->h_rowptr = rp;
    cudaStream_t st = nullptr;
    F->conn.upload(F->h_conn, st);
    F->rowptr.upload(rp, st);
    F->col.upload(cl, st);
    F->cptr.upload(cptr, st);
    F->cel.upload(cel, st);
    F->cij.upload(cij, st);
    F->nptr.upload(nptr, st);
    F->nel.upload(nel, st);
    F->nloc.upload(nloc, st);
    F->a.upload(std::vector<double>(a, a + N), st);
    F->b.upload(std::vector<double>(b, b + N), st);
    F->emat.upload(emat, st);
    F->a22.alloc(nnz);
    F->a21.alloc(4 * N);
    F->ecoef.alloc(2 * N);
    HM_CUDA(cudaStreamSynchronize(st));
    *out = F.release();
    HM_API_END
}

extern "C" void hm_flow_destroy(hm_flow* f) { delete f; }

extern "C" hm_status hm_flow_assemble(hm_flow* f, const hm_flow_params* prm, const double* dn_dev,
                                      const double* dp_dev, const double* pn_dev, void* stream) {
    HM_API_BEGIN
    if (!f || !prm) hm::fail(HM_EINVAL, "flow_assemble: NULL argument");
    hm::flow_assemble(*f, *prm, dn_dev, dp_dev, pn_dev, (cudaStream_t)stream);
    HM_API_END
}

extern "C" hm_status hm_flow_export(const hm_flow* f, int64_t* nnz_out, int64_t* rowptr, int32_t* col, double* a22,
                                    double* a21, void* stream) {
    HM_API_BEGIN
    if (!f) hm::fail(HM_EINVAL, "flow_export: NULL flow");
    cudaStream_t st = (cudaStream_t)stream;
    if (nnz_out) *nnz_out = f->nnz;
    if (rowptr) std::copy(f->h_rowptr.begin(), f->h_rowptr.end(), rowptr);
    if (col) HM_CUDA(cudaMemcpyAsync(col, f->col.p, f->col.bytes(), cudaMemcpyDeviceToHost, st));
    if ((a22 || a21) && !f->assembled) hm::fail(HM_EINVAL, "flow_export: not assembled");
    if (a22) HM_CUDA(cudaMemcpyAsync(a22, f->a22.p, f->a22.bytes(), cudaMemcpyDeviceToHost, st));
    if (a21) HM_CUDA(cudaMemcpyAsync(a21, f->a21.p, f->a21.bytes(), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    HM_API_END
}

extern "C" hm_status hm_coupled_matvec(const hm_hmat* h, const hm_flow* f, const double* k_dev,
                                       const double* cep_dev, double shift, const double* x_dev, double* y_dev,
                                       void* stream) {
    HM_API_BEGIN
    if (!h || !f || !x_dev || !y_dev) hm::fail(HM_EINVAL, "coupled_matvec: NULL argument");
    if (!f->assembled) hm::fail(HM_EINVAL, "coupled_matvec: the flow matrices are not assembled");
    if (3 * f->N != h->h.ndof) hm::fail(HM_EINVAL, "coupled_matvec: the flow mesh and the H-matrix differ in size");
    if (!std::isfinite(shift)) hm::fail(HM_ENAN, "coupled_matvec: shift is not finite");
    hm::coupled_apply(const_cast<hm::HMat&>(h->h), *f, k_dev, cep_dev, shift, x_dev, y_dev, (cudaStream_t)stream);
    HM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    HM_API_END
}

extern "C" hm_status hm_coupled_solve(const hm_hmat* h, const hm_flow* f, const double* k_dev,
                                      const double* cep_dev, double shift, const double* b_dev, double* x_dev,
                                      const hm_coupled_opts* opt, hm_coupled_info* info, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_coupled_solve");
    if (!h || !f) hm::fail(HM_EINVAL, "coupled_solve: NULL argument");
    if (!std::isfinite(shift)) hm::fail(HM_ENAN, "coupled_solve: shift is not finite");
    hm_coupled_opts o{};
    if (opt) o = *opt;
    if (!opt) o.inner_precond = HM_PRECOND_BLOCKJ;
    if (o.inner_precond == HM_PRECOND_LEARNED) hm::fail(HM_EINVAL, "coupled_solve: no learned inner preconditioner");
    hm::coupled_solve(const_cast<hm::HMat&>(h->h), *f, k_dev, cep_dev, shift, b_dev, x_dev, o, info,
                      (cudaStream_t)stream);
    HM_API_END
}
