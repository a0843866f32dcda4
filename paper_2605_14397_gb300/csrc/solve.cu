// Tangent solve A x = b, A = E - diag(k) - C^ep - shift I (eq. jac_mech: C^ep block
// diagonal with 3x3 blocks, or diagonal as k; eta/dt = shift): restarted flexible GMRES(m)
// with right preconditioning, on the device.
//
// The paper solves its A11 system with a Krylov method (BiCGSTAB or GMRES) and a Jacobi
// preconditioner (Sec. 3.3.1).  Here:
//   * Krylov vectors, Hessenberg matrix, Gram-Schmidt and Givens rotations in FP64;
//     Arnoldi by classical Gram-Schmidt applied twice (CGS2); x0 = 0;
//   * flexible variant (the preconditioned vectors z_j = M^-1 v_j are kept), so the
//     preconditioner may be inexact, FP32, or nonlinear (the learned correction);
//   * block-Jacobi preconditioner: the inverse of every diagonal leaf block of A,
//     from the stored FP32 near-field tile minus the diagonal, by Gauss-Jordan with
//     partial pivoting in shared memory (FP32);
//   * every kernel of a restart cycle reads a per-RHS `done` flag set by the Givens step
//     when the residual estimate meets the tolerance, so a cycle of m iterations is
//     launched without host synchronisation; the host synchronises once per cycle;
//   * point-Jacobi preconditioner (the paper's): the inverse of every element's 3x3
//     diagonal block of A;
//   * mode F64: products with the FP32 factors in compensated FP64 throughout;
//     mode MIXED: iterative refinement (outer residual in compensated FP64 with the
//     FP32 factors; corrections by FGMRES on the BF16-factor operator, FP32 products);
//     mode PLAIN32: the same refinement with the corrections on the FP32 factors.
// Vectors are kept in cluster order internally (RHS-major, stride 3N).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "hmat_impl.h"
#include "ilu_dev.h"
#include "learned.h"

namespace hm {

namespace {

constexpr int ROW_NT = 256;
constexpr int ROWS_PER_CTA = 1024;  // 4 rows per thread
constexpr int VSLACK = 64;          // elements after each buffer read by rounded copies
constexpr int BJ_MAX_ROWS_SMEM = 224;

struct CycleState {
    int done;     // 1: stop iterating this RHS in the current cycle
    int iters;    // iterations completed in the current cycle
    int brk;      // breakdown seen
    int pad_;
    double tol;   // absolute tolerance on the residual estimate
    double inv;   // 1 / ||w|| of the last step
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- permutation, diagonal

// flag |= 1 if any of v[0..n) is NaN or infinite
__global__ void k_nonfinite(const double* __restrict__ v, int64_t n, int* __restrict__ flag) {
    int bad = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(v[q]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_to_cluster(const double* __restrict__ u, double* __restrict__ c, const int32_t* __restrict__ perm,
                             int64_t ndof, int nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, r = q % ndof;
    c[q] = u[k * ndof + 3 * (int64_t)perm[r / 3] + r % 3];
}

__global__ void k_to_user(const double* __restrict__ c, double* __restrict__ u, const int32_t* __restrict__ perm,
                          int64_t ndof, int nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, r = q % ndof;
    u[k * ndof + 3 * (int64_t)perm[r / 3] + r % 3] = c[q];
}

__global__ void k_diag(const double* __restrict__ kel, double shift, const int32_t* __restrict__ perm, int64_t ndof,
                       double* __restrict__ d) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= ndof) return;
    d[r] = (kel ? kel[perm[r / 3]] : 0.0) + shift;
}

// The interface term with a block-diagonal C^ep (eq. jac_mech): d[r] = k + C^ep_ii +
// shift on the diagonal (cluster DOF order) and blk = C^ep with a zero diagonal, 9 per
// element in cluster element order (C^ep in user element order, row-major per element).
__global__ void k_blockdiag(const double* __restrict__ kel, const double* __restrict__ cep, double shift,
                            const int32_t* __restrict__ perm, int64_t nel, double* __restrict__ d,
                            double* __restrict__ blk) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nel) return;
    const int64_t e = perm[q];
    const double kv = kel ? kel[e] : 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        d[3 * q + i] = kv + cep[9 * e + 4 * i] + shift;
#pragma unroll
        for (int j = 0; j < 3; ++j) blk[9 * q + 3 * i + j] = i == j ? 0.0 : cep[9 * e + 3 * i + j];
    }
}

// off-diagonal part of the interface term in row i of element-local block products
__device__ __forceinline__ double blk_row(const double* __restrict__ blk, const double* __restrict__ zk, int64_t i) {
    const int64_t e = i / 3;
    const double* B = blk + 9 * e + 3 * (i % 3);
    const double* z = zk + 3 * e;
    return B[0] * z[0] + B[1] * z[1] + B[2] * z[2];
}

// ---------------------------------------------------------------- block-Jacobi

// Inverse of B = E_ll - diag(d_l) for every leaf l (one CTA each), Gauss-Jordan with
// partial pivoting; B^-1 stored column-major with the leaf's padded row count.
__global__ void __launch_bounds__(512) k_bj_build(const LeafDesc* __restrict__ leaves,
                                                  const int64_t* __restrict__ self_off,
                                                  const float* __restrict__ near, const double* __restrict__ d,
                                                  const double* __restrict__ blk, float* __restrict__ binv,
                                                  const int64_t* __restrict__ binv_off, float* __restrict__ gscratch,
                                                  int use_smem, int* __restrict__ err) {
    extern __shared__ float sm[];
    const LeafDesc L = leaves[blockIdx.x];
    const int n = 3 * L.n;
    float* A = use_smem ? sm : gscratch + binv_off[blockIdx.x];  // row-major n x n
    __shared__ float colk[384];
    __shared__ int piv[384];
    __shared__ float s_v[16];
    __shared__ int s_i[16];
    const int tid = threadIdx.x, nt = blockDim.x;
    const float* E = near + self_off[blockIdx.x];
    for (int q = tid; q < n * n; q += nt) {
        const int r = q / n, c = q % n;
        float v = E[(int64_t)c * L.ld + r];
        if (r == c) v -= (float)d[3 * (int64_t)L.begin + r];
        if (blk && r / 3 == c / 3) v -= (float)blk[9 * ((int64_t)L.begin + r / 3) + 3 * (r % 3) + c % 3];
        A[q] = v;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // pivot: largest |A[i][k]|, i >= k
        float bv = -1.f;
        int bi = k;
        for (int i = k + tid; i < n; i += nt) {
            const float v = fabsf(A[i * n + k]);
            if (v > bv) { bv = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { s_v[tid >> 5] = bv; s_i[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            float b = -1.f;
            int ib = k;
            for (int w = 0; w < nt / 32; ++w)
                if (s_v[w] > b || (s_v[w] == b && s_i[w] < ib)) { b = s_v[w]; ib = s_i[w]; }
            piv[k] = ib;
            if (!(b > 0.f)) atomicOr(err, 1);
        }
        __syncthreads();
        const int p = piv[k];
        if (p != k)
            for (int c = tid; c < n; c += nt) {
                const float t = A[k * n + c];
                A[k * n + c] = A[p * n + c];
                A[p * n + c] = t;
            }
        __syncthreads();
        const float pv = A[k * n + k];
        const float pinv = pv != 0.f ? 1.f / pv : 0.f;
        for (int i = tid; i < n; i += nt) colk[i] = A[i * n + k];
        __syncthreads();
        for (int c = tid; c < n; c += nt) A[k * n + c] = (c == k ? 1.f : A[k * n + c]) * pinv;
        __syncthreads();
        for (int q = tid; q < n * n; q += nt) {
            const int i = q / n, c = q % n;
            if (i == k) continue;
            A[q] = (c == k ? 0.f : A[q]) - A[k * n + c] * colk[i];
        }
        __syncthreads();
    }
    // undo the row interchanges by column interchanges, last first
    for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int i = tid; i < n; i += nt) {
                const float t = A[i * n + k];
                A[i * n + k] = A[i * n + p];
                A[i * n + p] = t;
            }
        __syncthreads();
    }
    float* out = binv + binv_off[blockIdx.x];
    for (int q = tid; q < n * n; q += nt) {
        const int r = q / n, c = q % n;
        out[(int64_t)c * L.ld + r] = A[q];
    }
}

// The same inverse for leaves of at most BJR_ROWS rows, with the matrix held in registers:
// 512 threads, thread (tr, tc) = (t / 32, t % 32) owns rows tr + 16 a (a < AR) and columns
// tc + 32 b (b < BC), the tile sized by the largest leaf of the launch.  Gauss-Jordan by
// in-place sweeps with partial pivoting and no row interchanges: step k picks the unused
// row p_k with the largest |A[i][k]| (ties: the lowest row) and sweeps on (p_k, k) -- the
// pivot row divided by the pivot, every other row i minus A[i][k] times it, column k
// replaced by -A[i][k] / pivot and 1 / pivot.  After n sweeps row p_k holds the
// coefficients of unknown k against equations p_0 .. p_(n-1), so A^-1[k][m] = W[p_k][q]
// with p_q = m.
// A sweep is one uniform rank-1 update A -= c' r'^T, r' the pivot row over the pivot
// (r'[k] = 1 / pivot), c' column k (c'[p] = -1), followed by two fix-ups: column k minus
// its old values, and row p set to r'.  Every warp finds the pivot itself (shuffles over
// the column in shared memory, the taken rows a bit mask per lane), and the column and
// the scaled pivot row are double-buffered, so a step needs two barriers.
constexpr int BJR_ROWS = 192;

// Steps k = 32 KB .. 32 KB + 31 of the sweep: column k lives in register column KB, a
// compile-time index, so only lane k % 32 of each warp touches it.  Returns false when the
// remaining column has no non-zero entry in an unused row (a singular block), with the
// same decision in every thread.
template <int AR, int BC, int KB>
__device__ __forceinline__ bool bjr_steps(float (&A)[AR][BC], unsigned& used, int n, int t, int tr, int tc,
                                          float (*colk)[16 * AR], float (*rp)[32 * BC], int* pk, int* pinv,
                                          int* err) {
    constexpr int M = (16 * AR + 31) / 32;  // row slots per lane in the pivot search
    for (int kc = 0; kc < 32; ++kc) {
        const int k = 32 * KB + kc;
        if (k >= n) return true;
        const int buf = k & 1;
        if (tc == kc) {
#pragma unroll
            for (int a = 0; a < AR; ++a) colk[buf][tr + 16 * a] = A[a][KB];
        }
        __syncthreads();
        float bv = -1.f;
        int bi = 0x7fffffff;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int i = tc + 32 * m;
            if (i < n && !((used >> m) & 1u)) {
                const float v = fabsf(colk[buf][i]);
                if (v > bv) {  // rows ascend within a lane: the lowest row wins ties
                    bv = v;
                    bi = i;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (!(bv > 0.f)) {  // every warp sees the same column: a uniform exit
            if (t == 0) atomicOr(err, 1);
            return false;
        }
        const int p = bi, ap = p >> 4;
        if (tc == (p & 31)) used |= 1u << (p >> 5);
        if (t == 0) {
            pk[k] = p;
            pinv[p] = k;
        }
        if (tr == (p & 15)) {  // the warp of the pivot row: r' = row p / pivot, r'[k] = 1 / pivot
            const float pinvv = 1.0f / colk[buf][p];
#pragma unroll
            for (int a = 0; a < AR; ++a)
                if (a == ap)
#pragma unroll
                    for (int b = 0; b < BC; ++b)
                        rp[buf][tc + 32 * b] = (b == KB && tc == kc) ? pinvv : A[a][b] * pinvv;
        }
        __syncthreads();
        float r[BC];
#pragma unroll
        for (int b = 0; b < BC; ++b) r[b] = rp[buf][tc + 32 * b];
#pragma unroll
        for (int a = 0; a < AR; ++a) {
            const int i = tr + 16 * a;
            const float c = (i == p) ? -1.f : colk[buf][i];
#pragma unroll
            for (int b = 0; b < BC; ++b) A[a][b] = fmaf(-c, r[b], A[a][b]);
        }
        if (tc == kc) {  // column k: -c[i] / pivot (the sweep left c[i] on top)
#pragma unroll
            for (int a = 0; a < AR; ++a) A[a][KB] -= colk[buf][tr + 16 * a];
        }
        if (tr == (p & 15)) {  // row p: r'
#pragma unroll
            for (int a = 0; a < AR; ++a)
                if (a == ap)
#pragma unroll
                    for (int b = 0; b < BC; ++b) A[a][b] = r[b];
        }
    }
    return true;
}

template <int AR, int BC, int KB>
struct BjrSweep {
    static __device__ __forceinline__ bool run(float (&A)[AR][BC], unsigned& used, int n, int t, int tr, int tc,
                                               float (*colk)[16 * AR], float (*rp)[32 * BC], int* pk, int* pinv,
                                               int* err) {
        if (!bjr_steps<AR, BC, KB>(A, used, n, t, tr, tc, colk, rp, pk, pinv, err)) return false;
        return BjrSweep<AR, BC, KB + 1>::run(A, used, n, t, tr, tc, colk, rp, pk, pinv, err);
    }
};
template <int AR, int BC>
struct BjrSweep<AR, BC, BC> {
    static __device__ __forceinline__ bool run(float (&)[AR][BC], unsigned&, int, int, int, int, float (*)[16 * AR],
                                               float (*)[32 * BC], int*, int*, int*) {
        return true;
    }
};

template <int AR, int BC>
__global__ void __launch_bounds__(512, 1) k_bj_build_reg(const LeafDesc* __restrict__ leaves,
                                                         const int64_t* __restrict__ self_off,
                                                         const float* __restrict__ near, const double* __restrict__ d,
                                                         const double* __restrict__ blk, float* __restrict__ binv,
                                                         const int64_t* __restrict__ binv_off, int* __restrict__ err) {
    extern __shared__ float wsm[];  // n x n staging (row-major): the block, then W
    __shared__ float colk[2][16 * AR], rp[2][32 * BC];
    __shared__ int pk[BJR_ROWS], pinv[BJR_ROWS];
    const LeafDesc L = leaves[blockIdx.x];
    const int n = 3 * L.n;
    const int t = threadIdx.x, tr = t >> 5, tc = t & 31;
    const float* E = near + self_off[blockIdx.x];
    // the leaf's block of E - diag(d) - C^ep, read column by column (coalesced)
    for (int q = t; q < n * n; q += 512) {
        const int j = q / n, i = q % n;
        float v = E[(int64_t)j * L.ld + i];
        if (i == j) v -= (float)d[3 * (int64_t)L.begin + i];
        if (blk && i / 3 == j / 3) v -= (float)blk[9 * ((int64_t)L.begin + i / 3) + 3 * (i % 3) + j % 3];
        wsm[i * n + j] = v;
    }
    __syncthreads();
    float A[AR][BC];
#pragma unroll
    for (int a = 0; a < AR; ++a)
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            const int i = tr + 16 * a, j = tc + 32 * b;
            A[a][b] = (i < n && j < n) ? wsm[i * n + j] : 0.f;
        }
    unsigned used = 0;  // bit m: row tc + 32 m is a pivot row already
    const bool ok = BjrSweep<AR, BC, 0>::run(A, used, n, t, tr, tc, colk, rp, pk, pinv, err);
    __syncthreads();  // every thread is past its last read of wsm
    if (!ok) return;
#pragma unroll
    for (int a = 0; a < AR; ++a)
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            const int i = tr + 16 * a, j = tc + 32 * b;
            if (i < n && j < n) wsm[i * n + j] = A[a][b];
        }
    __syncthreads();
    float* out = binv + binv_off[blockIdx.x];
    for (int q = t; q < n * n; q += 512) {
        const int c = q / n, rr = q % n;
        out[(int64_t)c * L.ld + rr] = wsm[pk[rr] * n + pinv[c]];
    }
}

template <int AR, int BC>
void bj_build_reg_launch(HMat& H, SolveWS& W, size_t smem, cudaStream_t st) {
    static bool attr_done[64] = {};
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        HM_CUDA(cudaFuncSetAttribute(k_bj_build_reg<AR, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float) * BJR_ROWS * BJR_ROWS)));
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    k_bj_build_reg<AR, BC><<<H.n_leaves, 512, smem, st>>>(H.leaves.p, W.self_off.p, H.near.p, W.dc.p, W.blk,
                                                           W.binv.p, W.binv_off.p, W.err.p);
}

// z = M^-1 v per leaf (block-Jacobi), or z = v; also the FP32 copy zf (RHS-interleaved)
__global__ void __launch_bounds__(256) k_bj_apply(const LeafDesc* __restrict__ leaves, const float* __restrict__ binv,
                                                  const int64_t* __restrict__ binv_off, const double* __restrict__ v,
                                                  double* __restrict__ z, float* __restrict__ zf, int64_t ndof, int nr,
                                                  const CycleState* __restrict__ cs, int identity,
                                                  const float* __restrict__ dsc) {
    __shared__ double red[8][384];
    const LeafDesc L = leaves[blockIdx.x];
    const int n = 3 * L.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = 3 * (int64_t)L.begin;
    for (int k = 0; k < nr; ++k) {
        if (cs[k].done) continue;
        const double* vk = v + k * ndof + base;
        double* zk = z + k * ndof + base;
        if (identity) {
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                zk[r] = vk[r];
                if (zf) zf[(base + r) * nr + k] = (float)vk[r];
            }
            continue;
        }
        // FP32 arithmetic: the flexible Krylov method tolerates an inexact preconditioner
        const float* B = binv + binv_off[blockIdx.x];
        float acc[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = 0.f;
        // two columns per pass: twice the loads in flight
        int c = w;
        for (; c + 8 < n; c += 16) {
            const float vc0 = (float)vk[c], vc1 = (float)vk[c + 8];
            const float* col0 = B + (int64_t)c * L.ld;
            const float* col1 = col0 + (int64_t)8 * L.ld;
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const int r = lane + 32 * i;
                if (r < n) acc[i] = fmaf(__ldg(col1 + r), vc1, fmaf(__ldg(col0 + r), vc0, acc[i]));
            }
        }
        for (; c < n; c += 8) {
            const float vc = (float)vk[c];
            const float* col = B + (int64_t)c * L.ld;
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const int r = lane + 32 * i;
                if (r < n) acc[i] = fmaf(__ldg(col + r), vc, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const int r = lane + 32 * i;
            if (r < 384) red[w][r] = acc[i];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            double s = 0.0;
            for (int q = 0; q < 8; ++q) s += red[q][r];
            if (dsc) s *= (double)dsc[3 * (int64_t)blockIdx.x + r % 3];  // learned correction D
            zk[r] = s;
            if (zf) zf[(base + r) * nr + k] = (float)s;
        }
        __syncthreads();
    }
}

// out = N v per row leaf: the near-field tiles of the leaf except its own diagonal block
// (columns whose operand lies in the leaf).  The work is cut into items, a run of at most
// NOD_CMAX near columns of one row leaf, so that the leaves where many near blocks meet
// (a crack crossing a fault) do not set the kernel's length; one CTA per item, a thread
// per row.  The operand v32 (FP32, RHS-interleaved [ndof][nr]) of NOD_CH columns at a
// time is staged in shared memory with the leaf's own columns zeroed, and every row
// reads its FP32 coefficients column by column (coalesced over the rows, NOD_UN loads in
// flight).  An item that covers its whole leaf writes out; the items of a longer leaf
// write FP32 partial sums, added in item order by k_near_sum (deterministic).  Products
// and sums in FP32: a preconditioner only has to be a fixed operator, and the FP64 pipe
// of this GPU is far too slow for one FMA per near-field entry.
constexpr int NOD_NT = 192, NOD_CH = 128, NOD_UN = 8, NOD_CMAX = 1024;
struct NearItem {
    int32_t leaf, c0, c1;
    int32_t prow;  // first partial row of the item; -1: the item writes out directly
};
template <int NRP>
__global__ void __launch_bounds__(NOD_NT) k_near_offdiag(const LeafDesc* __restrict__ leaves,
                                                         const NearItem* __restrict__ items,
                                                         const float* __restrict__ near,
                                                         const int32_t* __restrict__ zidx,
                                                         const float* __restrict__ v32, double* __restrict__ out,
                                                         float* __restrict__ part, int64_t ndof, int nr,
                                                         const CycleState* __restrict__ cs) {
    __shared__ __align__(16) float sv[NOD_CH * NRP];
    const NearItem it = items[blockIdx.x];
    const LeafDesc L = leaves[it.leaf];
    const int n = 3 * L.n;
    const int64_t lo = 3 * (int64_t)L.begin, hi = lo + n;
    const float* D = near + L.near_off;
    const int32_t* Z = zidx + L.near_cbase;
    for (int r0 = 0; r0 < n; r0 += NOD_NT) {
        const int r = r0 + threadIdx.x;
        float acc[NRP];
#pragma unroll
        for (int k = 0; k < NRP; ++k) acc[k] = 0.f;
        for (int c0 = it.c0; c0 < it.c1; c0 += NOD_CH) {
            const int cn = min(NOD_CH, it.c1 - c0);
            __syncthreads();
            for (int q = threadIdx.x; q < cn * NRP; q += NOD_NT) {
                const int c = q / NRP, k = q % NRP;
                const int64_t z = Z[c0 + c];
                sv[q] = (k < nr && (z < lo || z >= hi)) ? v32[z * nr + k] : 0.f;
            }
            __syncthreads();
            if (r < n) {
                const float* Dc = D + (int64_t)c0 * L.ld + r;
                int c = 0;
                for (; c + NOD_UN <= cn; c += NOD_UN) {
                    float a[NOD_UN];
#pragma unroll
                    for (int u = 0; u < NOD_UN; ++u) a[u] = __ldg(Dc + (int64_t)(c + u) * L.ld);
#pragma unroll
                    for (int u = 0; u < NOD_UN; ++u)
#pragma unroll
                        for (int k = 0; k < NRP; ++k) acc[k] = fmaf(a[u], sv[(c + u) * NRP + k], acc[k]);
                }
                for (; c < cn; ++c) {
                    const float a = __ldg(Dc + (int64_t)c * L.ld);
#pragma unroll
                    for (int k = 0; k < NRP; ++k) acc[k] = fmaf(a, sv[c * NRP + k], acc[k]);
                }
            }
        }
        if (r < n) {
#pragma unroll
            for (int k = 0; k < NRP; ++k) {
                if (k >= nr) continue;
                if (it.prow >= 0)
                    part[((int64_t)it.prow + r) * nr + k] = acc[k];
                else if (!cs || !cs[k].done)
                    out[k * ndof + lo + r] = (double)acc[k];
            }
        }
    }
}

// out rows of the leaves cut into several items: the items' partial sums added in order;
// msum[3 l'] = leaf, msum[3 l' + 1] = first partial row, msum[3 l' + 2] = items
__global__ void k_near_sum(const LeafDesc* __restrict__ leaves, const int32_t* __restrict__ msum,
                           const float* __restrict__ part, double* __restrict__ out, int64_t ndof, int nr,
                           const CycleState* __restrict__ cs) {
    const LeafDesc L = leaves[msum[3 * blockIdx.x]];
    const int64_t prow = msum[3 * blockIdx.x + 1];
    const int m = msum[3 * blockIdx.x + 2];
    const int n = 3 * L.n;
    for (int q = threadIdx.x; q < n * nr; q += blockDim.x) {
        const int r = q / nr, k = q % nr;
        if (cs && cs[k].done) continue;
        float s = 0.f;
        for (int j = 0; j < m; ++j) s += part[(prow + (int64_t)j * n + r) * nr + k];
        out[k * ndof + 3 * (int64_t)L.begin + r] = (double)s;
    }
}

// the item list of the near product: host vectors, built once per matrix
struct NearPlan {
    std::vector<NearItem> items;
    std::vector<int32_t> msum;
    int64_t part_rows = 0;
};
NearPlan near_plan(const HMat& H) {
    NearPlan P;
    for (int l = 0; l < H.n_leaves; ++l) {
        const LeafDesc& L = H.h_leaves[l];
        const int m = std::max(1, (L.near_cols + NOD_CMAX - 1) / NOD_CMAX);
        if (m == 1) {
            P.items.push_back(NearItem{l, 0, L.near_cols, -1});
            continue;
        }
        P.msum.insert(P.msum.end(), {l, (int32_t)P.part_rows, m});
        for (int j = 0; j < m; ++j) {
            const int c0 = (int)((int64_t)L.near_cols * j / m), c1 = (int)((int64_t)L.near_cols * (j + 1) / m);
            P.items.push_back(NearItem{l, c0, c1, (int32_t)(P.part_rows + (int64_t)j * 3 * L.n)});
        }
        P.part_rows += (int64_t)m * 3 * L.n;
    }
    return P;
}

struct NearDev {
    const NearItem* items;
    int n_items;
    const int32_t* msum;
    int n_multi;
    float* part;
};

void near_offdiag_launch(HMat& H, const NearDev& P, const float* v32, double* out, int nr, const CycleState* cs,
                         cudaStream_t st) {
    const int64_t n = H.ndof;
#define HM_NEAR_LAUNCH(NRP)                                                                                  \
    k_near_offdiag<NRP><<<P.n_items, NOD_NT, 0, st>>>(H.leaves.p, P.items, H.near.p, H.near_zidx.p, v32, out, \
                                                      P.part, n, nr, cs)
    if (nr == 1)
        HM_NEAR_LAUNCH(1);
    else if (nr == 2)
        HM_NEAR_LAUNCH(2);
    else if (nr <= 4)
        HM_NEAR_LAUNCH(4);
    else if (nr <= 8)
        HM_NEAR_LAUNCH(8);
    else
        HM_NEAR_LAUNCH(16);
#undef HM_NEAR_LAUNCH
    HM_LAUNCH_CHECK();
    if (P.n_multi) {
        k_near_sum<<<P.n_multi, 192, 0, st>>>(H.leaves.p, P.msum, P.part, out, n, nr, cs);
        HM_LAUNCH_CHECK();
    }
}

// z -= gamma d o u (the damped near correction), d per (leaf, component); also the FP32
// RHS-interleaved copy zf
__global__ void k_near_update(double* __restrict__ z, const double* __restrict__ u, const float* __restrict__ dsc,
                              const int32_t* __restrict__ leaf_of, double gamma, float* __restrict__ zf,
                              int64_t ndof, int nr, const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, i = q % ndof;
    if (cs && cs[k].done) return;
    const double s = z[q] - gamma * (double)dsc[3 * (int64_t)leaf_of[i / 3] + i % 3] * u[q];
    z[q] = s;
    if (zf) zf[i * nr + k] = (float)s;
}

// Point Jacobi (the paper's Jacobi preconditioner of the A11 system, Sec. 3.3.1): the
// inverse of every element's 3x3 diagonal block of A = E - diag(d), read from the leaf's
// self tile of the FP32 near field.  One CTA per leaf, one thread per element; the 3x3
// inverse by cofactors in FP64, stored row-major in FP32.
__global__ void k_j3_build(const LeafDesc* __restrict__ leaves, const int64_t* __restrict__ self_off,
                           const float* __restrict__ near, const double* __restrict__ d,
                           const double* __restrict__ blk, float* __restrict__ j3, int* __restrict__ err) {
    const LeafDesc L = leaves[blockIdx.x];
    const float* T = near + self_off[blockIdx.x];
    for (int e = threadIdx.x; e < L.n; e += blockDim.x) {
        const int64_t p = (int64_t)L.begin + e;
        double a[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                a[i][j] = (double)T[(int64_t)(3 * e + j) * L.ld + 3 * e + i];
                if (i == j) a[i][j] -= d[3 * p + i];
                if (blk) a[i][j] -= blk[9 * p + 3 * i + j];
            }
        const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
        const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
        const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
        const double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
        const double nrm = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]) + fabs(a[0][1]) + fabs(a[1][0]) +
                           fabs(a[0][2]) + fabs(a[2][0]) + fabs(a[1][2]) + fabs(a[2][1]);
        if (!(fabs(det) > 1e-30 * nrm * nrm * nrm) || !isfinite(det)) {
            atomicOr(err, 1);
            continue;
        }
        const double id = 1.0 / det;
        double inv[3][3];
        inv[0][0] = c00 * id;
        inv[1][0] = c01 * id;
        inv[2][0] = c02 * id;
        inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
        inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
        inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
        inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
        inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
        inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
        float* o = j3 + 9 * p;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) o[3 * i + j] = (float)inv[i][j];
    }
}

// z = M^-1 v with the 3x3 point-Jacobi inverses (one thread per element and RHS); also
// the FP32 copy zf (RHS-interleaved)
__global__ void k_j3_apply(const float* __restrict__ j3, const double* __restrict__ v, double* __restrict__ z,
                           float* __restrict__ zf, int64_t nel, int64_t ndof, int nr,
                           const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nel * nr) return;
    const int64_t k = q / nel, p = q % nel;
    if (cs[k].done) return;
    const double* vk = v + k * ndof + 3 * p;
    const float* B = j3 + 9 * p;
    const float v0 = (float)vk[0], v1 = (float)vk[1], v2 = (float)vk[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float s = fmaf(B[3 * i + 2], v2, fmaf(B[3 * i + 1], v1, B[3 * i] * v0));
        z[k * ndof + 3 * p + i] = s;
        if (zf) zf[(3 * p + i) * nr + k] = s;
    }
}

// interleave a set of FP64 vectors for the product: out[dof * nr + k] = in[k * ndof + dof]
// F64 product operand: out[dof * nr + k] = (hi, lo) float split of in[k * ndof + dof]
__global__ void k_interleave_split(const double* __restrict__ in, float2* __restrict__ out, int64_t ndof, int nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t r = q / nr, k = q % nr;
    const double v = in[k * ndof + r];
    const float h = (float)v;
    out[q] = make_float2(h, (float)(v - (double)h));
}

__global__ void k_to_f32_interleaved(const double* __restrict__ in, float* __restrict__ out, int64_t ndof, int nr) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t r = q / nr, k = q % nr;
    out[q] = (float)in[k * ndof + r];
}

// ---------------------------------------------------------------- Arnoldi (CGS2)

template <class Y>
__device__ __forceinline__ double yval(const Y* y, int64_t i) { return (double)y[i]; }

// pass 1: w = y - d .* z (stored), partial dots with V_0..V_j
template <class Y>
__global__ void __launch_bounds__(ROW_NT) k_arn_first(const Y* __restrict__ y, const double* __restrict__ d,
                                                      const double* __restrict__ blk,
                                                      const double* __restrict__ z, double* __restrict__ w,
                                                      const double* __restrict__ V, int64_t ndof, int nr, int j,
                                                      int64_t vstride, double* __restrict__ part,
                                                      const CycleState* __restrict__ cs) {
    __shared__ double sp[ROW_NT / 32][132];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS_PER_CTA;
    for (int k = 0; k < nr; ++k) {
        if (cs[k].done) continue;
        double wl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = r0 + threadIdx.x + u * ROW_NT;
            double v = 0.0;
            if (i < ndof) {
                v = yval(y, k * ndof + i) - d[i] * z[k * ndof + i];
                if (blk) v -= blk_row(blk, z + k * ndof, i);
                w[k * ndof + i] = v;
            }
            wl[u] = v;
        }
        for (int jj = 0; jj <= j; ++jj) {
            const double* Vj = V + ((int64_t)jj * nr + k) * vstride;
            double s = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = r0 + threadIdx.x + u * ROW_NT;
                if (i < ndof) s += Vj[i] * wl[u];
            }
            s = warp_sum_d(s);
            if (lane == 0) sp[wp][jj] = s;
        }
        __syncthreads();
        for (int jj = threadIdx.x; jj <= j; jj += ROW_NT) {
            double s = 0.0;
            for (int q = 0; q < ROW_NT / 32; ++q) s += sp[q][jj];
            part[((int64_t)blockIdx.x * nr + k) * 132 + jj] = s;
        }
        __syncthreads();
    }
}

// sum the per-CTA partials: out[k][jj] = sum_b part[b][k][jj]
// warp-wide sum of one value's partials: lanes over the row blocks, then a butterfly
// (fixed order: deterministic)
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part, int nblk, int nr, int k, int jj) {
    const int lane = threadIdx.x & 31;
    double a0 = 0.0, a1 = 0.0;
    int b = lane;
    for (; b + 32 < nblk; b += 64) {
        a0 += part[((int64_t)b * nr + k) * 132 + jj];
        a1 += part[((int64_t)(b + 32) * nr + k) * 132 + jj];
    }
    if (b < nblk) a0 += part[((int64_t)b * nr + k) * 132 + jj];
    return warp_sum_d(a0 + a1);
}

// h[k][jj] = sum over row blocks, one warp per value (launched with 512 threads per RHS)
__global__ void k_reduce_parts(const double* __restrict__ part, int nblk, int nr, int nvals, double* __restrict__ out,
                               const CycleState* __restrict__ cs) {
    const int k = blockIdx.x;
    if (cs[k].done) return;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int jj = w; jj < nvals; jj += nw) {
        const double v = warp_sum_parts(part, nblk, nr, k, jj);
        if ((threadIdx.x & 31) == 0) out[k * 132 + jj] = v;
    }
}

// w -= V h (h = previous dots); then either partial dots with V (second pass) or
// the partial squared norm of w (last pass)
__global__ void __launch_bounds__(ROW_NT) k_arn_update(double* __restrict__ w, const double* __restrict__ V,
                                                       const double* __restrict__ h, int64_t ndof, int nr, int j,
                                                       int64_t vstride, double* __restrict__ part, int want_dots,
                                                       const CycleState* __restrict__ cs) {
    __shared__ double sp[ROW_NT / 32][132];
    __shared__ double sh[132];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS_PER_CTA;
    for (int k = 0; k < nr; ++k) {
        if (cs[k].done) continue;
        for (int jj = threadIdx.x; jj <= j; jj += ROW_NT) sh[jj] = h[k * 132 + jj];
        __syncthreads();
        double wl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = r0 + threadIdx.x + u * ROW_NT;
            double v = 0.0;
            if (i < ndof) {
                v = w[k * ndof + i];
                for (int jj = 0; jj <= j; ++jj) v -= V[((int64_t)jj * nr + k) * vstride + i] * sh[jj];
                w[k * ndof + i] = v;
            }
            wl[u] = v;
        }
        if (want_dots) {
            for (int jj = 0; jj <= j; ++jj) {
                const double* Vj = V + ((int64_t)jj * nr + k) * vstride;
                double s = 0.0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t i = r0 + threadIdx.x + u * ROW_NT;
                    if (i < ndof) s += Vj[i] * wl[u];
                }
                s = warp_sum_d(s);
                if (lane == 0) sp[wp][jj] = s;
            }
        } else {
            double s = wl[0] * wl[0] + wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
            s = warp_sum_d(s);
            if (lane == 0) sp[wp][0] = s;
        }
        __syncthreads();
        const int nv = want_dots ? j + 1 : 1;
        for (int jj = threadIdx.x; jj < nv; jj += ROW_NT) {
            double s = 0.0;
            for (int q = 0; q < ROW_NT / 32; ++q) s += sp[q][jj];
            part[((int64_t)blockIdx.x * nr + k) * 132 + jj] = s;
        }
        __syncthreads();
    }
}

// Hessenberg column j, Givens rotation, residual estimate, convergence and breakdown
__device__ void givens_one(int k, const double* __restrict__ h1, const double* __restrict__ h2,
                           const double* __restrict__ part, int nblk, int nr, int j, int m, double* __restrict__ Hm,
                           double* __restrict__ cs_, double* __restrict__ sn_, double* __restrict__ g,
                           CycleState* __restrict__ st, double nrm2) {
    const double hn = sqrt(nrm2);
    double* col = Hm + ((int64_t)k * m + j) * (m + 1);
    double* c = cs_ + (int64_t)k * (m + 1);
    double* s = sn_ + (int64_t)k * (m + 1);
    double* gk = g + (int64_t)k * (m + 1);
    double hsum = 0.0;
    for (int i = 0; i <= j; ++i) {
        col[i] = h1[k * 132 + i] + h2[k * 132 + i];
        hsum += col[i] * col[i];
    }
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = c[i] * col[i] + s[i] * col[i + 1];
        col[i + 1] = -s[i] * col[i] + c[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    st[k].iters = j + 1;
    if (!(den > 0.0) || !isfinite(den)) {
        st[k].brk = 1;
        st[k].done = 1;
        st[k].iters = j;  // this column cannot be used
        return;
    }
    c[j] = col[j] / den;
    s[j] = col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    gk[j + 1] = -s[j] * gk[j];
    gk[j] = c[j] * gk[j];
    st[k].inv = hn > 0.0 ? 1.0 / hn : 0.0;
    // converged estimate, or the Krylov space became invariant (happy breakdown)
    if (fabs(gk[j + 1]) <= st[k].tol || hn <= 1e-14 * sqrt(hsum + nrm2)) st[k].done = 1;
    if (j + 1 >= m) st[k].done = 1;
}

// one thread per right-hand side; *alldone = every RHS stopped (the product kernels of
// the remaining steps of the cycle then return at once)
__global__ void k_givens(const double* __restrict__ h1, const double* __restrict__ h2, const double* __restrict__ part,
                         int nblk, int nr, int j, int m, double* __restrict__ Hm, double* __restrict__ cs_,
                         double* __restrict__ sn_, double* __restrict__ g, CycleState* __restrict__ st,
                         int* __restrict__ alldone) {
    __shared__ double nrm[32];
    // ||w||^2 of every RHS first, the whole warp on each sum
    for (int q = 0; q < nr; ++q) {
        const double v = warp_sum_parts(part, nblk, nr, q, 0);
        if (threadIdx.x == 0) nrm[q] = v;
    }
    __syncwarp();
    const int k = threadIdx.x;
    if (k < nr && !st[k].done) givens_one(k, h1, h2, part, nblk, nr, j, m, Hm, cs_, sn_, g, st, nrm[k]);
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < nr; ++q) all &= st[q].done;
        *alldone = all;
    }
}

__global__ void k_scale_next(const double* __restrict__ w, double* __restrict__ V, int64_t ndof, int nr, int j,
                             int64_t vstride, const CycleState* __restrict__ st) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, i = q % ndof;
    if (st[k].done && st[k].iters < j + 1) return;  // stopped before this step
    V[((int64_t)(j + 1) * nr + k) * vstride + i] = w[q] * st[k].inv;
}

// start of a cycle: v0 = r / beta, g = beta e1
__global__ void k_cycle_start(const double* __restrict__ r, double* __restrict__ V, int64_t ndof, int nr,
                              int64_t vstride, const double* __restrict__ beta, int m, double* __restrict__ g) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)nr * (m + 1)) g[q] = (q % (m + 1) == 0) ? beta[q / (m + 1)] : 0.0;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, i = q % ndof;
    const double b = beta[k];
    V[k * vstride + i] = b > 0.0 ? r[q] / b : 0.0;
}

// y = H^-1 g (upper triangular, iters x iters), x += Z y
__global__ void k_lsq(const double* __restrict__ Hm, const double* __restrict__ g, double* __restrict__ y, int nr,
                      int m, const CycleState* __restrict__ st, const int* __restrict__ active) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    const int n = active[k] ? st[k].iters : 0;
    double* yk = y + (int64_t)k * (m + 1);
    for (int i = n - 1; i >= 0; --i) {
        double s = g[(int64_t)k * (m + 1) + i];
        for (int l = i + 1; l < n; ++l) s -= Hm[((int64_t)k * m + l) * (m + 1) + i] * yk[l];
        const double dgl = Hm[((int64_t)k * m + i) * (m + 1) + i];
        yk[i] = dgl != 0.0 ? s / dgl : 0.0;
    }
    for (int i = n; i <= m; ++i) yk[i] = 0.0;
}

__global__ void k_update_x(double* __restrict__ x, const double* __restrict__ Z, const double* __restrict__ y,
                           int64_t ndof, int nr, int m, int64_t vstride, const CycleState* __restrict__ st,
                           const int* __restrict__ active) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, i = q % ndof;
    if (!active[k]) return;
    const int n = st[k].iters;
    double s = x[q];
    for (int l = 0; l < n; ++l) s += Z[((int64_t)l * nr + k) * vstride + i] * y[k * (m + 1) + l];
    x[q] = s;
}

// r = b - (y - d .* x), partial ||r||^2
template <class Y>
__global__ void __launch_bounds__(ROW_NT) k_residual(const double* __restrict__ b, const Y* __restrict__ y,
                                                     const double* __restrict__ d, const double* __restrict__ blk,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ r, int64_t ndof, int nr,
                                                     double* __restrict__ part) {
    __shared__ double sp[ROW_NT / 32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS_PER_CTA;
    for (int k = 0; k < nr; ++k) {
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = r0 + threadIdx.x + u * ROW_NT;
            if (i < ndof) {
                const int64_t q = k * ndof + i;
                double v = b[q] - (yval(y, q) - d[i] * x[q]);
                if (blk) v += blk_row(blk, x + k * ndof, i);
                r[q] = v;
                s += v * v;
            }
        }
        s = warp_sum_d(s);
        if (lane == 0) sp[wp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < ROW_NT / 32; ++q) t += sp[q];
            part[(int64_t)blockIdx.x * nr + k] = t;
        }
        __syncthreads();
    }
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) x[q] += d[q];
}

}  // namespace


// ---------------------------------------------------------------- BiCGSTAB
// Right-preconditioned BiCGSTAB (van der Vorst, 1992), the Krylov method the paper uses
// for its A11 solves (Sec. 3.3.1), per RHS on the device: scalars per RHS in BcgScal,
// dot products reduced over row blocks in a fixed order.
struct BcgScal {
    double rho, alpha, omega, beta;
    int iters, maxit, pad0, pad1;
};

// partial sums of NQ dot products (a_q, b_q) per RHS over one row block
template <int NQ>
__global__ void __launch_bounds__(ROW_NT) k_bcg_dots(const double* __restrict__ a0, const double* __restrict__ b0,
                                                     const double* __restrict__ a1, const double* __restrict__ b1,
                                                     int64_t ndof, int nr, double* __restrict__ part,
                                                     const CycleState* __restrict__ cs) {
    __shared__ double sp[ROW_NT / 32][2];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS_PER_CTA;
    for (int k = 0; k < nr; ++k) {
        if (cs[k].done) continue;  // uniform over the block
        double acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = r0 + threadIdx.x + u * ROW_NT;
            if (i < ndof) {
                const int64_t o = k * ndof + i;
                acc[0] += a0[o] * b0[o];
                if (NQ > 1) acc[NQ - 1] += a1[o] * b1[o];
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double t = warp_sum_d(acc[q]);
            if (lane == 0) sp[wp][q] = t;
        }
        __syncthreads();
        if (threadIdx.x < NQ) {
            double t = 0.0;
            for (int w = 0; w < ROW_NT / 32; ++w) t += sp[w][threadIdx.x];
            part[((int64_t)blockIdx.x * nr + k) * 2 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// the stage's scalars from the reduced dots: warp k sums RHS k's partials (fixed order)
// stage 0: rho_new = (rh, r) -> beta, rho;  1: alpha = rho / (rh, v);
// stage 2: omega = (t, s) / (t, t);  3: ||r||^2 -> convergence, iteration count
__global__ void k_bcg_stage(int stage, const double* __restrict__ part, int nblk, int nr, BcgScal* __restrict__ sc,
                            CycleState* __restrict__ cs, int* __restrict__ alldone) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < nr && !cs[k].done) {
        double d0 = 0.0, d1 = 0.0;
        for (int b = lane; b < nblk; b += 32) {
            d0 += part[((int64_t)b * nr + k) * 2];
            d1 += part[((int64_t)b * nr + k) * 2 + 1];
        }
        d0 = warp_sum_d(d0);
        d1 = warp_sum_d(d1);
        if (lane == 0) {
            BcgScal& S = sc[k];
            CycleState& C = cs[k];
            if (stage == 0) {
                if (!(d0 != 0.0) || !isfinite(d0)) {
                    C.brk = 1;
                    C.done = 1;
                } else {
                    S.beta = S.iters == 0 ? 0.0 : (d0 / S.rho) * (S.alpha / S.omega);
                    S.rho = d0;
                }
            } else if (stage == 1) {
                if (!(d0 != 0.0) || !isfinite(d0)) {
                    C.brk = 1;
                    C.done = 1;
                } else {
                    S.alpha = S.rho / d0;
                }
            } else if (stage == 2) {
                S.omega = d1 > 0.0 ? d0 / d1 : 0.0;
            } else {
                ++S.iters;
                ++C.iters;
                if (sqrt(d0) <= C.tol) {
                    C.done = 1;
                } else if (!(S.omega != 0.0) || !isfinite(d0)) {
                    C.brk = 1;
                    C.done = 1;
                } else if (S.iters >= S.maxit) {
                    C.done = 1;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && stage == 3) {
        int all = 1;
        for (int q = 0; q < nr; ++q) all &= cs[q].done;
        *alldone = all;
    }
}

// p = r + beta (p - omega v)
__global__ void k_bcg_p(double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ v,
                        int64_t ndof, int nr, const BcgScal* __restrict__ sc, const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int k = (int)(q / ndof);
    if (cs[k].done) return;
    p[q] = r[q] + sc[k].beta * (p[q] - sc[k].omega * v[q]);
}

// s = r - alpha v
__global__ void k_bcg_s(double* __restrict__ s, const double* __restrict__ r, const double* __restrict__ v,
                        int64_t ndof, int nr, const BcgScal* __restrict__ sc, const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int k = (int)(q / ndof);
    if (cs[k].done) return;
    s[q] = r[q] - sc[k].alpha * v[q];
}

// x += alpha ph + omega sh;  r = s - omega t
__global__ void k_bcg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ ph,
                         const double* __restrict__ sh, const double* __restrict__ s, const double* __restrict__ t,
                         int64_t ndof, int nr, const BcgScal* __restrict__ sc, const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int k = (int)(q / ndof);
    if (cs[k].done) return;
    x[q] += sc[k].alpha * ph[q] + sc[k].omega * sh[q];
    r[q] = s[q] - sc[k].omega * t[q];
}

// out = y - d .* z - blk z  (the tangent applied to z, y = E z)
template <class Y>
__global__ void k_tangent(const Y* __restrict__ y, const double* __restrict__ d, const double* __restrict__ blk,
                          const double* __restrict__ z, double* __restrict__ out, int64_t ndof, int nr,
                          const CycleState* __restrict__ cs) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= ndof * nr) return;
    const int64_t k = q / ndof, i = q % ndof;
    if (cs[k].done) return;
    double v = yval(y, q) - d[i] * z[q];
    if (blk) v -= blk_row(blk, z + k * ndof, i);
    out[q] = v;
}

// ---------------------------------------------------------------- workspace

struct SolveWS {
    int nr = 0, m = 0;
    int64_t ndof = 0, vstride = 0;
    DevBuf<double> V, Z, w, r, xc, bc, dc, corr, y64, zi, Hm, cs, sn, g, ylsq, part, h1, h2;
    DevBuf<float> zf, y32, binv, bjscratch, dsc, j3;
    bool dsc_on = false;  // apply the learned per-leaf scalings after block-Jacobi
    DevBuf<double> blkbuf;  // off-diagonal C^ep blocks, cluster element order
    DevBuf<double> bcg;     // BiCGSTAB vectors: rh, p, v, ph, s, sh, t (nr x 3N each)
    // what the preconditioner in the workspace was built for (hm_solve_opts.reuse_precond)
    struct PcKey {
        bool valid = false;
        const double* kel = nullptr;
        const double* cep = nullptr;
        double shift = 0.0, ilu_p = 0.0;
        int precond = -1;
        const void* lp = nullptr;
        bool same(const PcKey& o) const {
            return valid && o.kel == kel && o.cep == cep && o.shift == shift && o.ilu_p == ilu_p &&
                   o.precond == precond && o.lp == lp;
        }
    } pc_key;
    DevBuf<BcgScal> bsc;
    // the learned near correction (HM_LP_NEAR): scratch N z and B^-1 N z, the leaf of
    // every cluster element, and gamma
    bool near_on = false;
    double near_gamma = 1.0;
    DevBuf<double> nt, nu;
    DevBuf<float> nv32;  // FP32 RHS-interleaved copy of B^-1 v, the operand of N
    DevBuf<NearItem> near_items;  // the work items of N v (near_plan)
    DevBuf<int32_t> near_msum;
    DevBuf<float> near_part;
    int64_t near_part_rows = -1;  // -1: no plan yet
    DevBuf<int32_t> leaf_of;
    const double* blk = nullptr;  // blkbuf.p when the tangent has a block-diagonal C^ep
    DevBuf<int64_t> binv_off, self_off;
    DevBuf<CycleState> st;
    DevBuf<int> active, err, alldone;
    int* h_flags = nullptr;  // pinned: all-done flag after the last two steps
    cudaEvent_t fev[2] = {nullptr, nullptr};
    ~SolveWS() {
        if (h_flags) cudaFreeHost(h_flags);
        for (cudaEvent_t e : fev)
            if (e) cudaEventDestroy(e);
    }
    int64_t binv_len = 0;
    bool bj_needs_global = false;
};

void solve_ws_free(SolveWS* w) { delete w; }

namespace {

int nblk_rows(int64_t ndof) { return (int)ceil_div(ndof, ROWS_PER_CTA); }

SolveWS& workspace(HMat& H, int nr, int m, cudaStream_t st) {
    if (!H.solve_ws) H.solve_ws = new SolveWS();
    SolveWS& W = *H.solve_ws;
    if (W.nr >= nr && W.m >= m && W.ndof == H.ndof) return W;
    W.pc_key.valid = false;  // the buffers below are reallocated
    W.nr = std::max(W.nr, nr);
    W.m = std::max(W.m, m);
    W.ndof = H.ndof;
    W.vstride = H.ndof;
    const int64_t vn = (int64_t)W.nr * H.ndof;
    W.V.alloc((size_t)(W.m + 1) * vn + VSLACK);
    W.Z.alloc((size_t)W.m * vn + VSLACK);
    W.w.alloc(vn + VSLACK);
    W.r.alloc(vn + VSLACK);
    W.xc.alloc(vn + VSLACK);
    W.bc.alloc(vn + VSLACK);
    W.corr.alloc(vn + VSLACK);
    W.y64.alloc(vn + VSLACK);
    W.zi.alloc(vn + VSLACK);
    W.dc.alloc(H.ndof + VSLACK);
    W.zf.alloc(vn + VSLACK);
    W.y32.alloc(vn + VSLACK);
    HM_CUDA(cudaMemsetAsync(W.zf.p, 0, W.zf.bytes(), st));
    HM_CUDA(cudaMemsetAsync(W.zi.p, 0, W.zi.bytes(), st));
    HM_CUDA(cudaMemsetAsync(W.V.p, 0, W.V.bytes(), st));
    HM_CUDA(cudaMemsetAsync(W.Z.p, 0, W.Z.bytes(), st));
    W.Hm.alloc((size_t)W.nr * W.m * (W.m + 1));
    W.cs.alloc((size_t)W.nr * (W.m + 1));
    W.sn.alloc((size_t)W.nr * (W.m + 1));
    W.g.alloc((size_t)W.nr * (W.m + 1));
    W.ylsq.alloc((size_t)W.nr * (W.m + 1));
    const int nb = nblk_rows(H.ndof);
    W.part.alloc((size_t)nb * W.nr * 132);
    W.h1.alloc((size_t)W.nr * 132);
    W.h2.alloc((size_t)W.nr * 132);
    W.st.alloc(W.nr);
    W.active.alloc(W.nr);
    W.err.alloc(1);
    W.alldone.alloc(1);
    if (!W.h_flags) {
        HM_CUDA(cudaHostAlloc((void**)&W.h_flags, 2 * sizeof(int), cudaHostAllocDefault));
        W.h_flags[0] = W.h_flags[1] = 0;
        for (cudaEvent_t& e : W.fev) HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // block-Jacobi layout: one ld x n block per leaf
    std::vector<int64_t> off(H.n_leaves);
    int64_t len = 0;
    bool glob = false;
    for (int l = 0; l < H.n_leaves; ++l) {
        off[l] = len;
        len += (int64_t)H.h_leaves[l].ld * 3 * H.h_leaves[l].n;
        if (3 * H.h_leaves[l].n > BJ_MAX_ROWS_SMEM) glob = true;
    }
    W.binv_len = len;
    W.binv.alloc(std::max<int64_t>(len, 1));
    W.j3.alloc((size_t)9 * H.N);
    W.binv_off.upload(off, st);
    W.self_off.upload(H.h_self_off, st);
    W.bj_needs_global = glob;
    if (glob) W.bjscratch.alloc(std::max<int64_t>(len, 1));
    return W;
}

unsigned g1(int64_t n) { return (unsigned)ceil_div(std::max<int64_t>(n, 1), 256); }

// y = A_op z for the Arnoldi step / residual: the product part (E z); the diagonal is
// applied by the consumer kernel.  dtype F64: compensated, input z (FP64); F32: input zf.
void apply_E(HMat& H, SolveWS& W, const double* z64, const float* z32, void* y, int nr, int dtype, int fac,
             cudaStream_t st, const int* skip = nullptr) {
    if (dtype == HM_F64) {
        k_interleave_split<<<g1(H.ndof * nr), 256, 0, st>>>(z64, (float2*)W.zi.p, H.ndof, nr);
        product_core(H, W.zi.p, y, nr, HM_F64, fac, st, skip);
    } else {
        product_core(H, z32, y, nr, HM_F32, fac, st, skip);
    }
}

struct CycleResult {
    std::vector<int> iters;
    std::vector<int> brk;
};

// One restart cycle of FGMRES on (E - diag d): rhs r (cluster order), solution x updated
// in place; beta[k] = ||r_k||; tol_abs[k] the target on the residual estimate.
// preconditioner applied in the Krylov loop
enum PcKind { PC_NONE = 0, PC_LEAF = 1, PC_POINT = 2, PC_ILU = 3 };

NearDev near_dev(SolveWS& W) {
    return NearDev{W.near_items.p, (int)W.near_items.n, W.near_msum.p, (int)(W.near_msum.n / 3), W.near_part.p};
}

// z = M^-1 v (cluster order, RHS-major), and its FP32 RHS-interleaved copy zf when the
// next product is an FP32 one; RHS whose CycleState is done are skipped
void precond_apply(HMat& H, SolveWS& W, PcKind pc, const double* v, double* z, float* zf, int nr, cudaStream_t st) {
    const int64_t n = H.ndof;
    if (pc == PC_LEAF && W.near_on) {
        // z = y - gamma d o B^-1 N y, y = B^-1 v
        k_bj_apply<<<H.n_leaves, 256, 0, st>>>(H.leaves.p, W.binv.p, W.binv_off.p, v, z, W.nv32.p, n, nr, W.st.p, 0,
                                               nullptr);
        near_offdiag_launch(H, near_dev(W), W.nv32.p, W.nt.p, nr, W.st.p, st);
        k_bj_apply<<<H.n_leaves, 256, 0, st>>>(H.leaves.p, W.binv.p, W.binv_off.p, W.nt.p, W.nu.p, nullptr, n, nr,
                                               W.st.p, 0, nullptr);
        k_near_update<<<g1(n * nr), 256, 0, st>>>(z, W.nu.p, W.dsc.p, W.leaf_of.p, W.near_gamma, zf, n, nr, W.st.p);
        HM_LAUNCH_CHECK();
        return;
    }
    if (pc == PC_POINT)
        k_j3_apply<<<g1(H.N * nr), 256, 0, st>>>(W.j3.p, v, z, zf, H.N, n, nr, W.st.p);
    else if (pc == PC_ILU)
        ilu_apply(H, v, z, zf, nr, &W.st.p->done, (int)(sizeof(CycleState) / sizeof(int)), st);
    else
        k_bj_apply<<<H.n_leaves, 256, 0, st>>>(H.leaves.p, W.binv.p, W.binv_off.p, v, z, zf, n, nr, W.st.p,
                                               pc == PC_LEAF ? 0 : 1, W.dsc_on ? W.dsc.p : nullptr);
    HM_LAUNCH_CHECK();
}

CycleResult fgmres_cycle(HMat& H, SolveWS& W, const double* beta_h, const double* tol_abs, const int* active_h,
                         int nr, int m, int dtype, int fac, PcKind pc, cudaStream_t st) {
    NvtxScope nvtx_("fgmres_cycle");
    const int64_t n = H.ndof;
    const int nb = nblk_rows(n);
    std::vector<CycleState> cs(nr);
    for (int k = 0; k < nr; ++k) {
        cs[k].done = active_h[k] ? 0 : 1;
        cs[k].iters = 0;
        cs[k].brk = 0;
        cs[k].pad_ = 0;
        cs[k].tol = tol_abs[k];
        cs[k].inv = 0.0;
    }
    HM_CUDA(cudaMemcpyAsync(W.st.p, cs.data(), nr * sizeof(CycleState), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(W.active.p, active_h, nr * sizeof(int), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(W.h1.p, beta_h, nr * sizeof(double), cudaMemcpyHostToDevice, st));
    k_cycle_start<<<g1(std::max<int64_t>(n * nr, (int64_t)nr * (m + 1))), 256, 0, st>>>(W.r.p, W.V.p, n, nr,
                                                                                      W.vstride, W.h1.p, m, W.g.p);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaMemsetAsync(W.alldone.p, 0, sizeof(int), st));
    for (int j = 0; j < m; ++j) {
        // the host runs at most two steps ahead of the device and stops issuing steps once
        // the flag copied after step j-2 says that every right-hand side has stopped
        if (j >= 2) {
            HM_CUDA(cudaEventSynchronize(W.fev[j % 2]));
            if (W.h_flags[j % 2]) break;
        }
        const double* vj = W.V.p + (int64_t)j * nr * W.vstride;
        double* zj = W.Z.p + (int64_t)j * nr * W.vstride;
        precond_apply(H, W, pc, vj, zj, dtype == HM_F32 ? W.zf.p : nullptr, nr, st);
        if (dtype == HM_F64) {
            apply_E(H, W, zj, nullptr, W.y64.p, nr, HM_F64, fac, st, W.alldone.p);
            k_arn_first<double><<<nb, ROW_NT, 0, st>>>(W.y64.p, W.dc.p, W.blk, zj, W.w.p, W.V.p, n, nr, j, W.vstride,
                                                       W.part.p, W.st.p);
        } else {
            apply_E(H, W, nullptr, W.zf.p, W.y32.p, nr, HM_F32, fac, st, W.alldone.p);
            k_arn_first<float><<<nb, ROW_NT, 0, st>>>(W.y32.p, W.dc.p, W.blk, zj, W.w.p, W.V.p, n, nr, j, W.vstride,
                                                      W.part.p, W.st.p);
        }
        HM_LAUNCH_CHECK();
        k_reduce_parts<<<nr, 512, 0, st>>>(W.part.p, nb, nr, j + 1, W.h1.p, W.st.p);
        k_arn_update<<<nb, ROW_NT, 0, st>>>(W.w.p, W.V.p, W.h1.p, n, nr, j, W.vstride, W.part.p, 1, W.st.p);
        k_reduce_parts<<<nr, 512, 0, st>>>(W.part.p, nb, nr, j + 1, W.h2.p, W.st.p);
        k_arn_update<<<nb, ROW_NT, 0, st>>>(W.w.p, W.V.p, W.h2.p, n, nr, j, W.vstride, W.part.p, 0, W.st.p);
        k_givens<<<1, 32, 0, st>>>(W.h1.p, W.h2.p, W.part.p, nb, nr, j, m, W.Hm.p, W.cs.p, W.sn.p, W.g.p, W.st.p,
                                   W.alldone.p);
        k_scale_next<<<g1(n * nr), 256, 0, st>>>(W.w.p, W.V.p, n, nr, j, W.vstride, W.st.p);
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaMemcpyAsync(W.h_flags + (j % 2), W.alldone.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaEventRecord(W.fev[j % 2], st));
    }
    k_lsq<<<1, 32, 0, st>>>(W.Hm.p, W.g.p, W.ylsq.p, nr, m, W.st.p, W.active.p);
    k_update_x<<<g1(n * nr), 256, 0, st>>>(W.xc.p, W.Z.p, W.ylsq.p, n, nr, m, W.vstride, W.st.p, W.active.p);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaMemcpyAsync(cs.data(), W.st.p, nr * sizeof(CycleState), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    CycleResult res;
    for (int k = 0; k < nr; ++k) {
        res.iters.push_back(active_h[k] ? cs[k].iters : 0);
        res.brk.push_back(cs[k].brk);
    }
    return res;
}

// r = rhs - (E - diag d) x with the given product; returns ||r_k|| on the host
std::vector<double> residual(HMat& H, SolveWS& W, const double* rhs, int nr, int dtype, int fac, cudaStream_t st,
                             bool x_zero = false) {
    const int64_t n = H.ndof;
    const int nb = nblk_rows(n);
    if (x_zero) {
        // x = 0 (the caller cleared W.xc): r = rhs without a product; the FP32 copy of x
        // is cleared as the product path would have left it
        HM_CUDA(cudaMemsetAsync(W.y64.p, 0, (size_t)n * nr * sizeof(double), st));
        if (dtype != HM_F64) HM_CUDA(cudaMemsetAsync(W.zf.p, 0, (size_t)n * nr * sizeof(float), st));
        k_residual<double><<<nb, ROW_NT, 0, st>>>(rhs, W.y64.p, W.dc.p, W.blk, W.xc.p, W.r.p, n, nr, W.part.p);
    } else if (dtype == HM_F64) {
        apply_E(H, W, W.xc.p, nullptr, W.y64.p, nr, HM_F64, fac, st);
        k_residual<double><<<nb, ROW_NT, 0, st>>>(rhs, W.y64.p, W.dc.p, W.blk, W.xc.p, W.r.p, n, nr, W.part.p);
    } else {
        // FP32 copy of x, interleaved, for the FP32 product
        k_to_f32_interleaved<<<g1(n * nr), 256, 0, st>>>(W.xc.p, W.zf.p, n, nr);
        apply_E(H, W, nullptr, W.zf.p, W.y32.p, nr, HM_F32, fac, st);
        k_residual<float><<<nb, ROW_NT, 0, st>>>(rhs, W.y32.p, W.dc.p, W.blk, W.xc.p, W.r.p, n, nr, W.part.p);
    }
    HM_LAUNCH_CHECK();
    std::vector<double> part((size_t)nb * nr);
    HM_CUDA(cudaMemcpyAsync(part.data(), W.part.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    std::vector<double> out(nr, 0.0);
    for (int k = 0; k < nr; ++k) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(size_t)b * nr + k];
        out[k] = std::sqrt(s);
    }
    return out;
}

// FGMRES(m) with restarts on rhs (cluster order) into W.xc (initial value kept; x_zero:
// the caller cleared it, and the first residual is rhs itself); stops at
// ||rhs - A x_k|| <= tol_abs[k] or when the iteration budget is spent.
// Returns per RHS the iterations used and the final residual norm.
void fgmres(HMat& H, SolveWS& W, const double* rhs, const std::vector<double>& tol_abs, int nr, int m, int max_its,
            int max_cycles, int dtype, int fac, PcKind pc, std::vector<int>& its, std::vector<double>& rn,
            std::vector<int>& brk, cudaStream_t st, bool x_zero) {
    its.assign(nr, 0);
    brk.assign(nr, 0);
    rn = residual(H, W, rhs, nr, dtype, fac, st, x_zero);
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        std::vector<int> active(nr, 0);
        bool any = false;
        for (int k = 0; k < nr; ++k) {
            active[k] = (rn[k] > tol_abs[k] && its[k] < max_its && !brk[k]) ? 1 : 0;
            any = any || active[k];
        }
        if (!any) break;
        int mm = m;
        for (int k = 0; k < nr; ++k)
            if (active[k]) mm = std::min(mm, std::max(1, max_its - its[k]));
        CycleResult cr = fgmres_cycle(H, W, rn.data(), tol_abs.data(), active.data(), nr, mm, dtype, fac, pc, st);
        for (int k = 0; k < nr; ++k) {
            its[k] += cr.iters[k];
            if (cr.brk[k] && cr.iters[k] == 0) brk[k] = 1;
        }
        rn = residual(H, W, rhs, nr, dtype, fac, st);
    }
}


// BiCGSTAB with restarts on rhs (cluster order) into W.xc (initial value kept): the
// recurrence's residual decides convergence, the true residual (recomputed after each
// run) decides a restart; same contract as fgmres.
void bicgstab(HMat& H, SolveWS& W, const double* rhs, const std::vector<double>& tol_abs, int nr, int max_its,
              int max_runs, int dtype, int fac, PcKind pc, std::vector<int>& its, std::vector<double>& rn,
              std::vector<int>& brk, cudaStream_t st, bool x_zero) {
    NvtxScope nvtx_("bicgstab");
    const int64_t n = H.ndof, vn = n * nr;
    const int nb = nblk_rows(n);
    if (W.bcg.n < (size_t)(7 * vn + VSLACK)) W.bcg.alloc((size_t)(7 * vn + VSLACK));
    if (W.bsc.n < (size_t)nr) W.bsc.alloc(nr);
    double* rh = W.bcg.p;
    double* p = rh + vn;
    double* v = p + vn;
    double* ph = v + vn;
    double* sv = ph + vn;
    double* sh = sv + vn;
    double* t = sh + vn;
    double* r = W.r.p;
    float* zf = dtype == HM_F32 ? W.zf.p : nullptr;
    void* y = dtype == HM_F64 ? (void*)W.y64.p : (void*)W.y32.p;
    its.assign(nr, 0);
    brk.assign(nr, 0);
    rn = residual(H, W, rhs, nr, dtype, fac, st, x_zero);  // W.r = rhs - A x
    auto tangent = [&](const double* z, double* out) {
        apply_E(H, W, z, zf, y, nr, dtype, fac, st, W.alldone.p);
        if (dtype == HM_F64)
            k_tangent<double><<<g1(vn), 256, 0, st>>>(W.y64.p, W.dc.p, W.blk, z, out, n, nr, W.st.p);
        else
            k_tangent<float><<<g1(vn), 256, 0, st>>>(W.y32.p, W.dc.p, W.blk, z, out, n, nr, W.st.p);
        HM_LAUNCH_CHECK();
    };
    auto stage = [&](int which, const double* a0, const double* b0, const double* a1, const double* b1) {
        if (a1)
            k_bcg_dots<2><<<nb, ROW_NT, 0, st>>>(a0, b0, a1, b1, n, nr, W.part.p, W.st.p);
        else
            k_bcg_dots<1><<<nb, ROW_NT, 0, st>>>(a0, b0, nullptr, nullptr, n, nr, W.part.p, W.st.p);
        k_bcg_stage<<<1, 32 * nr, 0, st>>>(which, W.part.p, nb, nr, W.bsc.p, W.st.p, W.alldone.p);
        HM_LAUNCH_CHECK();
    };
    for (int run = 0; run < max_runs; ++run) {
        std::vector<CycleState> cs(nr);
        std::vector<BcgScal> sc(nr);
        bool any = false;
        for (int k = 0; k < nr; ++k) {
            const bool act = rn[k] > tol_abs[k] && its[k] < max_its && !brk[k];
            any = any || act;
            cs[k] = CycleState{act ? 0 : 1, 0, 0, 0, tol_abs[k], 0.0};
            sc[k] = BcgScal{1.0, 1.0, 1.0, 0.0, 0, std::max(1, max_its - its[k]), 0, 0};
        }
        if (!any) break;
        HM_CUDA(cudaMemcpyAsync(W.st.p, cs.data(), nr * sizeof(CycleState), cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(W.bsc.p, sc.data(), nr * sizeof(BcgScal), cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(rh, r, vn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        HM_CUDA(cudaMemsetAsync(p, 0, vn * sizeof(double), st));
        HM_CUDA(cudaMemsetAsync(v, 0, vn * sizeof(double), st));
        HM_CUDA(cudaMemsetAsync(W.alldone.p, 0, sizeof(int), st));
        for (int j = 0; j < max_its; ++j) {
            // the host stays at most two iterations ahead and stops once every RHS has
            if (j >= 2) {
                HM_CUDA(cudaEventSynchronize(W.fev[j % 2]));
                if (W.h_flags[j % 2]) break;
            }
            stage(0, rh, r, nullptr, nullptr);                         // rho, beta
            k_bcg_p<<<g1(vn), 256, 0, st>>>(p, r, v, n, nr, W.bsc.p, W.st.p);
            HM_LAUNCH_CHECK();
            precond_apply(H, W, pc, p, ph, zf, nr, st);
            tangent(ph, v);
            stage(1, rh, v, nullptr, nullptr);                         // alpha
            k_bcg_s<<<g1(vn), 256, 0, st>>>(sv, r, v, n, nr, W.bsc.p, W.st.p);
            HM_LAUNCH_CHECK();
            precond_apply(H, W, pc, sv, sh, zf, nr, st);
            tangent(sh, t);
            stage(2, t, sv, t, t);                                      // omega
            k_bcg_xr<<<g1(vn), 256, 0, st>>>(W.xc.p, r, ph, sh, sv, t, n, nr, W.bsc.p, W.st.p);
            HM_LAUNCH_CHECK();
            stage(3, r, r, nullptr, nullptr);                          // ||r||, done
            HM_CUDA(cudaMemcpyAsync(W.h_flags + (j % 2), W.alldone.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaEventRecord(W.fev[j % 2], st));
        }
        HM_CUDA(cudaMemcpyAsync(cs.data(), W.st.p, nr * sizeof(CycleState), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < nr; ++k) {
            its[k] += cs[k].iters;
            if (cs[k].brk) brk[k] = 1;
        }
        rn = residual(H, W, rhs, nr, dtype, fac, st);
        for (int k = 0; k < nr; ++k)
            if (brk[k] && rn[k] > tol_abs[k] && cs[k].iters > 0) brk[k] = 0;  // a restart may still get on
    }
}

// block-Jacobi inverses of the leaf blocks of E - diag(W.dc)
void bj_build(HMat& H, SolveWS& W, cudaStream_t st) {
    HM_CUDA(cudaMemsetAsync(W.err.p, 0, sizeof(int), st));
    int max_rows = 0;
    for (const LeafDesc& L : H.h_leaves) max_rows = std::max(max_rows, 3 * L.n);
    if (max_rows <= BJR_ROWS) {
        const size_t smem = sizeof(float) * (size_t)max_rows * max_rows;
        // the register tile of the largest leaf: 16 AR rows, 32 BC columns
        if (max_rows <= 32)
            bj_build_reg_launch<2, 1>(H, W, smem, st);
        else if (max_rows <= 64)
            bj_build_reg_launch<4, 2>(H, W, smem, st);
        else if (max_rows <= 96)
            bj_build_reg_launch<6, 3>(H, W, smem, st);
        else if (max_rows <= 128)
            bj_build_reg_launch<8, 4>(H, W, smem, st);
        else if (max_rows <= 160)
            bj_build_reg_launch<10, 5>(H, W, smem, st);
        else
            bj_build_reg_launch<12, 6>(H, W, smem, st);
        HM_LAUNCH_CHECK();
        int e = 0;
        HM_CUDA(cudaMemcpyAsync(&e, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (e) fail(HM_EBREAKDOWN, "a diagonal leaf block of A is singular");
        return;
    }
    const size_t smem = W.bj_needs_global ? 0 : sizeof(float) * BJ_MAX_ROWS_SMEM * BJ_MAX_ROWS_SMEM;
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(k_bj_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bj_build<<<H.n_leaves, 512, smem, st>>>(H.leaves.p, W.self_off.p, H.near.p, W.dc.p, W.blk, W.binv.p,
                                              W.binv_off.p, W.bjscratch.p, W.bj_needs_global ? 0 : 1, W.err.p);
    HM_LAUNCH_CHECK();
    int e = 0;
    HM_CUDA(cudaMemcpyAsync(&e, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (e) fail(HM_EBREAKDOWN, "a diagonal leaf block of A is singular");
}

// device data of the near correction: the operand index of every near column, the leaf of
// every cluster element and N z / B^-1 N z scratch for nr RHS
void near_prepare(HMat& H, SolveWS& W, int nr, cudaStream_t st) {
    if (H.near_zidx.n != H.h_near_zidx.size()) H.near_zidx.upload(H.h_near_zidx, st);
    if (W.leaf_of.n != (size_t)H.N) {
        std::vector<int32_t> lo(H.N);
        for (int l = 0; l < H.n_leaves; ++l)
            for (int e = 0; e < H.h_leaves[l].n; ++e) lo[H.h_leaves[l].begin + e] = l;
        W.leaf_of.upload(lo, st);
    }
    if (W.near_part_rows < 0) {
        const NearPlan P = near_plan(H);
        W.near_items.upload(P.items, st);
        if (!P.msum.empty()) W.near_msum.upload(P.msum, st);
        W.near_part_rows = P.part_rows;
    }
    if (W.near_part.n < (size_t)W.near_part_rows * nr + 1) W.near_part.alloc((size_t)W.near_part_rows * nr + 1);
    const size_t len = (size_t)H.ndof * nr + VSLACK;
    if (W.nt.n < len) W.nt.alloc(len);
    if (W.nu.n < len) W.nu.alloc(len);
    if (W.nv32.n < len) W.nv32.alloc(len);
}

// the interface term of the tangent: diag(k) + C^ep + shift I into W.dc (and the
// off-diagonal C^ep entries into W.blk when cep is given)
void set_tangent(HMat& H, SolveWS& W, const double* kel, const double* cep, double shift, cudaStream_t st) {
    if (cep) {
        if (W.blkbuf.n < (size_t)9 * H.N) W.blkbuf.alloc((size_t)9 * H.N);
        k_blockdiag<<<g1(H.N), 256, 0, st>>>(kel, cep, shift, H.perm.p, H.N, W.dc.p, W.blkbuf.p);
        W.blk = W.blkbuf.p;
    } else {
        k_diag<<<g1(H.ndof), 256, 0, st>>>(kel, shift, H.perm.p, H.ndof, W.dc.p);
        W.blk = nullptr;
    }
    HM_LAUNCH_CHECK();
}

// point-Jacobi inverses of the 3x3 diagonal blocks of E - diag(W.dc) - W.blk
void j3_build(HMat& H, SolveWS& W, cudaStream_t st) {
    HM_CUDA(cudaMemsetAsync(W.err.p, 0, sizeof(int), st));
    k_j3_build<<<H.n_leaves, 64, 0, st>>>(H.leaves.p, W.self_off.p, H.near.p, W.dc.p, W.blk, W.j3.p, W.err.p);
    HM_LAUNCH_CHECK();
    int e = 0;
    HM_CUDA(cudaMemcpyAsync(&e, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (e) fail(HM_EBREAKDOWN, "a 3x3 diagonal block of A is singular");
}

}  // namespace

void to_cluster(HMat& H, const double* user, double* cluster, int nr, cudaStream_t st) {
    k_to_cluster<<<g1(H.ndof * nr), 256, 0, st>>>(user, cluster, H.perm.p, H.ndof, nr);
    HM_LAUNCH_CHECK();
}

void bj_solve_cluster(HMat& H, const double* kel, double shift, const double* v, double* z, int nr,
                      cudaStream_t st) {
    if (nr < 1 || nr > 16) fail(HM_EINVAL, "block-Jacobi solve: 1 to 16 right-hand sides");
    SolveWS& W = workspace(H, nr, 1, st);
    W.pc_key.valid = false;
    set_tangent(H, W, kel, nullptr, shift, st);
    bj_build(H, W, st);
    std::vector<CycleState> cs(nr, CycleState{0, 0, 0, 0, 0.0, 0.0});
    HM_CUDA(cudaMemcpyAsync(W.st.p, cs.data(), nr * sizeof(CycleState), cudaMemcpyHostToDevice, st));
    k_bj_apply<<<H.n_leaves, 256, 0, st>>>(H.leaves.p, W.binv.p, W.binv_off.p, v, z, nullptr, H.ndof, nr, W.st.p, 0,
                                           nullptr);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaStreamSynchronize(st));
}

void near_offdiag_cluster(HMat& H, const double* v, double* out, int nr, cudaStream_t st) {
    if (nr < 1 || nr > 16) fail(HM_EINVAL, "near product: 1 to 16 right-hand sides");
    SolveWS& W = workspace(H, nr, 1, st);
    near_prepare(H, W, nr, st);
    k_to_f32_interleaved<<<g1(H.ndof * nr), 256, 0, st>>>(v, W.nv32.p, H.ndof, nr);
    HM_LAUNCH_CHECK();
    near_offdiag_launch(H, near_dev(W), W.nv32.p, out, nr, nullptr, st);
}

// The ILU preconditioner of A = E - diag(k) - C^ep - shift I for a fraction p, built and
// factored, then copied to the host (see ilu_export).
void ilu_export_for(HMat& H, const double* kel, const double* cep, double shift, double p, int64_t* n_out,
                    int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr, int32_t* col,
                    double* a_val, double* lu_val, cudaStream_t st) {
    SolveWS& W = workspace(H, 1, 1, st);
    W.pc_key.valid = false;
    set_tangent(H, W, kel, cep, shift, st);
    ilu_prepare(H, p, cep != nullptr, st);
    if (lu_val) ilu_factor(H, W.dc.p, W.blk, st, W.err.p);
    ilu_export(H, n_out, nnz_out, n_colours_out, order, rowptr, col, a_val, lu_val, st);
}

// y = (E - diag(k) - C^ep - shift I) x for one user-ordered FP64 vector (compensated
// product with the FP32 factors)
void tangent_apply_user(HMat& H, const double* kel, const double* cep, double shift, const double* x, double* y,
                        cudaStream_t st) {
    if (!has_factors(H, 0)) fail(HM_EINVAL, "tangent product: the FP32 factors are required");
    SolveWS& W = workspace(H, 1, 1, st);
    const int64_t n = H.ndof;
    set_tangent(H, W, kel, cep, shift, st);
    CycleState c0{0, 0, 0, 0, 0.0, 0.0};
    HM_CUDA(cudaMemcpyAsync(W.st.p, &c0, sizeof(CycleState), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemsetAsync(W.alldone.p, 0, sizeof(int), st));
    k_to_cluster<<<g1(n), 256, 0, st>>>(x, W.xc.p, H.perm.p, n, 1);
    HM_LAUNCH_CHECK();
    apply_E(H, W, W.xc.p, nullptr, W.y64.p, 1, HM_F64, 0, st);
    k_tangent<double><<<g1(n), 256, 0, st>>>(W.y64.p, W.dc.p, W.blk, W.xc.p, W.w.p, n, 1, W.st.p);
    k_to_user<<<g1(n), 256, 0, st>>>(W.w.p, y, H.perm.p, n, 1);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaStreamSynchronize(st));  // the host struct c0 above is read by the copy
}

// diag(E - diag(k) - C^ep - shift I) per DOF in user order (E's diagonal from the FP32
// near-field self tiles)
__global__ void k_tangent_diag(const LeafDesc* __restrict__ leaves, const int64_t* __restrict__ self_off,
                               const float* __restrict__ near, const double* __restrict__ d,
                               const double* __restrict__ blk, const int32_t* __restrict__ perm,
                               double* __restrict__ out) {
    const LeafDesc L = leaves[blockIdx.x];
    const float* T = near + self_off[blockIdx.x];
    for (int r = threadIdx.x; r < 3 * L.n; r += blockDim.x) {
        const int64_t p = 3 * (int64_t)L.begin + r;
        out[3 * (int64_t)perm[p / 3] + r % 3] = (double)T[(int64_t)r * L.ld + r] - d[p];
    }
}

void tangent_diag_user(HMat& H, const double* kel, const double* cep, double shift, double* out, cudaStream_t st) {
    SolveWS& W = workspace(H, 1, 1, st);
    set_tangent(H, W, kel, cep, shift, st);
    k_tangent_diag<<<H.n_leaves, 128, 0, st>>>(H.leaves.p, W.self_off.p, H.near.p, W.dc.p, W.blk, H.perm.p, out);
    HM_LAUNCH_CHECK();
}

// z = (L U)^-1 r for user-ordered vectors with the last ILU factorization
void ilu_apply_user(HMat& H, const double* r, double* z, int nrhs, cudaStream_t st) {
    if (nrhs < 1 || nrhs > 16) fail(HM_EINVAL, "ilu_apply: 1 to 16 right-hand sides");
    if (!r || !z) fail(HM_EINVAL, "ilu_apply: NULL vector");
    if (!ilu_is_factored(H)) fail(HM_EINVAL, "ilu_apply: no ILU factorization on this H-matrix");
    SolveWS& W = workspace(H, nrhs, 1, st);
    k_to_cluster<<<g1(H.ndof * nrhs), 256, 0, st>>>(r, W.r.p, H.perm.p, H.ndof, nrhs);
    HM_LAUNCH_CHECK();
    ilu_apply(H, W.r.p, W.w.p, nullptr, nrhs, nullptr, 0, st);
    k_to_user<<<g1(H.ndof * nrhs), 256, 0, st>>>(W.w.p, z, H.perm.p, H.ndof, nrhs);
    HM_LAUNCH_CHECK();
}

// the preconditioner of the options for the tangent in W (W.dc, W.blk set), or the one
// already built for the same inputs when the options ask to reuse it
void build_precond(HMat& H, SolveWS& W, const double* kel, const double* cep, double shift, const hm_solve_opts& o,
                   PcKind pc, double ilu_p, const LPModel* lp, int nrhs, cudaStream_t st) {
    NvtxScope nvtx_("build_precond");
    SolveWS::PcKey key;
    key.valid = true;
    key.kel = kel;
    key.cep = cep;
    key.shift = shift;
    key.ilu_p = pc == PC_ILU ? ilu_p : 0.0;
    key.precond = o.precond;
    key.lp = lp;
    const bool reuse = o.reuse_precond && W.pc_key.same(key) && (pc != PC_ILU || ilu_is_factored(H));
    if (!reuse) {
        W.pc_key.valid = false;
        W.dsc_on = false;
        if (pc == PC_POINT) j3_build(H, W, st);
        if (pc == PC_ILU) {
            ilu_prepare(H, ilu_p, cep != nullptr, st);
            ilu_factor(H, W.dc.p, W.blk, st, W.err.p);
        }
        W.near_on = false;
        if (pc == PC_LEAF) {
            bj_build(H, W, st);
            if (o.precond == HM_PRECOND_LEARNED && !lp->fallback) {
                W.dsc.alloc((size_t)H.n_leaves * 3);
                lp_predict(const_cast<LPModel&>(*lp), H, kel, W.dsc.p, nullptr, st);
                if (lp->kind == LP_NEAR) {
                    near_prepare(H, W, nrhs, st);
                    W.near_on = true;
                    W.near_gamma = lp->gamma;
                } else {
                    W.dsc_on = true;
                }
            }
        }
        W.pc_key = key;
    }
    if (W.near_on) near_prepare(H, W, nrhs, st);  // scratch for this call's RHS count
}

PcKind pc_kind(int precond) {
    return (precond == HM_PRECOND_BLOCKJ || precond == HM_PRECOND_LEARNED)
               ? PC_LEAF
               : (precond == HM_PRECOND_JACOBI3 ? PC_POINT : (precond == HM_PRECOND_ILU ? PC_ILU : PC_NONE));
}

// z = M^-1 r with the preconditioner hm_gmres_solve builds for these options (user order)
void precond_apply_user(HMat& H, const double* kel, double shift, const hm_solve_opts& o, const LPModel* lp,
                        const double* r, double* z, int nrhs, cudaStream_t st) {
    if (nrhs < 1 || nrhs > 16) fail(HM_EINVAL, "precond_apply: 1 to 16 right-hand sides");
    if (!r || !z) fail(HM_EINVAL, "precond_apply: NULL vector");
    if (o.precond != HM_PRECOND_NONE && o.precond != HM_PRECOND_BLOCKJ && o.precond != HM_PRECOND_LEARNED &&
        o.precond != HM_PRECOND_JACOBI3 && o.precond != HM_PRECOND_ILU)
        fail(HM_EINVAL, "precond_apply: unknown preconditioner");
    if (o.precond == HM_PRECOND_LEARNED && !lp) fail(HM_EINVAL, "precond_apply: the learned preconditioner needs a model");
    if (o.precond == HM_PRECOND_LEARNED && o.cep_dev)
        fail(HM_EINVAL, "precond_apply: the learned preconditioner takes a diagonal interface term (k), not C^ep");
    const double ilu_p = o.ilu_p > 0.0 ? o.ilu_p : 0.01;
    if (o.precond == HM_PRECOND_ILU && !(ilu_p <= 1.0)) fail(HM_EINVAL, "precond_apply: ilu_p must lie in (0, 1]");
    SolveWS& W = workspace(H, nrhs, 1, st);
    const int64_t n = H.ndof;
    set_tangent(H, W, kel, o.cep_dev, shift, st);
    const PcKind pc = pc_kind(o.precond);
    build_precond(H, W, kel, o.cep_dev, shift, o, pc, ilu_p, lp, nrhs, st);
    std::vector<CycleState> cs(nrhs, CycleState{0, 0, 0, 0, 0.0, 0.0});
    HM_CUDA(cudaMemcpyAsync(W.st.p, cs.data(), nrhs * sizeof(CycleState), cudaMemcpyHostToDevice, st));
    k_to_cluster<<<g1(n * nrhs), 256, 0, st>>>(r, W.r.p, H.perm.p, n, nrhs);
    HM_LAUNCH_CHECK();
    precond_apply(H, W, pc, W.r.p, W.w.p, nullptr, nrhs, st);
    k_to_user<<<g1(n * nrhs), 256, 0, st>>>(W.w.p, z, H.perm.p, n, nrhs);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaStreamSynchronize(st));  // cs above is read by the copy
}

void gmres_solve(HMat& H, const double* kel, double shift, const double* b, double* x, int nrhs,
                 const hm_solve_opts& o, hm_solve_info* info, cudaStream_t st, const LPModel* lp) {
    const double* cep = o.cep_dev;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (nrhs < 1 || nrhs > 16) fail(HM_EINVAL, "gmres_solve: 1 to 16 right-hand sides");
    if (!b || !x) fail(HM_EINVAL, "gmres_solve: NULL vector");
    const double tol = o.tol > 0 ? o.tol : 1e-8;
    const int m = o.restart > 0 ? o.restart : 50;
    if (m > 128) fail(HM_EINVAL, "gmres_solve: restart must be <= 128");
    const int maxit = o.maxit > 0 ? o.maxit : 2000;
    const int mode = o.mode ? o.mode : HM_SOLVE_F64;
    if (mode != HM_SOLVE_F64 && mode != HM_SOLVE_MIXED && mode != HM_SOLVE_PLAIN32)
        fail(HM_EINVAL, "gmres_solve: unknown mode");
    if (o.method != HM_METHOD_FGMRES && o.method != HM_METHOD_BICGSTAB) fail(HM_EINVAL, "gmres_solve: unknown method");
    if (o.precond != HM_PRECOND_NONE && o.precond != HM_PRECOND_BLOCKJ && o.precond != HM_PRECOND_LEARNED &&
        o.precond != HM_PRECOND_JACOBI3 && o.precond != HM_PRECOND_ILU)
        fail(HM_EINVAL, "gmres_solve: unknown preconditioner");
    const double ilu_p = o.ilu_p > 0.0 ? o.ilu_p : 0.01;
    if (o.precond == HM_PRECOND_ILU && !(ilu_p <= 1.0)) fail(HM_EINVAL, "gmres_solve: ilu_p must lie in (0, 1]");
    if (o.precond == HM_PRECOND_LEARNED && !lp) fail(HM_EINVAL, "gmres_solve: the learned preconditioner needs a model");
    if (o.precond == HM_PRECOND_LEARNED && cep)
        fail(HM_EINVAL, "gmres_solve: the learned preconditioner takes a diagonal interface term (k), not C^ep");
    if (!has_factors(H, 0)) fail(HM_EINVAL, "gmres_solve: the FP32 factors are required (storage F32 or F32_BF16)");
    // refinement corrections: BF16 factors (mixed; FP32 if BF16 is not stored) or the
    // FP32 factors themselves (PLAIN32: the same refinement without the BF16 operator)
    const int inner_fac = mode == HM_SOLVE_PLAIN32 ? 0 : (has_factors(H, 1) ? 1 : 0);
    SolveWS& W = workspace(H, nrhs, m, st);
    const int64_t n = H.ndof;
    // the stiffness and the right-hand sides must be finite (a NaN would silently spread
    // through every Krylov vector)
    HM_CUDA(cudaMemsetAsync(W.err.p, 0, sizeof(int), st));
    if (kel) k_nonfinite<<<152, 256, 0, st>>>(kel, H.N, W.err.p);
    if (cep) k_nonfinite<<<152, 256, 0, st>>>(cep, 9 * H.N, W.err.p);
    k_nonfinite<<<152, 256, 0, st>>>(b, n * nrhs, W.err.p + 0);
    HM_LAUNCH_CHECK();
    {
        int e = 0;
        HM_CUDA(cudaMemcpyAsync(&e, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (e) fail(HM_ENAN, "gmres_solve: the stiffness k, C^ep or the right-hand side holds NaN or Inf");
    }
    set_tangent(H, W, kel, cep, shift, st);
    k_to_cluster<<<g1(n * nrhs), 256, 0, st>>>(b, W.bc.p, H.perm.p, n, nrhs);
    HM_LAUNCH_CHECK();
    const PcKind pc = pc_kind(o.precond);
    build_precond(H, W, kel, cep, shift, o, pc, ilu_p, lp, nrhs, st);
    // ||b||
    HM_CUDA(cudaMemsetAsync(W.xc.p, 0, (size_t)n * nrhs * sizeof(double), st));
    std::vector<double> bn = residual(H, W, W.bc.p, nrhs, HM_F64, 0, st, true);  // x = 0: r = b
    std::vector<double> tol_abs(nrhs);
    for (int k = 0; k < nrhs; ++k) tol_abs[k] = tol * bn[k];
    std::vector<int> its(nrhs, 0), outer(nrhs, 0), brk(nrhs, 0);
    std::vector<double> rn = bn;
    const bool bcg = o.method == HM_METHOD_BICGSTAB;
    if (mode == HM_SOLVE_F64) {
        if (bcg) {
            bicgstab(H, W, W.bc.p, tol_abs, nrhs, maxit, 8, HM_F64, 0, pc, its, rn, brk, st, true);
        } else {
            fgmres(H, W, W.bc.p, tol_abs, nrhs, m, maxit, 1 << 20, HM_F64, 0, pc, its, rn, brk, st, true);
            for (int k = 0; k < nrhs; ++k) outer[k] = (its[k] + m - 1) / m;
        }
    } else {
        const double itol = o.inner_tol > 0 ? o.inner_tol : 1e-2;
        const int max_outer = o.max_outer > 0 ? o.max_outer : 40;
        // x accumulates in W.xc; the correction solve runs on a saved copy
        DevBuf<double> xacc((size_t)n * nrhs);
        HM_CUDA(cudaMemsetAsync(xacc.p, 0, xacc.bytes(), st));
        std::vector<double> rr = bn;  // ||b - A x|| with the FP32 factors, compensated
        for (int it = 0; it < max_outer; ++it) {
            bool any = false;
            for (int k = 0; k < nrhs; ++k) any = any || (rr[k] > tol_abs[k] && its[k] < maxit);
            if (!any) break;
            // outer residual into W.r (current x in xacc)
            HM_CUDA(cudaMemcpyAsync(W.xc.p, xacc.p, xacc.bytes(), cudaMemcpyDeviceToDevice, st));
            rr = residual(H, W, W.bc.p, nrhs, HM_F64, 0, st, it == 0);
            bool need = false;
            for (int k = 0; k < nrhs; ++k) need = need || (rr[k] > tol_abs[k] && its[k] < maxit);
            if (!need) break;
            // correction: FGMRES on the BF16-factor operator, FP32 products, from 0
            HM_CUDA(cudaMemcpyAsync(W.corr.p, W.r.p, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice,
                                    st));
            HM_CUDA(cudaMemsetAsync(W.xc.p, 0, (size_t)n * nrhs * sizeof(double), st));
            std::vector<double> itol_abs(nrhs);
            for (int k = 0; k < nrhs; ++k) itol_abs[k] = rr[k] > tol_abs[k] ? itol * rr[k] : 1e300;
            std::vector<int> iits, ibrk;
            std::vector<double> irn;
            if (bcg)
                bicgstab(H, W, W.corr.p, itol_abs, nrhs, maxit, 2, HM_F32, inner_fac, pc, iits, irn, ibrk, st, true);
            else
                fgmres(H, W, W.corr.p, itol_abs, nrhs, m, maxit, 4, HM_F32, inner_fac, pc, iits, irn, ibrk, st, true);
            for (int k = 0; k < nrhs; ++k) {
                its[k] += iits[k];
                if (iits[k] > 0) outer[k]++;
            }
            k_axpy<<<g1(n * nrhs), 256, 0, st>>>(xacc.p, W.xc.p, n * nrhs);
            HM_LAUNCH_CHECK();
        }
        HM_CUDA(cudaMemcpyAsync(W.xc.p, xacc.p, xacc.bytes(), cudaMemcpyDeviceToDevice, st));
        rn = residual(H, W, W.bc.p, nrhs, HM_F64, 0, st);
    }
    k_to_user<<<g1(n * nrhs), 256, 0, st>>>(W.xc.p, x, H.perm.p, n, nrhs);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(clk::now() - t0).count();
    bool all_ok = true, any_brk = false;
    for (int k = 0; k < nrhs; ++k) {
        const double rel = bn[k] > 0 ? rn[k] / bn[k] : 0.0;
        const bool ok = rel <= tol;
        all_ok = all_ok && ok;
        any_brk = any_brk || (brk[k] && !ok);
        if (info) {
            info[k].iters = its[k];
            info[k].outer = outer[k];
            info[k].status = ok ? HM_OK : (brk[k] ? HM_EBREAKDOWN : HM_ENOCONV);
            info[k].pad_ = 0;
            info[k].relres = rel;
            info[k].seconds = secs;
        }
    }
    if (any_brk) fail(HM_EBREAKDOWN, "gmres_solve: Krylov breakdown before the tolerance");
    if (!all_ok) fail(HM_ENOCONV, "gmres_solve: tolerance not reached within maxit");
}

}  // namespace hm
