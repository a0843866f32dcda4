// Incomplete-LU preconditioner of the mechanical block on the device (Sec. 3.3.1): the
// tangent A = E - diag(k) - shift I is replaced, for preconditioning, by C^ep plus the
// fraction p of the near-field entries of E with the largest magnitude, and that sparse
// matrix is applied through its ILU(0) factors.
//
// Plan (once per H-matrix, p and kind of interface term; k, C^ep and shift change only
// values):
//   * selection: the ceil(p n) entries of largest |v| among the n entries of the FP32 near
//     tiles of inadmissible leaf pairs -- a radix select over the bit patterns of |v|
//     (three histogram passes), then a compaction of the entries above the threshold
//     and of the ties at it; ties are taken by (row, column) in cluster DOF order;
//   * ordering: the leaves coloured greedily by the coupling of the selected pattern and
//     listed colour by colour (leaf order within a colour, cluster order within a leaf):
//     leaves of one colour share no entry, so the factorization and the triangular solves
//     handle them in parallel, one CTA per leaf, and each solve is one launch per colour;
//   * CSR of the pattern in that order, the diagonal always present (E's entry if
//     selected, else 0; -k - shift is added per factorization); with a block-diagonal
//     C^ep (3x3 per element) every element's whole 3x3 block is present, since C^ep
//     belongs to the sparse matrix entirely.
// Factorization (per solve): ILU(0) in FP64, level by level of the lower triangle (a row
// waits for the rows its multipliers name), a warp per row (its multipliers in column
// order, the update from a finished row confined to the pattern).  Application: forward and backward substitution in FP64,
// colour by colour; the rows of one leaf are staged with their CSR block in shared memory
// and solved by one warp, their couplings to other colours gathered by the whole CTA.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "hmat_impl.h"
#include "ilu_dev.h"

namespace hm {

struct IluPlan {
    double p = 0.0;
    bool self_blocks = false;  // each element's 3x3 block forced into the pattern
    int64_t n = 0;        // DOFs
    int64_t nnz = 0;
    int64_t m_selected = 0;
    int n_colours = 0;
    std::vector<int32_t> h_order;      // new position -> cluster DOF position
    std::vector<int32_t> h_colour_first;  // [n_colours + 1] into the leaf schedule
    std::vector<int32_t> h_sched;      // leaves (ordinal) in colour order
    std::vector<int32_t> h_row0;       // new-order first row of each scheduled leaf
    int max_leaf_rows = 0;
    int64_t max_leaf_nnz = 0;
    std::vector<int32_t> h_level_first;  // [n_levels + 1] into level_rows
    DevBuf<int32_t> level_rows;        // rows grouped by level of the lower triangle
    DevBuf<int32_t> order, col, sched_row0, sched_nrows;
    // per leaf (at its rows' positions): local rows ordered by level inside the leaf, and
    // their levels, for the lower and the upper triangle
    DevBuf<uint8_t> lrow_lo, llev_lo, lrow_up, llev_up;
    DevBuf<int64_t> rowptr, diagpos;
    DevBuf<int64_t> selfpos;           // [3n]: positions of row a's entries in its element's block
    DevBuf<double> aval, lu;
    DevBuf<double> yv, zv;             // new-order work vectors, nr x n
    int nr_cap = 0;
    bool factored = false;
};

void ilu_plan_free(IluPlan* p) { delete p; }

namespace {

constexpr int SEL_NT = 256;

__device__ __forceinline__ uint32_t abits(float v) { return __float_as_uint(v) & 0x7fffffffu; }

// Histogram of bits [shift, shift + width) of |v| (binmask = 2^width - 1) over the
// near-field entries whose higher bits equal `prefix` (under `pmask`).  One CTA per leaf.
__global__ void __launch_bounds__(SEL_NT) k_sel_hist(const LeafDesc* __restrict__ leaves,
                                                     const int32_t* __restrict__ true_cols,
                                                     const float* __restrict__ near, uint32_t prefix, uint32_t pmask,
                                                     int shift, uint32_t binmask,
                                                     unsigned long long* __restrict__ hist) {
    __shared__ unsigned sh[2048];
    for (int i = threadIdx.x; i < 2048; i += SEL_NT) sh[i] = 0;
    __syncthreads();
    const LeafDesc L = leaves[blockIdx.x];
    const int rows = 3 * L.n;
    const int64_t cnt = (int64_t)true_cols[blockIdx.x] * rows;
    for (int64_t q = threadIdx.x; q < cnt; q += SEL_NT) {
        const int64_t c = q / rows, r = q % rows;
        const uint32_t b = abits(near[L.near_off + c * L.ld + r]);
        if ((b & pmask) == prefix) atomicAdd(&sh[(b >> shift) & binmask], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += SEL_NT)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// Entries with |v| above the threshold bits and those equal to it (row, column, value),
// appended through warp-aggregated counters (order irrelevant: sorted
// on the host).
__global__ void __launch_bounds__(SEL_NT) k_sel_compact(const LeafDesc* __restrict__ leaves,
                                                        const int32_t* __restrict__ true_cols,
                                                        const int32_t* __restrict__ zidx,
                                                        const float* __restrict__ near, uint32_t thr,
                                                        int32_t* __restrict__ gi, int32_t* __restrict__ gj,
                                                        float* __restrict__ gv, unsigned long long* __restrict__ cnt,
                                                        int64_t cap_gt, int32_t* __restrict__ ti,
                                                        int32_t* __restrict__ tj, float* __restrict__ tv,
                                                        int64_t cap_tie) {
    const LeafDesc L = leaves[blockIdx.x];
    const int rows = 3 * L.n;
    const int64_t tot = (int64_t)true_cols[blockIdx.x] * rows;
    const int lane = threadIdx.x & 31;
    for (int64_t q0 = 0; q0 < tot; q0 += SEL_NT) {
        const int64_t q = q0 + threadIdx.x;
        uint32_t b = 0;
        int64_t c = 0, r = 0;
        float v = 0.f;
        if (q < tot) {
            c = q / rows;
            r = q % rows;
            v = near[L.near_off + c * L.ld + r];
            b = abits(v);
        }
        const bool gt = q < tot && b > thr, eq = q < tot && b == thr;
        const unsigned mg = __ballot_sync(0xffffffffu, gt), me = __ballot_sync(0xffffffffu, eq);
        unsigned long long bg = 0, be = 0;
        if (lane == 0) {
            if (mg) bg = atomicAdd(cnt, (unsigned long long)__popc(mg));
            if (me) be = atomicAdd(cnt + 1, (unsigned long long)__popc(me));
        }
        bg = __shfl_sync(0xffffffffu, bg, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        const unsigned below = (1u << lane) - 1u;
        const int32_t row = 3 * L.begin + (int32_t)r;
        const int32_t colg = q < tot ? zidx[L.near_cbase + c] : 0;
        if (gt) {
            const int64_t pos = (int64_t)bg + __popc(mg & below);
            if (pos < cap_gt) {
                gi[pos] = row;
                gj[pos] = colg;
                gv[pos] = v;
            }
        }
        if (eq) {
            const int64_t pos = (int64_t)be + __popc(me & below);
            if (pos < cap_tie) {
                ti[pos] = row;
                tj[pos] = colg;
                tv[pos] = v;
            }
        }
    }
}

// lu = aval, then (k_ilu_diag) lu[diag(a)] -= d[order[a]] (d in cluster DOF order)
__global__ void k_ilu_init(const double* __restrict__ aval, double* __restrict__ lu, int64_t nnz) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < nnz) lu[q] = aval[q];
}

__global__ void k_ilu_diag(double* __restrict__ lu, const int64_t* __restrict__ diagpos,
                           const int32_t* __restrict__ order, const double* __restrict__ d, int64_t n) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < n) lu[diagpos[a]] -= d[order[a]];
}

// lu[block entries of row a] -= blk[element][row comp][col comp] (off the diagonal; blk
// in cluster element order with a zero diagonal)
__global__ void k_ilu_self(double* __restrict__ lu, const int64_t* __restrict__ selfpos,
                           const int32_t* __restrict__ order, const double* __restrict__ blk, int64_t n) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int32_t r = order[a];
    const int64_t e = r / 3;
    const int c = r % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (j != c) lu[selfpos[3 * a + j]] -= blk[9 * e + 3 * c + j];
}

// first position in [lo, hi) of col with col[pos] == c, else -1 (columns increasing)
__device__ __forceinline__ int64_t find_col(const int32_t* __restrict__ col, int64_t lo, int64_t hi, int32_t c) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c)
            lo = mid + 1;
        else
            hi = mid;
    }
    return -1;
}

// ILU(0) of a set of rows none of which depends on another (one level of the lower
// triangle): a warp per row, its multipliers in column order, each taking the finished row
// b of U times the multiplier off the row's entries in the pattern.
__global__ void __launch_bounds__(256) k_ilu_factor_rows(const int32_t* __restrict__ rows, int count,
                                                         const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const int64_t* __restrict__ diagpos, double* __restrict__ lu,
                                                         int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int wi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wi >= count) return;
    const int32_t a = rows[wi];
    const int64_t beg = rowptr[a], dp = diagpos[a], end = rowptr[a + 1];
    for (int64_t q = beg; q < dp; ++q) {
        const int32_t b = col[q];
        const double ub = lu[diagpos[b]];
        const double l = lu[q] / ub;
        if (!(ub != 0.0) || !isfinite(l)) {
            if (lane == 0) atomicOr(err, 1);
        }
        __syncwarp();
        if (lane == 0) lu[q] = l;
        const int64_t bend = rowptr[b + 1];
        for (int64_t t = diagpos[b] + 1 + lane; t < bend; t += 32) {
            const int64_t pos = find_col(col, q + 1, end, col[t]);
            if (pos >= 0) lu[pos] -= l * lu[t];
        }
        __syncwarp();
    }
}

// ---- application.  One CTA per leaf of a colour; shared memory holds the leaf's CSR
// block (values, columns), its rows' offsets into it, the staged solution of its rows and
// the leaf's rows ordered by level of the triangle inside the leaf (a row waits only for
// rows of the leaf its pattern names there, earlier for the lower, later for the upper
// factor; entries to other leaves were finished by earlier launches).  Each level is
// solved by the warps in parallel, a row per warp, between CTA barriers.
constexpr int ILU_ROWS = 192;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct LeafStage {
    double* xs;        // [ILU_ROWS] solution of the leaf's rows
    int32_t* rlo;      // [ILU_ROWS + 1] row starts relative to the block
    int32_t* rdp;      // [ILU_ROWS] diagonal positions relative to the block
    int32_t* bnd;      // [ILU_ROWS + 1] level boundaries in lrow
    uint8_t* lrow;     // [ILU_ROWS] rows (local) by level
    double* sval;      // [nnz] block values (staged) ...
    int32_t* scol;     // [nnz] ... and columns
};

__device__ __forceinline__ LeafStage leaf_stage(unsigned char* dsm, int64_t nnz_staged) {
    LeafStage L;
    L.xs = reinterpret_cast<double*>(dsm);
    L.rlo = reinterpret_cast<int32_t*>(L.xs + ILU_ROWS);
    L.rdp = L.rlo + ILU_ROWS + 1;
    L.bnd = L.rdp + ILU_ROWS;
    L.lrow = reinterpret_cast<uint8_t*>(L.bnd + ILU_ROWS + 1);
    L.sval = reinterpret_cast<double*>(dsm + 8 * ILU_ROWS + 4 * (3 * ILU_ROWS + 2) + ILU_ROWS + 8);
    L.scol = reinterpret_cast<int32_t*>(L.sval + nnz_staged);
    return L;
}

// bytes of shared memory before the staged block values (8-byte aligned)
constexpr int ILU_STAGE_HEAD = 8 * ILU_ROWS + 4 * (3 * ILU_ROWS + 2) + ILU_ROWS + 8;

// stage the leaf: block values and columns (if they fit), row offsets, levels; returns
// the number of levels
__device__ int stage_leaf(const LeafStage& S, int32_t r0, int rows, int64_t base, int64_t nnz, bool staged,
                          const int64_t* __restrict__ rowptr, const int64_t* __restrict__ diagpos,
                          const double* __restrict__ lu, const int32_t* __restrict__ col,
                          const uint8_t* __restrict__ lrow_g, const uint8_t* __restrict__ llev_g) {
    if (staged)
        for (int64_t q = threadIdx.x; q < nnz; q += blockDim.x) {
            S.sval[q] = lu[base + q];
            S.scol[q] = col[base + q];
        }
    for (int i = threadIdx.x; i <= rows; i += blockDim.x) S.rlo[i] = (int32_t)(rowptr[r0 + i] - base);
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        S.rdp[i] = (int32_t)(diagpos[r0 + i] - base);
        S.lrow[i] = lrow_g[r0 + i];
    }
    __syncthreads();
    // level boundaries: positions where the (sorted) level changes
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        const int lv = llev_g[r0 + i];
        if (i == 0 || llev_g[r0 + i - 1] != lv) S.bnd[lv] = i;
    }
    const int nlev = rows > 0 ? (int)llev_g[r0 + rows - 1] + 1 : 0;
    if (threadIdx.x == 0) S.bnd[nlev] = rows;
    __syncthreads();
    return nlev;
}

// forward substitution L y = v for the rows of the leaves of one colour (L unit lower):
// v is the cluster-order input, y the new-order result
__global__ void __launch_bounds__(256) k_ilu_fwd(const int32_t* __restrict__ row0s, const int32_t* __restrict__ nrows,
                                                 const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                 const int64_t* __restrict__ diagpos, const double* __restrict__ lu,
                                                 const uint8_t* __restrict__ lrow_g, const uint8_t* __restrict__ llev_g,
                                                 const int32_t* __restrict__ order, const double* __restrict__ v,
                                                 double* __restrict__ y, int64_t n, int nr, int smem_nnz,
                                                 const int* __restrict__ done, int done_stride) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int32_t r0 = row0s[blockIdx.x], rows = nrows[blockIdx.x];
    const int64_t base = rowptr[r0], nnz = rowptr[r0 + rows] - base;
    const bool staged = nnz <= smem_nnz;
    const LeafStage S = leaf_stage(dsm, staged ? nnz : 0);
    const int nlev = stage_leaf(S, r0, rows, base, nnz, staged, rowptr, diagpos, lu, col, lrow_g, llev_g);
    const double* cv = staged ? S.sval : lu + base;
    const int32_t* cc = staged ? S.scol : col + base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < nr; ++k) {
        if (done && done[k * done_stride]) continue;
        const double* vk = v + (int64_t)k * n;
        double* yk = y + (int64_t)k * n;
        // couplings to earlier colours (columns before the leaf), all rows at once
        for (int i = threadIdx.x; i < rows; i += blockDim.x) {
            double s = vk[order[r0 + i]];
            for (int q = S.rlo[i]; q < S.rdp[i] && cc[q] < r0; ++q) s -= cv[q] * yk[cc[q]];
            S.xs[i] = s;
        }
        __syncthreads();
        for (int lv = 0; lv < nlev; ++lv) {
            for (int p = S.bnd[lv] + w; p < S.bnd[lv + 1]; p += nw) {
                const int i = S.lrow[p];
                double part = 0.0;
                for (int q = S.rlo[i] + lane; q < S.rdp[i]; q += 32) {
                    const int32_t c = cc[q];
                    if (c >= r0) part += cv[q] * S.xs[c - r0];
                }
                part = warp_sum(part);
                if (lane == 0) S.xs[i] -= part;
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < rows; i += blockDim.x) yk[r0 + i] = S.xs[i];
        __syncthreads();
    }
}

// backward substitution U z = y for the rows of the leaves of one colour (reverse
// colour order on the host): z new-order, out / outf the cluster-order results
__global__ void __launch_bounds__(256) k_ilu_bwd(const int32_t* __restrict__ row0s, const int32_t* __restrict__ nrows,
                                                 const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                 const int64_t* __restrict__ diagpos, const double* __restrict__ lu,
                                                 const uint8_t* __restrict__ lrow_g, const uint8_t* __restrict__ llev_g,
                                                 const int32_t* __restrict__ order, const double* __restrict__ y,
                                                 double* __restrict__ z, double* __restrict__ out,
                                                 float* __restrict__ outf, int64_t n, int nr, int smem_nnz,
                                                 const int* __restrict__ done, int done_stride) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int32_t r0 = row0s[blockIdx.x], rows = nrows[blockIdx.x];
    const int32_t r1 = r0 + rows;
    const int64_t base = rowptr[r0], nnz = rowptr[r1] - base;
    const bool staged = nnz <= smem_nnz;
    const LeafStage S = leaf_stage(dsm, staged ? nnz : 0);
    const int nlev = stage_leaf(S, r0, rows, base, nnz, staged, rowptr, diagpos, lu, col, lrow_g, llev_g);
    const double* cv = staged ? S.sval : lu + base;
    const int32_t* cc = staged ? S.scol : col + base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < nr; ++k) {
        if (done && done[k * done_stride]) continue;
        const double* yk = y + (int64_t)k * n;
        double* zk = z + (int64_t)k * n;
        // couplings to later colours (columns after the leaf)
        for (int i = threadIdx.x; i < rows; i += blockDim.x) {
            double s = yk[r0 + i];
            for (int q = S.rlo[i + 1] - 1; q > S.rdp[i] && cc[q] >= r1; --q) s -= cv[q] * zk[cc[q]];
            S.xs[i] = s;
        }
        __syncthreads();
        for (int lv = 0; lv < nlev; ++lv) {
            for (int p = S.bnd[lv] + w; p < S.bnd[lv + 1]; p += nw) {
                const int i = S.lrow[p];
                const int dp = S.rdp[i];
                double part = 0.0;
                for (int q = dp + 1 + lane; q < S.rlo[i + 1]; q += 32) {
                    const int32_t c = cc[q];
                    if (c < r1) part += cv[q] * S.xs[c - r0];
                }
                part = warp_sum(part);
                if (lane == 0) S.xs[i] = (S.xs[i] - part) / cv[dp];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < rows; i += blockDim.x) {
            const int32_t a = r0 + i;
            zk[a] = S.xs[i];
            out[(int64_t)k * n + order[a]] = S.xs[i];
            if (outf) outf[(int64_t)order[a] * nr + k] = (float)S.xs[i];
        }
        __syncthreads();
    }
}

unsigned gsz(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

int64_t apply_smem_nnz(const IluPlan& P) {
    // at most 200 KB of staged CSR per leaf (12 bytes per entry) beside the row data
    const int64_t cap = (200 * 1024) / 12;
    return std::min<int64_t>(cap, P.max_leaf_nnz);
}

}  // namespace

void ilu_prepare(HMat& H, double p, bool self_blocks, cudaStream_t st) {
    if (!(p > 0.0 && p <= 1.0)) fail(HM_EINVAL, "ilu: p must lie in (0, 1]");
    if (H.ilu && H.ilu->p == p && H.ilu->self_blocks == self_blocks) return;
    if ((int64_t)H.h_near_true_cols.size() != H.n_leaves) fail(HM_EINVAL, "ilu: near-field layout unknown");
    if (H.ndof > INT32_MAX) fail(HM_EINVAL, "ilu: too many DOFs");
    ilu_plan_free(H.ilu);
    H.ilu = nullptr;
    IluPlan* P = new IluPlan();
    try {
        P->p = p;
        P->self_blocks = self_blocks;
        const int64_t n = H.ndof;
        P->n = n;
        const int nl = H.n_leaves;
        // candidate count
        int64_t n_cand = 0;
        for (int l = 0; l < nl; ++l) n_cand += (int64_t)H.h_near_true_cols[l] * 3 * H.h_leaves[l].n;
        const int64_t m = (int64_t)std::ceil(p * (double)n_cand);
        if (m < 1) fail(HM_EINVAL, "ilu: no near-field entries to select");
        DevBuf<int32_t> d_true, d_zidx;
        d_true.upload(H.h_near_true_cols, st);
        d_zidx.upload(H.h_near_zidx, st);
        // radix select of the m-th largest |v| over 31 bits: 11 + 11 + 9
        DevBuf<unsigned long long> hist(2048);
        std::vector<unsigned long long> h(2048);
        uint32_t prefix = 0, pmask = 0;
        int64_t above = 0;  // entries known to be larger than the current bucket
        const int shifts[3] = {20, 9, 0};
        const int widths[3] = {11, 11, 9};
        int64_t in_bucket = 0;
        for (int pass = 0; pass < 3; ++pass) {
            HM_CUDA(cudaMemsetAsync(hist.p, 0, hist.bytes(), st));
            k_sel_hist<<<nl, SEL_NT, 0, st>>>(H.leaves.p, d_true.p, H.near.p, prefix, pmask, shifts[pass],
                                              (1u << widths[pass]) - 1u, hist.p);
            HM_LAUNCH_CHECK();
            HM_CUDA(cudaMemcpyAsync(h.data(), hist.p, hist.bytes(), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            const int nb = 1 << widths[pass];
            int bucket = -1;
            for (int bkt = nb - 1; bkt >= 0; --bkt) {
                if (above + (int64_t)h[bkt] >= m) {
                    bucket = bkt;
                    in_bucket = (int64_t)h[bkt];
                    break;
                }
                above += (int64_t)h[bkt];
            }
            if (bucket < 0) fail(HM_EINVAL, "ilu: selection histogram inconsistent");
            prefix |= (uint32_t)bucket << shifts[pass];
            pmask |= (uint32_t)(nb - 1) << shifts[pass];
        }
        const uint32_t thr = prefix;      // bit pattern of the m-th largest |v|
        const int64_t n_gt = above;       // entries strictly larger
        const int64_t n_tie = in_bucket;  // entries equal to it
        const int64_t need_tie = m - n_gt;
        DevBuf<int32_t> gi(std::max<int64_t>(n_gt, 1)), gj(std::max<int64_t>(n_gt, 1)),
            ti(std::max<int64_t>(n_tie, 1)), tj(std::max<int64_t>(n_tie, 1));
        DevBuf<float> gv(std::max<int64_t>(n_gt, 1)), tv(std::max<int64_t>(n_tie, 1));
        DevBuf<unsigned long long> cnt(2);
        HM_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), st));
        k_sel_compact<<<nl, SEL_NT, 0, st>>>(H.leaves.p, d_true.p, d_zidx.p, H.near.p, thr, gi.p, gj.p, gv.p, cnt.p,
                                             n_gt, ti.p, tj.p, tv.p, n_tie);
        HM_LAUNCH_CHECK();
        unsigned long long hc[2];
        HM_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if ((int64_t)hc[0] != n_gt || (int64_t)hc[1] != n_tie) fail(HM_EINVAL, "ilu: selection counts inconsistent");
        std::vector<int32_t> I(m), J(m), TI(n_tie), TJ(n_tie);
        std::vector<float> Vf(n_gt), TV(n_tie);
        std::vector<double> V(m);
        if (n_gt > 0) {
            HM_CUDA(cudaMemcpyAsync(I.data(), gi.p, n_gt * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaMemcpyAsync(J.data(), gj.p, n_gt * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaMemcpyAsync(Vf.data(), gv.p, n_gt * 4, cudaMemcpyDeviceToHost, st));
        }
        if (n_tie > 0) {
            HM_CUDA(cudaMemcpyAsync(TI.data(), ti.p, n_tie * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaMemcpyAsync(TJ.data(), tj.p, n_tie * 4, cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaMemcpyAsync(TV.data(), tv.p, n_tie * 4, cudaMemcpyDeviceToHost, st));
        }
        HM_CUDA(cudaStreamSynchronize(st));
        for (int64_t q = 0; q < n_gt; ++q) V[q] = (double)Vf[q];
        // ties at the threshold: the first need_tie in (row, column) order
        std::vector<int64_t> o(n_tie);
        std::iota(o.begin(), o.end(), (int64_t)0);
        std::sort(o.begin(), o.end(),
                  [&](int64_t a, int64_t b) { return TI[a] != TI[b] ? TI[a] < TI[b] : TJ[a] < TJ[b]; });
        for (int64_t t = 0; t < need_tie; ++t) {
            I[n_gt + t] = TI[o[t]];
            J[n_gt + t] = TJ[o[t]];
            V[n_gt + t] = (double)TV[o[t]];
        }
        P->m_selected = m;
        int64_t mt = m;  // entries of the pattern besides the diagonal
        if (self_blocks) {
            // the off-diagonal entries of every element's 3x3 block not selected already
            std::vector<uint8_t> have((size_t)n * 3, 0);
            for (int64_t q = 0; q < m; ++q)
                if (I[q] / 3 == J[q] / 3) have[(size_t)3 * I[q] + J[q] % 3] = 1;
            for (int64_t r = 0; r < n; ++r)
                for (int j = 0; j < 3; ++j) {
                    const int64_t c = 3 * (r / 3) + j;
                    if (c == r || have[(size_t)3 * r + j]) continue;
                    I.push_back((int32_t)r);
                    J.push_back((int32_t)c);
                    V.push_back(0.0);
                    ++mt;
                }
        }
        // CSR in cluster order (diagonal added, no shift), colours, the colour order
        std::vector<int64_t> idx(mt);
        std::iota(idx.begin(), idx.end(), (int64_t)0);
        std::vector<double> zero(n, 0.0);
        std::vector<int64_t> rp(n + 1);
        std::vector<int32_t> cl(mt + n);
        std::vector<double> vl(mt + n);
        int64_t nnz = 0;
        hm_status s1 = hm_ilu_assemble((int32_t)n, mt, mt, idx.data(), I.data(), J.data(), V.data(), zero.data(),
                                       nullptr, rp.data(), cl.data(), vl.data(), &nnz);
        if (s1 != HM_OK) fail(s1, "ilu: assembling the selected pattern failed");
        std::vector<int32_t> leaf_of(n);
        for (int l = 0; l < nl; ++l)
            for (int r = 0; r < 3 * H.h_leaves[l].n; ++r) leaf_of[3 * H.h_leaves[l].begin + r] = l;
        std::vector<int32_t> colour(nl);
        int32_t nc = 0;
        hm_status s2 = hm_ilu_leaf_colours((int32_t)n, rp.data(), cl.data(), leaf_of.data(), nl, colour.data(), &nc);
        if (s2 != HM_OK) fail(s2, "ilu: colouring the leaves failed");
        P->n_colours = nc;
        // schedule: leaves by (colour, ordinal); rows leaf by leaf
        std::vector<int32_t> sched(nl);
        std::iota(sched.begin(), sched.end(), 0);
        std::stable_sort(sched.begin(), sched.end(), [&](int32_t a, int32_t b) { return colour[a] < colour[b]; });
        P->h_order.assign(n, 0);
        P->h_row0.assign(nl, 0);
        std::vector<int32_t> nrows(nl);
        P->h_colour_first.assign(nc + 1, nl);
        int64_t pos = 0;
        for (int s = 0; s < nl; ++s) {
            const int l = sched[s];
            if (s == 0 || colour[sched[s - 1]] != colour[l]) P->h_colour_first[colour[l]] = s;
            const LeafDesc& L = H.h_leaves[l];
            P->h_row0[s] = (int32_t)pos;
            nrows[s] = 3 * L.n;
            for (int r = 0; r < 3 * L.n; ++r) P->h_order[pos++] = 3 * L.begin + r;
            P->max_leaf_rows = std::max(P->max_leaf_rows, 3 * L.n);
        }
        if (P->max_leaf_rows > ILU_ROWS) fail(HM_EINVAL, "ilu: leaves of more than 64 elements are not supported");
        P->h_sched = sched;
        std::vector<int64_t> rp2(n + 1);
        std::vector<int32_t> cl2(mt + n);
        std::vector<double> vl2(mt + n);
        int64_t nnz2 = 0;
        hm_status s3 = hm_ilu_assemble((int32_t)n, mt, mt, idx.data(), I.data(), J.data(), V.data(), zero.data(),
                                       P->h_order.data(), rp2.data(), cl2.data(), vl2.data(), &nnz2);
        if (s3 != HM_OK) fail(s3, "ilu: assembling the ordered pattern failed");
        P->nnz = nnz2;
        std::vector<int64_t> dpos(n);
        for (int64_t a = 0; a < n; ++a) {
            dpos[a] = -1;
            for (int64_t q = rp2[a]; q < rp2[a + 1]; ++q)
                if (cl2[q] == a) dpos[a] = q;
        }
        if (self_blocks) {
            std::vector<int32_t> pos_of(n);
            for (int64_t a = 0; a < n; ++a) pos_of[P->h_order[a]] = (int32_t)a;
            std::vector<int64_t> spos((size_t)3 * n, -1);
            for (int64_t a = 0; a < n; ++a) {
                const int32_t r = P->h_order[a];
                for (int j = 0; j < 3; ++j) {
                    const int32_t c = pos_of[3 * (r / 3) + j];
                    for (int64_t q = rp2[a]; q < rp2[a + 1]; ++q)
                        if (cl2[q] == c) spos[(size_t)3 * a + j] = q;
                    if (spos[(size_t)3 * a + j] < 0) fail(HM_EINVAL, "ilu: an element block entry is missing");
                }
            }
            P->selfpos.upload(spos, st);
        }
        for (int s = 0; s < nl; ++s)
            P->max_leaf_nnz = std::max(P->max_leaf_nnz, rp2[P->h_row0[s] + nrows[s]] - rp2[P->h_row0[s]]);
        cl2.resize(nnz2);
        vl2.resize(nnz2);
        // levels of the lower triangle: the factorization runs level by level
        {
            std::vector<int32_t> lo(n), up(n);
            int32_t nlo = 0, nup = 0;
            hm_status s4 = hm_ilu_levels((int32_t)n, rp2.data(), cl2.data(), lo.data(), up.data(), &nlo, &nup);
            if (s4 != HM_OK) fail(s4, "ilu: levels of the pattern failed");
            std::vector<int32_t> cnt(nlo + 1, 0), rows_by(n);
            for (int64_t a = 0; a < n; ++a) ++cnt[lo[a] + 1];
            for (int q = 0; q < nlo; ++q) cnt[q + 1] += cnt[q];
            P->h_level_first = cnt;
            std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
            for (int64_t a = 0; a < n; ++a) rows_by[fill[lo[a]]++] = (int32_t)a;
            P->level_rows.upload(rows_by, st);
        }
        P->order.upload(P->h_order, st);
        P->rowptr.upload(rp2, st);
        P->col.upload(cl2, st);
        P->aval.upload(vl2, st);
        P->diagpos.upload(dpos, st);
        P->lu.alloc(nnz2);
        P->sched_row0.upload(P->h_row0, st);
        P->sched_nrows.upload(nrows, st);
        // levels inside each leaf (entries to other leaves are finished before)
        {
            std::vector<uint8_t> lrl(n), lvl(n), lru(n), lvu(n);
            std::vector<int> lev(ILU_ROWS);
            for (int s = 0; s < nl; ++s) {
                const int32_t r0 = P->h_row0[s], nr = nrows[s], r1 = r0 + nr;
                for (int pass = 0; pass < 2; ++pass) {
                    int maxl = 0;
                    for (int t = 0; t < nr; ++t) {
                        const int i = pass == 0 ? t : nr - 1 - t;
                        const int64_t a = r0 + i;
                        int l = 0;
                        for (int64_t q = rp2[a]; q < rp2[a + 1]; ++q) {
                            const int32_t c = cl2[q];
                            const bool dep = pass == 0 ? (c >= r0 && c < a) : (c > a && c < r1);
                            if (dep) l = std::max(l, lev[c - r0] + 1);
                        }
                        lev[i] = l;
                        maxl = std::max(maxl, l);
                    }
                    if (maxl > 255) fail(HM_EINVAL, "ilu: more than 256 levels inside a leaf");
                    std::vector<int> idx(nr);
                    std::iota(idx.begin(), idx.end(), 0);
                    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return lev[x] < lev[y]; });
                    for (int t = 0; t < nr; ++t) {
                        (pass == 0 ? lrl : lru)[r0 + t] = (uint8_t)idx[t];
                        (pass == 0 ? lvl : lvu)[r0 + t] = (uint8_t)lev[idx[t]];
                    }
                }
            }
            P->lrow_lo.upload(lrl, st);
            P->llev_lo.upload(lvl, st);
            P->lrow_up.upload(lru, st);
            P->llev_up.upload(lvu, st);
        }
        HM_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        delete P;
        throw;
    }
    H.ilu = P;
}

void ilu_factor(HMat& H, const double* d_cluster, const double* blk, cudaStream_t st, int* err_dev) {
    IluPlan& P = *H.ilu;
    if ((blk != nullptr) != P.self_blocks) fail(HM_EINVAL, "ilu: the plan was built for another interface term");
    k_ilu_init<<<gsz(P.nnz, 256), 256, 0, st>>>(P.aval.p, P.lu.p, P.nnz);
    k_ilu_diag<<<gsz(P.n, 256), 256, 0, st>>>(P.lu.p, P.diagpos.p, P.order.p, d_cluster, P.n);
    if (blk) k_ilu_self<<<gsz(P.n, 256), 256, 0, st>>>(P.lu.p, P.selfpos.p, P.order.p, blk, P.n);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaMemsetAsync(err_dev, 0, sizeof(int), st));
    const int nlev = (int)P.h_level_first.size() - 1;
    for (int l = 0; l < nlev; ++l) {
        const int f = P.h_level_first[l], cnt = P.h_level_first[l + 1] - f;
        if (cnt <= 0) continue;
        k_ilu_factor_rows<<<gsz(cnt, 8), 256, 0, st>>>(P.level_rows.p + f, cnt, P.rowptr.p, P.col.p, P.diagpos.p,
                                                        P.lu.p, err_dev);
        HM_LAUNCH_CHECK();
    }
    int e = 0;
    HM_CUDA(cudaMemcpyAsync(&e, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (e) fail(HM_EBREAKDOWN, "ilu: zero pivot in the incomplete factorization");
    P.factored = true;
}

void ilu_apply(HMat& H, const double* v, double* z, float* zf, int nr, const int* done, int done_stride,
               cudaStream_t st) {
    IluPlan& P = *H.ilu;
    if (!P.factored) fail(HM_EINVAL, "ilu: not factored");
    if (P.nr_cap < nr) {
        P.yv.alloc((size_t)P.n * nr);
        P.zv.alloc((size_t)P.n * nr);
        P.nr_cap = nr;
    }
    const int64_t snnz = apply_smem_nnz(P);
    const size_t smem = ILU_STAGE_HEAD + (size_t)snnz * 12;
    static bool attr_done[64] = {};
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        const int big = 200 * 1024 + ILU_STAGE_HEAD;
        HM_CUDA(cudaFuncSetAttribute(k_ilu_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        HM_CUDA(cudaFuncSetAttribute(k_ilu_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    for (int c = 0; c < P.n_colours; ++c) {
        const int f = P.h_colour_first[c], e = P.h_colour_first[c + 1];
        if (e <= f) continue;
        k_ilu_fwd<<<e - f, 256, smem, st>>>(P.sched_row0.p + f, P.sched_nrows.p + f, P.rowptr.p, P.col.p,
                                            P.diagpos.p, P.lu.p, P.lrow_lo.p, P.llev_lo.p, P.order.p, v, P.yv.p, P.n,
                                            nr, (int)snnz, done, done_stride);
        HM_LAUNCH_CHECK();
    }
    for (int c = P.n_colours - 1; c >= 0; --c) {
        const int f = P.h_colour_first[c], e = P.h_colour_first[c + 1];
        if (e <= f) continue;
        k_ilu_bwd<<<e - f, 256, smem, st>>>(P.sched_row0.p + f, P.sched_nrows.p + f, P.rowptr.p, P.col.p,
                                            P.diagpos.p, P.lu.p, P.lrow_up.p, P.llev_up.p, P.order.p, P.yv.p, P.zv.p,
                                            z, zf, P.n, nr, (int)snnz, done, done_stride);
        HM_LAUNCH_CHECK();
    }
}

bool ilu_is_factored(const HMat& H) { return H.ilu && H.ilu->factored; }

void ilu_export(HMat& H, int64_t* n_out, int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr,
                int32_t* col, double* a_val, double* lu_val, cudaStream_t st) {
    IluPlan& P = *H.ilu;
    if (n_out) *n_out = P.n;
    if (nnz_out) *nnz_out = P.nnz;
    if (n_colours_out) *n_colours_out = P.n_colours;
    if (order) std::copy(P.h_order.begin(), P.h_order.end(), order);
    if (rowptr) HM_CUDA(cudaMemcpyAsync(rowptr, P.rowptr.p, P.rowptr.bytes(), cudaMemcpyDeviceToHost, st));
    if (col) HM_CUDA(cudaMemcpyAsync(col, P.col.p, P.col.bytes(), cudaMemcpyDeviceToHost, st));
    if (a_val) HM_CUDA(cudaMemcpyAsync(a_val, P.aval.p, P.aval.bytes(), cudaMemcpyDeviceToHost, st));
    if (lu_val) {
        if (!P.factored) fail(HM_EINVAL, "ilu_export: not factored");
        HM_CUDA(cudaMemcpyAsync(lu_val, P.lu.p, P.lu.bytes(), cudaMemcpyDeviceToHost, st));
    }
    HM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace hm
