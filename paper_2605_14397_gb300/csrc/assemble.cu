// H-matrix assembly on the device: influence blocks, dense near-field tiles, adaptive
// cross approximation of the admissible blocks and packing into leaf-major streams.
//
// The paper keeps near-field blocks of E dense and approximates far-field blocks by
// low-rank products (Sec. 3.1, following the H-matrix literature it cites); it does not
// state the compression algorithm.  Used here: ACA with element pivots -- a pivot step
// takes the 3 rows of one receiver element and the 3 columns of one source element,
// and eliminates the 3x3 pivot block with complete pivoting, adding up to 3 rank-one
// terms.  A block is a candidate for stopping when two consecutive steps satisfy
//     sum ||u_l||^2 ||v_l||^2 (this step)  <=  eps^2 ||S_k||_F^2,
// ||S_k||_F being the Frobenius norm of the current approximation (updated exactly
// from the factor Gram products); it stops once four unused rows drawn at random have
// residuals that, scaled to the whole block, stay within the same bound -- a row that
// fails becomes the next pivot (partial-pivot ACA can otherwise miss a part of the
// block).  Every coefficient is evaluated in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

#include "ddkernel.cuh"
#include "hmat_impl.h"

namespace hm {

// ------------------------------------------------------------------ influence blocks

__global__ void k_influence_pairs(const ElemRec* __restrict__ el, const int64_t* __restrict__ ri,
                                  const int64_t* __restrict__ sj, int64_t npairs, int64_t N, double mu,
                                  double nu, double* __restrict__ out, int* __restrict__ err) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int64_t i = ri[p], j = sj[p];
    double blk[9];
    if (i < 0 || i >= N || j < 0 || j >= N) {
        atomicOr(err, 2);
        for (int k = 0; k < 9; ++k) out[9 * p + k] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    if (!dd_block(el[i], el[j], mu, nu, blk)) atomicOr(err, 1);
#pragma unroll
    for (int k = 0; k < 9; ++k) out[9 * p + k] = blk[k];
}

void influence_pairs(const hm_elements& e, double E, double nu, int64_t npairs, const int64_t* ri,
                     const int64_t* sj, double* out, cudaStream_t st) {
    if (npairs < 0) fail(HM_EINVAL, "influence_blocks: npairs < 0");
    if (npairs == 0) return;
    if (!ri || !sj || !out) fail(HM_EINVAL, "influence_blocks: NULL pointer");
    if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5)) fail(HM_EINVAL, "influence_blocks: need E > 0 and -1 < nu < 0.5");
    std::vector<ElemRec> h(e.N);
    for (int64_t i = 0; i < e.N; ++i) {
        for (int d = 0; d < 3; ++d) {
            h[i].c[d] = e.c[3 * i + d];
            h[i].s1[d] = e.s1[3 * i + d];
            h[i].s2[d] = e.s2[3 * i + d];
            h[i].n[d] = e.n[3 * i + d];
        }
        h[i].a = e.a[i];
        h[i].b = e.b[i];
        h[i].pad[0] = h[i].pad[1] = 0.0;
    }
    DevBuf<ElemRec> d_el;
    d_el.upload(h, st);
    DevBuf<int> d_err(1);
    HM_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
    const double mu = E / (2.0 * (1.0 + nu));
    const int nt = 128;
    k_influence_pairs<<<(unsigned)ceil_div(npairs, nt), nt, 0, st>>>(d_el.p, ri, sj, npairs, e.N, mu, nu, out,
                                                                    d_err.p);
    HM_LAUNCH_CHECK();
    int herr = 0;
    HM_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (herr & 2) fail(HM_EINVAL, "influence_blocks: element index out of range");
    if (herr & 1) fail(HM_ESINGULAR_GEOM, "influence_blocks: a receiver lies on a source element edge");
}

// ------------------------------------------------------------------ near field

struct NearJob {
    int32_t s_begin, s_n, t_begin, t_n;
    int32_t ld, pad_;
    int64_t off;
};

__global__ void __launch_bounds__(256) k_near_fill(const ElemRec* __restrict__ el, const NearJob* __restrict__ jobs,
                                                   float* __restrict__ near, double mu, double nu,
                                                   int* __restrict__ err) {
    const NearJob J = jobs[blockIdx.x];
    const int npair = J.s_n * J.t_n;
    for (int q = threadIdx.x; q < npair; q += blockDim.x) {
        const int i = q % J.s_n, j = q / J.s_n;
        double blk[9];
        if (!dd_block(el[J.s_begin + i], el[J.t_begin + j], mu, nu, blk)) atomicOr(err, 1);
        float* col = near + J.off + (int64_t)(3 * j) * J.ld + 3 * i;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int a = 0; a < 3; ++a) col[(int64_t)m * J.ld + a] = (float)blk[3 * a + m];
    }
}

// ------------------------------------------------------------------ ACA

struct AcaJob {
    int32_t s_begin, s_n, t_begin, t_n;
    int64_t ws_off;  // workspace: U (3 s_n x (R+3)) then V (3 t_n x (R+3)), FP64 column-major
};

constexpr int ACA_NT = 256;
constexpr int ACA_NW = ACA_NT / 32;

__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide argmax of (value, index); every thread gets the result
__device__ void block_argmax(double& v, int& i, double* sv, int* si) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    warp_argmax(v, i);
    __syncthreads();
    if (lane == 0) { sv[w] = v; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        v = lane < ACA_NW ? sv[lane] : -1.0;
        i = lane < ACA_NW ? si[lane] : 0x7fffffff;
        warp_argmax(v, i);
        if (lane == 0) { sv[0] = v; si[0] = i; }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
}

__device__ double block_sum(double v, double* sv) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sv[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < ACA_NW ? sv[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) sv[0] = v;
    }
    __syncthreads();
    return sv[0];
}

constexpr int ACA_CHECKS = 4;  // random rows that must confirm convergence

// An unused row element chosen by a hash of (block, check, rank); -1 if none is left.
__device__ int random_unused_row(const uint32_t* used, int n, unsigned blk, int check, int k, int* s_next) {
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t h = blk * 2654435761u ^ (uint32_t)(check + 1) * 40503u ^ (uint32_t)(k + 7) * 2246822519u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const int start = (int)(h % (uint32_t)n);
        int found = -1;
        for (int d = 0; d < n; ++d) {
            const int i = (start + d) % n;
            if (!(used[i >> 5] & (1u << (i & 31)))) { found = i; break; }
        }
        *s_next = found;
    }
    __syncthreads();
    return *s_next;
}

__global__ void __launch_bounds__(ACA_NT) k_aca(const ElemRec* __restrict__ el, const AcaJob* __restrict__ jobs,
                                                double* __restrict__ ws, int R, double eps, double mu, double nu,
                                                int32_t* __restrict__ rank_out, int32_t* __restrict__ status_out) {
    extern __shared__ uint32_t used[];  // one bit per row element of S
    __shared__ double sv[ACA_NW];
    __shared__ int si[ACA_NW];
    __shared__ double urow[3 * 132];    // U[l][3 ipiv + p] for l < k (R <= 128)
    __shared__ double vcol[3 * 132];    // V[l][3 jpiv + q]
    __shared__ double piv[3][3];
    __shared__ int s_pe, s_qe, s_go;
    __shared__ double s_pv;
    __shared__ double gram_u[132], gram_v[132];
    __shared__ int s_next;

    const AcaJob J = jobs[blockIdx.x];
    const int tid = threadIdx.x;
    const int mS = 3 * J.s_n, mT = 3 * J.t_n;
    double* U = ws + J.ws_off;
    double* V = U + (size_t)mS * (R + 3);
    double* Cc = U + (size_t)mS * R;  // 3 residual columns
    double* Rr = V + (size_t)mT * R;  // 3 residual rows
    const int nwords = (J.s_n + 31) >> 5;
    for (int w = tid; w < nwords; w += ACA_NT) used[w] = 0u;
    __syncthreads();

    int k = 0, status = 0, streak = 0, ipiv = 0, checks = 0;
    bool checking = false;
    double nrm2 = 0.0;
    const int kmax = min(R, min(mS, mT));
    for (int step = 0; step < J.s_n; ++step) {
        if (k + 3 > R && k < kmax) { status = 1; break; }
        // (1) residual rows of receiver element ipiv
        for (int l = tid; l < 3 * k; l += ACA_NT) urow[l] = U[(size_t)(l / 3) * mS + 3 * ipiv + (l % 3)];
        if (tid == 0) used[ipiv >> 5] |= 1u << (ipiv & 31);
        __syncthreads();
        const ElemRec er = el[J.s_begin + ipiv];
        for (int j = tid; j < J.t_n; j += ACA_NT) {
            double blk[9];
            dd_block(er, el[J.t_begin + j], mu, nu, blk);
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    double val = blk[3 * p + m];
                    for (int l = 0; l < k; ++l) val -= urow[3 * l + p] * V[(size_t)l * mT + 3 * j + m];
                    Rr[(size_t)p * mT + 3 * j + m] = val;
                }
        }
        __syncthreads();
        if (checking) {
            // a check row passes if its residual, scaled to all rows, is within eps
            double r2 = 0.0;
            for (int c = tid; c < 3 * mT; c += ACA_NT) {
                const double v = Rr[(size_t)(c / mT) * mT + (c % mT)];
                r2 += v * v;
            }
            r2 = block_sum(r2, sv);
            if (r2 * (double)J.s_n <= eps * eps * nrm2) {
                if (++checks >= ACA_CHECKS) break;
                ipiv = random_unused_row(used, J.s_n, blockIdx.x, checks, k, &s_next);
                if (ipiv < 0) break;
                continue;
            }
            // missed part of the block: resume the cross approximation from this row
            checking = false;
            checks = 0;
            streak = 0;
        }
        // (2) column pivot: largest residual entry of the three rows
        double av = -1.0;
        int ai = 0x7fffffff;
        for (int c = tid; c < 3 * mT; c += ACA_NT) {
            const double v = fabs(Rr[(size_t)(c / mT) * mT + (c % mT)]);
            if (v > av || (v == av && c < ai)) { av = v; ai = c; }
        }
        block_argmax(av, ai, sv, si);
        if (!(av > 0.0)) {
            // the rows are reproduced exactly; move to the next unused row element
            int nxt = -1;
            for (int i = 0; i < J.s_n; ++i)
                if (!(used[i >> 5] & (1u << (i & 31)))) { nxt = i; break; }
            if (nxt < 0) break;
            ipiv = nxt;
            __syncthreads();
            continue;
        }
        const int jpiv = (ai % mT) / 3;
        // (3) residual columns of source element jpiv
        for (int l = tid; l < 3 * k; l += ACA_NT) vcol[l] = V[(size_t)(l / 3) * mT + 3 * jpiv + (l % 3)];
        __syncthreads();
        const ElemRec es = el[J.t_begin + jpiv];
        for (int i = tid; i < J.s_n; i += ACA_NT) {
            double blk[9];
            dd_block(el[J.s_begin + i], es, mu, nu, blk);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double val = blk[3 * a + q];
                    for (int l = 0; l < k; ++l) val -= U[(size_t)l * mS + 3 * i + a] * vcol[3 * l + q];
                    Cc[(size_t)q * mS + 3 * i + a] = val;
                }
        }
        __syncthreads();
        // (4) complete-pivoting elimination of the 3x3 pivot block
        if (tid < 9) piv[tid / 3][tid % 3] = Rr[(size_t)(tid / 3) * mT + 3 * jpiv + (tid % 3)];
        __syncthreads();
        int rowdone = 0, coldone = 0, nr = 0;
        double p0 = 0.0, step2 = 0.0;
        for (int e = 0; e < 3 && k + nr < kmax; ++e) {
            if (tid == 0) {
                double best = -1.0;
                int pe = -1, qe = -1;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q)
                        if (!(rowdone & (1 << p)) && !(coldone & (1 << q)) && fabs(piv[p][q]) > best) {
                            best = fabs(piv[p][q]);
                            pe = p;
                            qe = q;
                        }
                if (e == 0) p0 = best;
                s_go = (best > 1e-12 * p0 && best > 0.0) ? 1 : 0;
                s_pe = pe;
                s_qe = qe;
                s_pv = pe >= 0 ? piv[pe][qe] : 0.0;
            }
            __syncthreads();
            if (!s_go) break;
            const int pe = s_pe, qe = s_qe;
            const double pv = s_pv;
            if (e == 0) p0 = fabs(pv);
            double* Un = U + (size_t)(k + nr) * mS;
            double* Vn = V + (size_t)(k + nr) * mT;
            const double inv = 1.0 / pv;
            for (int r = tid; r < mS; r += ACA_NT) Un[r] = Cc[(size_t)qe * mS + r] * inv;
            for (int c = tid; c < mT; c += ACA_NT) Vn[c] = Rr[(size_t)pe * mT + c];
            __syncthreads();
            rowdone |= 1 << pe;
            coldone |= 1 << qe;
            // eliminate from the remaining rows and columns
            for (int p = 0; p < 3; ++p) {
                if (rowdone & (1 << p)) continue;
                const double f = Un[3 * ipiv + p];
                for (int c = tid; c < mT; c += ACA_NT) Rr[(size_t)p * mT + c] -= f * Vn[c];
            }
            for (int q = 0; q < 3; ++q) {
                if (coldone & (1 << q)) continue;
                const double f = Vn[3 * jpiv + q];
                for (int r = tid; r < mS; r += ACA_NT) Cc[(size_t)q * mS + r] -= Un[r] * f;
            }
            __syncthreads();
            if (tid < 9) piv[tid / 3][tid % 3] = Rr[(size_t)(tid / 3) * mT + 3 * jpiv + (tid % 3)];
            // (5) norm update: ||S||^2 += ||u||^2 ||v||^2 + 2 sum_{l < new} (u.u_l)(v.v_l)
            const int lnew = k + nr;
            double su = 0.0, svv = 0.0;
            for (int r = tid; r < mS; r += ACA_NT) su += Un[r] * Un[r];
            for (int c = tid; c < mT; c += ACA_NT) svv += Vn[c] * Vn[c];
            const double nu2 = block_sum(su, sv);
            const double nv2 = block_sum(svv, sv);
            // Gram rows with the previous terms, one warp per previous term
            const int lane = tid & 31, w = tid >> 5;
            for (int l = w; l < lnew; l += ACA_NW) {
                const double* Ul = U + (size_t)l * mS;
                const double* Vl = V + (size_t)l * mT;
                double a = 0.0, b = 0.0;
                for (int r = lane; r < mS; r += 32) a += Un[r] * Ul[r];
                for (int c = lane; c < mT; c += 32) b += Vn[c] * Vl[c];
                a = warp_sum(a);
                b = warp_sum(b);
                if (lane == 0) { gram_u[l] = a; gram_v[l] = b; }
            }
            __syncthreads();
            double cross = 0.0;
            for (int l = 0; l < lnew; ++l) cross += gram_u[l] * gram_v[l];
            nrm2 += nu2 * nv2 + 2.0 * cross;
            step2 += nu2 * nv2;
            ++nr;
            __syncthreads();
        }
        if (nr == 0) {
            // pivot block numerically zero: treat the row element as exhausted
            int nxt = -1;
            for (int i = 0; i < J.s_n; ++i)
                if (!(used[i >> 5] & (1u << (i & 31)))) { nxt = i; break; }
            if (nxt < 0) break;
            ipiv = nxt;
            __syncthreads();
            continue;
        }
        k += nr;
        streak = (step2 <= eps * eps * nrm2) ? streak + 1 : 0;
        if (k >= kmax) break;
        if (streak >= 2) {
            // verify on unused rows drawn at random before accepting the approximation
            checking = true;
            ipiv = random_unused_row(used, J.s_n, blockIdx.x, checks, k, &s_next);
            if (ipiv < 0) break;
            continue;
        }
        // (6) next row pivot: unused element with the largest entry of the last u
        const double* Ul = U + (size_t)(k - 1) * mS;
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int i = tid; i < J.s_n; i += ACA_NT) {
            if (used[i >> 5] & (1u << (i & 31))) continue;
            const double v = fmax(fabs(Ul[3 * i]), fmax(fabs(Ul[3 * i + 1]), fabs(Ul[3 * i + 2])));
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        block_argmax(bv, bi, sv, si);
        if (bv < 0.0) break;  // every row element used
        ipiv = bi;
        __syncthreads();
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = k;
        status_out[blockIdx.x] = status;
    }
}


// ------------------------------------------------------------------ recompression
//
// The ACA factors are recompressed in FP64 (orthogonal factors also make the FP32/BF16
// rounding of the stored factors harmless: no cancellation between rank-one terms):
//   U = Q_U R_U, V = Q_V R_V  (classical Gram-Schmidt applied twice),
//   R_U R_V^T = W S Z^T       (one-sided Jacobi SVD, round-robin pairs),
//   keep the k leading singular triplets with sum_{j>=k} s_j^2 <= tau^2 sum_j s_j^2,
//   U <- Q_U (W S)_k,  V <- Q_V Z_k.

struct RecJob {
    int64_t ws_off;  // ACA workspace of the block (U then V)
    int64_t sm_off;  // small workspace: R_U, R_V, M, Z (r x r each) then the order (r)
    int32_t mS, mT, r, R;
};

__device__ void cgs2_qr(double* A, int m, int r, double* Rm, double* cbuf, double* sv) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int q = tid; q < r * r; q += ACA_NT) Rm[q] = 0.0;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        double* aj = A + (size_t)j * m;
        double o2 = 0.0;
        for (int row = tid; row < m; row += ACA_NT) o2 += aj[row] * aj[row];
        const double orig = sqrt(block_sum(o2, sv));
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = w; i < j; i += ACA_NW) {
                const double* qi = A + (size_t)i * m;
                double d = 0.0;
                for (int row = lane; row < m; row += 32) d += qi[row] * aj[row];
                d = warp_sum(d);
                if (lane == 0) cbuf[i] = d;
            }
            __syncthreads();
            for (int row = tid; row < m; row += ACA_NT) {
                double v = aj[row];
                for (int i = 0; i < j; ++i) v -= cbuf[i] * A[(size_t)i * m + row];
                aj[row] = v;
            }
            for (int i = tid; i < j; i += ACA_NT) Rm[(size_t)j * r + i] += cbuf[i];
            __syncthreads();
        }
        double n2 = 0.0;
        for (int row = tid; row < m; row += ACA_NT) n2 += aj[row] * aj[row];
        const double nrm = sqrt(block_sum(n2, sv));
        const bool keep = nrm > 1e-13 * orig && nrm > 0.0;
        const double sc = keep ? 1.0 / nrm : 0.0;
        for (int row = tid; row < m; row += ACA_NT) aj[row] *= sc;
        if (tid == 0) Rm[(size_t)j * r + j] = keep ? nrm : 0.0;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(ACA_NT) k_recompress(const RecJob* __restrict__ jobs, double* __restrict__ ws,
                                                       double* __restrict__ small, double tau,
                                                       int32_t* __restrict__ rank_out) {
    __shared__ double sv[ACA_NW];
    __shared__ double cbuf[132];
    __shared__ double sig[132];
    __shared__ int s_rot;
    const RecJob J = jobs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int r = J.r;
    if (r == 0) {
        if (tid == 0) rank_out[blockIdx.x] = 0;
        return;
    }
    double* U = ws + J.ws_off;
    double* V = U + (size_t)J.mS * (J.R + 3);
    double* RU = small + J.sm_off;
    double* RV = RU + (size_t)r * r;
    double* M = RV + (size_t)r * r;
    double* Z = M + (size_t)r * r;
    double* ord = Z + (size_t)r * r;
    cgs2_qr(U, J.mS, r, RU, cbuf, sv);
    cgs2_qr(V, J.mT, r, RV, cbuf, sv);
    // M = R_U R_V^T (column-major), Z = I
    for (int q = tid; q < r * r; q += ACA_NT) {
        const int i = q % r, j = q / r;
        double s = 0.0;
        for (int l = max(i, j); l < r; ++l) s += RU[(size_t)l * r + i] * RV[(size_t)l * r + j];
        M[q] = s;
        Z[q] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // one-sided Jacobi on the columns of M
    const int n = (r + 1) & ~1;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int t = 0; t < n - 1; ++t) {
            for (int k = w; k < n / 2; k += ACA_NW) {
                int p = (t + k) % (n - 1);
                int q = k == 0 ? n - 1 : (t - k + n - 1) % (n - 1);
                if (p >= r || q >= r) continue;
                if (p > q) { const int tt = p; p = q; q = tt; }
                double* mp = M + (size_t)p * r;
                double* mq = M + (size_t)q * r;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = lane; i < r; i += 32) {
                    a += mp[i] * mp[i];
                    b += mq[i] * mq[i];
                    g += mp[i] * mq[i];
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (g != 0.0 && fabs(g) > 1e-15 * sqrt(a * b)) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
                    double* zp = Z + (size_t)p * r;
                    double* zq = Z + (size_t)q * r;
                    for (int i = lane; i < r; i += 32) {
                        const double x = mp[i], y = mq[i];
                        mp[i] = c * x - s * y;
                        mq[i] = s * x + c * y;
                        const double u = zp[i], v = zq[i];
                        zp[i] = c * u - s * v;
                        zq[i] = s * u + c * v;
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (!rot) break;
    }
    // singular values, order by decreasing value, truncation rank
    for (int j = w; j < r; j += ACA_NW) {
        double a = 0.0;
        for (int i = lane; i < r; i += 32) a += M[(size_t)j * r + i] * M[(size_t)j * r + i];
        a = warp_sum(a);
        if (lane == 0) sig[j] = a;  // squared
    }
    __syncthreads();
    if (tid == 0) {
        int idx[132];
        for (int j = 0; j < r; ++j) idx[j] = j;
        for (int a = 0; a < r; ++a) {
            int best = a;
            for (int b = a + 1; b < r; ++b)
                if (sig[idx[b]] > sig[idx[best]]) best = b;
            const int t = idx[a];
            idx[a] = idx[best];
            idx[best] = t;
        }
        double tot = 0.0;
        for (int j = 0; j < r; ++j) tot += sig[j];
        int k = r;
        double tail = 0.0;
        while (k > 0 && tail + sig[idx[k - 1]] <= tau * tau * tot) {
            tail += sig[idx[k - 1]];
            --k;
        }
        for (int j = 0; j < r; ++j) ord[j] = (double)idx[j];
        rank_out[blockIdx.x] = k;
    }
}

struct ExpandJob {
    int64_t ws_off, sm_off;
    int64_t dst;  // compact store offset: U (mS x k) then V (mT x k), FP32 column-major
    int32_t mS, mT, r, k, R, pad_;
};

__global__ void k_expand(const ExpandJob* __restrict__ jobs, const double* __restrict__ ws,
                         const double* __restrict__ small, float* __restrict__ store) {
    const ExpandJob J = jobs[blockIdx.x];
    const int r = J.r, k = J.k;
    const double* Q = ws + J.ws_off;
    const double* QV = Q + (size_t)J.mS * (J.R + 3);
    const double* M = small + J.sm_off + 2 * (size_t)r * r;
    const double* Z = M + (size_t)r * r;
    const double* ord = Z + (size_t)r * r;
    float* dU = store + J.dst;
    float* dV = dU + (size_t)J.mS * k;
    for (int64_t q = threadIdx.x; q < (int64_t)J.mS * k; q += blockDim.x) {
        const int row = (int)(q % J.mS), j = (int)(q / J.mS);
        const int o = (int)ord[j];
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += Q[(size_t)i * J.mS + row] * M[(size_t)o * r + i];
        dU[q] = (float)s;
    }
    for (int64_t q = threadIdx.x; q < (int64_t)J.mT * k; q += blockDim.x) {
        const int row = (int)(q % J.mT), j = (int)(q / J.mT);
        const int o = (int)ord[j];
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += QV[(size_t)i * J.mT + row] * Z[(size_t)o * r + i];
        dV[q] = (float)s;
    }
}

// ------------------------------------------------------------------ packing

struct PackJob {
    int64_t src;     // first entry of the slice in the compact store
    int64_t dst;     // first entry in the stream
    int32_t src_ld;  // rows of the whole factor (3 |cluster|)
    int32_t rows;    // rows of the slice (3 |leaf|)
    int32_t dst_ld;  // padded rows of the leaf
    int32_t ncols;   // rank
};

__device__ __forceinline__ uint16_t f2bf(float f) {
    // round to nearest even
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

template <class T>
__global__ void k_pack(const float* __restrict__ store, const PackJob* __restrict__ jobs, T* __restrict__ out) {
    const PackJob J = jobs[blockIdx.x];
    const int64_t tot = (int64_t)J.rows * J.ncols;
    for (int64_t q = threadIdx.x; q < tot; q += blockDim.x) {
        const int r = (int)(q % J.rows);
        const int c = (int)(q / J.rows);
        const float v = store[J.src + (int64_t)c * J.src_ld + r];
        if constexpr (sizeof(T) == 2)
            out[J.dst + (int64_t)c * J.dst_ld + r] = f2bf(v);
        else
            out[J.dst + (int64_t)c * J.dst_ld + r] = v;
    }
}

// ------------------------------------------------------------------ driver

void assemble(const Tree& T, const hm_assemble_opts& opt, cudaStream_t st, HMat& H) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (!(opt.E > 0.0) || !(opt.nu > -1.0 && opt.nu < 0.5)) fail(HM_EINVAL, "assemble: need E > 0 and -1 < nu < 0.5");
    if (!(opt.aca_eps > 0.0 && opt.aca_eps < 1.0)) fail(HM_EINVAL, "assemble: aca_eps must be in (0, 1)");
    if (opt.storage != HM_F32 && opt.storage != HM_BF16) fail(HM_EINVAL, "assemble: storage must be HM_F32 or HM_BF16");
    const int R = opt.max_rank > 0 ? opt.max_rank : 96;
    if (R > 128) fail(HM_EINVAL, "assemble: max_rank must be <= 128");
    if (T.leaf_size > 128) fail(HM_EINVAL, "assemble: leaf_size must be <= 128");
    if (T.N > (int64_t)1 << 30) fail(HM_EINVAL, "assemble: too many elements");

    H.N = T.N;
    H.ndof = 3 * T.N;
    H.E = opt.E;
    H.nu = opt.nu;
    H.eps = opt.aca_eps;
    H.storage = opt.storage;
    const double mu = opt.E / (2.0 * (1.0 + opt.nu));
    const double eps_aca = 0.1 * opt.aca_eps;  // cross approximation target
    const double tau = 0.5 * opt.aca_eps;      // SVD truncation target

    H.elems.upload(T.elems, st);
    H.h_perm = T.perm;
    std::vector<int32_t> perm32(T.N);
    for (int64_t k = 0; k < T.N; ++k) perm32[k] = (int32_t)T.perm[k];
    H.perm.upload(perm32, st);

    const int nl = (int)T.leaves.size();
    H.n_leaves = nl;
    H.h_leaves.assign(nl, LeafDesc{});
    for (int l = 0; l < nl; ++l) {
        const int64_t q = T.leaves[l];
        LeafDesc& L = H.h_leaves[l];
        L.begin = (int32_t)T.begin[q];
        L.n = (int32_t)(T.end[q] - T.begin[q]);
        L.ld = (int32_t)round_up(3 * L.n, 8);
    }
    // leaves under each node (a contiguous ordinal range)
    const int64_t nn = (int64_t)T.begin.size();
    std::vector<int32_t> lfirst(nn), lcount(nn);
    for (int64_t q = nn - 1; q >= 0; --q) {
        if (T.left[q] < 0) {
            lfirst[q] = (int32_t)T.leaf_of_node[q];
            lcount[q] = 1;
        } else {
            lfirst[q] = lfirst[T.left[q]];
            lcount[q] = lcount[T.left[q]] + lcount[T.right[q]];
        }
    }

    // ---- far field: ACA + recompression in batches bounded by a workspace budget
    const int64_t nf = (int64_t)T.far.size();
    H.n_far = nf;
    H.h_far.assign(nf, FarDesc{});
    for (int64_t b = 0; b < nf; ++b) {
        const int64_t s = T.far[b][0], t = T.far[b][1];
        FarDesc& F = H.h_far[b];
        F.s_begin = (int32_t)T.begin[s];
        F.s_n = (int32_t)(T.end[s] - T.begin[s]);
        F.t_begin = (int32_t)T.begin[t];
        F.t_n = (int32_t)(T.end[t] - T.begin[t]);
    }
    const int64_t budget = (int64_t)4 << 30;  // bytes of FP64 ACA workspace per batch
    std::vector<int32_t> ranks(nf, 0), stat(nf, 0), fin(nf, 0);
    std::vector<char> dense_far(nf, 0);
    int64_t store_len = 0;
    std::vector<int64_t> fac_off(nf, 0);
    std::vector<DevBuf<float>> chunks;
    std::vector<int64_t> chunk_base;
    DevBuf<double> ws, small;
    DevBuf<int32_t> d_rank, d_stat;
    int64_t b0 = 0;
    while (b0 < nf) {
        std::vector<AcaJob> jobs;
        int64_t wlen = 0;
        int max_sn = 0;
        int64_t b1 = b0;
        while (b1 < nf) {
            const FarDesc& F = H.h_far[b1];
            const int64_t need = (int64_t)(3 * F.s_n + 3 * F.t_n) * (R + 3);
            if (!jobs.empty() && (wlen + need) * 8 > budget) break;
            AcaJob J;
            J.s_begin = F.s_begin;
            J.s_n = F.s_n;
            J.t_begin = F.t_begin;
            J.t_n = F.t_n;
            J.ws_off = wlen;
            jobs.push_back(J);
            wlen += need;
            max_sn = std::max(max_sn, F.s_n);
            ++b1;
        }
        const int64_t nb = b1 - b0;
        if ((size_t)wlen > ws.n) ws.alloc(wlen);
        DevBuf<AcaJob> d_jobs;
        d_jobs.upload(jobs, st);
        if ((int64_t)d_rank.n < nb) { d_rank.alloc(nb); d_stat.alloc(nb); }
        const size_t smem = sizeof(uint32_t) * (size_t)((max_sn + 31) / 32);
        if (smem > 96 * 1024) fail(HM_EINVAL, "assemble: cluster too large for the ACA kernel");
        if (smem > 48 * 1024)
            HM_CUDA(cudaFuncSetAttribute(k_aca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_aca<<<(unsigned)nb, ACA_NT, smem, st>>>(H.elems.p, d_jobs.p, ws.p, R, eps_aca, mu, opt.nu, d_rank.p,
                                                  d_stat.p);
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaMemcpyAsync(ranks.data() + b0, d_rank.p, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaMemcpyAsync(stat.data() + b0, d_stat.p, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        // recompress the converged blocks
        std::vector<RecJob> rj;
        std::vector<int64_t> rj_block;
        int64_t slen = 0;
        for (int64_t b = b0; b < b1; ++b) {
            const FarDesc& F = H.h_far[b];
            if (stat[b] != 0) {
                if ((int64_t)9 * F.s_n * F.t_n > ((int64_t)1 << 26)) {
                    char buf[256];
                    snprintf(buf, sizeof(buf), "assemble: ACA of far block %lld (%d x %d elements) exceeded rank %d",
                             (long long)b, F.s_n, F.t_n, R);
                    fail(HM_EBREAKDOWN, buf);
                }
                dense_far[b] = 1;  // not compressible to the cap: keep it dense
                continue;
            }
            RecJob J;
            J.ws_off = jobs[b - b0].ws_off;
            J.sm_off = slen;
            J.mS = 3 * F.s_n;
            J.mT = 3 * F.t_n;
            J.r = ranks[b];
            J.R = R;
            rj.push_back(J);
            rj_block.push_back(b);
            slen += 4LL * J.r * J.r + J.r;
        }
        std::vector<int32_t> krank(rj.size(), 0);
        if (!rj.empty()) {
            if ((size_t)slen > small.n) small.alloc(std::max<int64_t>(slen, 1));
            DevBuf<RecJob> d_rj;
            d_rj.upload(rj, st);
            k_recompress<<<(unsigned)rj.size(), ACA_NT, 0, st>>>(d_rj.p, ws.p, small.p, tau, d_rank.p);
            HM_LAUNCH_CHECK();
            HM_CUDA(cudaMemcpyAsync(krank.data(), d_rank.p, rj.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
        }
        // expand the low-rank blocks whose factors are smaller than the dense block
        std::vector<ExpandJob> ej;
        int64_t clen = 0;
        for (size_t q = 0; q < rj.size(); ++q) {
            const int64_t b = rj_block[q];
            const RecJob& J = rj[q];
            const int k = krank[q];
            if ((int64_t)k * (J.mS + J.mT) >= (int64_t)J.mS * J.mT) {
                dense_far[b] = 1;
                continue;
            }
            fin[b] = k;
            if (k == 0) continue;
            ExpandJob e;
            e.ws_off = J.ws_off;
            e.sm_off = J.sm_off;
            e.dst = clen;
            e.mS = J.mS;
            e.mT = J.mT;
            e.r = J.r;
            e.k = k;
            e.R = R;
            e.pad_ = 0;
            ej.push_back(e);
            fac_off[b] = store_len + clen;
            clen += (int64_t)k * (J.mS + J.mT);
        }
        chunks.emplace_back(std::max<int64_t>(clen, 1));
        chunk_base.push_back(store_len);
        if (!ej.empty()) {
            DevBuf<ExpandJob> d_ej;
            d_ej.upload(ej, st);
            k_expand<<<(unsigned)ej.size(), 256, 0, st>>>(d_ej.p, ws.p, small.p, chunks.back().p);
            HM_LAUNCH_CHECK();
            HM_CUDA(cudaStreamSynchronize(st));
        }
        store_len += clen;
        b0 = b1;
    }
    ws.release();
    small.release();
    H.facstore.alloc(std::max<int64_t>(store_len, 1));
    for (size_t c = 0; c < chunks.size(); ++c) {
        const int64_t len = (c + 1 < chunks.size() ? chunk_base[c + 1] : store_len) - chunk_base[c];
        if (len > 0)
            HM_CUDA(cudaMemcpyAsync(H.facstore.p + chunk_base[c], chunks[c].p, len * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
    }
    HM_CUDA(cudaStreamSynchronize(st));
    chunks.clear();

    // ---- near stream: near leaf pairs and the far blocks kept dense, by row leaf
    struct DenseTile {
        int32_t t_begin, t_n;
    };
    std::vector<std::vector<DenseTile>> tiles_by_row(nl);
    for (size_t b = 0; b < T.near.size(); ++b) {
        const int64_t s = T.near[b][0], t = T.near[b][1];
        tiles_by_row[T.leaf_of_node[s]].push_back({(int32_t)T.begin[t], (int32_t)(T.end[t] - T.begin[t])});
    }
    int64_t n_dense_far = 0;
    for (int64_t b = 0; b < nf; ++b) {
        if (!dense_far[b]) continue;
        ++n_dense_far;
        const int64_t s = T.far[b][0];
        for (int l = 0; l < lcount[s]; ++l)
            tiles_by_row[lfirst[s] + l].push_back({H.h_far[b].t_begin, H.h_far[b].t_n});
    }
    std::vector<NearJob> njobs;
    std::vector<int32_t> near_zidx;
    int64_t near_len = 0;
    H.near_entries = 0;
    for (int l = 0; l < nl; ++l) {
        LeafDesc& L = H.h_leaves[l];
        L.near_off = near_len;
        L.near_cbase = (int32_t)near_zidx.size();
        int cols = 0;
        for (const DenseTile& D : tiles_by_row[l]) {
            NearJob J;
            J.s_begin = L.begin;
            J.s_n = L.n;
            J.t_begin = D.t_begin;
            J.t_n = D.t_n;
            J.ld = L.ld;
            J.pad_ = 0;
            J.off = near_len + (int64_t)cols * L.ld;
            njobs.push_back(J);
            for (int c = 0; c < 3 * D.t_n; ++c) near_zidx.push_back(3 * D.t_begin + c);
            cols += 3 * D.t_n;
            H.near_entries += 9LL * L.n * D.t_n;
        }
        L.near_cols = cols;
        near_len += (int64_t)cols * L.ld;
    }
    H.n_near = (int64_t)T.near.size();
    H.n_dense_far = n_dense_far;
    H.near.alloc(std::max<int64_t>(near_len, 1));
    HM_CUDA(cudaMemsetAsync(H.near.p, 0, H.near.bytes(), st));
    DevBuf<int> d_err(1);
    HM_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
    if (!njobs.empty()) {
        DevBuf<NearJob> d_nj;
        d_nj.upload(njobs, st);
        k_near_fill<<<(unsigned)njobs.size(), 256, 0, st>>>(H.elems.p, d_nj.p, H.near.p, mu, opt.nu, d_err.p);
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaStreamSynchronize(st));
    }
    H.near_zidx.upload(near_zidx, st);

    // ---- ranks, partial-buffer and t-vector layout (low-rank blocks only)
    int64_t tb_len = 0, p_len = 0;
    H.far_entries = 0;
    H.rank_min = 1 << 30;
    H.rank_max = 0;
    double rsum = 0;
    int64_t nlr = 0;
    for (int64_t b = 0; b < nf; ++b) {
        FarDesc& F = H.h_far[b];
        F.rank = dense_far[b] ? 0 : fin[b];
        F.fac_off = fac_off[b];
        F.tb_off = tb_len;
        F.n_tleaves = lcount[T.far[b][1]];
        F.pbase = p_len;
        F.dense = dense_far[b];
        tb_len += F.rank;
        p_len += (int64_t)F.n_tleaves * F.rank;
        if (!dense_far[b]) {
            H.rank_min = std::min(H.rank_min, F.rank);
            H.rank_max = std::max(H.rank_max, F.rank);
            rsum += F.rank;
            ++nlr;
            H.far_entries += 3LL * F.rank * (F.s_n + F.t_n);
        }
    }
    if (nlr == 0) H.rank_min = 0;
    H.rank_mean = nlr ? rsum / (double)nlr : 0.0;
    H.tb_len = tb_len;
    H.p_len = p_len;

    std::vector<std::vector<int64_t>> far_by_row(nl), far_by_col(nl);
    for (int64_t b = 0; b < nf; ++b) {
        if (H.h_far[b].rank == 0) continue;
        const int64_t s = T.far[b][0], t = T.far[b][1];
        for (int l = 0; l < lcount[s]; ++l) far_by_row[lfirst[s] + l].push_back(b);
        for (int l = 0; l < lcount[t]; ++l) far_by_col[lfirst[t] + l].push_back(b);
    }

    // ---- U and V streams
    std::vector<PackJob> ujobs, vjobs;
    std::vector<int32_t> u_zidx, v_pidx;
    int64_t u_len = 0, v_len = 0;
    for (int l = 0; l < nl; ++l) {
        LeafDesc& L = H.h_leaves[l];
        L.u_off = u_len;
        L.u_cbase = (int32_t)u_zidx.size();
        int ucols = 0;
        for (int64_t b : far_by_row[l]) {
            const FarDesc& F = H.h_far[b];
            PackJob J;
            J.src = F.fac_off + 3LL * (L.begin - F.s_begin);
            J.dst = u_len + (int64_t)ucols * L.ld;
            J.src_ld = 3 * F.s_n;
            J.rows = 3 * L.n;
            J.dst_ld = L.ld;
            J.ncols = F.rank;
            ujobs.push_back(J);
            for (int c = 0; c < F.rank; ++c) u_zidx.push_back((int32_t)(F.tb_off + c));
            ucols += F.rank;
        }
        L.u_cols = ucols;
        u_len += (int64_t)ucols * L.ld;

        L.v_off = v_len;
        L.v_cbase = (int32_t)v_pidx.size();
        int vcols = 0;
        for (int64_t b : far_by_col[l]) {
            const FarDesc& F = H.h_far[b];
            const int64_t t = T.far[b][1];
            const int k = l - lfirst[t];  // which leaf of T
            PackJob J;
            J.src = F.fac_off + 3LL * F.s_n * F.rank + 3LL * (L.begin - F.t_begin);
            J.dst = v_len + (int64_t)vcols * L.ld;
            J.src_ld = 3 * F.t_n;
            J.rows = 3 * L.n;
            J.dst_ld = L.ld;
            J.ncols = F.rank;
            vjobs.push_back(J);
            for (int c = 0; c < F.rank; ++c) v_pidx.push_back((int32_t)(F.pbase + (int64_t)k * F.rank + c));
            vcols += F.rank;
        }
        L.v_cols = vcols;
        v_len += (int64_t)vcols * L.ld;
    }
    if (H.storage == HM_F32) {
        H.u32.alloc(std::max<int64_t>(u_len, 1));
        H.v32.alloc(std::max<int64_t>(v_len, 1));
        HM_CUDA(cudaMemsetAsync(H.u32.p, 0, H.u32.bytes(), st));
        HM_CUDA(cudaMemsetAsync(H.v32.p, 0, H.v32.bytes(), st));
    } else {
        H.u16.alloc(std::max<int64_t>(u_len, 1));
        H.v16.alloc(std::max<int64_t>(v_len, 1));
        HM_CUDA(cudaMemsetAsync(H.u16.p, 0, H.u16.bytes(), st));
        HM_CUDA(cudaMemsetAsync(H.v16.p, 0, H.v16.bytes(), st));
    }
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<PackJob>& pj = pass == 0 ? ujobs : vjobs;
        if (pj.empty()) continue;
        DevBuf<PackJob> d_p;
        d_p.upload(pj, st);
        if (H.storage == HM_F32)
            k_pack<float><<<(unsigned)pj.size(), 256, 0, st>>>(H.facstore.p, d_p.p, pass == 0 ? H.u32.p : H.v32.p);
        else
            k_pack<uint16_t><<<(unsigned)pj.size(), 256, 0, st>>>(H.facstore.p, d_p.p, pass == 0 ? H.u16.p : H.v16.p);
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaStreamSynchronize(st));
    }
    H.u_zidx.upload(u_zidx, st);
    H.v_pidx.upload(v_pidx, st);
    H.leaves.upload(H.h_leaves, st);
    H.far.upload(H.h_far, st);

    int herr = 0;
    HM_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (herr & 1) fail(HM_ESINGULAR_GEOM, "assemble: a collocation point lies on a source element edge");
    build_product_plan(H, st);
    ensure_product_scratch(H, 1, st);
    HM_CUDA(cudaStreamSynchronize(st));
    H.assemble_seconds = std::chrono::duration<double>(clk::now() - t0).count();
}

}  // namespace hm
