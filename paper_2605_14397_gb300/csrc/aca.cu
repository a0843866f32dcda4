// Compression of the admissible (far-field) blocks of E.
//
// The paper keeps near-field blocks of E dense and approximates far-field blocks by
// low-rank products (Sec. 3.1, following the H-matrix literature it cites); it does not
// state the compression algorithm.  Used here:
//
// Adaptive cross approximation with element pivots.  A step takes a receiver element,
// evaluates its 3 residual rows, picks the source element holding the largest residual
// entry among the element's not-yet-eliminated rows, evaluates its 3 residual columns
// and eliminates the 3x3 pivot block with complete pivoting: the first pivot is the
// largest entry; a further pivot is accepted only if it is at least PIVOT_GROWTH of the
// largest residual entry of its row and of its column (threshold pivoting, so that no
// rank-one term is much larger than the block).  Rows are retired one DOF at a time, so
// an element whose rows were not all eliminated can be a pivot again.
// A block is a candidate for stopping when two consecutive steps satisfy
//     sum ||u_l||^2 ||v_l||^2 (this step)  <=  eps^2 ||S_k||_F^2,
// ||S_k||_F being the Frobenius norm of the current approximation (updated exactly from
// the factor Gram products); it stops once ACA_CHECKS elements drawn at random have
// residual rows that, scaled to the whole block, stay within the same bound -- a row
// that fails becomes the next pivot.  Every coefficient is evaluated in FP64.
//
// Recompression in FP64 then orthogonalises the factors and truncates the rank (below).
#include <cmath>

#include "aca.h"
#include "ddkernel.cuh"

namespace hm {

namespace {

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

__device__ double block_max(double v, double* sv) {
    int dummy = 0;
    int* si = reinterpret_cast<int*>(sv + ACA_NW);
    block_argmax(v, dummy, sv, si);
    return v;
}

constexpr int ACA_CHECKS = 4;          // random elements that must confirm convergence
constexpr double PIVOT_GROWTH = 0.1;   // threshold for the 2nd and 3rd pivot of a step

__device__ __forceinline__ bool row_used(const uint32_t* used, int r) { return (used[r >> 5] >> (r & 31)) & 1u; }
__device__ __forceinline__ int free_rows(const uint32_t* used, int i) {
    return (row_used(used, 3 * i) ? 0 : 1) | (row_used(used, 3 * i + 1) ? 0 : 2) | (row_used(used, 3 * i + 2) ? 0 : 4);
}
__device__ __forceinline__ void mark_row(uint32_t* used, int r) { used[r >> 5] |= 1u << (r & 31); }

// An element with a row not yet eliminated, chosen by a hash of (block, check, rank);
// -1 if there is none.  Called by every thread of the CTA.
__device__ int random_free_element(const uint32_t* used, int n, unsigned blk, int check, int k, int* s_next) {
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
            if (free_rows(used, i)) { found = i; break; }
        }
        *s_next = found;
    }
    __syncthreads();
    return *s_next;
}

__global__ void __launch_bounds__(ACA_NT) k_aca(const ElemRec* __restrict__ el, const AcaJob* __restrict__ jobs,
                                                double* __restrict__ ws, int R, double eps, double mu, double nu,
                                                int32_t* __restrict__ rank_out, int32_t* __restrict__ status_out,
                                                unsigned long long* __restrict__ evals) {
    extern __shared__ __align__(16) double dyn[];
    double* urow = dyn;                  // U[l][3 ipiv + p] for l < k
    double* vcol = urow + 3 * (R + 3);   // V[l][3 jpiv + q]
    double* gram_u = vcol + 3 * (R + 3);
    double* gram_v = gram_u + (R + 3);
    uint32_t* used = reinterpret_cast<uint32_t*>(gram_v + (R + 3));  // one bit per DOF row of S
    __shared__ double sv[2 * ACA_NW];
    __shared__ int si[ACA_NW];
    __shared__ double piv[3][3];
    __shared__ int s_pe, s_qe, s_next;
    __shared__ double s_pv;

    const AcaJob J = jobs[blockIdx.x];
    const int tid = threadIdx.x;
    const int mS = 3 * J.s_n, mT = 3 * J.t_n;
    double* U = ws + J.ws_off;
    double* V = U + (size_t)mS * (R + 3);
    double* Cc = U + (size_t)mS * R;  // 3 residual columns
    double* Rr = V + (size_t)mT * R;  // 3 residual rows
    const int nwords = (mS + 31) >> 5;
    for (int w = tid; w < nwords; w += ACA_NT) used[w] = 0u;
    __syncthreads();

    int k = 0, status = 0, streak = 0, ipiv = 0, checks = 0;
    unsigned long long n_eval = 0;  // 3x3 blocks evaluated (thread 0's count)
    bool checking = false;
    double nrm2 = 0.0;
    const int kmax = min(R, min(mS, mT));
    for (int step = 0; step < mS + ACA_CHECKS + 1; ++step) {
        if (k + 3 > R && k < kmax) { status = 1; break; }
        // (1) residual rows of receiver element ipiv
        for (int l = tid; l < 3 * k; l += ACA_NT) urow[l] = U[(size_t)(l / 3) * mS + 3 * ipiv + (l % 3)];
        __syncthreads();
        const ElemRec& er = el[J.s_begin + ipiv];
        n_eval += J.t_n;
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
            // a check element passes if its residual rows, scaled to all rows, are within eps
            double r2 = 0.0;
            for (int c = tid; c < 3 * mT; c += ACA_NT) {
                const double v = Rr[(size_t)(c / mT) * mT + (c % mT)];
                r2 += v * v;
            }
            r2 = block_sum(r2, sv);
            if (r2 * (double)J.s_n <= eps * eps * nrm2) {
                if (tid == 0)
                    for (int p = 0; p < 3; ++p) mark_row(used, 3 * ipiv + p);
                if (++checks >= ACA_CHECKS) break;
                ipiv = random_free_element(used, J.s_n, blockIdx.x, checks, k, &s_next);
                if (ipiv < 0) break;
                continue;
            }
            // missed part of the block: resume the cross approximation from this element
            checking = false;
            checks = 0;
            streak = 0;
        }
        const int freemask = free_rows(used, ipiv);
        // (2) column pivot: largest residual entry among the element's free rows
        double av = -1.0;
        int ai = 0x7fffffff;
        for (int c = tid; c < 3 * mT; c += ACA_NT) {
            const int p = c / mT;
            if (!((freemask >> p) & 1)) continue;
            const double v = fabs(Rr[(size_t)p * mT + (c % mT)]);
            if (v > av || (v == av && c < ai)) { av = v; ai = c; }
        }
        block_argmax(av, ai, sv, si);
        if (!(av > 0.0)) {
            // the free rows are reproduced exactly: retire them, move to another element
            if (tid == 0)
                for (int p = 0; p < 3; ++p) mark_row(used, 3 * ipiv + p);
            ipiv = random_free_element(used, J.s_n, blockIdx.x, step + 100, k, &s_next);
            if (ipiv < 0) break;
            continue;
        }
        const int jpiv = (ai % mT) / 3;
        // (3) residual columns of source element jpiv
        for (int l = tid; l < 3 * k; l += ACA_NT) vcol[l] = V[(size_t)(l / 3) * mT + 3 * jpiv + (l % 3)];
        __syncthreads();
        const ElemRec& es = el[J.t_begin + jpiv];
        n_eval += J.s_n;
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
        // (4) elimination of the pivot block over the free rows, complete pivoting
        if (tid < 9) piv[tid / 3][tid % 3] = Rr[(size_t)(tid / 3) * mT + 3 * jpiv + (tid % 3)];
        __syncthreads();
        int rowdone = (~freemask) & 7, coldone = 0, nr = 0;
        double step2 = 0.0;
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
                s_pe = pe;
                s_qe = qe;
                s_pv = pe >= 0 ? piv[pe][qe] : 0.0;
            }
            __syncthreads();
            const int pe = s_pe, qe = s_qe;
            const double pv = s_pv;
            if (pe < 0 || !(fabs(pv) > 0.0)) break;
            if (e > 0) {
                double rm = 0.0, cm = 0.0;
                for (int c = tid; c < mT; c += ACA_NT) rm = fmax(rm, fabs(Rr[(size_t)pe * mT + c]));
                for (int r = tid; r < mS; r += ACA_NT) cm = fmax(cm, fabs(Cc[(size_t)qe * mS + r]));
                rm = block_max(rm, sv);
                cm = block_max(cm, sv);
                if (fabs(pv) < PIVOT_GROWTH * fmax(rm, cm)) break;
            }
            double* Un = U + (size_t)(k + nr) * mS;
            double* Vn = V + (size_t)(k + nr) * mT;
            const double inv = 1.0 / pv;
            for (int r = tid; r < mS; r += ACA_NT) Un[r] = Cc[(size_t)qe * mS + r] * inv;
            for (int c = tid; c < mT; c += ACA_NT) Vn[c] = Rr[(size_t)pe * mT + c];
            if (tid == 0) mark_row(used, 3 * ipiv + pe);
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
        k += nr;
        streak = (step2 <= eps * eps * nrm2) ? streak + 1 : 0;
        if (k >= kmax) {
            // full rank reproduces the block exactly; reaching the cap first is a failure
            if (kmax < min(mS, mT)) status = 1;
            break;
        }
        if (streak >= 2) {
            // verify on elements drawn at random before accepting the approximation
            checking = true;
            ipiv = random_free_element(used, J.s_n, blockIdx.x, checks, k, &s_next);
            if (ipiv < 0) break;
            continue;
        }
        // (6) next row pivot: the element whose free rows hold the largest entry of the last u
        const double* Ul = U + (size_t)(k - 1) * mS;
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int i = tid; i < J.s_n; i += ACA_NT) {
            const int fm = free_rows(used, i);
            if (!fm) continue;
            double v = 0.0;
            for (int p = 0; p < 3; ++p)
                if ((fm >> p) & 1) v = fmax(v, fabs(Ul[3 * i + p]));
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        block_argmax(bv, bi, sv, si);
        if (bv < 0.0) break;  // every row eliminated
        ipiv = bi;
        __syncthreads();
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = k;
        status_out[blockIdx.x] = status;
        if (evals) atomicAdd(evals, n_eval);
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

// One-sided Jacobi on the columns of the r x r matrix M (column-major), the rotations
// accumulated in Z: round-robin pairs, a warp per pair; stops after a sweep without a
// rotation (|g| <= thresh sqrt(a b) for every pair) or after max_sweeps.
template <typename T>
__device__ __forceinline__ void jacobi_sweeps(T* M, T* Z, int r, double thresh, int max_sweeps, int* s_rot) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = (r + 1) & ~1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) *s_rot = 0;
        __syncthreads();
        for (int t = 0; t < n - 1; ++t) {
            for (int k = w; k < n / 2; k += ACA_NW) {
                int p = (t + k) % (n - 1);
                int q = k == 0 ? n - 1 : (t - k + n - 1) % (n - 1);
                if (p >= r || q >= r) continue;
                if (p > q) { const int tt = p; p = q; q = tt; }
                T* mp = M + (size_t)p * r;
                T* mq = M + (size_t)q * r;
                T a = 0, b = 0, g = 0;
                for (int i = lane; i < r; i += 32) {
                    a += mp[i] * mp[i];
                    b += mq[i] * mq[i];
                    g += mp[i] * mq[i];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (g != T(0) && fabs((double)g) > thresh * sqrt((double)a * (double)b)) {
                    const T zeta = (b - a) / (T(2) * g);
                    const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                    const T c = T(1) / sqrt(T(1) + tt * tt), sn = c * tt;
                    T* zp = Z + (size_t)p * r;
                    T* zq = Z + (size_t)q * r;
                    for (int i = lane; i < r; i += 32) {
                        const T x = mp[i], y = mq[i];
                        mp[i] = c * x - sn * y;
                        mq[i] = sn * x + c * y;
                        const T u = zp[i], v = zq[i];
                        zp[i] = c * u - sn * v;
                        zq[i] = sn * u + c * v;
                    }
                    if (lane == 0) *s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int rot = *s_rot;
        __syncthreads();
        if (!rot) break;
    }
}

__global__ void __launch_bounds__(ACA_NT) k_recompress(const RecJob* __restrict__ jobs, double* __restrict__ ws,
                                                       double* __restrict__ small, double tau,
                                                       int32_t* __restrict__ rank_out) {
    const int J0R = jobs[blockIdx.x].R;
    extern __shared__ __align__(16) double dyn[];
    double* cbuf = dyn;               // R + 3
    double* sig = cbuf + (J0R + 3);   // R + 3
    int* idx = reinterpret_cast<int*>(sig + (J0R + 3));
    __shared__ double sv[ACA_NW];
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
    // one-sided Jacobi on the columns of M: sweeps on an FP32 copy to FP32 convergence,
    // then the accumulated rotations made orthonormal in FP64 (CGS2), M <- M Z in FP64
    // and FP64 sweeps to the end (one or two: the columns are nearly orthogonal already).
    // Z stays orthogonal and M = M_0 Z to FP64 rounding whatever the FP32 phase did; it
    // only spares most of the FP64 sweeps (the FP64 pipe bounds this kernel on GB300).
    float* Mf = reinterpret_cast<float*>(ord + r);
    float* Zf = Mf + (size_t)r * r;
    double f2 = 0.0;
    for (int q = tid; q < r * r; q += ACA_NT) f2 += M[q] * M[q];
    const double fn = sqrt(block_sum(f2, sv));  // rotations do not see the scale: M / ||M||_F in FP32
    for (int q = tid; q < r * r; q += ACA_NT) {
        Mf[q] = fn > 0.0 ? (float)(M[q] / fn) : 0.f;
        Zf[q] = (q % r == q / r) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps<float>(Mf, Zf, r, 1e-5, 15, &s_rot);
    int bad = 0;
    for (int q = tid; q < r * r; q += ACA_NT) bad |= !isfinite(Zf[q]);
    bad = __syncthreads_or(bad);
    for (int q = tid; q < r * r; q += ACA_NT) Z[q] = bad ? ((q % r == q / r) ? 1.0 : 0.0) : (double)Zf[q];
    __syncthreads();
    cgs2_qr(Z, r, r, RU, cbuf, sv);  // RU is free once M is formed
    // RV <- M Z, then back into M
    for (int q = tid; q < r * r; q += ACA_NT) {
        const int i = q % r, j = q / r;
        double acc = 0.0;
        for (int l = 0; l < r; ++l) acc += M[(size_t)l * r + i] * Z[(size_t)j * r + l];
        RV[q] = acc;
    }
    __syncthreads();
    for (int q = tid; q < r * r; q += ACA_NT) M[q] = RV[q];
    __syncthreads();
    jacobi_sweeps<double>(M, Z, r, 1e-15, 30, &s_rot);
    // singular values, order by decreasing value, truncation rank
    for (int j = w; j < r; j += ACA_NW) {
        double a = 0.0;
        for (int i = lane; i < r; i += 32) a += M[(size_t)j * r + i] * M[(size_t)j * r + i];
        a = warp_sum(a);
        if (lane == 0) sig[j] = a;  // squared
    }
    __syncthreads();
    if (tid == 0) {
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

// U <- Q_U (M columns in singular-value order)_k, V <- Q_V Z_k, rows of one item
__global__ void k_expand(const ExpandJob* __restrict__ jobs, const double* __restrict__ ws,
                         const double* __restrict__ small, float* __restrict__ store) {
    const ExpandJob J = jobs[blockIdx.x];
    const int r = J.r, k = J.k;
    const int m = J.side ? J.mT : J.mS;
    const double* Q = ws + J.ws_off + (J.side ? (size_t)J.mS * (J.R + 3) : 0);
    const double* M = small + J.sm_off + 2 * (size_t)r * r;
    const double* C = J.side ? M + (size_t)r * r : M;  // Z for V, M for U
    const double* ord = M + 2 * (size_t)r * r;
    float* d = store + J.dst + (J.side ? (size_t)J.mS * k : 0);
    for (int64_t q = threadIdx.x; q < (int64_t)J.rows * k; q += blockDim.x) {
        const int row = J.row0 + (int)(q % J.rows), j = (int)(q / J.rows);
        const int o = (int)ord[j];
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += Q[(size_t)i * m + row] * C[(size_t)o * r + i];
        d[(size_t)j * m + row] = (float)s;
    }
}


}  // namespace

void launch_aca(const ElemRec* el, const AcaJob* jobs, int njobs, int max_sn, double* ws, int R, double eps,
                double mu, double nu, int32_t* rank_out, int32_t* status_out, unsigned long long* evals,
                cudaStream_t st) {
    const size_t smem = sizeof(double) * (size_t)(8 * (R + 3)) + sizeof(uint32_t) * (size_t)((3 * max_sn + 31) / 32);
    if (smem > 200 * 1024) fail(HM_EINVAL, "assemble: cluster too large for the ACA kernel");
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(k_aca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_aca<<<(unsigned)njobs, ACA_NT, smem, st>>>(el, jobs, ws, R, eps, mu, nu, rank_out, status_out, evals);
    HM_LAUNCH_CHECK();
}

void launch_recompress(const RecJob* jobs, int njobs, int R, double* ws, double* small, double tau,
                       int32_t* rank_out, cudaStream_t st) {
    const size_t smem = sizeof(double) * 2 * (R + 3) + sizeof(int) * (R + 3);
    k_recompress<<<(unsigned)njobs, ACA_NT, smem, st>>>(jobs, ws, small, tau, rank_out);
    HM_LAUNCH_CHECK();
}

void launch_expand(const ExpandJob* jobs, int njobs, const double* ws, const double* small, float* store,
                   cudaStream_t st) {
    k_expand<<<(unsigned)njobs, 256, 0, st>>>(jobs, ws, small, store);
    HM_LAUNCH_CHECK();
}

}  // namespace hm
