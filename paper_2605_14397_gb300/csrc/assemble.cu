// H-matrix assembly on the device: influence blocks, dense near-field tiles, compression
// of the admissible blocks (aca.cu) and packing into the leaf-major streams of the
// product (hmat_impl.h).  The paper keeps near-field blocks of E dense and approximates
// far-field blocks by low-rank products (Sec. 3.1).  An admissible block whose factors
// would not be smaller than the block itself (or that does not compress below the rank
// cap) is kept dense, as extra near-field tiles of its row leaves.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <numeric>

#include "aca.h"
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
    for (int64_t i = 0; i < e.N; ++i) h[i] = make_elem_record(e, i);
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
    if (opt.storage != HM_F32 && opt.storage != HM_BF16 && opt.storage != HM_F32_BF16)
        fail(HM_EINVAL, "assemble: storage must be HM_F32, HM_BF16 or HM_F32_BF16");
    const int R = opt.max_rank > 0 ? opt.max_rank : 160;
    if (R > 256) fail(HM_EINVAL, "assemble: max_rank must be <= 256");
    if (T.leaf_size > 128) fail(HM_EINVAL, "assemble: leaf_size must be <= 128");
    if (T.N > (int64_t)1 << 30) fail(HM_EINVAL, "assemble: too many elements");

    H.N = T.N;
    H.ndof = 3 * T.N;
    H.E = opt.E;
    H.nu = opt.nu;
    H.eps = opt.aca_eps;
    H.storage = opt.storage;
    const double mu = opt.E / (2.0 * (1.0 + opt.nu));
    const double kappa = opt.trunc_factor > 0.0 ? opt.trunc_factor : HM_TRUNC_DEFAULT;
    if (!(kappa * opt.aca_eps < 0.5) || !std::isfinite(kappa))
        fail(HM_EINVAL, "assemble: trunc_factor * aca_eps must stay below 0.5");
    const double eps_aca = 0.1 * kappa * opt.aca_eps;  // cross approximation target
    const double tau = 0.5 * kappa * opt.aca_eps;      // SVD truncation target

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
        L.ld16 = bf16_ld(L.ld);
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

    // ---- far field: ACA + recompression in batches bounded by a workspace budget.
    // An admissible block whose cross approximation does not converge below the rank cap
    // is refined: replaced by the blocks of its children clusters (admissible as well:
    // smaller boxes, no smaller distance), appended to the list and compressed in a later
    // batch; a pair of leaves that still does not converge is stored dense.
    std::vector<std::array<int64_t, 2>> fnodes(T.far.begin(), T.far.end());
    H.h_far.clear();
    auto push_far = [&](int64_t s, int64_t t) {
        FarDesc F{};
        F.s_begin = (int32_t)T.begin[s];
        F.s_n = (int32_t)(T.end[s] - T.begin[s]);
        F.t_begin = (int32_t)T.begin[t];
        F.t_n = (int32_t)(T.end[t] - T.begin[t]);
        H.h_far.push_back(F);
    };
    for (const auto& st_ : fnodes) push_far(st_[0], st_[1]);
    const int64_t budget = (int64_t)4 << 30;  // bytes of FP64 ACA workspace per batch
    std::vector<int32_t> ranks(fnodes.size(), 0), stat(fnodes.size(), 0), fin(fnodes.size(), 0);
    std::vector<char> dense_far(fnodes.size(), 0);  // 1 dense, 2 refined into later blocks
    int64_t store_len = 0;
    std::vector<int64_t> fac_off(fnodes.size(), 0);
    std::vector<DevBuf<float>> chunks;
    std::vector<int64_t> chunk_base;
    DevBuf<double> ws, small;
    DevBuf<int32_t> d_rank, d_stat;
    DevBuf<unsigned long long> d_evals(1);
    HM_CUDA(cudaMemsetAsync(d_evals.p, 0, d_evals.bytes(), st));
    int64_t b0 = 0;
    while (b0 < (int64_t)H.h_far.size()) {
        const int64_t nf = (int64_t)H.h_far.size();
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
        launch_aca(H.elems.p, d_jobs.p, (int)nb, max_sn, ws.p, R, eps_aca, mu, opt.nu, d_rank.p, d_stat.p,
                   d_evals.p, st);
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
                const int64_t s = fnodes[b][0], t = fnodes[b][1];
                if (T.left[s] < 0 && T.left[t] < 0) {
                    dense_far[b] = 1;  // a pair of leaves not compressible to the cap: dense
                    continue;
                }
                dense_far[b] = 2;
                const int64_t cs[2] = {T.left[s] < 0 ? s : T.left[s], T.left[s] < 0 ? -1 : T.right[s]};
                const int64_t ct[2] = {T.left[t] < 0 ? t : T.left[t], T.left[t] < 0 ? -1 : T.right[t]};
                for (int64_t a : cs)
                    for (int64_t c : ct) {
                        if (a < 0 || c < 0) continue;
                        fnodes.push_back({a, c});
                        push_far(a, c);
                        ranks.push_back(0);
                        stat.push_back(0);
                        fin.push_back(0);
                        dense_far.push_back(0);
                        fac_off.push_back(0);
                    }
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
            slen += 5LL * J.r * J.r + J.r;  // R_U, R_V, M, Z, order, FP32 copies of M and Z
        }
        std::vector<int32_t> krank(rj.size(), 0);
        if (!rj.empty()) {
            if ((size_t)slen > small.n) small.alloc(std::max<int64_t>(slen, 1));
            DevBuf<RecJob> d_rj;
            d_rj.upload(rj, st);
            launch_recompress(d_rj.p, (int)rj.size(), R, ws.p, small.p, tau, d_rank.p, st);
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
            constexpr int EXPAND_ROWS = 512;  // rows per item: a large block spreads over many CTAs
            for (int side = 0; side < 2; ++side) {
                const int m = side ? J.mT : J.mS;
                for (int r0 = 0; r0 < m; r0 += EXPAND_ROWS) {
                    e.side = side;
                    e.row0 = r0;
                    e.rows = std::min(EXPAND_ROWS, m - r0);
                    ej.push_back(e);
                }
            }
            fac_off[b] = store_len + clen;
            clen += (int64_t)k * (J.mS + J.mT);
        }
        chunks.emplace_back(std::max<int64_t>(clen, 1));
        chunk_base.push_back(store_len);
        if (!ej.empty()) {
            DevBuf<ExpandJob> d_ej;
            d_ej.upload(ej, st);
            launch_expand(d_ej.p, (int)ej.size(), ws.p, small.p, chunks.back().p, st);
            HM_CUDA(cudaStreamSynchronize(st));
        }
        store_len += clen;
        b0 = b1;
    }
    ws.release();
    small.release();
    {
        unsigned long long ev = 0;
        HM_CUDA(cudaMemcpyAsync(&ev, d_evals.p, sizeof(ev), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        H.aca_blocks = (int64_t)ev;
    }
    const int64_t nf = (int64_t)H.h_far.size();
    H.n_far = nf;
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
    H.h_near_true_cols.assign(nl, 0);
    for (int l = 0; l < nl; ++l)
        for (const DenseTile& D : tiles_by_row[l]) H.h_near_true_cols[l] += 3 * D.t_n;
    int64_t n_dense_far = 0;
    H.n_refined = 0;
    for (int64_t b = 0; b < nf; ++b) {
        if (dense_far[b] == 2) ++H.n_refined;
        if (dense_far[b] != 1) continue;
        ++n_dense_far;
        const int64_t s = fnodes[b][0];
        for (int l = 0; l < lcount[s]; ++l)
            tiles_by_row[lfirst[s] + l].push_back({H.h_far[b].t_begin, H.h_far[b].t_n});
    }
    std::vector<NearJob> njobs;
    std::vector<int32_t> near_zidx;
    int64_t near_len = 0;
    H.near_entries = 0;
    H.h_self_off.assign(nl, -1);
    for (int l = 0; l < nl; ++l) {
        LeafDesc& L = H.h_leaves[l];
        L.near_off = near_len;
        L.near_cbase = (int32_t)near_zidx.size();
        int cols = 0;
        for (const DenseTile& D : tiles_by_row[l]) {
            if (D.t_begin == L.begin && D.t_n == L.n) H.h_self_off[l] = near_len + (int64_t)cols * L.ld;
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
    H.h_near_zidx = std::move(near_zidx);

    // ---- ranks, partial-buffer and t-vector layout (low-rank blocks only)
    int64_t tb_len = 0, p_len = 0, poff_len = 0, uoff_len = 0;
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
        F.n_tleaves = lcount[fnodes[b][1]];
        F.pbase = poff_len;
        poff_len += F.n_tleaves;
        F.n_sleaves = lcount[fnodes[b][0]];
        F.ubase = uoff_len;
        uoff_len += F.n_sleaves;
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
    H.p_len = p_len;

    std::vector<std::vector<int64_t>> far_by_row(nl), far_by_col(nl);
    for (int64_t b = 0; b < nf; ++b) {
        if (H.h_far[b].rank == 0) continue;
        const int64_t s = fnodes[b][0], t = fnodes[b][1];
        for (int l = 0; l < lcount[s]; ++l) far_by_row[lfirst[s] + l].push_back(b);
        for (int l = 0; l < lcount[t]; ++l) far_by_col[lfirst[t] + l].push_back(b);
    }

    // ---- U and V streams
    // (the BF16 streams hold the same slices with their own padding, bf16_ld)
    std::vector<PackJob> ujobs, vjobs, ujobs16, vjobs16;
    std::vector<int32_t> u_zidx, v_pidx;
    H.h_poff.assign(std::max<int64_t>(poff_len, 1), 0);
    H.h_uoff.assign(std::max<int64_t>(uoff_len, 1), 0);
    int64_t u_len = 0, v_len = 0, u_len16 = 0, v_len16 = 0;
    auto as16 = [](PackJob J, int64_t base16, int cols, int ld16) {
        J.dst = base16 + (int64_t)cols * ld16;
        J.dst_ld = ld16;
        return J;
    };
    for (int l = 0; l < nl; ++l) {
        LeafDesc& L = H.h_leaves[l];
        L.u_off = u_len;
        L.u_off16 = u_len16;
        L.u_cbase = (int32_t)u_zidx.size();
        int ucols = 0;
        for (int64_t b : far_by_row[l]) {
            const FarDesc& F = H.h_far[b];
            const int64_t s = fnodes[b][0];
            const int32_t ustart = (int32_t)u_zidx.size();  // this leaf's copy of t_b
            H.h_uoff[F.ubase + (l - lfirst[s])] = ustart;
            PackJob J;
            J.src = F.fac_off + 3LL * (L.begin - F.s_begin);
            J.dst = u_len + (int64_t)ucols * L.ld;
            J.src_ld = 3 * F.s_n;
            J.rows = 3 * L.n;
            J.dst_ld = L.ld;
            J.ncols = F.rank;
            ujobs.push_back(J);
            ujobs16.push_back(as16(J, u_len16, ucols, L.ld16));
            for (int c = 0; c < F.rank; ++c) u_zidx.push_back(ustart + c);
            ucols += F.rank;
        }
        L.u_cols = ucols;
        u_len += (int64_t)ucols * L.ld;
        u_len16 += (int64_t)ucols * L.ld16;

        L.v_off = v_len;
        L.v_off16 = v_len16;
        L.v_cbase = (int32_t)v_pidx.size();
        int vcols = 0;
        for (int64_t b : far_by_col[l]) {
            const FarDesc& F = H.h_far[b];
            const int64_t t = fnodes[b][1];
            const int k = l - lfirst[t];  // which leaf of T
            PackJob J;
            J.src = F.fac_off + 3LL * F.s_n * F.rank + 3LL * (L.begin - F.t_begin);
            J.dst = v_len + (int64_t)vcols * L.ld;
            J.src_ld = 3 * F.t_n;
            J.rows = 3 * L.n;
            J.dst_ld = L.ld;
            J.ncols = F.rank;
            vjobs.push_back(J);
            vjobs16.push_back(as16(J, v_len16, vcols, L.ld16));
            const int32_t start = (int32_t)v_pidx.size();  // partials in V-stream order
            H.h_poff[F.pbase + k] = start;
            for (int c = 0; c < F.rank; ++c) v_pidx.push_back(start + c);
            vcols += F.rank;
        }
        L.v_cols = vcols;
        v_len += (int64_t)vcols * L.ld;
        v_len16 += (int64_t)vcols * L.ld16;
    }
    const bool want32 = has_factors(H, 0), want16 = has_factors(H, 1);
    if (want32) {
        H.u32.alloc(std::max<int64_t>(u_len, 1));
        H.v32.alloc(std::max<int64_t>(v_len, 1));
        HM_CUDA(cudaMemsetAsync(H.u32.p, 0, H.u32.bytes(), st));
        HM_CUDA(cudaMemsetAsync(H.v32.p, 0, H.v32.bytes(), st));
    }
    if (want16) {
        H.u16.alloc(std::max<int64_t>(u_len16, 1));
        H.v16.alloc(std::max<int64_t>(v_len16, 1));
        HM_CUDA(cudaMemsetAsync(H.u16.p, 0, H.u16.bytes(), st));
        HM_CUDA(cudaMemsetAsync(H.v16.p, 0, H.v16.bytes(), st));
    }
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<PackJob>& pj = pass == 0 ? ujobs : vjobs;
        const std::vector<PackJob>& pj16 = pass == 0 ? ujobs16 : vjobs16;
        if (pj.empty()) continue;
        DevBuf<PackJob> d_p, d_p16;
        if (want32) {
            d_p.upload(pj, st);
            k_pack<float><<<(unsigned)pj.size(), 256, 0, st>>>(H.facstore.p, d_p.p, pass == 0 ? H.u32.p : H.v32.p);
        }
        if (want16) {
            d_p16.upload(pj16, st);
            k_pack<uint16_t><<<(unsigned)pj16.size(), 256, 0, st>>>(H.facstore.p, d_p16.p,
                                                                     pass == 0 ? H.u16.p : H.v16.p);
        }
        HM_LAUNCH_CHECK();
        HM_CUDA(cudaStreamSynchronize(st));
    }
    H.tb_len = (int64_t)u_zidx.size();
    if (H.tb_len > INT32_MAX) fail(HM_EINVAL, "assemble: too many U columns");
    (void)tb_len;
    H.h_u_zidx = std::move(u_zidx);
    H.uoff.upload(H.h_uoff, st);
    H.h_v_pidx = std::move(v_pidx);
    H.poff.upload(H.h_poff, st);
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
