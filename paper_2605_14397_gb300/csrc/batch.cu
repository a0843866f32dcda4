// Batching of independent faults, graph-replayed products and the leaf-size autotuner.
//
// Independent faults do not interact (block-diagonal operator), so a batch is the
// concatenation of the faults' H-matrices in one arena: element records, coefficient
// streams, leaf and block descriptors and operand index arrays are appended with
// offsets, and one product plan (one chunk work list per phase) is cut over all of them.
// One persistent launch per phase then streams every fault's coefficients, with the
// byte-balanced split of the work list keeping all SMs busy however unequal the faults
// are.  Each fault keeps the material it was assembled with (per-fault nu).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <string>

#include "hmat_impl.h"
#include "tree.h"

namespace hm {

namespace {

template <class T>
void append_dev(DevBuf<T>& dst, const std::vector<const DevBuf<T>*>& src, cudaStream_t st) {
    size_t tot = 0;
    for (const DevBuf<T>* s : src) tot += s->n;
    dst.alloc(std::max<size_t>(tot, 1));
    size_t off = 0;
    for (const DevBuf<T>* s : src) {
        if (s->n) HM_CUDA(cudaMemcpyAsync(dst.p + off, s->p, s->bytes(), cudaMemcpyDeviceToDevice, st));
        off += s->n;
    }
}

}  // namespace

void merge(const std::vector<const HMat*>& hs, cudaStream_t st, HMat& M) {
    if (hs.empty()) fail(HM_EINVAL, "batch: no H-matrices");
    const int storage = hs[0]->storage;
    int64_t N = 0;
    for (const HMat* h : hs) {
        if (!h) fail(HM_EINVAL, "batch: NULL H-matrix");
        if (h->storage != storage) fail(HM_EINVAL, "batch: all H-matrices must use the same factor storage");
        N += h->N;
    }
    if (N > ((int64_t)1 << 29)) fail(HM_EINVAL, "batch: too many elements");
    M.N = N;
    M.ndof = 3 * N;
    M.storage = storage;
    M.E = hs[0]->E;
    M.nu = hs[0]->nu;
    M.eps = hs[0]->eps;
    for (const HMat* h : hs) {
        if (h->E != M.E) M.E = NAN;
        if (h->nu != M.nu) M.nu = NAN;
        M.eps = std::max(M.eps, h->eps);
    }

    int64_t pos = 0, near_b = 0, u_b = 0, v_b = 0, u16_b = 0, v16_b = 0, tb_b = 0, p_b = 0, fac_b = 0, po_b = 0,
            uo_b = 0;
    int32_t nz_b = 0, uz_b = 0, vp_b = 0;
    M.h_leaves.clear();
    M.h_far.clear();
    M.h_perm.clear();
    M.h_near_zidx.clear();
    M.h_u_zidx.clear();
    M.h_v_pidx.clear();
    M.h_self_off.clear();
    M.h_near_true_cols.clear();
    M.h_poff.clear();
    M.h_uoff.clear();
    M.n_near = M.n_far = M.n_dense_far = M.n_refined = 0;
    M.near_entries = M.far_entries = 0;
    M.assemble_seconds = 0.0;
    M.aca_blocks = 0;
    std::vector<int32_t> perm32;
    perm32.reserve(N);
    for (const HMat* h : hs) {
        if (M.h_near_zidx.size() + h->h_near_zidx.size() > (size_t)INT32_MAX ||
            M.h_u_zidx.size() + h->h_u_zidx.size() > (size_t)INT32_MAX ||
            M.h_v_pidx.size() + h->h_v_pidx.size() > (size_t)INT32_MAX || tb_b + h->tb_len > INT32_MAX ||
            p_b + h->p_len > INT32_MAX)
            fail(HM_EINVAL, "batch: operand index space exceeds 32 bits");
        for (int64_t k = 0; k < h->N; ++k) {
            M.h_perm.push_back(h->h_perm[k] + pos);
            perm32.push_back((int32_t)(h->h_perm[k] + pos));
        }
        for (LeafDesc L : h->h_leaves) {
            L.begin += (int32_t)pos;
            L.near_off += near_b;
            L.u_off += u_b;
            L.v_off += v_b;
            L.u_off16 += u16_b;
            L.v_off16 += v16_b;
            L.near_cbase += nz_b;
            L.u_cbase += uz_b;
            L.v_cbase += vp_b;
            M.h_leaves.push_back(L);
        }
        for (FarDesc F : h->h_far) {
            F.s_begin += (int32_t)pos;
            F.t_begin += (int32_t)pos;
            F.pbase += po_b;
            F.ubase += uo_b;
            F.tb_off += tb_b;
            F.fac_off += fac_b;
            M.h_far.push_back(F);
        }
        for (int32_t z : h->h_near_zidx) M.h_near_zidx.push_back(z + (int32_t)(3 * pos));
        for (int32_t z : h->h_u_zidx) M.h_u_zidx.push_back(z + (int32_t)tb_b);
        for (int32_t z : h->h_v_pidx) M.h_v_pidx.push_back(z + (int32_t)p_b);
        for (int64_t o : h->h_self_off) M.h_self_off.push_back(o < 0 ? o : o + near_b);
        for (int32_t c : h->h_near_true_cols) M.h_near_true_cols.push_back(c);
        for (int32_t o : h->h_poff) M.h_poff.push_back(o + (int32_t)p_b);
        po_b += (int64_t)h->h_poff.size();
        for (int32_t o : h->h_uoff) M.h_uoff.push_back(o + (int32_t)tb_b);
        uo_b += (int64_t)h->h_uoff.size();
        pos += h->N;
        near_b += (int64_t)h->near.n;
        u_b += (int64_t)h->u32.n;
        v_b += (int64_t)h->v32.n;
        u16_b += (int64_t)h->u16.n;
        v16_b += (int64_t)h->v16.n;
        tb_b += h->tb_len;
        p_b += h->p_len;
        fac_b += (int64_t)h->facstore.n;
        nz_b += (int32_t)h->h_near_zidx.size();
        uz_b += (int32_t)h->h_u_zidx.size();
        vp_b += (int32_t)h->h_v_pidx.size();
        M.n_near += h->n_near;
        M.n_far += h->n_far;
        M.n_dense_far += h->n_dense_far;
        M.n_refined += h->n_refined;
        M.near_entries += h->near_entries;
        M.far_entries += h->far_entries;
        M.assemble_seconds += h->assemble_seconds;
        M.aca_blocks += h->aca_blocks;
    }
    M.n_leaves = (int)M.h_leaves.size();
    M.tb_len = tb_b;
    M.p_len = p_b;
    M.rank_min = 1 << 30;
    M.rank_max = 0;
    double rsum = 0.0;
    int64_t nlr = 0;
    for (const FarDesc& F : M.h_far) {
        if (F.dense) continue;
        M.rank_min = std::min(M.rank_min, F.rank);
        M.rank_max = std::max(M.rank_max, F.rank);
        rsum += F.rank;
        ++nlr;
    }
    if (nlr == 0) M.rank_min = 0;
    M.rank_mean = nlr ? rsum / (double)nlr : 0.0;

    std::vector<const DevBuf<ElemRec>*> se;
    std::vector<const DevBuf<float>*> sn, su32, sv32, sfac;
    std::vector<const DevBuf<uint16_t>*> su16, sv16;
    for (const HMat* h : hs) {
        se.push_back(&h->elems);
        sn.push_back(&h->near);
        su32.push_back(&h->u32);
        sv32.push_back(&h->v32);
        su16.push_back(&h->u16);
        sv16.push_back(&h->v16);
        sfac.push_back(&h->facstore);
    }
    append_dev(M.elems, se, st);
    append_dev(M.near, sn, st);
    append_dev(M.facstore, sfac, st);
    if (has_factors(M, 0)) {
        append_dev(M.u32, su32, st);
        append_dev(M.v32, sv32, st);
    }
    if (has_factors(M, 1)) {
        append_dev(M.u16, su16, st);
        append_dev(M.v16, sv16, st);
    }
    M.perm.upload(perm32, st);
    M.poff.upload(M.h_poff, st);
    M.uoff.upload(M.h_uoff, st);
    M.leaves.upload(M.h_leaves, st);
    M.far.upload(M.h_far, st);
    build_product_plan(M, st);
    ensure_product_scratch(M, 1, st);
    HM_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ graph replay

void graphs_clear(HMat& H) {
    for (HMat::GraphEntry& g : H.graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    H.graphs.clear();
}

// y = E x through a CUDA graph of the whole product (gather, the three streaming
// kernels, scatter), instantiated on first use for this (x, y, nrhs, dtype) and
// replayed on `st` afterwards: one launch of host work per product.
void matvec_graph(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st) {
    if (H.timing) {  // per-phase events cannot live inside a replayed graph
        matvec(H, x, y, nrhs, dtype, st);
        return;
    }
    for (const HMat::GraphEntry& g : H.graphs)
        if (g.x == x && g.y == y && g.nrhs == nrhs && g.dtype == dtype) {
            HM_CUDA(cudaGraphLaunch(g.exec, st));
            return;
        }
    // one eager product first: it sizes the scratch and sets the kernels' attributes
    matvec(H, x, y, nrhs, dtype, st);
    if (!H.cap_stream) HM_CUDA(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    // the capture stream must see the eager product's scratch writes in order
    cudaEvent_t ev;
    HM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HM_CUDA(cudaEventRecord(ev, st));
    HM_CUDA(cudaStreamWaitEvent(H.cap_stream, ev, 0));
    HM_CUDA(cudaStreamSynchronize(H.cap_stream));
    cudaEventDestroy(ev);
    cudaGraph_t graph = nullptr;
    HM_CUDA(cudaStreamBeginCapture(H.cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
        matvec(H, x, y, nrhs, dtype, H.cap_stream);
    } catch (...) {
        cudaStreamEndCapture(H.cap_stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    HM_CUDA(cudaStreamEndCapture(H.cap_stream, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    HM_CUDA(e);
    H.graphs.push_back(HMat::GraphEntry{x, y, nrhs, dtype, exec});
    HM_CUDA(cudaGraphLaunch(exec, st));
}

// ------------------------------------------------------------------ tile shapes

void set_tile_shape(HMat& H, const hm_tile_shape& t, cudaStream_t st) {
    if (t.chunk_bytes < 2048 || t.chunk_bytes > 32768 || t.chunk_bytes % 16)
        fail(HM_EINVAL, "tile shape: chunk_bytes must be a multiple of 16 in [2048, 32768]");
    if (t.chunk_cols < 8 || t.chunk_cols > 128) fail(HM_EINVAL, "tile shape: chunk_cols must lie in [8, 128]");
    if (t.ring != 4 && t.ring != 6) fail(HM_EINVAL, "tile shape: ring must be 4 or 6");
    if (t.warps != 8 && t.warps != 16) fail(HM_EINVAL, "tile shape: warps must be 8 or 16");
    HM_CUDA(cudaStreamSynchronize(st));
    graphs_clear(H);
    H.shape.chunk_bytes = t.chunk_bytes;
    H.shape.chunk_cols = t.chunk_cols;
    H.shape.ring = t.ring;
    H.shape.warps = t.warps;
    build_product_plan(H, st);
    // the split-leaf slots depend on the plan: size the product scratch again
    const int cap = std::max(H.nrhs_cap, 1);
    H.nrhs_cap = 0;
    ensure_product_scratch(H, cap, st);
    HM_CUDA(cudaStreamSynchronize(st));
}

namespace {

// average time of `reps` single-RHS FP32-vector products (FP32 factors when stored)
double time_product(HMat& H, int reps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    DevBuf<float> x(H.ndof), y(H.ndof);
    HM_CUDA(cudaMemsetAsync(x.p, 0, x.bytes(), st));
    for (int w = 0; w < 3; ++w) matvec(H, x.p, y.p, 1, HM_F32, st);
    HM_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) matvec(H, x.p, y.p, 1, HM_F32, st);
    HM_CUDA(cudaEventRecord(e1, st));
    HM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    HM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (product_error_flags(H, st)) fail(HM_ETIMEOUT, "tile-shape timing: a product wait gave up");
    return ms / reps;
}

std::string shape_json(const hm_tile_shape& t) {
    char buf[160];
    snprintf(buf, sizeof(buf), "\"chunk_bytes\": %d, \"chunk_cols\": %d, \"ring\": %d, \"warps\": %d", t.chunk_bytes,
             t.chunk_cols, t.ring, t.warps);
    return buf;
}

struct Events {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Events() {
        HM_CUDA(cudaEventCreate(&e0));
        HM_CUDA(cudaEventCreate(&e1));
    }
    ~Events() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace

// Time the single-RHS product of H under every shape, keep the fastest on H.
std::string tune_tile_shape(HMat& H, const hm_tile_shape* shapes, int n, int reps, cudaStream_t st) {
    if (!shapes || n < 1) fail(HM_EINVAL, "tune_tile_shape: empty shape list");
    if (reps < 1) reps = 20;
    Events ev;
    std::string js = "{\"candidates\": [";
    double best = 1e300;
    int ib = 0;
    for (int i = 0; i < n; ++i) {
        set_tile_shape(H, shapes[i], st);
        const double ms = time_product(H, reps, st, ev.e0, ev.e1);
        char buf[64];
        snprintf(buf, sizeof(buf), ", \"ms\": %.6f}", ms);
        js += (i ? ", {" : "{") + shape_json(shapes[i]) + buf;
        if (ms < best) {
            best = ms;
            ib = i;
        }
    }
    set_tile_shape(H, shapes[ib], st);
    char buf[64];
    snprintf(buf, sizeof(buf), ", \"ms\": %.6f}, \"tuned\": %d}", best, n);
    js += "], \"best\": {" + shape_json(shapes[ib]) + buf;
    return js;
}

// ------------------------------------------------------------------ autotuner

// Time the product for every (leaf size, eta) candidate on this geometry and pick the
// fastest: the leaf size sets the near-field tile and factor-slice shapes the product
// streams, eta the split between dense tiles and low-rank blocks.  Every candidate meets
// the same per-block accuracy aca_eps, so only time (and memory) differ.  Candidates are
// tried in order until budget_ms has elapsed (at least one is always timed).
std::string autotune(const hm_elements& el, const hm_assemble_opts& opt, const int* leaves, int n_leaf,
                     const double* etas, int n_eta, const hm_tile_shape* shapes, int n_shapes, int budget_ms,
                     cudaStream_t st) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (n_leaf < 1 || n_eta < 1 || !leaves || !etas) fail(HM_EINVAL, "autotune: empty candidate list");
    hm_tile_shape def{32768, 128, 4, 16};
    if (!shapes || n_shapes < 1) {
        shapes = &def;
        n_shapes = 1;
    }
    std::string js = "{\"n_elements\": " + std::to_string(el.N) + ", \"candidates\": [";
    double best = 1e300;
    int best_leaf = 0, best_shape = 0;
    double best_eta = 0.0;
    int tried = 0;
    Events ev;
    for (int i = 0; i < n_leaf; ++i)
        for (int j = 0; j < n_eta; ++j) {
            const double el_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
            if (tried > 0 && el_ms > budget_ms) break;
            Tree T;
            build_tree(el, leaves[i], etas[j], T);
            HMat H;
            assemble(T, opt, st, H);
            for (int q = 0; q < n_shapes; ++q) {
                const double el2 = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
                if (tried > 0 && el2 > budget_ms) break;
                set_tile_shape(H, shapes[q], st);
                const double per = time_product(H, 20, st, ev.e0, ev.e1);
                char buf[320];
                snprintf(buf, sizeof(buf),
                         "%s{\"leaf\": %d, \"eta\": %.6g, \"ms\": %.6f, \"stored_bytes\": %lld, "
                         "\"assemble_s\": %.4f, \"rank_mean\": %.4f, ",
                         tried ? ", " : "", leaves[i], etas[j], per, (long long)H.stored_bytes(),
                         H.assemble_seconds, H.rank_mean);
                js += buf + shape_json(shapes[q]) + "}";
                if (per < best) {
                    best = per;
                    best_leaf = leaves[i];
                    best_eta = etas[j];
                    best_shape = q;
                }
                ++tried;
            }
        }
    char buf[200];
    snprintf(buf, sizeof(buf), "], \"best\": {\"leaf\": %d, \"eta\": %.6g, \"ms\": %.6f, ", best_leaf, best_eta, best);
    js += buf + shape_json(shapes[best_shape]) + "}, \"tuned\": " + std::to_string(tried) + "}";
    return js;
}

}  // namespace hm
