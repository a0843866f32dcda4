// extern "C" boundary of libhmat: argument checks, handle ownership, status codes.
#include <cmath>
#include <cstring>
#include <string>

#include "hmat_impl.h"
#include "learned.h"
#include "tree.h"

struct hm_tree {
    hm::Tree t;
};

namespace hm {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

std::string autotune(const hm_elements& el, const hm_assemble_opts& opt, const int* leaves, int n_leaf,
                     const double* etas, int n_eta, const hm_tile_shape* shapes, int n_shapes, int budget_ms,
                     cudaStream_t st);
void influence_pairs(const hm_elements& e, double E, double nu, int64_t npairs, const int64_t* ri,
                     const int64_t* sj, double* out, cudaStream_t st);

static void check_elements(const hm_elements* el) {
    if (!el) fail(HM_EINVAL, "NULL element description");
    if (el->N <= 0) fail(HM_EINVAL, "element count must be positive");
    if (!el->c || !el->s1 || !el->s2 || !el->n || !el->a || !el->b) fail(HM_EINVAL, "NULL geometry array");
    validate_elements(*el, "elements");
}

}  // namespace hm

extern "C" {

const char* hm_last_error(void) { return hm::g_last_error.c_str(); }

int hm_version(void) { return 200; }

hm_status hm_influence_blocks(const hm_elements* el, double E, double nu, int64_t npairs, const int64_t* ri_dev,
                              const int64_t* sj_dev, double* out_dev, void* stream) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    hm::check_elements(el);
    hm::influence_pairs(*el, E, nu, npairs, ri_dev, sj_dev, out_dev, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_build_cluster_tree(const hm_elements* el, int leaf_size, double eta, hm_tree** out) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    if (!out) hm::fail(HM_EINVAL, "build_cluster_tree: NULL output handle");
    *out = nullptr;
    hm::check_elements(el);
    hm_tree* t = new hm_tree();
    try {
        hm::build_tree(*el, leaf_size, eta, t->t);
    } catch (...) {
        delete t;
        throw;
    }
    *out = t;
    HM_API_END
}

hm_status hm_tree_get_info(const hm_tree* t, hm_tree_info* info) {
    HM_API_BEGIN
    if (!t || !info) hm::fail(HM_EINVAL, "tree_get_info: NULL argument");
    info->n_elements = t->t.N;
    info->n_nodes = (int64_t)t->t.begin.size();
    info->n_leaves = (int64_t)t->t.leaves.size();
    info->n_near = (int64_t)t->t.near.size();
    info->n_far = (int64_t)t->t.far.size();
    info->leaf_size = t->t.leaf_size;
    info->depth = t->t.depth;
    info->eta = t->t.eta;
    HM_API_END
}

hm_status hm_tree_export(const hm_tree* t, int64_t* perm, int64_t* begin, int64_t* end, int64_t* left,
                         int64_t* right, int64_t* near, int64_t* far) {
    HM_API_BEGIN
    if (!t) hm::fail(HM_EINVAL, "tree_export: NULL tree");
    const hm::Tree& T = t->t;
    if (perm) std::memcpy(perm, T.perm.data(), T.perm.size() * sizeof(int64_t));
    if (begin) std::memcpy(begin, T.begin.data(), T.begin.size() * sizeof(int64_t));
    if (end) std::memcpy(end, T.end.data(), T.end.size() * sizeof(int64_t));
    if (left) std::memcpy(left, T.left.data(), T.left.size() * sizeof(int64_t));
    if (right) std::memcpy(right, T.right.data(), T.right.size() * sizeof(int64_t));
    if (near)
        for (size_t b = 0; b < T.near.size(); ++b) { near[2 * b] = T.near[b][0]; near[2 * b + 1] = T.near[b][1]; }
    if (far)
        for (size_t b = 0; b < T.far.size(); ++b) { far[2 * b] = T.far[b][0]; far[2 * b + 1] = T.far[b][1]; }
    HM_API_END
}

void hm_tree_destroy(hm_tree* t) { delete t; }

hm_status hm_assemble_hmat(const hm_tree* t, const hm_elements* el, const hm_assemble_opts* opt, void* stream,
                           hm_hmat** out) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_assemble_hmat");
    hm::g_last_error.clear();
    if (!out) hm::fail(HM_EINVAL, "assemble_hmat: NULL output handle");
    *out = nullptr;
    if (!t || !opt) hm::fail(HM_EINVAL, "assemble_hmat: NULL tree or options");
    if (el) {
        hm::check_elements(el);
        if (el->N != t->t.N) hm::fail(HM_EINVAL, "assemble_hmat: element count differs from the tree's");
    }
    hm_hmat* h = new hm_hmat();
    try {
        hm::assemble(t->t, *opt, (cudaStream_t)stream, h->h);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    HM_API_END
}

hm_status hm_hmat_get_info(const hm_hmat* hh, hm_hmat_info* info) {
    HM_API_BEGIN
    if (!hh || !info) hm::fail(HM_EINVAL, "hmat_get_info: NULL argument");
    const hm::HMat& H = hh->h;
    info->n_dof = H.ndof;
    info->near_entries = H.near_entries;
    info->far_entries = H.far_entries;
    info->stored_bytes = H.stored_bytes();
    const int64_t fb = H.storage == HM_BF16 ? 2 : 4;
    info->algorithmic_bytes = 4 * H.near_entries + fb * H.far_entries + 2 * 4 * H.ndof;
    info->rank_min = H.rank_min;
    info->rank_max = H.rank_max;
    info->rank_mean = H.rank_mean;
    info->assemble_seconds = H.assemble_seconds;
    info->storage = H.storage;
    info->pad_ = 0;
    info->n_far_dense = H.n_dense_far;
    info->n_far_lowrank = H.n_far - H.n_dense_far - H.n_refined;
    info->n_far_refined = H.n_refined;
    info->n_leaves = H.n_leaves;
    info->u_entries = info->v_entries = 0;
    for (const hm::FarDesc& F : H.h_far) {
        info->u_entries += 3LL * F.rank * F.s_n;
        info->v_entries += 3LL * F.rank * F.t_n;
    }
    info->tb_len = H.tb_len;
    info->p_len = H.p_len;
    info->coeff_blocks = H.aca_blocks + H.near_entries / 9;
    HM_API_END
}

hm_status hm_hmat_far_factors(const hm_hmat* hh, int64_t b, int32_t* rank_out, double* U, double* V) {
    HM_API_BEGIN
    if (!hh) hm::fail(HM_EINVAL, "hmat_far_factors: NULL H-matrix");
    const hm::HMat& H = hh->h;
    if (b < 0 || b >= H.n_far) hm::fail(HM_EINVAL, "hmat_far_factors: block index out of range");
    const hm::FarDesc& F = H.h_far[b];
    if (rank_out) *rank_out = F.dense == 1 ? -1 : (F.dense == 2 ? -2 : F.rank);
    if ((U || V) && !F.dense) {
        const int64_t nu = 3LL * F.s_n * F.rank, nv = 3LL * F.t_n * F.rank;
        std::vector<float> buf(nu + nv);
        if (nu + nv > 0)
            HM_CUDA(cudaMemcpy(buf.data(), H.facstore.p + F.fac_off, (nu + nv) * sizeof(float), cudaMemcpyDeviceToHost));
        if (U)
            for (int64_t q = 0; q < nu; ++q) U[q] = buf[q];
        if (V)
            for (int64_t q = 0; q < nv; ++q) V[q] = buf[nu + q];
    }
    HM_API_END
}

void hm_hmat_destroy(hm_hmat* h) { delete h; }

hm_status hm_matvec(const hm_hmat* hh, const void* x_dev, void* y_dev, int nrhs, int dtype, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_matvec");
    if (!hh) hm::fail(HM_EINVAL, "matvec: NULL H-matrix");
    if (x_dev == y_dev) hm::fail(HM_EINVAL, "matvec: x and y must not overlap");
    hm::matvec(const_cast<hm::HMat&>(hh->h), x_dev, y_dev, nrhs, dtype, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_matvec_factors(const hm_hmat* hh, const void* x_dev, void* y_dev, int nrhs, int dtype, int factors,
                            void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_matvec_factors");
    if (!hh) hm::fail(HM_EINVAL, "matvec_factors: NULL H-matrix");
    if (x_dev == y_dev) hm::fail(HM_EINVAL, "matvec_factors: x and y must not overlap");
    hm::matvec(const_cast<hm::HMat&>(hh->h), x_dev, y_dev, nrhs, dtype, (cudaStream_t)stream, factors);
    HM_API_END
}

hm_status hm_matvec_host(const hm_hmat* hh, const void* x_host, void* y_host, int nrhs, int dtype, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_matvec_host");
    if (!hh) hm::fail(HM_EINVAL, "matvec_host: NULL H-matrix");
    if (x_host == y_host) hm::fail(HM_EINVAL, "matvec_host: x and y must not overlap");
    hm::matvec_host(const_cast<hm::HMat&>(hh->h), x_host, y_host, nrhs, dtype, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_hmat_timing(const hm_hmat* hh, int enable) {
    HM_API_BEGIN
    if (!hh) hm::fail(HM_EINVAL, "hmat_timing: NULL H-matrix");
    hm::timing_enable(const_cast<hm::HMat&>(hh->h), enable != 0);
    HM_API_END
}

hm_status hm_hmat_timing_read(const hm_hmat* hh, double* out6) {
    HM_API_BEGIN
    if (!hh || !out6) hm::fail(HM_EINVAL, "hmat_timing_read: NULL argument");
    hm::timing_read(const_cast<hm::HMat&>(hh->h), out6);
    HM_API_END
}

hm_status hm_gmres_solve(const hm_hmat* hh, const double* k_dev, double shift, const double* b_dev, double* x_dev,
                         int nrhs, const hm_solve_opts* opt, hm_solve_info* info, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_gmres_solve");
    hm::g_last_error.clear();
    if (!hh) hm::fail(HM_EINVAL, "gmres_solve: NULL H-matrix");
    hm_solve_opts o{};
    if (opt) o = *opt;
    if (!opt) {
        o.precond = HM_PRECOND_BLOCKJ;
        o.mode = HM_SOLVE_F64;
    }
    if (!std::isfinite(shift)) hm::fail(HM_ENAN, "gmres_solve: shift is not finite");
    hm::gmres_solve(const_cast<hm::HMat&>(hh->h), k_dev, shift, b_dev, x_dev, nrhs, o, info, (cudaStream_t)stream,
                    o.lp ? &o.lp->m : nullptr);
    HM_API_END
}

hm_status hm_precond_apply(const hm_hmat* hh, const double* k_dev, double shift, const hm_solve_opts* opt,
                           const double* r_dev, double* z_dev, int nrhs, void* stream) {
    HM_API_BEGIN
    if (!hh || !opt) hm::fail(HM_EINVAL, "precond_apply: NULL argument");
    if (!std::isfinite(shift)) hm::fail(HM_ENAN, "precond_apply: shift is not finite");
    hm::precond_apply_user(const_cast<hm::HMat&>(hh->h), k_dev, shift, *opt, opt->lp ? &opt->lp->m : nullptr, r_dev,
                           z_dev, nrhs, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_ilu_export(const hm_hmat* hh, const double* k_dev, const double* cep_dev, double shift, double p,
                        int64_t* n_out, int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr,
                        int32_t* col, double* a_val, double* lu_val, void* stream) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    if (!hh) hm::fail(HM_EINVAL, "ilu_export: NULL H-matrix");
    if (!(p > 0.0 && p <= 1.0)) hm::fail(HM_EINVAL, "ilu_export: p must lie in (0, 1]");
    if (!std::isfinite(shift)) hm::fail(HM_ENAN, "ilu_export: shift is not finite");
    hm::ilu_export_for(const_cast<hm::HMat&>(hh->h), k_dev, cep_dev, shift, p, n_out, nnz_out, n_colours_out, order,
                       rowptr, col, a_val, lu_val, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_ilu_apply(const hm_hmat* hh, const double* r_dev, double* z_dev, int nrhs, void* stream) {
    HM_API_BEGIN
    if (!hh) hm::fail(HM_EINVAL, "ilu_apply: NULL H-matrix");
    if (r_dev == z_dev) hm::fail(HM_EINVAL, "ilu_apply: r and z must not overlap");
    hm::ilu_apply_user(const_cast<hm::HMat&>(hh->h), r_dev, z_dev, nrhs, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_batch_create(const hm_hmat* const* hs, int nf, void* stream, hm_hmat** out) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    if (!out) hm::fail(HM_EINVAL, "batch_create: NULL output handle");
    *out = nullptr;
    if (!hs || nf < 1) hm::fail(HM_EINVAL, "batch_create: need at least one H-matrix");
    std::vector<const hm::HMat*> parts(nf);
    for (int f = 0; f < nf; ++f) {
        if (!hs[f]) hm::fail(HM_EINVAL, "batch_create: NULL H-matrix in the list");
        parts[f] = &hs[f]->h;
    }
    hm_hmat* m = new hm_hmat();
    try {
        hm::merge(parts, (cudaStream_t)stream, m->h);
    } catch (...) {
        delete m;
        throw;
    }
    *out = m;
    HM_API_END
}

hm_status hm_matvec_graph(const hm_hmat* hh, const void* x_dev, void* y_dev, int nrhs, int dtype, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_matvec_graph");
    if (!hh) hm::fail(HM_EINVAL, "matvec_graph: NULL H-matrix");
    if (!x_dev || !y_dev) hm::fail(HM_EINVAL, "matvec_graph: NULL vector");
    if (x_dev == y_dev) hm::fail(HM_EINVAL, "matvec_graph: x and y must not overlap");
    if (nrhs < 1) hm::fail(HM_EINVAL, "matvec_graph: nrhs must be >= 1");
    if (dtype != HM_F32 && dtype != HM_F64) hm::fail(HM_EINVAL, "matvec_graph: dtype must be HM_F32 or HM_F64");
    hm::matvec_graph(const_cast<hm::HMat&>(hh->h), x_dev, y_dev, nrhs, dtype, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_autotune(const hm_elements* el, const hm_assemble_opts* opt, const int* leaf_sizes, int n_leaf,
                      const double* etas, int n_eta, const hm_tile_shape* shapes, int n_shapes, int budget_ms,
                      char* json_out, size_t cap, void* stream) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    hm::check_elements(el);
    if (!opt) hm::fail(HM_EINVAL, "autotune: NULL assembly options");
    if (!json_out || cap == 0) hm::fail(HM_EINVAL, "autotune: NULL output buffer");
    if (!leaf_sizes || !etas || n_leaf < 1 || n_eta < 1) hm::fail(HM_EINVAL, "autotune: empty candidate list");
    for (int i = 0; i < n_leaf; ++i)
        if (leaf_sizes[i] < 1 || leaf_sizes[i] > 128) hm::fail(HM_EINVAL, "autotune: leaf sizes must be in [1, 128]");
    for (int j = 0; j < n_eta; ++j)
        if (!(etas[j] > 0.0) || !std::isfinite(etas[j])) hm::fail(HM_EINVAL, "autotune: eta must be positive");
    if (n_shapes < 0 || (n_shapes > 0 && !shapes)) hm::fail(HM_EINVAL, "autotune: bad shape list");
    const std::string js = hm::autotune(*el, *opt, leaf_sizes, n_leaf, etas, n_eta, shapes, n_shapes, budget_ms,
                                        (cudaStream_t)stream);
    if (js.size() + 1 > cap) hm::fail(HM_EINVAL, "autotune: output buffer too small (need " +
                                                     std::to_string(js.size() + 1) + " bytes)");
    std::memcpy(json_out, js.c_str(), js.size() + 1);
    HM_API_END
}

hm_status hm_hmat_set_tile_shape(hm_hmat* hh, const hm_tile_shape* shape, void* stream) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    if (!hh || !shape) hm::fail(HM_EINVAL, "hmat_set_tile_shape: NULL argument");
    hm::set_tile_shape(hh->h, *shape, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_hmat_get_tile_shape(const hm_hmat* hh, hm_tile_shape* shape) {
    HM_API_BEGIN
    if (!hh || !shape) hm::fail(HM_EINVAL, "hmat_get_tile_shape: NULL argument");
    shape->chunk_bytes = hh->h.shape.chunk_bytes;
    shape->chunk_cols = hh->h.shape.chunk_cols;
    shape->ring = hh->h.shape.ring;
    shape->warps = hh->h.shape.warps;
    HM_API_END
}

hm_status hm_tune_tile_shape(hm_hmat* hh, const hm_tile_shape* shapes, int n_shapes, int reps, char* json_out,
                             size_t cap, void* stream) {
    HM_API_BEGIN
    hm::g_last_error.clear();
    if (!hh) hm::fail(HM_EINVAL, "tune_tile_shape: NULL H-matrix");
    if (!json_out || cap == 0) hm::fail(HM_EINVAL, "tune_tile_shape: NULL output buffer");
    const std::string js = hm::tune_tile_shape(hh->h, shapes, n_shapes, reps, (cudaStream_t)stream);
    if (js.size() + 1 > cap)
        hm::fail(HM_EINVAL, "tune_tile_shape: output buffer too small (need " + std::to_string(js.size() + 1) +
                                " bytes)");
    std::memcpy(json_out, js.c_str(), js.size() + 1);
    HM_API_END
}

hm_status hm_hmat_set_wait(hm_hmat* hh, double limit_s, int64_t withhold_chunk) {
    HM_API_BEGIN
    if (!hh) hm::fail(HM_EINVAL, "hmat_set_wait: NULL H-matrix");
    if (!(limit_s >= 1e-6 && limit_s <= 10.0)) hm::fail(HM_EINVAL, "hmat_set_wait: limit must lie in [1e-6, 10] s");
    if (withhold_chunk < -1) hm::fail(HM_EINVAL, "hmat_set_wait: withhold_chunk must be -1 or a chunk index");
    hm::graphs_clear(hh->h);  // captured products hold the old arguments
    hh->h.wait_ns = (uint64_t)(limit_s * 1e9);
    hh->h.withhold_chunk = withhold_chunk;
    HM_API_END
}

hm_status hm_hmat_check(const hm_hmat* hh, void* stream) {
    HM_API_BEGIN
    if (!hh) hm::fail(HM_EINVAL, "hmat_check: NULL H-matrix");
    const int e = hm::product_error_flags(const_cast<hm::HMat&>(hh->h), (cudaStream_t)stream);
    if (e) {
        char buf[128];
        snprintf(buf, sizeof(buf), "hmat_check: a product kernel gave up waiting (flags 0x%x)", e);
        hm::fail(HM_ETIMEOUT, buf);
    }
    HM_API_END
}

}  // extern "C"
