// Device-resident H-matrix: storage layout and work lists.
//
// Layout (all coefficient streams are "leaf-major": everything one leaf cluster of the
// row or column side consumes is one contiguous, column-major block, so a product
// streams each byte once, in order):
//   near stream   for leaf s: [ D_st for t in near(s) ]        ld_s x (sum 3|t|) FP32
//   U stream      for leaf s: [ U_b[s] for b in far, s in S_b ] ld_s x (sum r_b)   FP32|BF16
//   V stream      for leaf t: [ V_b[t] for b in far, t in T_b ] ld_t x (sum r_b)   FP32|BF16
// where ld = 3|leaf| rounded up to 8 entries (the BF16 copies of U and V pad further to an
// odd number of 16-byte lines, see bf16_ld, and have their own offsets) and the rows of
// a slice are the leaf's DOFs in cluster order.
//
// The product y = E x runs as
//   gather     xc = x[perm]                       (cluster order, RHS interleaved)
//   phase 1    P = V_t^T xc_t                      per leaf t (one partial per V column)
//   reduce     tb_b = sum over the leaves t of T_b of the partials of b
//   phase 2    yc_s = [D_s | U_s] z_s,  z = xc (near columns) or tb (U columns)
//   scatter    y[perm] = yc
// A near tile, a U slice and a V slice each read (or write) a contiguous range of
// xc / tb / P, so the operands of a pipeline chunk are one bulk copy.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "common.h"
#include "tree.h"

namespace hm {

struct LeafDesc {
    int32_t begin;     // first cluster position
    int32_t n;         // elements
    int32_t ld;        // padded rows of the FP32 streams (3 n rounded up to 8)
    int32_t ld16;      // padded rows of the BF16 streams (see bf16_ld)
    int64_t near_off;  // entry offset into the near stream
    int64_t u_off;     // entry offset into the U stream (FP32)
    int64_t v_off;     // entry offset into the V stream (FP32)
    int32_t near_cols, u_cols, v_cols;
    int32_t near_cbase, u_cbase, v_cbase;  // first index into the host zidx / pidx arrays
    int32_t pad2_;
    int64_t u_off16, v_off16;  // entry offsets into the BF16 U and V streams
};

// Padded rows of a BF16 stream slice: a multiple of 8 whose 16-byte line count is odd.
// The tensor-core kernels read eight slice columns at once (ldmatrix, one 16-byte line
// per column); with an odd number of lines per column those eight lines fall into eight
// different shared-memory bank groups, where a stride of a multiple of 128 bytes (192
// rows) would put all eight into one.
inline int32_t bf16_ld(int32_t ld) { return (ld / 8) % 2 == 1 ? ld : ld + 8; }

struct FarDesc {
    int32_t s_begin, s_n, t_begin, t_n;  // clusters (positions, element counts)
    int32_t rank;
    int32_t n_tleaves;                   // leaves of T (partials per output)
    int64_t pbase;                       // first of its n_tleaves entries in the partial offset table:
                                         // partial l of the k-th leaf of T is P[poff[pbase + k] + l]
    int64_t tb_off;                      // offset of the block in the compact t order (blocks
                                         // back to back; kept for reference)
    int64_t fac_off;                     // compact factor store offset (U then V)
    int32_t dense;                       // 1: kept dense (its tiles live in the near stream),
                                         // 2: refined into its children blocks (listed later)
    int32_t n_sleaves;                   // leaves of S (copies of t_b)
    int64_t ubase;                       // first of its n_sleaves entries in the t-copy table: the
                                         // k-th leaf of S reads t_b at tb[uoff[ubase + k] ...]
};

// One pipeline chunk: whole columns of one tile or factor slice of one leaf, at most one
// stage of bytes and 64 columns.
struct Chunk {
    int64_t src;    // first entry in its stream
    int64_t zoff;   // first operand index: xc (near), tb (U) or output partial (V)
    int32_t leaf;   // leaf ordinal
    int32_t ncols;
    int32_t kind;   // 0 near tile (FP32), 1 U factor, 2 V factor
    int32_t ld;     // padded rows of the leaf
};

// Row leaves whose phase-2 columns are split over several persistent CTAs.
struct LeafSplit {
    int32_t w_first;    // first CTA holding columns of the leaf
    int32_t nparts;     // CTAs holding columns of the leaf (1 = not split)
    int32_t slot_base;  // first partial slot
    int32_t pad_;
};

struct SolveWS;                  // solver workspace (solve.cu)
void solve_ws_free(SolveWS* w);
struct IluPlan;                  // ILU(0) preconditioner of the tangent (ilu_dev.cu)
void ilu_plan_free(IluPlan* p);

struct HMat {
    SolveWS* solve_ws = nullptr;
    int64_t N = 0, ndof = 0;
    double E = 1.0, nu = 0.25, eps = 1e-6;
    int storage = HM_F32;
    int n_leaves = 0;
    int64_t n_far = 0, n_near = 0, n_dense_far = 0, n_refined = 0;
    int64_t tb_len = 0, p_len = 0;  // tb_len: t entries with their copies (U columns)
    int64_t near_entries = 0, far_entries = 0;
    int rank_min = 0, rank_max = 0;
    double rank_mean = 0.0, assemble_seconds = 0.0;
    int64_t aca_blocks = 0;  // 3x3 influence blocks evaluated by the cross approximation

    std::vector<LeafDesc> h_leaves;
    std::vector<FarDesc> h_far;
    std::vector<int64_t> h_perm;

    DevBuf<ElemRec> elems;        // cluster order
    DevBuf<int32_t> perm;         // cluster position -> user element
    DevBuf<LeafDesc> leaves;
    DevBuf<FarDesc> far;
    DevBuf<float> near;           // near stream
    DevBuf<float> u32, v32;       // factor streams (FP32 storage)
    DevBuf<uint16_t> u16, v16;    // factor streams (BF16 storage)
    DevBuf<float> facstore;       // compact FP32 factors per far block (U then V)
    // operand index of every column (host; consecutive runs become the z ranges of the
    // product chunks): xc index (near), tb index (U), partial index (V)
    std::vector<int32_t> h_near_zidx, h_u_zidx, h_v_pidx;
    DevBuf<int32_t> near_zidx;    // device copy of h_near_zidx (made on first use)
    // V columns write their partials in V-stream order, so the slices of one column leaf
    // form one contiguous output range (whole pipeline chunks); poff locates each far
    // block's slice in every leaf of its column cluster
    std::vector<int32_t> h_poff;
    DevBuf<int32_t> poff;
    // t_b is written once for every leaf of the row cluster S, at the position of that
    // leaf's U slice in U-stream order, so a leaf's U columns read one contiguous range of
    // tb and its chunks span blocks; uoff locates each copy
    std::vector<int32_t> h_uoff;
    DevBuf<int32_t> uoff;
    // single-RHS reduction order: the n_red_big blocks with many leaves of T first (a CTA
    // each), then the rest (a warp each); blocks without factors are left out
    DevBuf<int32_t> red_order;
    int64_t n_red_big = 0, n_red = 0;

    // tile shape of the product: bytes and columns of a pipeline chunk (at most one 32 KB
    // stage and 128 columns), ring depth (4 or 6 stages) and consumer warps (16 or 8) of
    // the single-RHS FP32-vector product; the plans below are cut with it
    struct TileShape {
        int chunk_bytes = 32768, chunk_cols = 128, ring = 4, warps = 16;
    } shape;
    // persistent product plans: [0] with the FP32 factors, [1] with the BF16 factors
    int grid = 0;
    int ld_max = 0;
    struct Plan {
        bool ready = false;
        int n_slots = 0;
        DevBuf<Chunk> ch1, ch2;
        DevBuf<int32_t> cta1, cta2;
        DevBuf<LeafSplit> split;
    } plan[2];
    DevBuf<int32_t> counters;
    DevBuf<int> err;
    uint64_t wait_ns = 2000000000ull;  // limit of the product's bounded waits
    int64_t withhold_chunk = -1;       // test switch of hm_hmat_set_wait (-1: off)
    std::vector<int64_t> h_self_off;  // near-stream offset of each leaf's diagonal tile
    // per leaf: the first columns of its near block that belong to inadmissible leaf pairs
    // (the near field proper; admissible blocks stored dense follow them)
    std::vector<int32_t> h_near_true_cols;
    IluPlan* ilu = nullptr;           // ILU preconditioner plan (ilu_dev.cu), built on demand
    DevBuf<float> slotsf;
    DevBuf<double> slotsd;

    // per-phase timing (CUDA events, 6 per product) and host-vector staging
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double t_acc[5] = {0, 0, 0, 0, 0};
    int64_t t_count = 0;
    DevBuf<unsigned char> xs, ys;

    // instantiated product graphs, one per (x, y, nrhs, dtype), captured on cap_stream
    struct GraphEntry {
        const void* x;
        void* y;
        int nrhs, dtype;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;

    HMat() = default;
    HMat(const HMat&) = delete;
    HMat& operator=(const HMat&) = delete;
    ~HMat() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (GraphEntry& g : graphs) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        solve_ws_free(solve_ws);
        ilu_plan_free(ilu);
    }

    // product scratch, sized for nrhs_cap right-hand sides
    int nrhs_cap = 0;
    DevBuf<double> xc, yc;        // cluster-order vectors (F64 path) [nrhs][ndof]
    DevBuf<float> xcf, ycf;       // (F32 path)
    DevBuf<double> P, tb;         // partials / t vectors (F64 path uses hi+lo pairs as double)
    DevBuf<float> Pf, tbf;

    int64_t stored_bytes() const {
        return (int64_t)near.bytes() + (int64_t)u32.bytes() + (int64_t)v32.bytes() + (int64_t)u16.bytes() +
               (int64_t)v16.bytes();
    }
};

void assemble(const Tree& T, const hm_assemble_opts& opt, cudaStream_t st, HMat& H);
void ensure_product_scratch(HMat& H, int nrhs, cudaStream_t st);
void build_product_plan(HMat& H, cudaStream_t st);
int product_error_flags(HMat& H, cudaStream_t st);
void timing_enable(HMat& H, bool on);
void timing_read(HMat& H, double out[6]);
void matvec_host(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st);
void matvec(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st, int factors = 0);
// Product on cluster-ordered operands: xc is RHS-interleaved (xc[dof * nr + k]) with at
// least 32 readable elements after its end, yc is RHS-major (yc[k * ndof + dof]).
// fac: 0 FP32 factors, 1 BF16 factors.  dtype HM_F32: float vectors; HM_F64: xc holds
// every double pre-split into (hi, lo) floats (float2, written by the gather or the
// solver), yc doubles.
void product_core(HMat& H, const void* xc, void* yc, int nr, int dtype, int fac, cudaStream_t st,
                  const int* skip = nullptr);
// Concatenate independent H-matrices into one (block-diagonal operator, one work list).
void merge(const std::vector<const HMat*>& hs, cudaStream_t st, HMat& M);
// tile shape of the product (plans rebuilt) and its tuning over a candidate list
void set_tile_shape(HMat& H, const hm_tile_shape& t, cudaStream_t st);
std::string tune_tile_shape(HMat& H, const hm_tile_shape* shapes, int n, int reps, cudaStream_t st);
void graphs_clear(HMat& H);
void matvec_graph(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st);
struct LPModel;
void ilu_export_for(HMat& H, const double* kel, const double* cep, double shift, double p, int64_t* n_out,
                    int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr, int32_t* col,
                    double* a_val, double* lu_val, cudaStream_t st);
void ilu_apply_user(HMat& H, const double* r, double* z, int nrhs, cudaStream_t st);
// y = (E - diag(k) - C^ep - shift I) x, one user-ordered FP64 vector (synchronises)
void tangent_apply_user(HMat& H, const double* kel, const double* cep, double shift, const double* x, double* y,
                        cudaStream_t st);
// the diagonal of that tangent per DOF, user order (FP32 near-field entries of E)
void tangent_diag_user(HMat& H, const double* kel, const double* cep, double shift, double* out, cudaStream_t st);
void gmres_solve(HMat& H, const double* kel, double shift, const double* b, double* x, int nrhs,
                 const hm_solve_opts& o, hm_solve_info* info, cudaStream_t st, const LPModel* lp = nullptr);
// z = M^-1 r with the preconditioner of gmres_solve for these options (user order)
void precond_apply_user(HMat& H, const double* kel, double shift, const hm_solve_opts& o, const LPModel* lp,
                        const double* r, double* z, int nrhs, cudaStream_t st);
inline bool has_factors(const HMat& H, int fac) {
    return fac == 0 ? (H.storage == HM_F32 || H.storage == HM_F32_BF16)
                    : (H.storage == HM_BF16 || H.storage == HM_F32_BF16);
}

}  // namespace hm

// C handle of an assembled H-matrix (include/hmat.h)
struct hm_hmat {
    hm::HMat h;
};
