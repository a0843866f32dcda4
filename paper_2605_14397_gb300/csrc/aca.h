// Compression of admissible blocks: adaptive cross approximation with element pivots,
// FP64 recompression, expansion into the compact FP32 factor store.
#pragma once

#include <cstdint>

#include "common.h"

namespace hm {

struct AcaJob {
    int32_t s_begin, s_n, t_begin, t_n;
    int64_t ws_off;  // workspace: U (3 s_n x (R+3)) then V (3 t_n x (R+3)), FP64 column-major
};

struct RecJob {
    int64_t ws_off;  // ACA workspace of the block (U then V)
    int64_t sm_off;  // small workspace: R_U, R_V, M, Z (r x r each), the order (r), FP32 M and Z
    int32_t mS, mT, r, R;
};

// One item of the expansion: rows [row0, row0 + rows) of one factor (side 0: U, 1: V)
// of one block, so that the largest blocks are spread over many CTAs.
struct ExpandJob {
    int64_t ws_off, sm_off;
    int64_t dst;  // compact store offset of the block: U (mS x k) then V (mT x k), FP32 column-major
    int32_t mS, mT, r, k, R, side, row0, rows;
};

// ACA of every job (one CTA each) to relative accuracy eps; rank_out / status_out per
// job (status 1: the rank cap R was reached before convergence).
void launch_aca(const ElemRec* el, const AcaJob* jobs, int njobs, int max_sn, double* ws, int R, double eps,
                double mu, double nu, int32_t* rank_out, int32_t* status_out, unsigned long long* evals,
                cudaStream_t st);
// Recompress the ACA factors of every job; rank_out receives the truncated rank.
void launch_recompress(const RecJob* jobs, int njobs, int R, double* ws, double* small, double tau,
                       int32_t* rank_out, cudaStream_t st);
// Write the truncated factors of every job into the compact FP32 store.
void launch_expand(const ExpandJob* jobs, int njobs, const double* ws, const double* small, float* store,
                   cudaStream_t st);

}  // namespace hm
