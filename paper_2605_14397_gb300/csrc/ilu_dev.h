// ILU(0) preconditioner of the tangent on the device (ilu_dev.cu; Sec. 3.3.1).
#pragma once

#include "hmat_impl.h"

namespace hm {

// Plan for the fraction p of the near-field entries (selection, leaf-colour order, CSR),
// with every element's 3x3 block in the pattern if self_blocks (a block-diagonal C^ep);
// kept on the H-matrix and rebuilt only when p or self_blocks changes.
void ilu_prepare(HMat& H, double p, bool self_blocks, cudaStream_t st);
// ILU(0) of the sparse approximation minus diag(d) (d per DOF in cluster order, k + C^ep's
// diagonal + shift) minus the off-diagonal block entries blk (9 per element in cluster
// order, zero diagonal; NULL without C^ep, which must match the plan); HM_EBREAKDOWN on a
// zero pivot.  err_dev: one int of device scratch.
void ilu_factor(HMat& H, const double* d_cluster, const double* blk, cudaStream_t st, int* err_dev);
// z = (L U)^-1 v for nr right-hand sides (cluster order, RHS-major with stride 3N); zf, if
// given, receives the FP32 copy RHS-interleaved; done[k * done_stride] != 0 skips RHS k.
void ilu_apply(HMat& H, const double* v, double* z, float* zf, int nr, const int* done, int done_stride,
               cudaStream_t st);
bool ilu_is_factored(const HMat& H);
// Sizes, order (new position -> cluster DOF position), CSR pattern, values before and
// after the factorization, to host arrays (any may be NULL).
void ilu_export(HMat& H, int64_t* n_out, int64_t* nnz_out, int32_t* n_colours_out, int32_t* order, int64_t* rowptr,
                int32_t* col, double* a_val, double* lu_val, cudaStream_t st);

}  // namespace hm
