// ILU(0) preconditioner of the tangent on the device (ilu_dev.cu; Sec. 3.3.1).
#pragma once

#include "hmat_impl.h"

namespace hm {

// Plan for the fraction p of the near-field entries (selection, leaf-colour order, CSR);
// kept on the H-matrix and rebuilt only when p changes.
void ilu_prepare(HMat& H, double p, cudaStream_t st);
// ILU(0) of the sparse approximation minus diag(d) (d per DOF in cluster order, k + shift);
// HM_EBREAKDOWN on a zero pivot.  err_dev: one int of device scratch.
void ilu_factor(HMat& H, const double* d_cluster, cudaStream_t st, int* err_dev);
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
