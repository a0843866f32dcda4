// Learned block-Jacobi correction: model state and the entry points the solver uses.
//
// Two kinds of correction of B^-1 by d = 1 + 0.5 tanh(o) per (leaf, component):
//   scale:  M^-1 r = D B^-1 r;
//   near:   M^-1 r = y - gamma D B^-1 N y,  y = B^-1 r,  N = the near-field blocks of E off
//           the diagonal leaf blocks (a damped first Neumann term of the near coupling).
// d comes from the output o
// of a two-hidden-layer tanh network evaluated per leaf on eight leaf features (the
// stiffness distribution of the leaf relative to E/h, its size, planarity and distance to
// another fracture plane).  B is the leaf block-Jacobi preconditioner of A = E - diag(k)
// (the Jacobi preconditioner of Sec. 3.3.1 taken per leaf).  The network is trained on
// the device by Adam on the approximate-inverse loss over solved systems: sum |x - D y|^2
// (scale) or sum |(y - x) - D w|^2, w = B^-1 N y (near), which separate into
// per-(leaf, component) sums (see learned.cu); gamma is chosen by the caller on
// validation systems (GMRES iterations as the judge).
#pragma once

#include <cstdint>
#include <vector>

#include "hmat_impl.h"

namespace hm {

constexpr int LP_FEATURES = 8;
constexpr int LP_OUT = 3;
constexpr int LP_SAMPLE_Q = 9;  // q_xy[3], q_yy[3], q_xx[3]

inline int64_t lp_param_count(int H) {
    return (int64_t)H * LP_FEATURES + H + (int64_t)H * H + H + LP_OUT * H + LP_OUT;
}

enum { LP_SCALE = 0, LP_NEAR = 1 };

struct LPModel {
    int H = 32;
    int kind = LP_SCALE;     // LP_SCALE or LP_NEAR
    double gamma = 1.0;      // LP_NEAR: factor on the predicted d
    int64_t P = 0;
    int fallback = 0;        // 1: the solver applies plain block-Jacobi
    int64_t steps = 0;       // Adam steps taken
    double last_loss = 0.0;
    std::vector<float> theta_h, m_h, v_h;  // host mirror of parameters and Adam moments
    // training samples (host; uploaded before training): one row per (system, leaf)
    std::vector<float> X_h;  // S x 8
    std::vector<float> Q_h;  // S x 9, already divided by the system's sum |x|^2
    int n_groups = 0;        // systems (or sample batches) added: the loss averages over them

    // device state, allocated on first use
    bool dev_ready = false;
    bool samples_dirty = true;
    DevBuf<float> theta, m, v, grad;
    DevBuf<float> X, Q, act;  // samples and per-sample activations / deltas
    DevBuf<double> gsum;
};

// per-leaf scalings d (n_leaves x 3, device) of the model for this H-matrix and k
// (k_dev: N doubles, user order, or NULL); features_out (n_leaves x 8, device, FP64) if
// not NULL.
void lp_predict(LPModel& M, HMat& H, const double* k_dev, float* d_out, double* features_out, cudaStream_t st);

// block-Jacobi solve z = B^-1 v for cluster-ordered vectors (nr x 3N), with B built for
// A = E - diag(k) - shift I (solve.cu)
void bj_solve_cluster(HMat& H, const double* kel, double shift, const double* v, double* z, int nr,
                      cudaStream_t st);
// out = N v for cluster-ordered vectors (nr x 3N): the near-field tiles of E off the
// diagonal leaf blocks, FP32 coefficients, FP64 vectors (solve.cu)
void near_offdiag_cluster(HMat& H, const double* v, double* out, int nr, cudaStream_t st);
void to_cluster(HMat& H, const double* user, double* cluster, int nr, cudaStream_t st);

}  // namespace hm

struct hm_lp {
    hm::LPModel m;
};
