// Learned block-Jacobi correction on the device: leaf features, the network's forward
// and backward passes, the training statistics and Adam (learned.h states the model).
//
// Training loss over the samples s = (system, leaf) with targets q = S / T_system:
//   loss = (1 / n_groups) sum_s sum_a  q_xx - 2 d_a q_xy + d_a^2 q_yy
// where S = (S_xy, S_yy, S_xx) are the leaf/component sums of x y, y y, x x over the
// system's right-hand sides (x the solution, y = B^-1 b) and T the system's sum x x.
// Everything is deterministic: per-sample activations and deltas are stored, parameter
// gradients are reduced per fixed chunk of samples and the chunks summed in order.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>

#include "learned.h"

namespace hm {

namespace {

constexpr int FEAT_NT = 128;
constexpr int SAMPLE_CHUNK = 256;

// ---------------------------------------------------------------- features (FP64)

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
    return s;
}

__device__ __forceinline__ double block_min_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = sh[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) s = fmin(s, sh[q]);
    return s;
}

// Features 0-6 per leaf (one CTA each), and the leaf centroid, mean normal and mean
// element size for feature 7.
__global__ void __launch_bounds__(FEAT_NT) k_lp_leaf(const LeafDesc* __restrict__ leaves,
                                                    const ElemRec* __restrict__ el, const int32_t* __restrict__ perm,
                                                    const double* __restrict__ kel, double E,
                                                    double* __restrict__ feat, double* __restrict__ geo) {
    __shared__ double sh[FEAT_NT / 32];
    const LeafDesc L = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    double s_kap = 0.0, s_soft = 0.0, mn = 1e300, mx = -1e300, s_h = 0.0;
    double c[3] = {0, 0, 0}, nn[3] = {0, 0, 0};
    for (int i = tid; i < L.n; i += FEAT_NT) {
        const ElemRec& e = el[L.begin + i];
        const double h = sqrt(4.0 * e.a * e.b);
        const double kv = kel ? kel[perm[L.begin + i]] : 0.0;
        const double s = kv * h / E;
        const double kap = log10(s + 1e-6);
        s_kap += kap;
        s_soft += s < 0.5 ? 1.0 : 0.0;
        mn = fmin(mn, kap);
        mx = fmax(mx, kap);
        s_h += h;
        for (int q = 0; q < 3; ++q) {
            c[q] += e.c[q];
            nn[q] += e.n[q];
        }
    }
    const double n = (double)L.n;
    const double mu = block_sum_d(s_kap, sh) / n;
    const double soft = block_sum_d(s_soft, sh) / n;
    const double hbar = block_sum_d(s_h, sh) / n;
    double cm[3], nm[3];
    for (int q = 0; q < 3; ++q) {
        cm[q] = block_sum_d(c[q], sh) / n;
        nm[q] = block_sum_d(nn[q], sh) / n;
    }
    mn = block_min_d(mn, sh);
    mx = -block_min_d(-mx, sh);
    // second pass: standard deviation about the mean
    double s2 = 0.0;
    for (int i = tid; i < L.n; i += FEAT_NT) {
        const ElemRec& e = el[L.begin + i];
        const double h = sqrt(4.0 * e.a * e.b);
        const double kv = kel ? kel[perm[L.begin + i]] : 0.0;
        const double d = log10(kv * h / E + 1e-6) - mu;
        s2 += d * d;
    }
    const double var = block_sum_d(s2, sh) / n;
    if (tid == 0) {
        double* f = feat + (size_t)blockIdx.x * LP_FEATURES;
        f[0] = mu;
        f[1] = sqrt(var);
        f[2] = mn;
        f[3] = mx;
        f[4] = soft;
        f[5] = log10(n);
        f[6] = sqrt(nm[0] * nm[0] + nm[1] * nm[1] + nm[2] * nm[2]);
        double* g = geo + (size_t)blockIdx.x * 7;
        for (int q = 0; q < 3; ++q) {
            g[q] = cm[q];
            g[3 + q] = nm[q];
        }
        g[6] = hbar;
    }
}

// Feature 7: distance from the leaf centroid to the nearest centroid of a leaf whose mean
// normal points another way, relative to the mean element size.
__global__ void __launch_bounds__(FEAT_NT) k_lp_distance(const double* __restrict__ geo, int nl,
                                                        double* __restrict__ feat) {
    __shared__ double sh[FEAT_NT / 32];
    const double* g = geo + (size_t)blockIdx.x * 7;
    const double nl2 = sqrt(g[3] * g[3] + g[4] * g[4] + g[5] * g[5]);
    double best = 1e300;
    for (int m = threadIdx.x; m < nl; m += FEAT_NT) {
        if (m == (int)blockIdx.x) continue;
        const double* o = geo + (size_t)m * 7;
        const double dot = fabs(g[3] * o[3] + g[4] * o[4] + g[5] * o[5]);
        const double no = sqrt(o[3] * o[3] + o[4] * o[4] + o[5] * o[5]);
        if (dot < 0.99 * nl2 * no) {
            const double dx = g[0] - o[0], dy = g[1] - o[1], dz = g[2] - o[2];
            best = fmin(best, sqrt(dx * dx + dy * dy + dz * dz));
        }
    }
    best = block_min_d(best, sh);
    if (threadIdx.x == 0) {
        const double d = best < 1e299 ? best : 1000.0 * g[6];
        feat[(size_t)blockIdx.x * LP_FEATURES + 7] = log10(1.0 + d / g[6]);
    }
}

// ---------------------------------------------------------------- network (FP32)

struct Net {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

template <int H>
__device__ __forceinline__ Net net_view(const float* th) {
    Net n;
    n.W1 = th;
    n.b1 = n.W1 + H * LP_FEATURES;
    n.W2 = n.b1 + H;
    n.b2 = n.W2 + H * H;
    n.W3 = n.b2 + H;
    n.b3 = n.W3 + LP_OUT * H;
    return n;
}

// forward of one sample: a1, a2 (H each) and t = tanh(o) (3)
template <int H>
__device__ __forceinline__ void net_forward(const Net& n, const float* x, float* a1, float* a2, float* t) {
    for (int i = 0; i < H; ++i) {
        float z = n.b1[i];
#pragma unroll
        for (int j = 0; j < LP_FEATURES; ++j) z = fmaf(n.W1[i * LP_FEATURES + j], x[j], z);
        a1[i] = tanhf(z);
    }
    for (int i = 0; i < H; ++i) {
        float z = n.b2[i];
        for (int j = 0; j < H; ++j) z = fmaf(n.W2[i * H + j], a1[j], z);
        a2[i] = tanhf(z);
    }
    for (int a = 0; a < LP_OUT; ++a) {
        float z = n.b3[a];
        for (int j = 0; j < H; ++j) z = fmaf(n.W3[a * H + j], a2[j], z);
        t[a] = tanhf(z);
    }
}

// d per leaf from FP64 features (inference)
template <int H>
__global__ void k_lp_forward(const float* __restrict__ theta, int64_t P, const double* __restrict__ feat, int nl,
                             float* __restrict__ d) {
    extern __shared__ float th[];
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const Net n = net_view<H>(th);
    float x[LP_FEATURES], a1[H], a2[H], t[LP_OUT];
#pragma unroll
    for (int j = 0; j < LP_FEATURES; ++j) x[j] = (float)feat[(size_t)l * LP_FEATURES + j];
    net_forward<H>(n, x, a1, a2, t);
#pragma unroll
    for (int a = 0; a < LP_OUT; ++a) d[(size_t)l * LP_OUT + a] = 1.0f + 0.5f * t[a];
}

// Forward and backward of every training sample (one thread each): stores the row
// [a1 (H) | a2 (H) | dloss/dz1 (H) | dloss/dz2 (H) | dloss/do (3)] and the sample's loss.
template <int H>
__global__ void k_lp_fwdbwd(const float* __restrict__ theta, int64_t P, const float* __restrict__ X,
                            const float* __restrict__ Q, int64_t S, float scale, float* __restrict__ act,
                            double* __restrict__ loss) {
    extern __shared__ float th[];
    for (int64_t p = threadIdx.x; p < P; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S) return;
    const Net n = net_view<H>(th);
    float x[LP_FEATURES], a1[H], a2[H], t[LP_OUT];
#pragma unroll
    for (int j = 0; j < LP_FEATURES; ++j) x[j] = X[s * LP_FEATURES + j];
    net_forward<H>(n, x, a1, a2, t);
    const float* q = Q + s * LP_SAMPLE_Q;
    float go[LP_OUT];
    double l = 0.0;
#pragma unroll
    for (int a = 0; a < LP_OUT; ++a) {
        const float d = 1.0f + 0.5f * t[a];
        const float qxy = q[a], qyy = q[3 + a], qxx = q[6 + a];
        l += (double)qxx - 2.0 * (double)d * qxy + (double)d * d * qyy;
        const float gd = 2.0f * (d * qyy - qxy) * scale;
        go[a] = gd * 0.5f * (1.0f - t[a] * t[a]);
    }
    loss[s] = l * scale;
    float* row = act + s * (4 * H + LP_OUT);
    float gz2[H];
    for (int j = 0; j < H; ++j) {
        float g = 0.f;
#pragma unroll
        for (int a = 0; a < LP_OUT; ++a) g = fmaf(go[a], n.W3[a * H + j], g);
        gz2[j] = g * (1.0f - a2[j] * a2[j]);
    }
    for (int j = 0; j < H; ++j) {
        float g = 0.f;
        for (int i = 0; i < H; ++i) g = fmaf(gz2[i], n.W2[i * H + j], g);
        row[2 * H + j] = g * (1.0f - a1[j] * a1[j]);
    }
    for (int j = 0; j < H; ++j) {
        row[j] = a1[j];
        row[H + j] = a2[j];
        row[3 * H + j] = gz2[j];
    }
#pragma unroll
    for (int a = 0; a < LP_OUT; ++a) row[4 * H + a] = go[a];
}

// Partial parameter gradients: thread = parameter, blockIdx.y = chunk of samples;
// part[chunk * P + p] = sum over the chunk's samples of (delta x input) for p.
template <int H>
__global__ void k_lp_param_grad(const float* __restrict__ X, const float* __restrict__ act, int64_t S, int64_t P,
                                double* __restrict__ part) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    constexpr int R = 4 * H + LP_OUT;
    // decode p: which delta (offset in the row) times which input (X column, act column or 1)
    int dcol, icol;
    bool from_x = false, bias = false;
    int64_t q = p;
    if (q < H * LP_FEATURES) {
        dcol = 2 * H + (int)(q / LP_FEATURES);
        icol = (int)(q % LP_FEATURES);
        from_x = true;
    } else if ((q -= H * LP_FEATURES) < H) {
        dcol = 2 * H + (int)q;
        icol = 0;
        bias = true;
    } else if ((q -= H) < H * H) {
        dcol = 3 * H + (int)(q / H);
        icol = (int)(q % H);  // a1
    } else if ((q -= H * H) < H) {
        dcol = 3 * H + (int)q;
        icol = 0;
        bias = true;
    } else if ((q -= H) < LP_OUT * H) {
        dcol = 4 * H + (int)(q / H);
        icol = H + (int)(q % H);  // a2
    } else {
        q -= LP_OUT * H;
        dcol = 4 * H + (int)q;
        icol = 0;
        bias = true;
    }
    const int64_t s0 = (int64_t)blockIdx.y * SAMPLE_CHUNK, s1 = min(S, s0 + SAMPLE_CHUNK);
    double acc = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
        const float dv = act[s * R + dcol];
        const float iv = bias ? 1.0f : (from_x ? X[s * LP_FEATURES + icol] : act[s * R + icol]);
        acc += (double)dv * (double)iv;
    }
    part[(int64_t)blockIdx.y * P + p] = acc;
}

// grad[p] = sum of the chunk partials in chunk order
__global__ void k_lp_grad_sum(const double* __restrict__ part, int64_t P, int nchunk, double* __restrict__ gsum,
                              float* __restrict__ grad) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * P + p];
    gsum[p] = s;
    grad[p] = (float)s;
}

// total loss, one CTA, fixed order
__global__ void k_lp_loss_sum(const double* __restrict__ loss, int64_t S, double* __restrict__ out) {
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) s += loss[i];
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// Adam (Kingma and Ba, 2015), step t >= 1
__global__ void k_lp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                          const float* __restrict__ g, int64_t P, float lr, float c1, float c2) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mm = b1 * m[p] + (1.0f - b1) * g[p];
    const float vv = b2 * v[p] + (1.0f - b2) * g[p] * g[p];
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Per (leaf, component) sums over the right-hand sides of x y, y y, x x (cluster order,
// RHS-major vectors), FP64: S[leaf][0..8] = [S_xy | S_yy | S_xx].
__global__ void __launch_bounds__(FEAT_NT) k_lp_stats(const LeafDesc* __restrict__ leaves,
                                                     const double* __restrict__ x, const double* __restrict__ y,
                                                     int64_t ndof, int nr, double* __restrict__ S) {
    __shared__ double sh[FEAT_NT / 32];
    const LeafDesc L = leaves[blockIdx.x];
    const int n = 3 * L.n;
    double v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = 0.0;
    for (int k = 0; k < nr; ++k)
        for (int r = threadIdx.x; r < n; r += FEAT_NT) {
            const int64_t i = k * ndof + 3 * (int64_t)L.begin + r;
            const double xv = x[i], yv = y[i];
            const int a = r % 3;
            // component-selected accumulation without dynamic register indexing
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (c == a) {
                    v[c] += xv * yv;
                    v[3 + c] += yv * yv;
                    v[6 + c] += xv * xv;
                }
        }
    for (int q = 0; q < 9; ++q) {
        const double t = block_sum_d(v[q], sh);
        if (threadIdx.x == 0) S[(size_t)blockIdx.x * 9 + q] = t;
    }
}


// x = y - x (the near correction fits D w to the part y - x that B^-1 gets wrong)
__global__ void k_lp_diff(const double* __restrict__ y, double* __restrict__ x, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = y[i] - x[i];
}

// ---------------------------------------------------------------- host side

template <class F>
void with_h(int H, F&& f) {
    if (H == 16)
        f(std::integral_constant<int, 16>{});
    else if (H == 32)
        f(std::integral_constant<int, 32>{});
    else if (H == 64)
        f(std::integral_constant<int, 64>{});
    else
        fail(HM_EINVAL, "learned correction: hidden width must be 16, 32 or 64");
}

void lp_device_init(LPModel& M, cudaStream_t st) {
    if (M.dev_ready) return;
    M.theta.alloc(M.P);
    M.m.alloc(M.P);
    M.v.alloc(M.P);
    M.grad.alloc(M.P);
    M.gsum.alloc(M.P + 1);
    HM_CUDA(cudaMemcpyAsync(M.theta.p, M.theta_h.data(), M.P * sizeof(float), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(M.m.p, M.m_h.data(), M.P * sizeof(float), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(M.v.p, M.v_h.data(), M.P * sizeof(float), cudaMemcpyHostToDevice, st));
    M.dev_ready = true;
}

void lp_sync_host(LPModel& M, cudaStream_t st) {
    HM_CUDA(cudaMemcpyAsync(M.theta_h.data(), M.theta.p, M.P * sizeof(float), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(M.m_h.data(), M.m.p, M.P * sizeof(float), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(M.v_h.data(), M.v.p, M.P * sizeof(float), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
}

int64_t n_samples(const LPModel& M) { return (int64_t)M.X_h.size() / LP_FEATURES; }

void lp_upload_samples(LPModel& M, cudaStream_t st) {
    if (!M.samples_dirty) return;
    const int64_t S = n_samples(M);
    if (S == 0) fail(HM_EINVAL, "learned correction: no training samples");
    M.X.upload(M.X_h, st);
    M.Q.upload(M.Q_h, st);
    M.act.alloc((size_t)S * (4 * M.H + LP_OUT));
    M.samples_dirty = false;
}

// loss and gradient at the current parameters (gradient left in M.grad / M.gsum)
double lp_loss_grad(LPModel& M, cudaStream_t st) {
    lp_device_init(M, st);
    lp_upload_samples(M, st);
    const int64_t S = n_samples(M);
    const int nchunk = (int)ceil_div(S, SAMPLE_CHUNK);
    DevBuf<double> part((size_t)nchunk * M.P), loss((size_t)S);
    const float scale = 1.0f / (float)std::max(M.n_groups, 1);
    with_h(M.H, [&](auto hc) {
        constexpr int H = decltype(hc)::value;
        const size_t smem = (size_t)M.P * sizeof(float);
        if (smem > 48 * 1024)
            HM_CUDA(cudaFuncSetAttribute(k_lp_fwdbwd<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lp_fwdbwd<H><<<(unsigned)ceil_div(S, 128), 128, smem, st>>>(M.theta.p, M.P, M.X.p, M.Q.p, S, scale,
                                                                     M.act.p, loss.p);
        HM_LAUNCH_CHECK();
        dim3 g((unsigned)ceil_div(M.P, 128), (unsigned)nchunk);
        k_lp_param_grad<H><<<g, 128, 0, st>>>(M.X.p, M.act.p, S, M.P, part.p);
        HM_LAUNCH_CHECK();
    });
    k_lp_grad_sum<<<(unsigned)ceil_div(M.P, 256), 256, 0, st>>>(part.p, M.P, nchunk, M.gsum.p, M.grad.p);
    k_lp_loss_sum<<<1, 256, 0, st>>>(loss.p, S, M.gsum.p + M.P);
    HM_LAUNCH_CHECK();
    double l = 0.0;
    HM_CUDA(cudaMemcpyAsync(&l, M.gsum.p + M.P, sizeof(double), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    return l;
}

double lp_train(LPModel& M, int steps, double lr, cudaStream_t st) {
    double l = 0.0;
    for (int it = 0; it < steps; ++it) {
        l = lp_loss_grad(M, st);
        ++M.steps;
        const float c1 = 1.0f - powf(0.9f, (float)M.steps), c2 = 1.0f - powf(0.999f, (float)M.steps);
        k_lp_adam<<<(unsigned)ceil_div(M.P, 256), 256, 0, st>>>(M.theta.p, M.m.p, M.v.p, M.grad.p, M.P, (float)lr,
                                                               c1, c2);
        HM_LAUNCH_CHECK();
    }
    lp_sync_host(M, st);
    M.last_loss = l;
    return l;
}

void lp_features(HMat& H, const double* k_dev, double* feat, cudaStream_t st) {
    DevBuf<double> geo((size_t)H.n_leaves * 7);
    const double E = std::isfinite(H.E) ? H.E : 1.0;
    k_lp_leaf<<<H.n_leaves, FEAT_NT, 0, st>>>(H.leaves.p, H.elems.p, H.perm.p, k_dev, E, feat, geo.p);
    k_lp_distance<<<H.n_leaves, FEAT_NT, 0, st>>>(geo.p, H.n_leaves, feat);
    HM_LAUNCH_CHECK();
    HM_CUDA(cudaStreamSynchronize(st));
}

void lp_add_system(LPModel& M, HMat& H, const double* k_dev, const double* b, const double* x, int nr,
                   cudaStream_t st) {
    if (nr < 1 || nr > 16) fail(HM_EINVAL, "lp_add_system: 1 to 16 right-hand sides");
    if (!b || !x) fail(HM_EINVAL, "lp_add_system: NULL vector");
    const int64_t n = H.ndof;
    DevBuf<double> bc((size_t)n * nr), xc((size_t)n * nr), yc((size_t)n * nr);
    DevBuf<double> feat((size_t)H.n_leaves * LP_FEATURES), S((size_t)H.n_leaves * 9);
    to_cluster(H, b, bc.p, nr, st);
    to_cluster(H, x, xc.p, nr, st);
    bj_solve_cluster(H, k_dev, 0.0, bc.p, yc.p, nr, st);
    if (M.kind == LP_NEAR) {
        // the statistics of (y - x, w), w = B^-1 N y: the loss |(y - x) - d w|^2
        DevBuf<double> t((size_t)n * nr), w((size_t)n * nr);
        near_offdiag_cluster(H, yc.p, t.p, nr, st);
        bj_solve_cluster(H, k_dev, 0.0, t.p, w.p, nr, st);
        k_lp_diff<<<(unsigned)ceil_div((int64_t)n * nr, 256), 256, 0, st>>>(yc.p, xc.p, (int64_t)n * nr);
        k_lp_stats<<<H.n_leaves, FEAT_NT, 0, st>>>(H.leaves.p, xc.p, w.p, n, nr, S.p);
    } else {
        k_lp_stats<<<H.n_leaves, FEAT_NT, 0, st>>>(H.leaves.p, xc.p, yc.p, n, nr, S.p);
    }
    HM_LAUNCH_CHECK();
    lp_features(H, k_dev, feat.p, st);
    std::vector<double> hf((size_t)H.n_leaves * LP_FEATURES), hs((size_t)H.n_leaves * 9);
    HM_CUDA(cudaMemcpyAsync(hf.data(), feat.p, hf.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(hs.data(), S.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    double T = 0.0;
    for (int l = 0; l < H.n_leaves; ++l)
        for (int a = 0; a < 3; ++a) T += hs[(size_t)l * 9 + 6 + a];
    if (!(T > 0.0) || !std::isfinite(T)) fail(HM_EINVAL, "lp_add_system: the solution is zero or not finite");
    for (int l = 0; l < H.n_leaves; ++l) {
        for (int j = 0; j < LP_FEATURES; ++j) M.X_h.push_back((float)hf[(size_t)l * LP_FEATURES + j]);
        for (int q = 0; q < 9; ++q) M.Q_h.push_back((float)(hs[(size_t)l * 9 + q] / T));
    }
    ++M.n_groups;
    M.samples_dirty = true;
}

}  // namespace

void lp_predict(LPModel& M, HMat& H, const double* k_dev, float* d_out, double* features_out, cudaStream_t st) {
    lp_device_init(M, st);
    DevBuf<double> own;
    double* feat = features_out;
    if (!feat) {
        own.alloc((size_t)H.n_leaves * LP_FEATURES);
        feat = own.p;
    }
    lp_features(H, k_dev, feat, st);
    with_h(M.H, [&](auto hc) {
        constexpr int H_ = decltype(hc)::value;
        const size_t smem = (size_t)M.P * sizeof(float);
        if (smem > 48 * 1024)
            HM_CUDA(cudaFuncSetAttribute(k_lp_forward<H_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_lp_forward<H_><<<(unsigned)ceil_div(H.n_leaves, 128), 128, smem, st>>>(M.theta.p, M.P, feat, H.n_leaves,
                                                                                d_out);
        HM_LAUNCH_CHECK();
    });
    HM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace hm

// ---------------------------------------------------------------- C ABI

namespace {
const char LP_MAGIC1[8] = {'H', 'M', 'L', 'P', '0', '0', '0', '1'};  // scale kind only
const char LP_MAGIC[8] = {'H', 'M', 'L', 'P', '0', '0', '0', '2'};   // + kind and gamma
hm::LPModel& model(hm_lp* lp) {
    if (!lp) hm::fail(HM_EINVAL, "learned correction: NULL handle");
    return lp->m;
}
}  // namespace

extern "C" {

int64_t hm_lp_param_count(int hidden) {
    return (hidden == 16 || hidden == 32 || hidden == 64) ? hm::lp_param_count(hidden) : -1;
}

hm_status hm_lp_create(int hidden, const double* theta0, hm_lp** out) {
    HM_API_BEGIN
    if (!out) hm::fail(HM_EINVAL, "lp_create: NULL output handle");
    *out = nullptr;
    if (hm_lp_param_count(hidden) < 0) hm::fail(HM_EINVAL, "lp_create: hidden width must be 16, 32 or 64");
    if (!theta0) hm::fail(HM_EINVAL, "lp_create: NULL initial parameters");
    hm_lp* lp = new hm_lp();
    hm::LPModel& M = lp->m;
    M.H = hidden;
    M.P = hm::lp_param_count(hidden);
    M.theta_h.resize(M.P);
    M.m_h.assign(M.P, 0.0f);
    M.v_h.assign(M.P, 0.0f);
    for (int64_t p = 0; p < M.P; ++p) {
        if (!std::isfinite(theta0[p])) {
            delete lp;
            hm::fail(HM_ENAN, "lp_create: non-finite initial parameter");
        }
        M.theta_h[p] = (float)theta0[p];
    }
    *out = lp;
    HM_API_END
}

hm_status hm_lp_add_samples(hm_lp* lp, const double* features, const double* q, int64_t n) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    if (n < 1 || !features || !q) hm::fail(HM_EINVAL, "lp_add_samples: need n >= 1 samples");
    for (int64_t i = 0; i < n * hm::LP_FEATURES; ++i) M.X_h.push_back((float)features[i]);
    for (int64_t i = 0; i < n * hm::LP_SAMPLE_Q; ++i) M.Q_h.push_back((float)q[i]);
    ++M.n_groups;
    M.samples_dirty = true;
    HM_API_END
}

hm_status hm_lp_add_system(hm_lp* lp, const hm_hmat* h, const double* k_dev, const double* b_dev,
                           const double* x_dev, int nrhs, void* stream) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    if (!h) hm::fail(HM_EINVAL, "lp_add_system: NULL H-matrix");
    hm::lp_add_system(M, const_cast<hm::HMat&>(h->h), k_dev, b_dev, x_dev, nrhs, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_lp_clear_samples(hm_lp* lp) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    M.X_h.clear();
    M.Q_h.clear();
    M.n_groups = 0;
    M.samples_dirty = true;
    HM_API_END
}

hm_status hm_lp_loss_grad(hm_lp* lp, double* loss_out, double* grad_out, void* stream) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    const cudaStream_t st = (cudaStream_t)stream;
    const double l = hm::lp_loss_grad(M, st);
    if (loss_out) *loss_out = l;
    if (grad_out) {
        HM_CUDA(cudaMemcpyAsync(grad_out, M.gsum.p, M.P * sizeof(double), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    HM_API_END
}

hm_status hm_lp_train(hm_lp* lp, int steps, double lr, double* loss_out, void* stream) {
    HM_API_BEGIN
    hm::NvtxScope nvtx_("hm_lp_train");
    hm::LPModel& M = model(lp);
    if (steps < 1) hm::fail(HM_EINVAL, "lp_train: steps must be >= 1");
    if (!(lr > 0.0) || !std::isfinite(lr)) hm::fail(HM_EINVAL, "lp_train: learning rate must be positive");
    const double l = hm::lp_train(M, steps, lr, (cudaStream_t)stream);
    if (loss_out) *loss_out = l;
    HM_API_END
}

hm_status hm_lp_predict(hm_lp* lp, const hm_hmat* h, const double* k_dev, double* features_out, double* d_out,
                        void* stream) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    if (!h) hm::fail(HM_EINVAL, "lp_predict: NULL H-matrix");
    hm::HMat& H = const_cast<hm::HMat&>(h->h);
    const cudaStream_t st = (cudaStream_t)stream;
    hm::DevBuf<float> d((size_t)H.n_leaves * hm::LP_OUT);
    hm::DevBuf<double> f((size_t)H.n_leaves * hm::LP_FEATURES);
    hm::lp_predict(M, H, k_dev, d.p, f.p, st);
    if (features_out)
        HM_CUDA(cudaMemcpyAsync(features_out, f.p, f.bytes(), cudaMemcpyDeviceToHost, st));
    if (d_out) {
        std::vector<float> hd(d.n);
        HM_CUDA(cudaMemcpyAsync(hd.data(), d.p, d.bytes(), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < hd.size(); ++i) d_out[i] = hd[i];
    }
    HM_CUDA(cudaStreamSynchronize(st));
    HM_API_END
}

hm_status hm_lp_get_params(const hm_lp* lp, double* theta_out) {
    HM_API_BEGIN
    if (!lp || !theta_out) hm::fail(HM_EINVAL, "lp_get_params: NULL argument");
    for (int64_t p = 0; p < lp->m.P; ++p) theta_out[p] = lp->m.theta_h[p];
    HM_API_END
}

hm_status hm_lp_set_kind(hm_lp* lp, int kind, double gamma) {
    HM_API_BEGIN
    hm::LPModel& M = model(lp);
    if (kind != HM_LP_SCALE && kind != HM_LP_NEAR) hm::fail(HM_EINVAL, "lp_set_kind: unknown kind");
    if (!(gamma > 0.0) || !std::isfinite(gamma)) hm::fail(HM_EINVAL, "lp_set_kind: gamma must be positive");
    if (kind != M.kind && !M.X_h.empty()) hm::fail(HM_EINVAL, "lp_set_kind: samples of the other kind are held");
    M.kind = kind;
    M.gamma = gamma;
    HM_API_END
}

hm_status hm_lp_set_fallback(hm_lp* lp, int fallback) {
    HM_API_BEGIN
    model(lp).fallback = fallback ? 1 : 0;
    HM_API_END
}

hm_status hm_lp_get_info(const hm_lp* lp, hm_lp_info* info) {
    HM_API_BEGIN
    if (!lp || !info) hm::fail(HM_EINVAL, "lp_get_info: NULL argument");
    const hm::LPModel& M = lp->m;
    info->hidden = M.H;
    info->fallback = M.fallback;
    info->n_params = M.P;
    info->n_samples = (int64_t)M.X_h.size() / hm::LP_FEATURES;
    info->n_groups = M.n_groups;
    info->steps = M.steps;
    info->last_loss = M.last_loss;
    info->kind = M.kind;
    info->gamma = M.gamma;
    HM_API_END
}

hm_status hm_lp_save(const hm_lp* lp, const char* path) {
    HM_API_BEGIN
    if (!lp || !path) hm::fail(HM_EINVAL, "lp_save: NULL argument");
    const hm::LPModel& M = lp->m;
    FILE* f = fopen(path, "wb");
    if (!f) hm::fail(HM_EINVAL, std::string("lp_save: cannot open ") + path);
    const int32_t hdr[2] = {M.H, M.fallback};
    const int64_t steps = M.steps;
    const int32_t kind = M.kind;
    const double gamma = M.gamma;
    bool ok = fwrite(LP_MAGIC, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 2, f) == 2 &&
              fwrite(&steps, sizeof(int64_t), 1, f) == 1 && fwrite(&kind, sizeof(int32_t), 1, f) == 1 &&
              fwrite(&gamma, sizeof(double), 1, f) == 1 &&
              fwrite(M.theta_h.data(), sizeof(float), M.P, f) == (size_t)M.P &&
              fwrite(M.m_h.data(), sizeof(float), M.P, f) == (size_t)M.P &&
              fwrite(M.v_h.data(), sizeof(float), M.P, f) == (size_t)M.P;
    ok = (fclose(f) == 0) && ok;
    if (!ok) hm::fail(HM_EINVAL, std::string("lp_save: write failed: ") + path);
    HM_API_END
}

hm_status hm_lp_load(const char* path, hm_lp** out) {
    HM_API_BEGIN
    if (!path || !out) hm::fail(HM_EINVAL, "lp_load: NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) hm::fail(HM_EINVAL, std::string("lp_load: cannot open ") + path);
    char magic[8];
    int32_t hdr[2];
    int64_t steps = 0;
    int32_t kind = hm::LP_SCALE;
    double gamma = 1.0;
    bool ok = fread(magic, 1, 8, f) == 8;
    const bool v2 = ok && std::memcmp(magic, LP_MAGIC, 8) == 0;
    ok = ok && (v2 || std::memcmp(magic, LP_MAGIC1, 8) == 0) && fread(hdr, sizeof(int32_t), 2, f) == 2 &&
         fread(&steps, sizeof(int64_t), 1, f) == 1 && hm_lp_param_count(hdr[0]) > 0;
    if (ok && v2)
        ok = fread(&kind, sizeof(int32_t), 1, f) == 1 && fread(&gamma, sizeof(double), 1, f) == 1 &&
             (kind == hm::LP_SCALE || kind == hm::LP_NEAR) && gamma > 0.0 && std::isfinite(gamma);
    hm_lp* lp = nullptr;
    if (ok) {
        lp = new hm_lp();
        hm::LPModel& M = lp->m;
        M.H = hdr[0];
        M.fallback = hdr[1] ? 1 : 0;
        M.kind = kind;
        M.gamma = gamma;
        M.steps = steps;
        M.P = hm::lp_param_count(M.H);
        M.theta_h.resize(M.P);
        M.m_h.resize(M.P);
        M.v_h.resize(M.P);
        ok = fread(M.theta_h.data(), sizeof(float), M.P, f) == (size_t)M.P &&
             fread(M.m_h.data(), sizeof(float), M.P, f) == (size_t)M.P &&
             fread(M.v_h.data(), sizeof(float), M.P, f) == (size_t)M.P;
        char extra;
        ok = ok && fread(&extra, 1, 1, f) == 0;
    }
    fclose(f);
    if (!ok) {
        delete lp;
        hm::fail(HM_EINVAL, std::string("lp_load: not a learned-correction file: ") + path);
    }
    *out = lp;
    HM_API_END
}

void hm_lp_destroy(hm_lp* lp) { delete lp; }

}  // extern "C"
