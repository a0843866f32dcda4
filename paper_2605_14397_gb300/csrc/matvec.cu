// H-matrix product y = E x on the device (the product of Sec. 3.1 on the stored
// H-matrix).
//
//   gather   xc = x[perm]                          cluster order, RHS interleaved
//   phase 1  P = V_t^T xc_t                        every V column (one per rank per leaf)
//   reduce   tb_b = sum of the partials of block b over the leaves of its column cluster
//   phase 2  yc_s = [D_s | U_s] z_s, z = xc (near columns) or tb (U columns)
//   scatter  y[perm] = yc
//
// Phases 1 and 2 are persistent kernels, one CTA per SM.  Their coefficient streams are
// cut into chunks of whole columns of one tile or factor slice (at most 32 KB and 128
// columns) and the chunk list is split into equal byte ranges, one per CTA ("stream-K"):
// every SM streams the same number of bytes.  One producer thread moves each chunk --
// its coefficients and, in phase 2, the contiguous range of operands it multiplies --
// with two cp.async.bulk (TMA) copies into a 4-stage shared-memory ring guarded by
// mbarriers; 8 or 16 consumer warps each take columns of the chunk, lanes over rows,
// and touch no global memory except at leaf boundaries.  A row leaf whose columns fall
// into several CTAs is finished by the last of them (atomic arrival count, partials
// summed in CTA order), so the result is deterministic.
//
// Arithmetic modes over the same FP32/BF16 coefficient streams:
//   F32: float vectors, FP32 accumulation;
//   F64: double vectors; each coefficient a multiplies z = zh + zl (zh = fl32(z),
//        zl = fl32(z - zh)) in the compensated dot product of Ogita, Rump and Oishi
//        (2005): TwoProduct via fmaf, TwoSum of the running sum, rounding errors summed
//        apart, the two parts combined in FP64 -- the stored operator applied to FP64
//        vectors to about 1e-13 relative while the coefficients stream at 4 (or 2) bytes.
#include <algorithm>
#include <type_traits>

#include "hmat_impl.h"
#include "pipeline.cuh"

namespace hm {

namespace {

constexpr int STAGES = 4;
constexpr int STAGE_BYTES = 32768;   // coefficients of one chunk
constexpr int MAX_CHUNK_COLS = 128;
constexpr int BAR_BYTES = 128;
// zeroed bytes after phase 1's ring: a single-RHS column read of up to 32 * 12 rows of
// 4 bytes that starts in the last stage ends inside them
constexpr int P1_TAIL = 2048;
constexpr int VEC_SLACK = 32;        // elements after xc / tb so rounded-up copies stay inside

struct FF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <int MODE>
struct AccT;
// type: accumulator; vec: output vectors (y, partials); zin: the x / t operands as the
// kernels read them -- in F64 mode each double is stored pre-split into (hi, lo) floats
// by the gather and the reduction, so the streaming kernels do no FP64 arithmetic
template <>
struct AccT<0> {
    using type = float;
    using vec = float;
    using zin = float;
};
template <>
struct AccT<1> {
    using type = FF;
    using vec = double;
    using zin = float2;
};

// z operand: one float, or the (hi, lo) split of a double
struct Z32 {
    float h;
};
struct Z64 {
    float h, l;
};

__device__ __forceinline__ Z32 make_z(float v) { return Z32{v}; }
__device__ __forceinline__ Z64 make_z(float2 v) { return Z64{v.x, v.y}; }
__device__ __forceinline__ float2 split_d(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
template <class Zin>
__device__ __forceinline__ Zin zin_zero();
template <>
__device__ __forceinline__ float zin_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 zin_zero<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ void acc_zero(float& a) { a = 0.f; }
__device__ __forceinline__ void acc_zero(FF& a) { a.hi = 0.f; a.lo = 0.f; }

__device__ __forceinline__ void acc_fma(float& acc, float a, Z32 z) { acc = fmaf(a, z.h, acc); }
// two FP32 accumulators against one coefficient: one packed FMA (sm_100-class FFMA2,
// each half rounded like fmaf), half the instructions of the multi-RHS loops
__device__ __forceinline__ void acc_fma2(float& a0, float& a1, float v, Z32 z0, Z32 z1) {
    const float2 r = __ffma2_rn(make_float2(v, v), make_float2(z0.h, z1.h), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}
// the RHS of one coefficient: pairs for FP32 accumulators, one by one otherwise
template <int NR, class A, class Z>
__device__ __forceinline__ void acc_fma_rhs(A* acc, float v, const Z* z, int stride) {
    if constexpr (std::is_same<A, float>::value && NR % 2 == 0) {
#pragma unroll
        for (int k = 0; k < NR; k += 2) acc_fma2(acc[k * stride], acc[(k + 1) * stride], v, z[k], z[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < NR; ++k) acc_fma(acc[k * stride], v, z[k]);
    }
}
__device__ __forceinline__ void acc_fma(FF& acc, float a, Z64 z) {
    const float p = a * z.h;
    const float pe = fmaf(a, z.h, -p);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo += e + pe + a * z.l;
}

__device__ __forceinline__ void acc_add(float& a, float b) { a += b; }
__device__ __forceinline__ void acc_add(FF& a, const FF& b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    a.hi = s;
    a.lo += e + b.lo;
}

__device__ __forceinline__ float acc_shfl(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ FF acc_shfl(const FF& v, int o) {
    return FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// Sum each of the NR accumulators over the warp, spread over the lanes: halving
// exchanges (each lane sends the half of its values it does not keep, NR - 1 shuffles in
// all) and then plain butterflies over the remaining lane bits.  Afterwards acc[0] of lane
// l holds the warp sum of right-hand side k(l) (returned); lanes with the low log2(32/NR)
// bits clear are the first holder of each k.
template <int NR, class Acc>
__device__ __forceinline__ int warp_reduce_scatter(Acc (&acc)[NR], int lane) {
    int k = 0;
#pragma unroll
    for (int h = NR / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const Acc lo = acc[j], hi = acc[j + h];
            Acc mine = up ? hi : lo;
            acc_add(mine, acc_shfl(up ? lo : hi, o));
            acc[j] = mine;
        }
        if (up) k += h;
    }
#pragma unroll
    for (int o = 16 / NR; o > 0; o >>= 1) acc_add(acc[0], acc_shfl(acc[0], o));
    return k;
}

__device__ __forceinline__ float acc_value(float a) { return a; }
__device__ __forceinline__ double acc_value(const FF& a) { return (double)a.hi + (double)a.lo; }

// z operands of one column for NR right-hand sides (p: the column's nr interleaved
// values in shared memory).  With nr == NR (a multiple of 4 for floats, of 2 for
// doubles) the values are 16-byte aligned and read as vectors.
template <int NR>
__device__ __forceinline__ void load_z(Z32 (&z)[NR], const float* p, int nr) {
    if constexpr (NR % 4 == 0) {
        if (nr == NR) {
#pragma unroll
            for (int q = 0; q < NR / 4; ++q) {
                const float4 f = reinterpret_cast<const float4*>(p)[q];
                z[4 * q] = Z32{f.x};
                z[4 * q + 1] = Z32{f.y};
                z[4 * q + 2] = Z32{f.z};
                z[4 * q + 3] = Z32{f.w};
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) z[k] = make_z(k < nr ? p[k] : 0.f);
}
template <int NR>
__device__ __forceinline__ void load_z(Z64 (&z)[NR], const float2* p, int nr) {
    if constexpr (NR % 2 == 0) {
        if (nr == NR) {
#pragma unroll
            for (int q = 0; q < NR / 2; ++q) {
                const float4 f = reinterpret_cast<const float4*>(p)[q];
                z[2 * q] = Z64{f.x, f.y};
                z[2 * q + 1] = Z64{f.z, f.w};
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) z[k] = make_z(k < nr ? p[k] : make_float2(0.f, 0.f));
}

__device__ __forceinline__ float coef(const float* p, int i) { return p[i]; }
__device__ __forceinline__ float coef(const uint16_t* p, int i) { return __uint_as_float(((uint32_t)p[i]) << 16); }

// ---- tensor-core helpers (mma.sync m16n8k16 BF16 x BF16 -> FP32, ldmatrix fragments)
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// round to nearest even BF16 bits
__device__ __forceinline__ uint32_t bf16_bits(float v) {
    const uint32_t u = __float_as_uint(v);
    return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float bf16_value(uint32_t b) { return __uint_as_float(b << 16); }

// Programmatic dependent launch: the kernels of a product after the gather are launched
// so that they may start while their predecessor drains; each waits for it (and its
// memory) with griddepcontrol.wait before touching what it produced, and lets its own
// successor launch early with griddepcontrol.launch_dependents.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// xc[dof * nr + k] = x[k * ndof + user dof]
template <class V>
__global__ void k_gather(const V* __restrict__ x, V* __restrict__ xc, const int32_t* __restrict__ perm, int64_t N,
                         int nrhs) {
    pdl_trigger();
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ndof = 3 * N;
    if (q >= ndof * nrhs) return;
    const int64_t r = q / nrhs, k = q % nrhs;
    const int64_t p = r / 3, m = r % 3;
    xc[q] = x[k * ndof + 3 * (int64_t)perm[p] + m];
}

// F64 gather: xc[dof * nr + k] = (hi, lo) split of x[k * ndof + user dof]
__global__ void k_gather_split(const double* __restrict__ x, float2* __restrict__ xc,
                               const int32_t* __restrict__ perm, int64_t N, int nrhs) {
    pdl_trigger();
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ndof = 3 * N;
    if (q >= ndof * nrhs) return;
    const int64_t r = q / nrhs, k = q % nrhs;
    const int64_t p = r / 3, m = r % 3;
    xc[q] = split_d(x[k * ndof + 3 * (int64_t)perm[p] + m]);
}

// y[k * ndof + user dof] = yc[k * ndof + dof]
template <class V>
__global__ void k_scatter(const V* __restrict__ yc, V* __restrict__ y, const int32_t* __restrict__ perm, int64_t N,
                          int nrhs) {
    pdl_wait();
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ndof = 3 * N;
    if (q >= ndof * nrhs) return;
    const int64_t k = q / ndof, r = q % ndof;
    const int64_t p = r / 3, m = r % 3;
    y[k * ndof + 3 * (int64_t)perm[p] + m] = yc[q];
}

__device__ __forceinline__ float to_zin(float v, float*) { return v; }
__device__ __forceinline__ float2 to_zin(double v, float2*) { return split_d(v); }
// BF16 high part in the low 16 bits, BF16 of the remainder in the high 16 bits: the B
// operand of the single-RHS tensor-core phase 2
__device__ __forceinline__ uint32_t to_zin(float v, uint32_t*) {
    const uint32_t hb = bf16_bits(v);
    return hb | (bf16_bits(v - bf16_value(hb)) << 16);
}

// tb[(tb_off + l) nr + k] = sum_q P[(poff[pbase + q] + l) nr + k], one CTA (128 threads)
// (VEC4: FP32 with nr a multiple of 4, each slice read as float4)
// per block: the n = r nr entries times G = 128 / n interleaved groups of leaf partials,
// four independent loads in flight per thread, groups combined in a fixed order.  In F64
// mode the sums are stored as (hi, lo) float pairs, the form phase 2 reads.
template <class V, class Zt, bool VEC4>
__global__ void __launch_bounds__(128) k_reduce_tb(const FarDesc* __restrict__ far, const int32_t* __restrict__ poff,
                                                   const int32_t* __restrict__ uoff, const V* __restrict__ P,
                                                   Zt* __restrict__ tb, int nrhs, const int* __restrict__ skip) {
    __shared__ V sp[128];
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    const FarDesc F = far[blockIdx.x];
    const int n = F.rank * nrhs;
    if (n == 0) return;
    // first partial of the block in each leaf of T, staged in shared memory when it fits so
    // that the partial loads do not wait on their index loads
    constexpr int SPO = 2048;
    __shared__ int32_t spo[SPO];
    const int32_t* po = poff + F.pbase;
    if (F.n_tleaves <= SPO) {
        for (int q = threadIdx.x; q < F.n_tleaves; q += 128) spo[q] = po[q];
        __syncthreads();
        po = spo;
    }
    auto at = [&](int q) -> int64_t { return (int64_t)po[q] * nrhs; };
    if constexpr (VEC4) {
        {
            // several RHS: each slice is rank * nrhs contiguous floats, read as float4
            const int n4 = n >> 2;
            const float4* P4 = reinterpret_cast<const float4*>(P);
            for (int e = threadIdx.x; e < n4; e += 128) {
                float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
                int q = 0;
                for (; q + 3 < F.n_tleaves; q += 4) {
                    const float4 v0 = P4[(at(q) >> 2) + e], v1 = P4[(at(q + 1) >> 2) + e];
                    const float4 v2 = P4[(at(q + 2) >> 2) + e], v3 = P4[(at(q + 3) >> 2) + e];
                    s0.x += v0.x; s0.y += v0.y; s0.z += v0.z; s0.w += v0.w;
                    s1.x += v1.x; s1.y += v1.y; s1.z += v1.z; s1.w += v1.w;
                    s2.x += v2.x; s2.y += v2.y; s2.z += v2.z; s2.w += v2.w;
                    s3.x += v3.x; s3.y += v3.y; s3.z += v3.z; s3.w += v3.w;
                }
                for (; q < F.n_tleaves; ++q) {
                    const float4 v0 = P4[(at(q) >> 2) + e];
                    s0.x += v0.x; s0.y += v0.y; s0.z += v0.z; s0.w += v0.w;
                }
                const float4 t = make_float4((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y),
                                             (s0.z + s1.z) + (s2.z + s3.z), (s0.w + s1.w) + (s2.w + s3.w));
                for (int c = 0; c < F.n_sleaves; ++c) {  // one copy per leaf of S
                    float* o = reinterpret_cast<float*>(tb) + (int64_t)uoff[F.ubase + c] * nrhs + 4 * e;
                    o[0] = t.x;
                    o[1] = t.y;
                    o[2] = t.z;
                    o[3] = t.w;
                }
            }
            return;
        }
    }
    if (n >= 128) {
        for (int e = threadIdx.x; e < n; e += 128) {
            V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            int q = 0;
            for (; q + 3 < F.n_tleaves; q += 4) {
                s0 += P[at(q) + e];
                s1 += P[at(q + 1) + e];
                s2 += P[at(q + 2) + e];
                s3 += P[at(q + 3) + e];
            }
            for (; q < F.n_tleaves; ++q) s0 += P[at(q) + e];
            const Zt t = to_zin((s0 + s1) + (s2 + s3), tb);
            for (int c = 0; c < F.n_sleaves; ++c) tb[(int64_t)uoff[F.ubase + c] * nrhs + e] = t;
        }
        return;
    }
    const int G = 128 / n;
    const int e = threadIdx.x % n, g = threadIdx.x / n;
    V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    if (g < G) {
        int q = g;
        for (; q + 3 * G < F.n_tleaves; q += 4 * G) {
            s0 += P[at(q) + e];
            s1 += P[at(q + G) + e];
            s2 += P[at(q + 2 * G) + e];
            s3 += P[at(q + 3 * G) + e];
        }
        for (; q < F.n_tleaves; q += G) s0 += P[at(q) + e];
    }
    sp[threadIdx.x] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (threadIdx.x < n) {
        V s = 0;
        for (int q = 0; q < G; ++q) s += sp[q * n + threadIdx.x];
        const Zt t = to_zin(s, tb);
        for (int c = 0; c < F.n_sleaves; ++c) tb[(int64_t)uoff[F.ubase + c] * nrhs + threadIdx.x] = t;
    }
}

// 16 right-hand sides with BF16 U slices on tensor cores: the sums of t (float4 slices,
// k_reduce_pack16_mix below), each value split into BF16
// hi + lo (hi = bf16(t), lo = bf16(t - hi)) and stored as the B operand of phase 2:
// 64 bytes per rank entry l, four 16-byte pieces (RHS 0-7 hi, RHS 0-7 lo, RHS 8-15 hi,
// RHS 8-15 lo), piece q stored at position q ^ ((l >> 1) & 3), so that the eight
// consecutive entries one ldmatrix row group reads fall into eight different bank groups.
__device__ __forceinline__ int tb16_piece_pos(int64_t l, int q) { return q ^ (int)((l >> 1) & 3); }

// The same reduction for one RHS in one launch of 256-thread CTAs over a block order
// (red_order) that lists the blocks with more than RED_WARP_LEAVES leaves of T first.
// Each of those gets a CTA: its offset table staged in shared memory, 256 / r groups of
// threads over the leaves, four partials per thread in flight.  The many small blocks get
// a warp each, eight per CTA -- four times the blocks in flight of a CTA per block, whose
// launch was bound by the latency of short load chains rather than by bytes: lanes take
// the rank entries, one load fetches 32 offset-table entries which shuffles broadcast.
// Every block sums its partials in a fixed order.
constexpr int RED_WARP_LEAVES = 32;
template <class V, class Zt>
__global__ void __launch_bounds__(256) k_reduce_mix(const FarDesc* __restrict__ far,
                                                    const int32_t* __restrict__ poff,
                                                    const int32_t* __restrict__ uoff,
                                                    const int32_t* __restrict__ order, int64_t n_big, int64_t n_all,
                                                    const V* __restrict__ P, Zt* __restrict__ tb,
                                                    const int* __restrict__ skip) {
    __shared__ V sp[256];
    constexpr int SPO = 2048;
    __shared__ int32_t spo[SPO];
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    if ((int64_t)blockIdx.x < n_big) {
        const FarDesc F = far[order[blockIdx.x]];
        const int r = F.rank, nt = F.n_tleaves;  // r <= 256 (rank cap)
        const int32_t* po = poff + F.pbase;
        if (nt <= SPO) {
            for (int q = threadIdx.x; q < nt; q += 256) spo[q] = po[q];
            __syncthreads();
            po = spo;
        }
        const int G = 256 / r;
        const int e = threadIdx.x % r, g = threadIdx.x / r;
        V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        if (g < G) {
            int q = g;
            for (; q + 3 * G < nt; q += 4 * G) {
                s0 += P[(int64_t)po[q] + e];
                s1 += P[(int64_t)po[q + G] + e];
                s2 += P[(int64_t)po[q + 2 * G] + e];
                s3 += P[(int64_t)po[q + 3 * G] + e];
            }
            for (; q < nt; q += G) s0 += P[(int64_t)po[q] + e];
        }
        sp[threadIdx.x] = (s0 + s1) + (s2 + s3);
        __syncthreads();
        if (threadIdx.x < r) {
            V s = 0;
            for (int q = 0; q < G; ++q) s += sp[q * r + threadIdx.x];
            const Zt t = to_zin(s, tb);
            for (int c = 0; c < F.n_sleaves; ++c) tb[uoff[F.ubase + c] + threadIdx.x] = t;
        }
        return;
    }
    const int64_t k = n_big + ((int64_t)blockIdx.x - n_big) * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n_all) return;
    const int64_t b = order[k];
    const int r = far[b].rank, nt = far[b].n_tleaves;
    const int32_t* po = poff + far[b].pbase;
    const int ns = far[b].n_sleaves;
    const int32_t* uo = uoff + far[b].ubase;
    for (int e0 = 0; e0 < r; e0 += 32) {
        const int e = e0 + lane;
        const bool on = e < r;
        V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int q0 = 0; q0 < nt; q0 += 32) {
            const int m = min(32, nt - q0);
            const int32_t mine = lane < m ? po[q0 + lane] : 0;
            int q = 0;
            for (; q + 3 < m; q += 4) {
                const int32_t o0 = __shfl_sync(0xffffffffu, mine, q), o1 = __shfl_sync(0xffffffffu, mine, q + 1);
                const int32_t o2 = __shfl_sync(0xffffffffu, mine, q + 2), o3 = __shfl_sync(0xffffffffu, mine, q + 3);
                if (on) {
                    s0 += P[(int64_t)o0 + e];
                    s1 += P[(int64_t)o1 + e];
                    s2 += P[(int64_t)o2 + e];
                    s3 += P[(int64_t)o3 + e];
                }
            }
            for (; q < m; ++q) {
                const int32_t o0 = __shfl_sync(0xffffffffu, mine, q);
                if (on) s0 += P[(int64_t)o0 + e];
            }
        }
        if (on) {
            const Zt t = to_zin((s0 + s1) + (s2 + s3), tb);
            for (int c = 0; c < ns; ++c) tb[uo[c] + e] = t;  // one copy per leaf of S
        }
    }
}

// 16 RHS packed for TC16 over the same block order as k_reduce_mix: blocks with more
// than RED_WARP_LEAVES leaves of T a 256-thread CTA each (float4 groups x subsets of the
// leaves, partials meeting in shared memory in subset order), the others a warp each,
// eight per CTA (lanes over the float4 groups, 32 offsets per load broadcast by
// shuffles, four partials in flight).  Every block sums in a fixed order.
__device__ __forceinline__ void store_pack16(uint16_t* __restrict__ tb, const int32_t* __restrict__ uo, int ns,
                                             int e, float4 a) {
    const float t[4] = {a.x, a.y, a.z, a.w};
    uint32_t hb[4], lb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        hb[i] = bf16_bits(t[i]);
        lb[i] = bf16_bits(t[i] - bf16_value(hb[i]));
    }
    const int k0 = (e & 3) * 4;                  // first of the four RHS
    const int qh = 2 * (k0 >> 3), off = k0 & 7;  // hi piece of these RHS, offset inside it
    for (int c = 0; c < ns; ++c) {               // one copy per leaf of S
        const int64_t l = (int64_t)uo[c] + e / 4;
        uint16_t* row = tb + 32 * l;             // 64 bytes
        *reinterpret_cast<uint2*>(row + 8 * tb16_piece_pos(l, qh) + off) =
            make_uint2(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16));
        *reinterpret_cast<uint2*>(row + 8 * tb16_piece_pos(l, qh + 1) + off) =
            make_uint2(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16));
    }
}

__device__ __forceinline__ void add4(float4& s, const float4 v) {
    s.x += v.x;
    s.y += v.y;
    s.z += v.z;
    s.w += v.w;
}

__global__ void __launch_bounds__(256) k_reduce_pack16_mix(const FarDesc* __restrict__ far,
                                                           const int32_t* __restrict__ poff,
                                                           const int32_t* __restrict__ uoff,
                                                           const int32_t* __restrict__ order, int64_t n_big,
                                                           int64_t n_all, const float* __restrict__ P,
                                                           uint16_t* __restrict__ tb, const int* __restrict__ skip) {
    __shared__ float4 sp[256];
    constexpr int SPO = 2048;
    __shared__ int32_t spo[SPO];
    pdl_wait();
    pdl_trigger();
    if (skip && *(volatile const int*)skip) return;
    const float4* P4 = reinterpret_cast<const float4*>(P);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((int64_t)blockIdx.x < n_big) {
        const FarDesc F = far[order[blockIdx.x]];
        const int n4 = 4 * F.rank, nt = F.n_tleaves;
        const int32_t* po = poff + F.pbase;
        if (nt <= SPO) {
            for (int q = threadIdx.x; q < nt; q += 256) spo[q] = po[q];
            __syncthreads();
            po = spo;
        }
        for (int e0 = 0; e0 < n4; e0 += 256) {
            const int r = min(256, n4 - e0);
            const int G = 256 / r;
            const int e = e0 + threadIdx.x % r, g = threadIdx.x / r;
            float4 s0 = z4, s1 = z4, s2 = z4, s3 = z4;
            if (g < G) {
                int q = g;
                for (; q + 3 * G < nt; q += 4 * G) {
                    add4(s0, P4[(int64_t)po[q] * 4 + e]);
                    add4(s1, P4[(int64_t)po[q + G] * 4 + e]);
                    add4(s2, P4[(int64_t)po[q + 2 * G] * 4 + e]);
                    add4(s3, P4[(int64_t)po[q + 3 * G] * 4 + e]);
                }
                for (; q < nt; q += G) add4(s0, P4[(int64_t)po[q] * 4 + e]);
            }
            add4(s0, s1);
            add4(s2, s3);
            add4(s0, s2);
            sp[threadIdx.x] = s0;
            __syncthreads();
            if (threadIdx.x < r) {
                float4 a = sp[threadIdx.x];
                for (int q = 1; q < G; ++q) add4(a, sp[q * r + threadIdx.x]);
                store_pack16(tb, uoff + F.ubase, F.n_sleaves, e0 + threadIdx.x, a);
            }
            __syncthreads();
        }
        return;
    }
    const int64_t k = n_big + ((int64_t)blockIdx.x - n_big) * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n_all) return;
    const int64_t b = order[k];
    const int n4 = 4 * far[b].rank, nt = far[b].n_tleaves;
    const int32_t* po = poff + far[b].pbase;
    // up to RP passes of 32 groups at once: their loads for one leaf are independent
    constexpr int RP = 4;
    for (int e0 = 0; e0 < n4; e0 += 32 * RP) {
        float4 acc[2][RP];  // even and odd leaves: two more loads in flight
#pragma unroll
        for (int p = 0; p < RP; ++p) acc[0][p] = acc[1][p] = z4;
        for (int q0 = 0; q0 < nt; q0 += 32) {
            const int m = min(32, nt - q0);
            const int32_t mine = lane < m ? po[q0 + lane] : 0;
            int q = 0;
            for (; q + 1 < m; q += 2) {
                const int64_t o0 = (int64_t)__shfl_sync(0xffffffffu, mine, q) * 4;
                const int64_t o1 = (int64_t)__shfl_sync(0xffffffffu, mine, q + 1) * 4;
#pragma unroll
                for (int p = 0; p < RP; ++p) {
                    const int e = e0 + 32 * p + lane;
                    if (e < n4) {
                        add4(acc[0][p], P4[o0 + e]);
                        add4(acc[1][p], P4[o1 + e]);
                    }
                }
            }
            if (q < m) {
                const int64_t o0 = (int64_t)__shfl_sync(0xffffffffu, mine, q) * 4;
#pragma unroll
                for (int p = 0; p < RP; ++p) {
                    const int e = e0 + 32 * p + lane;
                    if (e < n4) add4(acc[0][p], P4[o0 + e]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            const int e = e0 + 32 * p + lane;
            add4(acc[0][p], acc[1][p]);
            if (e < n4) store_pack16(tb, uoff + far[b].ubase, far[b].n_sleaves, e, acc[0][p]);
        }
    }
}

struct StreamArgs {
    const Chunk* chunks;
    const int32_t* cta_begin;
    const LeafDesc* leaves;
    const LeafSplit* split;
    const float* near;
    const void* ucoef;
    const void* vcoef;
    const void* xc;
    const void* tb;
    void* out;    // yc (phase 2) or P (phase 1)
    void* slots;  // phase-2 partials of split leaves
    int32_t* counters;
    int* err;
    int64_t ndof;
    int nr;       // right-hand sides in this launch (<= NR); also the interleave stride
    int ld_max;
    const int* skip;  // optional device flag: when set, the kernels return at once
    uint64_t wait_ns; // limit of every bounded wait of the copy ring
    // test switch (hm_hmat_set_wait): the producer of phase 2 stops before this chunk of
    // the plan (its copy and every later one of the CTA are never issued), so that the
    // consumers' waits run out; -1: off
    int64_t withhold;
};

template <class V, int NR>
struct ZRange {
    static constexpr int ALIGN = 16 / (int)sizeof(V);  // elements per 16 bytes
    static constexpr int BYTES = ((MAX_CHUNK_COLS * NR + 2 * ALIGN) * (int)sizeof(V) + 127) / 128 * 128;
};

// ---- producer: one thread streams this CTA's chunks (and their operands) through the ring
// (WAIT_T: wait for the preceding kernel -- the reduction producing t -- only before the
// first chunk whose operand is t; near tiles read x, complete before that kernel began)
template <class C, class V, int NR, bool WITH_Z, bool WAIT_T = false, int ST = STAGES>
__device__ __forceinline__ void produce(const StreamArgs& a, unsigned char* smem_stage, int stage_stride,
                                        uint64_t* full, uint64_t* empty, int c0, int c1) {
    using ZR = ZRange<V, NR>;
    bool waited = false;
    int issued = c1 - c0;  // copies issued (all of them unless the test switch stops early)
    Chunk nxt = c0 < c1 ? a.chunks[c0] : Chunk{};
    for (int i = c0; i < c1; ++i) {
        if (WITH_Z && i == a.withhold) {
            issued = i - c0;
            break;
        }
        const Chunk ch = nxt;
        if (i + 1 < c1) nxt = a.chunks[i + 1];
        if constexpr (WAIT_T) {
            if (!waited && ch.kind != 0) {
                pdl_wait();
                waited = true;
            }
        }
        const int q = i - c0, s = q % ST;
        const uint32_t ph = (uint32_t)(q / ST) & 1u;
        if (q >= ST) mbar_wait(empty + s, ph ^ 1u, a.err, 4, a.wait_ns);
        unsigned char* stg = smem_stage + (size_t)s * stage_stride;
        const void* src;
        uint32_t bytes;
        if (ch.kind == 0) {
            src = a.near + ch.src;
            bytes = (uint32_t)ch.ncols * ch.ld * 4u;
        } else {
            const C* base = (const C*)(ch.kind == 1 ? a.ucoef : a.vcoef);
            src = base + ch.src;
            bytes = (uint32_t)ch.ncols * ch.ld * (uint32_t)sizeof(C);
        }
        if constexpr (WITH_Z) {
            const V* zsrc = (const V*)(ch.kind == 0 ? a.xc : a.tb);
            const int64_t z0 = ch.zoff * a.nr;
            const int64_t a0 = z0 & ~(int64_t)(ZR::ALIGN - 1);
            const int64_t a1 = (z0 + (int64_t)ch.ncols * a.nr + ZR::ALIGN - 1) & ~(int64_t)(ZR::ALIGN - 1);
            const uint32_t zbytes = (uint32_t)((a1 - a0) * (int64_t)sizeof(V));
            mbar_arrive_expect_tx(full + s, bytes + zbytes);
            bulk_g2s(stg, zsrc + a0, zbytes, full + s);
            bulk_g2s(stg + ZR::BYTES, src, bytes, full + s);
        } else {
            mbar_arrive_expect_tx(full + s, bytes);
            bulk_g2s(stg, src, bytes, full + s);
        }
    }
    if constexpr (WAIT_T) {
        if (!waited) pdl_wait();
    }
    // no copy may still be in flight when the CTA exits
    const int n = issued;
    for (int q = std::max(0, n - ST); q < n; ++q)
        mbar_wait(full + (q % ST), (uint32_t)(q / ST) & 1u, a.err, 8, a.wait_ns);
}

template <int ST = STAGES>
__device__ __forceinline__ void init_ring(uint64_t* full, uint64_t* empty, int ncw) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, ncw);
        }
        mbar_fence_init();
    }
    __syncthreads();
}

// ---- phase 2: y = [D | U] z per row leaf
// RS > 1 splits each column's rows over RS warps (RPL / RS rows per lane each), so that
// many right-hand sides fit in registers with more warps in flight.
//
// BF16 U slices with one RHS (TC2) run on tensor cores: A = the slice (rows x columns,
// column-major in shared memory, so ldmatrix.trans gives the row-major fragments), B
// column 0 = the BF16 high part of t, column 1 the low part (the reduction stores t in
// that packed form), so d(col 0) + d(col 1) = U t for 16 rows.  Warp w = (kg, mg) takes
// the k-tiles kg, kg + 4 of each slice and keeps m-tiles mg, mg + 4, mg + 8 of the leaf
// in registers; at the flush each warp adds them to its own row of the reduction buffer.
template <int MODE, class C, int NR, int RPL, int NCW, int RS, int ST = STAGES>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) k_phase2(StreamArgs a) {
    constexpr bool TC2 = MODE == 0 && NR == 1 && RS == 1 && NCW == 16 && RPL == 6 &&
                         std::is_same<C, uint16_t>::value;
    // BF16 U slices with 16 RHS (TC16, when the launch has exactly 16): warp w < 12 owns
    // m-tile w (rows 16 w .. 16 w + 15 of the leaf) and both n-tiles (RHS 0-7, 8-15); A as
    // in TC2, B = t in the packed BF16 (hi, lo) form of k_reduce_pack16_mix read with
    // ldmatrix.trans, two mma per n-tile and k-tile.  The CUDA-core accumulators keep the
    // near tiles; the tensor-core results join them at the flush through ty.
    constexpr bool TC16 = MODE == 0 && NR == 16 && RS == 2 && NCW == 16 && RPL == 6 &&
                          std::is_same<C, uint16_t>::value;
    constexpr int TC16_MT = 12, TY_LD = 196;  // m-tiles (192 rows); ty row stride (bank spread)
    constexpr int TKG = 4, TMG = 4, TMT = 3;  // k-groups x m-groups = NCW; m-tiles per warp
    static_assert(!TC2 || (TKG * TMG == NCW && TMG * TMT * 16 >= 32 * RPL && TKG * 2 * 16 >= MAX_CHUNK_COLS),
                  "tensor-core phase 2 covers every row and column");
    using Acc = typename AccT<MODE>::type;
    using Vv = typename AccT<MODE>::vec;
    using ZR = ZRange<Vv, NR>;
    constexpr int STRIDE = ZR::BYTES + STAGE_BYTES;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)smem;
    uint64_t* empty = full + ST;
    int* s_flag = (int*)(empty + ST);
    uint16_t* zline = (uint16_t*)(smem + 112);  // a zeroed 16-byte line (ldmatrix rows outside a slice)
    static_assert(2 * ST * 8 + 4 <= 112 && 112 + 16 <= BAR_BYTES, "barrier area layout");
    unsigned char* stage = smem + BAR_BYTES;
    constexpr int RPW = RPL / RS;  // rows per lane of one warp
    constexpr int NG = NCW / RS;   // column groups
    static_assert(RPL % RS == 0 && NCW % RS == 0, "row split must divide rows and warps");
    // FP32 vectors with 16 RHS on leaves of up to 64 elements reduce 8 RHS per pass of the
    // flush (4 barriers per leaf instead of 32); the other variants one RHS per pass (their
    // reduction buffer would not fit beside the ring)
    constexpr int KP = (MODE == 0 && NR == 16 && RPL == 6) ? 8 : 1;
    Acc* red = (Acc*)(stage + (size_t)ST * STRIDE);  // [KP][NG][32 RPL]
    float* ty = (float*)(red + (size_t)KP * NG * 32 * RPL);  // TC16: the leaf's tensor-core sums [16 RHS][TY_LD]

    if (a.skip && *(volatile const int*)a.skip) return;  // every right-hand side already converged
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 8) zline[threadIdx.x] = 0;
    init_ring<ST>(full, empty, NCW);
    const int c0 = a.cta_begin[blockIdx.x], c1 = a.cta_begin[blockIdx.x + 1];
    pdl_trigger();
    if (w == NCW) {
        // the t operand ranges come from the reduction: the producer waits for it before the
        // first U chunk, so the near tiles ahead of it stream while the reduction runs
        if (lane == 0) produce<C, Vv, NR, true, true, ST>(a, stage, STRIDE, full, empty, c0, c1);
        return;
    }
    Vv* yc = (Vv*)a.out;
    Vv* slots = (Vv*)a.slots;
    const int g = w / RS, rbase = (w % RS) * 32 * RPW;
    Acc acc[NR][RPW];
    float dt[TMT][4];  // TC2: this warp's m-tiles of the leaf (tensor-core part)
    const bool tc16 = TC16 && a.nr == 16;
    int cur = -1;
    LeafDesc L{};

    auto flush = [&]() {
        const LeafSplit sp = a.split[cur];
        const int rows = 3 * L.n;
        const bool whole = sp.nparts == 1;
        const int64_t slot = whole ? 0 : (int64_t)(sp.slot_base + (int)blockIdx.x - sp.w_first);
        // KP right-hand sides per reduction pass through red (k unrolled at compile time: a
        // runtime index into acc would move it to local memory)
#pragma unroll
        for (int k0 = 0; k0 < NR; k0 += KP) {
            if (k0 >= a.nr) break;
#pragma unroll
            for (int kk = 0; kk < KP; ++kk)
#pragma unroll
                for (int i = 0; i < RPW; ++i)
                    red[((size_t)kk * NG + g) * (32 * RPL) + rbase + lane + 32 * i] = acc[k0 + kk][i];
            if constexpr (TC2) {
                // lanes 4 c hold rows 16 mt + c (d0 + d1) and 16 mt + c + 8 (d2 + d3)
                __syncwarp();
                if ((lane & 3) == 0) {
#pragma unroll
                    for (int j = 0; j < TMT; ++j) {
                        Acc* rw = red + (size_t)g * (32 * RPL) + (w % TMG + TMG * j) * 16 + (lane >> 2);
                        rw[0] += dt[j][0] + dt[j][1];
                        rw[8] += dt[j][2] + dt[j][3];
                    }
                }
            }
            consumer_sync(NCW * 32);
            for (int e = threadIdx.x; e < KP * rows; e += NCW * 32) {
                const int kk = e / rows, r = e - kk * rows, k = k0 + kk;
                if (k >= a.nr) continue;
                const Acc* rk = red + (size_t)kk * NG * (32 * RPL);
                Acc s = rk[r];
                for (int q = 1; q < NG; ++q) acc_add(s, rk[(size_t)q * (32 * RPL) + r]);
                if constexpr (TC16) {
                    if (tc16) acc_add(s, ty[(size_t)k * TY_LD + r]);
                }
                if (whole)
                    yc[(int64_t)k * a.ndof + 3 * (int64_t)L.begin + r] = (Vv)acc_value(s);
                else
                    slots[(slot * NR + k) * a.ld_max + r] = (Vv)acc_value(s);
            }
            consumer_sync(NCW * 32);
        }
        if (!whole) {
            __threadfence();
            consumer_sync(NCW * 32);
            if (threadIdx.x == 0) {
                const int old = atomicAdd(a.counters + cur, 1);
                *s_flag = (old == sp.nparts - 1);
            }
            consumer_sync(NCW * 32);
            if (*s_flag) {
                __threadfence();
                for (int k = 0; k < a.nr; ++k)
                    for (int r = threadIdx.x; r < rows; r += NCW * 32) {
                        Vv s = 0;
                        for (int p = 0; p < sp.nparts; ++p)
                            s += __ldcg(slots + ((int64_t)(sp.slot_base + p) * NR + k) * a.ld_max + r);
                        yc[(int64_t)k * a.ndof + 3 * (int64_t)L.begin + r] = s;
                    }
                if (threadIdx.x == 0) a.counters[cur] = 0;
            }
            consumer_sync(NCW * 32);
        }
    };

    Chunk nxt = c0 < c1 ? a.chunks[c0] : Chunk{};
    for (int i = c0; i < c1; ++i) {
        const Chunk ch = nxt;
        if (i + 1 < c1) nxt = a.chunks[i + 1];
        const int q = i - c0, s = q % ST;
        if (ch.leaf != cur) {
            if (cur >= 0) flush();
            cur = ch.leaf;
            L = a.leaves[cur];
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int j = 0; j < RPW; ++j) acc_zero(acc[k][j]);
#pragma unroll
            for (int j = 0; j < TMT; ++j) dt[j][0] = dt[j][1] = dt[j][2] = dt[j][3] = 0.f;
            if constexpr (TC16) {
                // the entries of ty this lane accumulates (its m-tile, see below) start at 0
                if (tc16 && w < TC16_MT) {
                    const int r0 = 16 * w + (lane >> 2), c0 = 2 * (lane & 3);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        float* col = ty + (size_t)(8 * nt + c0) * TY_LD;
                        col[r0] = col[TY_LD + r0] = col[r0 + 8] = col[TY_LD + r0 + 8] = 0.f;
                    }
                }
            }
        }
        mbar_wait(full + s, (uint32_t)(q / ST) & 1u, a.err, 1, a.wait_ns);
        const unsigned char* stg = stage + (size_t)s * STRIDE;
        const int64_t z0 = ch.zoff * a.nr;
        using Zin = typename AccT<MODE>::zin;  // same size as Vv
        const Zin* zb = (const Zin*)stg + (z0 - (z0 & ~(int64_t)(ZR::ALIGN - 1)));
        const unsigned char* buf = stg + ZR::BYTES;
        const int rows = 3 * L.n;
        if constexpr (TC16) {
            if (tc16 && ch.kind != 0) {
                if (w < TC16_MT && 16 * w < rows) {
                    float d16[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                    const uint16_t* ub = (const uint16_t*)buf;
                    const int ld = ch.ld, ncols = ch.ncols;
                    const int j8 = lane >> 3, i8 = lane & 7;
                    const int m0 = 16 * w + (j8 & 1) * 8;
                    const uint32_t zaddr = smem_u32(zline);
                    const uint32_t tbase = smem_u32(stg);  // packed t of the chunk: 64 B per column
                    for (int kt = 0; kt * 16 < ncols; ++kt) {
                        // A: this lane addresses slice column kt 16 + (j8 / 2) 8 + i8, rows m0 ..
                        const int kc = kt * 16 + (j8 >> 1) * 8 + i8;
                        const uint32_t aaddr = (kc < ncols && m0 < ld) ? smem_u32(ub + (size_t)kc * ld + m0) : zaddr;
                        uint32_t a0, a1, a2, a3;
                        ldsm_x4_t(aaddr, a0, a1, a2, a3);
                        // B: matrix j8 = (k half j8 % 2, n-tile j8 / 2), row i8 = column kb of t
                        const int kb = kt * 16 + (j8 & 1) * 8 + i8;
                        const int64_t lg = ch.zoff + kb;
                        const uint32_t rowaddr = tbase + 64u * (uint32_t)kb;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {  // BF16 high parts of t, then the low parts
                            const uint32_t badd =
                                kb < ncols ? rowaddr + 16u * (uint32_t)tb16_piece_pos(lg, 2 * (j8 >> 1) + h) : zaddr;
                            uint32_t b0, b1, b2, b3;
                            ldsm_x4_t(badd, b0, b1, b2, b3);
                            mma_bf16(d16[0], a0, a1, a2, a3, b0, b1);
                            mma_bf16(d16[1], a0, a1, a2, a3, b2, b3);
                        }
                    }
                    // d16: rows 16 w + lane / 4 (c0, c1) and + 8 (c2, c3), RHS 8 nt + 2 (lane % 4)
                    // + {0, 1}; summed over the leaf's chunks in ty, read by the flush
                    const int r0 = 16 * w + (lane >> 2), c0 = 2 * (lane & 3);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        float* col = ty + (size_t)(8 * nt + c0) * TY_LD;
                        col[r0] += d16[nt][0];
                        col[TY_LD + r0] += d16[nt][1];
                        col[r0 + 8] += d16[nt][2];
                        col[TY_LD + r0 + 8] += d16[nt][3];
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty + s);
                continue;
            }
        }
        if constexpr (TC2) {
            if (ch.kind != 0) {
                const uint32_t* zw = (const uint32_t*)zb;  // packed (hi, lo) of t per column
                const uint16_t* ub = (const uint16_t*)buf;
                const int ld = ch.ld, ncols = ch.ncols;
                const int kg = w / TMG, mg = w % TMG, n = lane >> 2;
                const int j8 = lane >> 3, i8 = lane & 7;
                const uint32_t sel = n == 0 ? 0x5410u : 0x7632u;
                const uint32_t zaddr = smem_u32(zline);
#pragma unroll
                for (int tk = 0; tk < 2; ++tk) {
                    const int kt = kg + TKG * tk;
                    if (kt * 16 >= ncols) break;
                    // B: rows k0 + 2 (lane % 4) + {0, 1} and the same + 8; column n
                    uint32_t b[2];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int k0 = kt * 16 + hh * 8 + 2 * (lane & 3);
                        const uint32_t w0 = k0 < ncols ? zw[k0] : 0u;
                        const uint32_t w1 = k0 + 1 < ncols ? zw[k0 + 1] : 0u;
                        b[hh] = n < 2 ? __byte_perm(w0, w1, sel) : 0u;
                    }
                    // A: this lane supplies the address of slice column kt*16 + (j8/2)*8 + i8
                    const int kc = kt * 16 + (j8 >> 1) * 8 + i8;
#pragma unroll
                    for (int j = 0; j < TMT; ++j) {
                        const int m0 = (mg + TMG * j) * 16 + (j8 & 1) * 8;
                        const uint32_t addr = (kc < ncols && m0 < ld) ? smem_u32(ub + (size_t)kc * ld + m0) : zaddr;
                        uint32_t a0, a1, a2, a3;
                        ldsm_x4_t(addr, a0, a1, a2, a3);
                        mma_bf16(dt[j], a0, a1, a2, a3, b[0], b[1]);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty + s);
                continue;
            }
        }
        // Rows at or beyond `rows` read whatever follows the column in shared memory (the
        // next column, stage or the reduction buffer: always inside the allocation); their
        // accumulators are never flushed, so no bound check is needed per coefficient.
        // With several RHS a warp skips its row blocks past the leaf (leaves of fewer than
        // 64 elements), a warp-uniform test; with one RHS the loop stays branch-free.
        const int nact = NR == 1 ? RPW : max(0, min(RPW, (rows - rbase + 31) >> 5));
        for (int c = g; c < ch.ncols && nact > 0; c += NG) {
            decltype(make_z(zin_zero<Zin>())) zv[NR];
            if constexpr (NR == 1)
                zv[0] = make_z(zb[c]);
            else
                load_z<NR>(zv, zb + (size_t)c * a.nr, a.nr);
            if (ch.kind == 0) {
                const float* col = (const float*)buf + (size_t)c * ch.ld + rbase + lane;
#pragma unroll
                for (int ii = 0; ii < RPW; ++ii) {
                    if (NR > 1 && ii >= nact) break;
                    const float v = col[32 * ii];
                    acc_fma_rhs<NR>(&acc[0][ii], v, zv, RPW);
                }
            } else {
                const C* col = (const C*)buf + (size_t)c * ch.ld + rbase + lane;
#pragma unroll
                for (int ii = 0; ii < RPW; ++ii) {
                    if (NR > 1 && ii >= nact) break;
                    const float v = coef(col, 32 * ii);
                    acc_fma_rhs<NR>(&acc[0][ii], v, zv, RPW);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
    }
    if (cur >= 0) flush();
}

// ---- phase 1: P = V_t^T xc_t, one partial per V column
template <int MODE, class C, int NR, int RPL, int NCW, int ST = STAGES>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) k_phase1(StreamArgs a) {
    using Acc = typename AccT<MODE>::type;
    using Vv = typename AccT<MODE>::vec;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)smem;
    uint64_t* empty = full + ST;
    unsigned char* stage = smem + BAR_BYTES;

    if (a.skip && *(volatile const int*)a.skip) return;  // every right-hand side already converged
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (NR == 1) {
        // The single-RHS loop reads whole 32 RPL-row columns without bound checks: rows past
        // a leaf meet x = 0, columns past a chunk are clamped to its last one.  Every byte
        // such a read can reach (the ring and the tail after it) must then be finite, so the
        // ring is zeroed once before the first copy lands in it.
        uint4* z = reinterpret_cast<uint4*>(stage);
        for (int i = threadIdx.x; i < (ST * STAGE_BYTES + P1_TAIL) / 16; i += blockDim.x)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // before the copies write it
    }
    init_ring<ST>(full, empty, NCW);
    const int c0 = a.cta_begin[blockIdx.x], c1 = a.cta_begin[blockIdx.x + 1];
    pdl_trigger();
    if (w == NCW) {
        // the V coefficients are constant: the copies start while the gather drains
        if (lane == 0) produce<C, Vv, NR, false, false, ST>(a, stage, STAGE_BYTES, full, empty, c0, c1);
        return;
    }
    pdl_wait();  // x in cluster order comes from the preceding kernel
    Vv* P = (Vv*)a.out;
    int cur = -1;
    int rows = 0;
    using Zin = typename AccT<MODE>::zin;
    const Zin* xs = (const Zin*)a.xc;
    constexpr bool PAIR = std::is_same<C, uint16_t>::value && NR == 1 && RPL == 6;
    decltype(make_z(zin_zero<Zin>())) xr[NR][RPL];
    Chunk nxt = c0 < c1 ? a.chunks[c0] : Chunk{};
    for (int i = c0; i < c1; ++i) {
        const Chunk ch = nxt;
        if (i + 1 < c1) nxt = a.chunks[i + 1];
        const int q = i - c0, s = q % ST;
        if (ch.leaf != cur) {
            cur = ch.leaf;
            const LeafDesc L = a.leaves[cur];
            rows = 3 * L.n;
#pragma unroll
            for (int ii = 0; ii < RPL; ++ii) {
                // BF16 single-RHS columns are read two rows per 32-bit word: lane holds rows
                // 2 lane + 64 (ii / 2) + ii % 2; otherwise rows lane + 32 ii
                const int r = PAIR ? 2 * lane + 64 * (ii >> 1) + (ii & 1) : lane + 32 * ii;
#pragma unroll
                for (int k = 0; k < NR; ++k)
                    xr[k][ii] = make_z((r < rows && k < a.nr) ? xs[(3 * (int64_t)L.begin + r) * a.nr + k]
                                                              : zin_zero<Zin>());
            }
        }
        mbar_wait(full + s, (uint32_t)(q / ST) & 1u, a.err, 1, a.wait_ns);
        const C* buf = (const C*)(stage + (size_t)s * STAGE_BYTES);
        if constexpr (NR == 1) {
            // Four columns (w, w + NCW, w + 2 NCW, w + 3 NCW) per pass: their four warp sums
            // share one reduce-scatter (6 shuffles instead of 20) and the loads of four
            // columns are in flight together.
            // (no per-coefficient bound checks: see the ring zeroing at the kernel start)
            constexpr int CG = 4;
            for (int c = w; c < ch.ncols; c += CG * NCW) {
                Acc acc[CG];
                const C* colp[CG];
#pragma unroll
                for (int j = 0; j < CG; ++j) {
                    acc_zero(acc[j]);
                    colp[j] = buf + (size_t)min(c + j * NCW, ch.ncols - 1) * ch.ld;
                }
                if constexpr (PAIR) {
#pragma unroll
                    for (int jj = 0; jj < RPL / 2; ++jj) {
#pragma unroll
                        for (int j = 0; j < CG; ++j) {
                            const uint32_t wv = reinterpret_cast<const uint32_t*>(colp[j])[lane + 32 * jj];
                            acc_fma(acc[j], __uint_as_float(wv << 16), xr[0][2 * jj]);
                            acc_fma(acc[j], __uint_as_float(wv & 0xffff0000u), xr[0][2 * jj + 1]);
                        }
                    }
                } else {
#pragma unroll
                    for (int ii = 0; ii < RPL; ++ii) {
#pragma unroll
                        for (int j = 0; j < CG; ++j) acc_fma(acc[j], coef(colp[j], lane + 32 * ii), xr[0][ii]);
                    }
                }
                const int j = warp_reduce_scatter<CG>(acc, lane);
                const int cj = c + j * NCW;
                if ((lane & (32 / CG - 1)) == 0 && cj < ch.ncols) P[ch.zoff + cj] = (Vv)acc_value(acc[0]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + s);
            continue;
        }
        for (int c = w; c < ch.ncols; c += NCW) {
            const C* col = buf + (size_t)c * ch.ld;
            Acc acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc_zero(acc[k]);
#pragma unroll
            for (int ii = 0; ii < RPL; ++ii) {
                const int r = lane + 32 * ii;
                const float v = r < rows ? coef(col, r) : 0.f;
                if constexpr (std::is_same<Acc, float>::value && NR % 2 == 0) {
#pragma unroll
                    for (int k = 0; k < NR; k += 2) acc_fma2(acc[k], acc[k + 1], v, xr[k][ii], xr[k + 1][ii]);
                } else {
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc_fma(acc[k], v, xr[k][ii]);
                }
            }
            const int k = warp_reduce_scatter<NR>(acc, lane);
            if ((lane & (32 / NR - 1)) == 0 && k < a.nr) P[(ch.zoff + c) * a.nr + k] = (Vv)acc_value(acc[0]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
    }
}

// ---- phase 1 on tensor cores: BF16 V factors, 16 right-hand sides
//
// P (columns x 16) = V_chunk^T X_leaf as mma.sync m16n8k16 BF16 x BF16 -> FP32: the A
// operand is V^T (row m = V column, k = leaf row; a column of the stream is contiguous in
// shared memory, so ldmatrix reads A fragments directly), the B operand the leaf's rows
// of x, each value split into BF16 hi + lo (two products, x kept to ~16 bits), kept in
// registers for the whole leaf.  Warp w takes n-tile w % 2 (8 RHS) and m-tiles
// w / 2, w / 2 + NCW / 2, ...; a lane whose ldmatrix row lies outside the chunk reads a
// zeroed 16-byte line instead, so no access leaves the chunk.
constexpr int TC_KT = 12;  // k-tiles of 16 rows: leaves of up to 192 rows

template <int NCW>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) k_phase1_tc(StreamArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) uint16_t zline[8];
    uint64_t* full = (uint64_t*)smem;
    uint64_t* empty = full + STAGES;
    unsigned char* stage = smem + BAR_BYTES;

    if (a.skip && *(volatile const int*)a.skip) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < 8) zline[threadIdx.x] = 0;
    init_ring(full, empty, NCW);
    const int c0 = a.cta_begin[blockIdx.x], c1 = a.cta_begin[blockIdx.x + 1];
    pdl_trigger();
    if (w == NCW) {
        if (lane == 0) produce<uint16_t, float, 16, false>(a, stage, STAGE_BYTES, full, empty, c0, c1);
        return;
    }
    pdl_wait();
    const float* xc = (const float*)a.xc;
    float* P = (float*)a.out;
    const int nt = w & 1;
    const uint32_t zaddr = smem_u32(zline);
    int cur = -1, rows = 0;
    uint32_t bh[TC_KT][2], bl[TC_KT][2];
    Chunk nxt = c0 < c1 ? a.chunks[c0] : Chunk{};
    for (int i = c0; i < c1; ++i) {
        const Chunk ch = nxt;
        if (i + 1 < c1) nxt = a.chunks[i + 1];
        const int q = i - c0, s = q % STAGES;
        if (ch.leaf != cur) {
            cur = ch.leaf;
            const LeafDesc L = a.leaves[cur];
            rows = 3 * L.n;
            // B fragments: b0b1 = X[k0 + 2 (lane % 4) + {0, 1}][n], b2b3 = the same 8 rows on
            // (n = nt * 8 + lane / 4), low half the smaller k
            const int n = nt * 8 + (lane >> 2);
#pragma unroll
            for (int kt = 0; kt < TC_KT; ++kt)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t hi2 = 0, lo2 = 0;
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int k = kt * 16 + hh * 8 + 2 * (lane & 3) + e;
                        const float x = k < rows ? xc[(3 * (int64_t)L.begin + k) * 16 + n] : 0.f;
                        const uint32_t hb = bf16_bits(x);
                        const uint32_t lb = bf16_bits(x - bf16_value(hb));
                        hi2 |= hb << (16 * e);
                        lo2 |= lb << (16 * e);
                    }
                    bh[kt][hh] = hi2;
                    bl[kt][hh] = lo2;
                }
        }
        mbar_wait(full + s, (uint32_t)(q / STAGES) & 1u, a.err, 1, a.wait_ns);
        const uint16_t* buf = (const uint16_t*)(stage + (size_t)s * STAGE_BYTES);
        const int ld = ch.ld, ncols = ch.ncols;
        const int mtiles = (ncols + 15) >> 4;
        const int j8 = lane >> 3, i8 = lane & 7;
        for (int mt = w >> 1; mt < mtiles; mt += NCW / 2) {
            const int m = mt * 16 + (j8 & 1) * 8 + i8;  // this lane's ldmatrix row (a V column)
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < TC_KT; ++kt) {
                const int k = kt * 16 + (j8 >> 1) * 8;
                if (kt * 16 >= ld) break;
                const uint32_t addr = (m < ncols && k < ld) ? smem_u32(buf + (size_t)m * ld + k) : zaddr;
                uint32_t a0, a1, a2, a3;
                ldsm_x4(addr, a0, a1, a2, a3);
                mma_bf16(d, a0, a1, a2, a3, bh[kt][0], bh[kt][1]);
                mma_bf16(d, a0, a1, a2, a3, bl[kt][0], bl[kt][1]);
            }
            // d0, d1: column mt*16 + lane/4, RHS nt*8 + 2 (lane % 4) + {0, 1}; d2, d3: column + 8
            const int col = mt * 16 + (lane >> 2), rhs = nt * 8 + 2 * (lane & 3);
            if (col < ncols)
                *reinterpret_cast<float2*>(P + (ch.zoff + col) * 16 + rhs) = make_float2(d[0], d[1]);
            if (col + 8 < ncols)
                *reinterpret_cast<float2*>(P + (ch.zoff + col + 8) * 16 + rhs) = make_float2(d[2], d[3]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
    }
}

// launch with programmatic stream serialisation (the kernel may start before its
// predecessor on the stream completes; it synchronises through griddepcontrol.wait)
template <class... P, class... A>
void launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HM_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

constexpr int EV_PER_PRODUCT = 6;
constexpr int EV_POOL = EV_PER_PRODUCT * 1024;

void timing_accumulate(HMat& H) {
    if (H.ev_used == 0) return;
    HM_CUDA(cudaEventSynchronize(H.ev[H.ev_used - 1]));
    for (int s = 0; s < H.ev_used; s += EV_PER_PRODUCT) {
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            HM_CUDA(cudaEventElapsedTime(&ms, H.ev[s + i], H.ev[s + i + 1]));
            H.t_acc[i] += ms;
        }
        ++H.t_count;
    }
    H.ev_used = 0;
}

// phase boundary idx (0 before the gather ... 5 after the scatter) of one product
void mark(HMat& H, int idx, cudaStream_t st) {
    if (!H.timing) return;
    if (idx == 0 && H.ev_used + EV_PER_PRODUCT > (int)H.ev.size()) timing_accumulate(H);
    HM_CUDA(cudaEventRecord(H.ev[H.ev_used + idx], st));
    if (idx == EV_PER_PRODUCT - 1) H.ev_used += EV_PER_PRODUCT;
}

// consumer warps of phase 1 and phase 2, and phase 2's row split, per right-hand-side
// count: as many warps as the per-thread registers (accumulators and operands) allow
template <int MODE>
constexpr int ncw1_for(int NR) {
    return NR > 4 ? 8 : 16;
}
template <int MODE>
constexpr int ncw2_for(int NR) {
    return NR > 1 && MODE == 1 ? 8 : 16;
}
constexpr int rs_for(int NR) { return NR > 4 ? 2 : 1; }

// ST: ring depth; NCW1V / NCW2V: consumer warps of phase 1 / phase 2 (0: the default for
// the right-hand-side count).  The tile-shape variants the autotuner chooses from use
// other values for the single-RHS FP32-vector product.
template <int MODE, class C, int NR, int RPL, int ST = STAGES, int NCW1V = 0, int NCW2V = 0>
void launch_phases(HMat& H, const HMat::Plan& PL, const StreamArgs& base, bool timed, cudaStream_t st) {
    constexpr int NCW = NCW1V ? NCW1V : ncw1_for<MODE>(NR), NCW2 = NCW2V ? NCW2V : ncw2_for<MODE>(NR),
                  RS = rs_for(NR);
    using Acc = typename AccT<MODE>::type;
    using V = typename AccT<MODE>::vec;
    const size_t smem1 = BAR_BYTES + (size_t)ST * STAGE_BYTES + P1_TAIL;
    // BF16 factors with 16 RHS on leaves of up to 192 rows: phase 1 on tensor cores
    constexpr bool kTensorPhase1 = MODE == 0 && NR == 16 && std::is_same<C, uint16_t>::value && RPL == 6;
    // BF16 factors with one RHS: the U slices of phase 2 on tensor cores, which read t in
    // packed BF16 (hi, lo) form (phase 1 stays on the CUDA cores: one mma.sync per 16 x 16
    // tile did not keep up with the stream there)
    constexpr bool kTensorPhase2x1 = MODE == 0 && NR == 1 && std::is_same<C, uint16_t>::value && RPL == 6;
    static_assert(!kTensorPhase2x1 || (NCW2 == 16 && rs_for(NR) == 1),
                  "the single-RHS tensor-core phase 2 assumes 16 consumer warps without row split");
    // BF16 factors with 16 RHS: the U slices of phase 2 on tensor cores as well, reading t
    // in the packed BF16 form of k_reduce_pack16_mix
    constexpr bool kTensorPhase2x16 = MODE == 0 && NR == 16 && std::is_same<C, uint16_t>::value && RPL == 6;
    constexpr int KP = (MODE == 0 && NR == 16 && RPL == 6) ? 8 : 1;  // RHS per flush pass of k_phase2
    const size_t smem2 = BAR_BYTES + (size_t)ST * (ZRange<V, NR>::BYTES + STAGE_BYTES) +
                         (size_t)KP * (NCW2 / RS) * 32 * RPL * sizeof(Acc) + (kTensorPhase2x16 ? 16 * 196 * 4 : 0);
    // shared-memory opt-in, once per device for each instantiation
    static bool attr_done[64] = {};
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        HM_CUDA(cudaFuncSetAttribute(k_phase1<MODE, C, NR, RPL, NCW, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem1));
        if constexpr (kTensorPhase1)
            HM_CUDA(cudaFuncSetAttribute(k_phase1_tc<NCW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
        HM_CUDA(cudaFuncSetAttribute(k_phase2<MODE, C, NR, RPL, NCW2, RS, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (H.n_far > 0 && H.p_len > 0) {
        StreamArgs a = base;
        a.chunks = PL.ch1.p;
        a.cta_begin = PL.cta1.p;
        a.out = MODE == 0 ? (void*)H.Pf.p : (void*)H.P.p;
        bool tc = false;
        if constexpr (kTensorPhase1) tc = base.nr == 16;
        if (tc)
            launch_pdl(k_phase1_tc<NCW>, dim3(H.grid), dim3((NCW + 1) * 32), smem1, st, a);
        else
            launch_pdl(k_phase1<MODE, C, NR, RPL, NCW, ST>, dim3(H.grid), dim3((NCW + 1) * 32), smem1, st, a);
        HM_LAUNCH_CHECK();
        if (timed) mark(H, 2, st);
        using Zt = typename AccT<MODE>::zin;
        // several FP32 RHS in multiples of 4: the float4 variant (nrhs 1 keeps the scalar one);
        // BF16 factors with one RHS: t packed as BF16 (hi, lo) for the tensor-core phase 2
        // one RHS: big blocks a CTA each, the others a warp each (red_order)
        const unsigned gm = (unsigned)std::max<int64_t>(1, H.n_red_big + (H.n_red - H.n_red_big + 7) / 8);
        if constexpr (kTensorPhase2x1)
            launch_pdl(k_reduce_mix<V, uint32_t>, dim3(gm), dim3(256), 0, st, (const FarDesc*)H.far.p,
                       (const int32_t*)H.poff.p, (const int32_t*)H.uoff.p, (const int32_t*)H.red_order.p,
                       H.n_red_big, H.n_red,
                       (const V*)a.out, (uint32_t*)base.tb, base.skip);
        else if (kTensorPhase2x16 && base.nr == 16)
            launch_pdl(k_reduce_pack16_mix, dim3(gm), dim3(256), 0, st, (const FarDesc*)H.far.p,
                       (const int32_t*)H.poff.p, (const int32_t*)H.uoff.p, (const int32_t*)H.red_order.p,
                       H.n_red_big, H.n_red, (const float*)a.out, (uint16_t*)base.tb, base.skip);
        else if (base.nr == 1)
            launch_pdl(k_reduce_mix<V, Zt>, dim3(gm), dim3(256), 0, st, (const FarDesc*)H.far.p,
                       (const int32_t*)H.poff.p, (const int32_t*)H.uoff.p, (const int32_t*)H.red_order.p,
                       H.n_red_big, H.n_red,
                       (const V*)a.out, (Zt*)base.tb, base.skip);
        else if (MODE == 0 && (base.nr & 3) == 0)
            launch_pdl(k_reduce_tb<V, Zt, MODE == 0>, dim3((unsigned)H.n_far), dim3(128), 0, st,
                       (const FarDesc*)H.far.p, (const int32_t*)H.poff.p, (const int32_t*)H.uoff.p, (const V*)a.out,
                       (Zt*)base.tb, base.nr, base.skip);
        else
            launch_pdl(k_reduce_tb<V, Zt, false>, dim3((unsigned)H.n_far), dim3(128), 0, st,
                       (const FarDesc*)H.far.p, (const int32_t*)H.poff.p, (const int32_t*)H.uoff.p, (const V*)a.out,
                       (Zt*)base.tb, base.nr, base.skip);
        HM_LAUNCH_CHECK();
        if (timed) mark(H, 3, st);
    } else if (timed) {
        mark(H, 2, st);
        mark(H, 3, st);
    }
    StreamArgs a = base;
    a.chunks = PL.ch2.p;
    a.cta_begin = PL.cta2.p;
    a.split = PL.split.p;
    launch_pdl(k_phase2<MODE, C, NR, RPL, NCW2, RS, ST>, dim3(H.grid), dim3((NCW2 + 1) * 32), smem2, st, a);
    HM_LAUNCH_CHECK();
    if (timed) mark(H, 4, st);
}

template <int MODE, class C, int NR>
void launch_rpl(HMat& H, const HMat::Plan& PL, const StreamArgs& a, bool timed, cudaStream_t st) {
    if (H.ld_max <= 192)
        launch_phases<MODE, C, NR, 6>(H, PL, a, timed, st);
    else
        launch_phases<MODE, C, NR, 12>(H, PL, a, timed, st);
}

// The single-RHS FP32-vector product with the ring depth and consumer-warp count of the
// H-matrix's tile shape (leaves of up to 64 elements); false if the shape is the default.
// BF16 factors keep 16 warps in phase 2 (its tensor-core U slices assume them).
template <class C>
bool launch_shape_variant(HMat& H, const HMat::Plan& PL, const StreamArgs& a, bool timed, cudaStream_t st) {
    const int ring = H.shape.ring, warps = H.shape.warps;
    if (H.ld_max > 192 || (ring == STAGES && warps == 16)) return false;
    constexpr bool b16 = std::is_same<C, uint16_t>::value;
    if (ring == 6 && warps == 16)
        launch_phases<0, C, 1, 6, 6>(H, PL, a, timed, st);
    else if (ring == STAGES && warps == 8)
        launch_phases<0, C, 1, 6, STAGES, 8, b16 ? 16 : 8>(H, PL, a, timed, st);
    else if (ring == 6 && warps == 8)
        launch_phases<0, C, 1, 6, 6, 8, b16 ? 16 : 8>(H, PL, a, timed, st);
    else
        fail(HM_EINVAL, "product: unsupported tile shape");
    return true;
}

template <int MODE, class C>
void launch_nr(HMat& H, const HMat::Plan& PL, const StreamArgs& a, int nrhs, bool timed, cudaStream_t st) {
    if (nrhs == 1)
        launch_rpl<MODE, C, 1>(H, PL, a, timed, st);
    else if (nrhs <= 4)
        launch_rpl<MODE, C, 4>(H, PL, a, timed, st);
    else
        launch_rpl<MODE, C, 16>(H, PL, a, timed, st);
}

// phase 1, reduction and phase 2 on cluster-ordered operands (see hmat_impl.h)
void run_core(HMat& H, const void* xc, void* yc, int nr, int dtype, int fac, bool timed, cudaStream_t st,
              const int* skip = nullptr) {
    if (!has_factors(H, fac)) fail(HM_EINVAL, "product: the requested factor precision is not stored");
    const HMat::Plan& PL = H.plan[fac];
    StreamArgs a{};
    a.leaves = H.leaves.p;
    a.near = H.near.p;
    a.ucoef = fac == 1 ? (const void*)H.u16.p : (const void*)H.u32.p;
    a.vcoef = fac == 1 ? (const void*)H.v16.p : (const void*)H.v32.p;
    a.counters = H.counters.p;
    a.err = H.err.p;
    a.ndof = H.ndof;
    a.nr = nr;
    a.ld_max = H.ld_max;
    a.skip = skip;
    a.wait_ns = H.wait_ns;
    a.withhold = H.withhold_chunk;
    a.xc = xc;
    a.out = yc;
    if (dtype == HM_F32) {
        a.tb = H.tbf.p;
        a.slots = H.slotsf.p;
        if (nr == 1 && (fac == 1 ? launch_shape_variant<uint16_t>(H, PL, a, timed, st)
                                 : launch_shape_variant<float>(H, PL, a, timed, st)))
            return;
        if (fac == 1)
            launch_nr<0, uint16_t>(H, PL, a, nr, timed, st);
        else
            launch_nr<0, float>(H, PL, a, nr, timed, st);
    } else {
        a.tb = H.tb.p;
        a.slots = H.slotsd.p;
        if (fac == 1)
            launch_nr<1, uint16_t>(H, PL, a, nr, timed, st);
        else
            launch_nr<1, float>(H, PL, a, nr, timed, st);
    }
}

}  // namespace

void build_plan_for(HMat& H, HMat::Plan& PLAN, int esz, int G, cudaStream_t st);

void build_product_plan(HMat& H, cudaStream_t st) {
    int dev = 0, nsm = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    H.grid = std::max(1, nsm);
    const int G = H.grid;
    H.ld_max = 0;
    for (const LeafDesc& L : H.h_leaves) H.ld_max = std::max(H.ld_max, L.ld);
    for (int fac = 0; fac < 2; ++fac)
        if (has_factors(H, fac)) build_plan_for(H, H.plan[fac], fac == 1 ? 2 : 4, G, st);
    H.counters.alloc(H.n_leaves);
    HM_CUDA(cudaMemsetAsync(H.counters.p, 0, H.counters.bytes(), st));
    // single-RHS reduction order: blocks with many leaves of T first, factorless ones out
    std::vector<int32_t> big, small;
    for (int64_t b = 0; b < H.n_far; ++b) {
        const FarDesc& F = H.h_far[b];
        if (F.rank <= 0) continue;
        if (F.rank > 256) fail(HM_EINVAL, "product plan: rank above 256");
        (F.n_tleaves > RED_WARP_LEAVES ? big : small).push_back((int32_t)b);
    }
    H.n_red_big = (int64_t)big.size();
    H.n_red = H.n_red_big + (int64_t)small.size();
    big.insert(big.end(), small.begin(), small.end());
    if (big.empty()) big.push_back(0);
    H.red_order.upload(big, st);
    H.err.alloc(1);
    HM_CUDA(cudaMemsetAsync(H.err.p, 0, sizeof(int), st));
}

void build_plan_for(HMat& H, HMat::Plan& PLAN, int esz, int G, cudaStream_t st) {

    // cut a segment into chunks: runs of consecutive operand indices, bounded in size
    auto cut = [&](std::vector<Chunk>& out, std::vector<int64_t>& bytes, int leaf, int kind, int64_t src,
                   const std::vector<int32_t>& idx, int cbase, int ncols, int ld, int elem) {
        const int per = std::max(1, std::min(H.shape.chunk_cols, H.shape.chunk_bytes / (ld * elem)));
        int c = 0;
        while (c < ncols) {
            int n = 1;
            while (c + n < ncols && n < per && idx[cbase + c + n] == idx[cbase + c] + n) ++n;
            Chunk ch;
            ch.src = src + (int64_t)c * ld;
            ch.zoff = idx[cbase + c];
            ch.leaf = leaf;
            ch.ncols = n;
            ch.kind = kind;
            ch.ld = ld;
            out.push_back(ch);
            bytes.push_back((int64_t)n * ld * elem);
            c += n;
        }
    };
    auto split_ranges = [&](const std::vector<int64_t>& bytes, std::vector<int32_t>& cta) {
        int64_t tot = 0;
        for (int64_t b : bytes) tot += b;
        cta.assign(G + 1, (int32_t)bytes.size());
        int64_t acc = 0;
        int w = 0;
        cta[0] = 0;
        for (size_t i = 0; i < bytes.size(); ++i) {
            // chunk i goes to the CTA whose share contains its first byte
            while (w + 1 <= G && acc >= (tot * (int64_t)(w + 1)) / G) {
                ++w;
                cta[w] = (int32_t)i;
            }
            acc += bytes[i];
        }
        for (int q = w + 1; q <= G; ++q) cta[q] = (int32_t)bytes.size();
        // A chunk larger than a share would leave the CTAs whose shares it covers without
        // a chunk; such an empty CTA inside a row leaf split over several CTAs would be
        // counted as a part of it and never arrive.  So every CTA gets at least one chunk
        // (with fewer chunks than CTAs, one each and the empty CTAs last).
        const int32_t n = (int32_t)bytes.size();
        if (n < G) {
            for (int q = 0; q <= G; ++q) cta[q] = std::min(q, n);
        } else {
            for (int q = 1; q < G; ++q) cta[q] = std::max(cta[q], cta[q - 1] + 1);
            for (int q = G - 1; q >= 1; --q) cta[q] = std::min(cta[q], cta[q + 1] - 1);
        }
    };

    std::vector<Chunk> c1, c2;
    std::vector<int64_t> b1, b2;
    const int nl = H.n_leaves;
    for (int l = 0; l < nl; ++l) {
        const LeafDesc& L = H.h_leaves[l];
        cut(c2, b2, l, 0, L.near_off, H.h_near_zidx, L.near_cbase, L.near_cols, L.ld, 4);
        // the BF16 streams have their own offsets and padding (bf16_ld)
        const bool b16 = esz == 2;
        cut(c2, b2, l, 1, b16 ? L.u_off16 : L.u_off, H.h_u_zidx, L.u_cbase, L.u_cols, b16 ? L.ld16 : L.ld, esz);
        cut(c1, b1, l, 2, b16 ? L.v_off16 : L.v_off, H.h_v_pidx, L.v_cbase, L.v_cols, b16 ? L.ld16 : L.ld, esz);
    }
    std::vector<int32_t> cta1, cta2;
    split_ranges(b1, cta1);
    split_ranges(b2, cta2);
    // split row leaves
    std::vector<LeafSplit> sp(nl, LeafSplit{0, 0, 0, 0});
    std::vector<int> first(nl, -1), last(nl, -1);
    for (int w = 0; w < G; ++w)
        for (int i = cta2[w]; i < cta2[w + 1]; ++i) {
            const int l = c2[i].leaf;
            if (first[l] < 0) first[l] = w;
            last[l] = w;
        }
    int slots = 0;
    for (int l = 0; l < nl; ++l) {
        if (first[l] < 0) fail(HM_EINVAL, "product plan: a leaf has no columns");
        sp[l].w_first = first[l];
        sp[l].nparts = last[l] - first[l] + 1;
        sp[l].slot_base = sp[l].nparts > 1 ? slots : 0;
        if (sp[l].nparts > 1) slots += sp[l].nparts;
    }
    PLAN.n_slots = slots;
    PLAN.ch1.upload(c1, st);
    PLAN.ch2.upload(c2, st);
    PLAN.cta1.upload(cta1, st);
    PLAN.cta2.upload(cta2, st);
    PLAN.split.upload(sp, st);
    PLAN.ready = true;
}

void ensure_product_scratch(HMat& H, int nrhs, cudaStream_t st) {
    if (nrhs <= H.nrhs_cap) return;
    graphs_clear(H);  // captured products refer to the scratch being replaced
    const int cap = nrhs <= 1 ? 1 : (nrhs <= 4 ? 4 : 16);
    const size_t nv = (size_t)H.ndof * cap + VEC_SLACK;
    const size_t np = (size_t)std::max<int64_t>(H.p_len, 1) * cap + VEC_SLACK;
    const size_t nt = (size_t)std::max<int64_t>(H.tb_len, 1) * cap + VEC_SLACK;
    H.xc.alloc(nv);
    H.yc.alloc(nv);
    H.xcf.alloc(nv);
    H.ycf.alloc(nv);
    H.P.alloc(np);
    H.tb.alloc(nt);
    H.Pf.alloc(np);
    H.tbf.alloc(nt);
    // the slack read by rounded-up operand copies is never used, but keep it defined
    HM_CUDA(cudaMemsetAsync(H.xc.p, 0, H.xc.bytes(), st));
    HM_CUDA(cudaMemsetAsync(H.xcf.p, 0, H.xcf.bytes(), st));
    HM_CUDA(cudaMemsetAsync(H.tb.p, 0, H.tb.bytes(), st));
    HM_CUDA(cudaMemsetAsync(H.tbf.p, 0, H.tbf.bytes(), st));
    int slots = 1;
    for (const HMat::Plan& p : H.plan) slots = std::max(slots, p.n_slots);
    const size_t sl = (size_t)slots * 16 * std::max(H.ld_max, 1);
    H.slotsf.alloc(sl);
    H.slotsd.alloc(sl);
    H.nrhs_cap = cap;
}

void product_core(HMat& H, const void* xc, void* yc, int nr, int dtype, int fac, cudaStream_t st, const int* skip) {
    if (nr < 1 || nr > 16) fail(HM_EINVAL, "product: 1 to 16 right-hand sides per pass");
    ensure_product_scratch(H, nr, st);
    run_core(H, xc, yc, nr, dtype, fac, false, st, skip);
}

void matvec(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st, int factors) {
    if (nrhs < 1) fail(HM_EINVAL, "matvec: nrhs must be >= 1");
    if (!x || !y) fail(HM_EINVAL, "matvec: NULL vector");
    if (dtype != HM_F32 && dtype != HM_F64) fail(HM_EINVAL, "matvec: dtype must be HM_F32 or HM_F64");
    if (factors != 0 && factors != HM_F32 && factors != HM_BF16)
        fail(HM_EINVAL, "matvec: factors must be 0, HM_F32 or HM_BF16");
    // FP32 factors when stored, unless the caller asks for a stored precision
    const int fac = factors == HM_BF16 ? 1 : (factors == HM_F32 ? 0 : (has_factors(H, 0) ? 0 : 1));
    if (!has_factors(H, fac)) fail(HM_EINVAL, "matvec: the requested factor precision is not stored");
    ensure_product_scratch(H, std::min(nrhs, 16), st);
    // at most 16 right-hand sides per pass of the coefficient streams
    for (int k0 = 0; k0 < nrhs; k0 += 16) {
        const int nr = std::min(16, nrhs - k0);
        const int64_t tot = H.ndof * nr;
        const unsigned gb = (unsigned)ceil_div(tot, 256);
        mark(H, 0, st);
        if (dtype == HM_F32) {
            const float* xf = (const float*)x + (int64_t)k0 * H.ndof;
            float* yf = (float*)y + (int64_t)k0 * H.ndof;
            k_gather<float><<<gb, 256, 0, st>>>(xf, H.xcf.p, H.perm.p, H.N, nr);
            mark(H, 1, st);
            run_core(H, H.xcf.p, H.ycf.p, nr, dtype, fac, true, st);
            launch_pdl(k_scatter<float>, dim3(gb), dim3(256), 0, st, (const float*)H.ycf.p, yf,
                       (const int32_t*)H.perm.p, (int64_t)H.N, nr);
        } else {
            const double* xd = (const double*)x + (int64_t)k0 * H.ndof;
            double* yd = (double*)y + (int64_t)k0 * H.ndof;
            k_gather_split<<<gb, 256, 0, st>>>(xd, (float2*)H.xc.p, H.perm.p, H.N, nr);
            mark(H, 1, st);
            run_core(H, H.xc.p, H.yc.p, nr, dtype, fac, true, st);
            launch_pdl(k_scatter<double>, dim3(gb), dim3(256), 0, st, (const double*)H.yc.p, yd,
                       (const int32_t*)H.perm.p, (int64_t)H.N, nr);
        }
        HM_LAUNCH_CHECK();
        mark(H, 5, st);
    }
}

void matvec_host(HMat& H, const void* x, void* y, int nrhs, int dtype, cudaStream_t st) {
    if (nrhs < 1) fail(HM_EINVAL, "matvec_host: nrhs must be >= 1");
    if (!x || !y) fail(HM_EINVAL, "matvec_host: NULL vector");
    if (dtype != HM_F32 && dtype != HM_F64) fail(HM_EINVAL, "matvec_host: dtype must be HM_F32 or HM_F64");
    const size_t bytes = (size_t)H.ndof * nrhs * (dtype == HM_F32 ? 4 : 8);
    if (H.xs.n < bytes) {
        H.xs.alloc(bytes);
        H.ys.alloc(bytes);
    }
    HM_CUDA(cudaMemcpyAsync(H.xs.p, x, bytes, cudaMemcpyHostToDevice, st));
    matvec(H, H.xs.p, H.ys.p, nrhs, dtype, st);
    HM_CUDA(cudaMemcpyAsync(y, H.ys.p, bytes, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
}

void timing_enable(HMat& H, bool on) {
    if (on) {
        if (H.ev.empty()) {
            H.ev.resize(EV_POOL);
            for (auto& e : H.ev) HM_CUDA(cudaEventCreate(&e));
        }
        for (double& t : H.t_acc) t = 0.0;
        H.t_count = 0;
        H.ev_used = 0;
    } else {
        timing_accumulate(H);
    }
    H.timing = on;
}

void timing_read(HMat& H, double out[6]) {
    timing_accumulate(H);
    for (int i = 0; i < 5; ++i) out[i] = H.t_acc[i];
    out[5] = (double)H.t_count;
}

// Error flags raised by the product kernels since the last check (0 if none); clears them.
int product_error_flags(HMat& H, cudaStream_t st) {
    int e = 0;
    HM_CUDA(cudaMemcpyAsync(&e, H.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (e) {
        HM_CUDA(cudaMemsetAsync(H.err.p, 0, sizeof(int), st));
        // a product that gave up waiting may leave split-leaf arrival counts behind
        HM_CUDA(cudaMemsetAsync(H.counters.p, 0, H.counters.bytes(), st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    return e;
}

}  // namespace hm
