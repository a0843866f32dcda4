// hm_influence_blocks_noalloc: the influence-block evaluation of hm_influence_blocks
// without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc at the point where they evaluate
// coefficients -- for example code running under a caching or pooled allocator that
// owns all device memory and forbids side allocations, code on a latency-critical path
// where cudaMalloc/cudaFree would synchronise the device, or hosts that embed this
// library with a fixed device-memory budget.  hm_influence_blocks copies the element
// geometry into a freshly allocated device buffer on every call; this variant uses a
// fixed scratch array in the module's global memory instead.
//
// Scratch: one file-scope __device__ array of NOALLOC_SCRATCH_BYTES (8 MiB) that every
// GPU which loads the library holds until the process exits.  Its first 256 bytes hold
// the error word; the rest holds the element geometry as structure-of-arrays doubles
// (c, s1, s2, n: 3N each; a, b: N each), i.e. 112 bytes per element, so at most
// NOALLOC_MAX_ELEMENTS = 65,536 elements.  Every call shares the array and leaves the
// last call's contents in it; the error word is cleared at the start of each call.
// Calls whose work overlaps on the GPU (several host threads, or several streams)
// race on the array: serialise them.
#include <mutex>

#include "ddkernel.cuh"

namespace hm {

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;
constexpr int64_t NOALLOC_MAX_ELEMENTS = 65536;
constexpr size_t NOALLOC_HEADER = 256;
static_assert(NOALLOC_HEADER + (size_t)NOALLOC_MAX_ELEMENTS * 14 * sizeof(double) <= NOALLOC_SCRATCH_BYTES,
              "scratch too small for the element limit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up once per device).
void* scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (dev < 0 || dev >= MAX_DEVICES) fail(HM_EINVAL, "influence_blocks_noalloc: device ordinal out of range");
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        HM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

__device__ __forceinline__ void load_elem(const double* g, int64_t N, int64_t i, ElemRec& r) {
    const double* c = g;
    const double* s1 = g + 3 * N;
    const double* s2 = g + 6 * N;
    const double* n = g + 9 * N;
    const double* a = g + 12 * N;
    const double* b = g + 13 * N;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r.c[d] = c[3 * i + d];
        r.s1[d] = s1[3 * i + d];
        r.s2[d] = s2[3 * i + d];
        r.n[d] = n[3 * i + d];
    }
    r.a = a[i];
    r.b = b[i];
#pragma unroll
    for (int q = 0; q < 6; ++q) r.tv[q] = 0.0;
    r.shape = HM_SHAPE_RECT;
    r.area = 4.0 * r.a * r.b;
}

// Same arithmetic as the allocating entry point; geometry read from the scratch array.
__global__ void k_influence_pairs_noalloc(const int64_t* __restrict__ ri, const int64_t* __restrict__ sj,
                                          int64_t npairs, int64_t N, double mu, double nu,
                                          double* __restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    int* err = reinterpret_cast<int*>(g_noalloc_scratch);
    const double* geom = reinterpret_cast<const double*>(g_noalloc_scratch + NOALLOC_HEADER);
    const int64_t i = ri[p], j = sj[p];
    double blk[9];
    if (i < 0 || i >= N || j < 0 || j >= N) {
        atomicOr(err, 2);
        for (int k = 0; k < 9; ++k) out[9 * p + k] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    ElemRec er, es;
    load_elem(geom, N, i, er);
    load_elem(geom, N, j, es);
    if (!dd_block(er, es, mu, nu, blk)) atomicOr(err, 1);
#pragma unroll
    for (int k = 0; k < 9; ++k) out[9 * p + k] = blk[k];
}

}  // namespace

}  // namespace hm

extern "C" hm_status hm_influence_blocks_noalloc(const hm_elements* el, double E, double nu, int64_t npairs,
                                                 const int64_t* ri_dev, const int64_t* sj_dev, double* out_dev,
                                                 void* stream) {
    HM_API_BEGIN
    using namespace hm;
    if (!el) fail(HM_EINVAL, "influence_blocks_noalloc: NULL element description");
    if (el->N <= 0) fail(HM_EINVAL, "influence_blocks_noalloc: element count must be positive");
    if (el->N > NOALLOC_MAX_ELEMENTS)
        fail(HM_EINVAL, "influence_blocks_noalloc: " + std::to_string(el->N) +
                            " elements exceed the fixed scratch limit of 65536 elements (use hm_influence_blocks)");
    if (!el->c || !el->s1 || !el->s2 || !el->n || !el->a || !el->b)
        fail(HM_EINVAL, "influence_blocks_noalloc: NULL geometry array");
    if (el->shape)
        for (int64_t i = 0; i < el->N; ++i)
            if (el->shape[i] != HM_SHAPE_RECT) fail(HM_EINVAL, "influence_blocks_noalloc: rectangles only");
    if (npairs < 0) fail(HM_EINVAL, "influence_blocks_noalloc: npairs < 0");
    if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5))
        fail(HM_EINVAL, "influence_blocks_noalloc: need E > 0 and -1 < nu < 0.5");
    if (npairs == 0) return HM_OK;
    if (!ri_dev || !sj_dev || !out_dev) fail(HM_EINVAL, "influence_blocks_noalloc: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(dev));
    const int64_t N = el->N;
    double* g = reinterpret_cast<double*>(base + NOALLOC_HEADER);
    HM_CUDA(cudaMemsetAsync(base, 0, sizeof(int), st));  // error word starts at zero
    const size_t v3 = (size_t)3 * N * sizeof(double), v1 = (size_t)N * sizeof(double);
    HM_CUDA(cudaMemcpyAsync(g, el->c, v3, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(g + 3 * N, el->s1, v3, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(g + 6 * N, el->s2, v3, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(g + 9 * N, el->n, v3, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(g + 12 * N, el->a, v1, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(g + 13 * N, el->b, v1, cudaMemcpyHostToDevice, st));
    const double mu = E / (2.0 * (1.0 + nu));
    const int nt = 128;
    k_influence_pairs_noalloc<<<(unsigned)ceil_div(npairs, nt), nt, 0, st>>>(ri_dev, sj_dev, npairs, N, mu, nu,
                                                                            out_dev);
    HM_LAUNCH_CHECK();
    int herr = 0;
    HM_CUDA(cudaMemcpyAsync(&herr, base, sizeof(int), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (herr & 2) fail(HM_EINVAL, "influence_blocks_noalloc: element index out of range");
    if (herr & 1) fail(HM_ESINGULAR_GEOM, "influence_blocks_noalloc: a receiver lies on a source element edge");
    HM_API_END
}
