// Internal helpers shared by the translation units of libhmat: error reporting,
// CUDA error checks and an owning device buffer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hmat.h"

namespace hm {

// Scoped NVTX range: names the library's phases (assembly, products, solves, GMRES
// cycles) on a profiler's timeline; NVTX is header-only and costs a few nanoseconds
// when no tool is attached.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

// Exception carrying an hm_status; converted to a return code at the C boundary.
struct Error : public std::runtime_error {
    hm_status code;
    Error(hm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

[[noreturn]] inline void fail(hm_status code, const std::string& msg) { throw Error(code, msg); }

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
    if (e != cudaSuccess) {
        char buf[512];
        snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
        throw Error(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, buf);
    }
}
#define HM_CUDA(x) ::hm::cuda_check((x), #x, __FILE__, __LINE__)
#define HM_LAUNCH_CHECK() ::hm::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// Owning device allocation (cudaMalloc / cudaFree).
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        HM_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
    void upload(const std::vector<T>& h, cudaStream_t s) {
        if (h.size() != n) alloc(h.size());
        if (n) HM_CUDA(cudaMemcpyAsync(p, h.data(), bytes(), cudaMemcpyHostToDevice, s));
    }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Element record in cluster order on the device (176 bytes).
struct __align__(16) ElemRec {
    double c[3];
    double s1[3];
    double s2[3];
    double n[3];
    double a, b;    // rectangle: half sides along s1, s2; triangle: both sqrt(area) / 2
    double tv[6];   // triangle: its vertices in the (s1, s2) frame about c
    double shape;   // HM_SHAPE_RECT or HM_SHAPE_TRI
    double area;
};
static_assert(sizeof(ElemRec) == 176, "ElemRec is eleven 16-byte words");

}  // namespace hm

// Status-returning wrapper used by every extern "C" function.
#define HM_API_BEGIN try {
#define HM_API_END                                                   \
    }                                                                \
    catch (const ::hm::Error& e) {                                   \
        ::hm::set_last_error(e.what());                              \
        return e.code;                                               \
    }                                                                \
    catch (const std::bad_alloc&) {                                  \
        ::hm::set_last_error("host allocation failed");              \
        return HM_ENOMEM;                                            \
    }                                                                \
    catch (const std::exception& e) {                                \
        ::hm::set_last_error(e.what());                              \
        return HM_EINVAL;                                            \
    }                                                                \
    return HM_OK;
