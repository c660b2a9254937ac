// Shared helpers of libmsbicg: status handling, device buffers, complex
// arithmetic for double2/float2, warp/block reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/msbicg.h"

namespace msb {

// ----------------------------------------------------------------------------
// Errors: internal code throws msb::Error; the C ABI layer converts it into a
// status + thread-local message.
// ----------------------------------------------------------------------------
struct Error : std::runtime_error {
    msb_status status;
    Error(msb_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] inline void fail(msb_status s, const std::string& m) { throw Error(s, m); }

inline void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
    if (e != cudaSuccess) {
        msb_status s = (e == cudaErrorMemoryAllocation) ? MSB_ENOMEM : MSB_ECUDA;
        fail(s, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                    std::to_string(line) + ")");
    }
}
#define MSB_CUDA(x) ::msb::cuda_check((x), #x, __FILE__, __LINE__)
#define MSB_LAUNCH_CHECK() ::msb::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)
#define MSB_REQUIRE(cond, msg) \
    do { if (!(cond)) ::msb::fail(MSB_EINVAL, msg); } while (0)

// Number of SMs of the current device (cached per device).
int sm_count();
// Launch counter, used for the gpu_launches claim of the bench.
extern thread_local int64_t g_launches;
inline void count_launch(int64_t n = 1) { g_launches += n; }

// ----------------------------------------------------------------------------
// Device buffer (RAII).  Tracks the bytes a call allocated.
// ----------------------------------------------------------------------------
extern thread_local int64_t g_alloc_bytes;

template <typename T>
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
        MSB_CUDA(cudaMalloc(&p, count * sizeof(T)));
        n = count;
        g_alloc_bytes += int64_t(count * sizeof(T));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const T* h, size_t count, cudaStream_t s = 0) {
        MSB_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void zero(cudaStream_t s = 0) {
        if (n) MSB_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    size_t bytes() const { return n * sizeof(T); }
};

// Pinned host buffer.
template <typename T>
struct HostBuf {
    T* p = nullptr;
    size_t n = 0;
    HostBuf() = default;
    explicit HostBuf(size_t count) {
        if (count) MSB_CUDA(cudaMallocHost(&p, count * sizeof(T)));
        n = count;
    }
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf() { if (p) cudaFreeHost(p); }
};

// ----------------------------------------------------------------------------
// Complex arithmetic on CUDA vector types.  Real scalar type S, complex C.
// ----------------------------------------------------------------------------
template <typename S> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <typename S> using cplx_t = typename Cplx<S>::type;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a + b * c
template <typename C> __host__ __device__ __forceinline__ C cfma(C b, C c, C a) {
    return mk(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
__host__ __device__ __forceinline__ float2 cfma(float2 b, float2 c, float2 a) {
    return make_float2(fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y)));
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm for a / b.
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __device__ __forceinline__ C from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
    return make_float2(float(a.x), float(a.y));
}

// ----------------------------------------------------------------------------
// Reductions.  Deterministic: fixed shuffle tree inside a block, and partials
// per block summed in index order by a single CTA afterwards.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum NV doubles over the block; result valid in thread 0.  `sm` needs
// NV * 32 doubles.  All threads of the block must call it.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[i * 32 + wid] = v[i];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = lane < nw ? sm[i * 32 + lane] : 0.0;
            v[i] = warp_sum(x);
        }
    }
    __syncthreads();
}

inline int div_up(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// Grid size for a grid-stride kernel over n items: a multiple of the SM count.
inline int grid_for(int64_t n, int block, int per_sm = 4) {
    int64_t want = (n + block - 1) / block;
    int64_t cap = int64_t(sm_count()) * per_sm;
    if (want < 1) want = 1;
    return int(want < cap ? want : cap);
}

}  // namespace msb
