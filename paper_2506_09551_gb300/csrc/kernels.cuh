// Device helpers shared by the solver, Lanczos and map kernels.
#pragma once

#include <functional>

#include "operator.cuh"

namespace msb {

// c * v for a complex scalar c = (cr, ci): complex v -> complex product;
// real v -> cr * v (callers pass ci = 0 for real vectors).
__device__ __forceinline__ double2 cscale(double cr, double ci, double2 v) {
    return make_double2(cr * v.x - ci * v.y, cr * v.y + ci * v.x);
}
__device__ __forceinline__ float2 cscale(double cr, double ci, float2 v) {
    const float a = float(cr), b = float(ci);
    return make_float2(a * v.x - b * v.y, a * v.y + b * v.x);
}
__device__ __forceinline__ double cscale(double cr, double, double v) { return cr * v; }
__device__ __forceinline__ float cscale(double cr, double, float v) { return float(cr) * v; }

// Bilinear product term u * v (no conjugation) accumulated into (re, im) in FP64.
__device__ __forceinline__ void bil_acc(double2 u, double2 v, double& re, double& im) {
    re = fma(u.x, v.x, fma(-u.y, v.y, re));
    im = fma(u.x, v.y, fma(u.y, v.x, im));
}
// Compensated accumulation of products in the FP32 pipe.  GB300 issues FP64 at
// 1/64 of the FP32 rate, so per-element FP64 work would bound the FP32 path.
// hi + lo carries the running sum of x*y to about 2^-48 relative: the product
// is split exactly with an FMA (TwoProduct) and added with Knuth's TwoSum; the
// _rn intrinsics keep the compiler from contracting the error terms away.
// The pair is converted to FP64 once per thread (df_value).
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ double df_value(float hi, float lo) { return double(hi) + double(lo); }

// (hi, lo) += (bh, bl) in float-float arithmetic (TwoSum of the high parts).
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, bl));
}

// Block sum of per-thread float-float pairs with FP32 arithmetic only (warp
// shuffles, then one warp over the warp sums); thread 0 gets hi + lo as a
// double.  sm: 64 floats.  Every thread of the block must call it.
__device__ __forceinline__ double block_sum_df(float hi, float lo, float* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
        df_add(hi, lo, oh, ol);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        sm[2 * wid] = hi;
        sm[2 * wid + 1] = lo;
    }
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        hi = lane < nw ? sm[2 * lane] : 0.f;
        lo = lane < nw ? sm[2 * lane + 1] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            df_add(hi, lo, oh, ol);
        }
        r = double(hi) + double(lo);
    }
    return r;
}

// Compensated accumulators of a bilinear product (re, im) and a squared norm.
struct DF4 { float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f, nh = 0.f, nl = 0.f; };
__device__ __forceinline__ void bil_acc_df(float2 u, float2 v, DF4& a) {
    df_add_prod(a.rh, a.rl, u.x, v.x);
    df_add_prod(a.rh, a.rl, -u.y, v.y);
    df_add_prod(a.ih, a.il, u.x, v.y);
    df_add_prod(a.ih, a.il, u.y, v.x);
}
__device__ __forceinline__ void norm_acc_df(float2 v, DF4& a) {
    df_add_prod(a.nh, a.nl, v.x, v.x);
    df_add_prod(a.nh, a.nl, v.y, v.y);
}
// Compensated Hermitian product term conj(u) * v (FP32 vectors) into a DF4.
__device__ __forceinline__ void her_acc_df(float2 u, float2 v, DF4& a) {
    df_add_prod(a.rh, a.rl, u.x, v.x);
    df_add_prod(a.rh, a.rl, u.y, v.y);
    df_add_prod(a.ih, a.il, u.x, v.y);
    df_add_prod(a.ih, a.il, -u.y, v.x);
}
// Hermitian product term conj(u) * v accumulated into (re, im).
__device__ __forceinline__ void her_acc(double2 u, double2 v, double& re, double& im) {
    re = fma(u.x, v.x, fma(u.y, v.y, re));
    im = fma(u.x, v.y, fma(-u.y, v.x, im));
}
__device__ __forceinline__ void her_acc(float2 u, float2 v, double& re, double& im) {
    her_acc(make_double2(u.x, u.y), make_double2(v.x, v.y), re, im);
}
__device__ __forceinline__ double norm2(double2 u) { return fma(u.x, u.x, u.y * u.y); }
__device__ __forceinline__ double norm2(float2 u) {
    const double a = u.x, b = u.y;
    return fma(a, a, b * b);
}
__device__ __forceinline__ double norm2(double u) { return u * u; }

// Sum of the n partials written by a producer kernel (stride NV, component i),
// computed by one CTA in a fixed order.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* part, int n, double (&out)[NV], double* sm) {
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] += part[int64_t(b) * NV + i];
    }
    block_sum<NV>(out, sm);
}

// Store per-block partials (thread 0 holds the block sum after block_sum).
template <int NV>
__device__ __forceinline__ void store_partials(double (&v)[NV], double* sm, double* part) {
    block_sum<NV>(v, sm);
    if (threadIdx.x == 0) {
        const int64_t base = (int64_t(blockIdx.y) * gridDim.x + blockIdx.x) * NV;
#pragma unroll
        for (int i = 0; i < NV; ++i) part[base + i] = v[i];
    }
}

// CUDA device sanity check used by every compute entry point.
void require_device();
msb_status guard(const char* fn, const std::function<void()>& body);

}  // namespace msb
