// common.cuh -- shared device helpers of the ivis engine (complex arithmetic, ES kernel,
// block reductions).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ivis {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
// float2 sums and differences as paired FP32 operations (add/sub.rn.f32x2: the two IEEE
// round-to-nearest results of the scalar forms, in one instruction)
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 f2_from_bits(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(r);
}
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(r);
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Exponential-of-semicircle kernel (Barnett, Magland & af Klinteberg 2019):
// psi(t) = exp(beta (sqrt(1 - z^2) - 1)), z = t / (w/2), zero for |z| > 1.
__device__ __forceinline__ float es_kernel(float z, float beta) {
    float a = 1.0f - z * z;
    return a >= 0.0f ? expf(beta * (sqrtf(a) - 1.0f)) : 0.0f;
}
__device__ __forceinline__ double es_kernel(double z, double beta) {
    double a = 1.0 - z * z;
    return a >= 0.0 ? exp(beta * (sqrt(a) - 1.0)) : 0.0;
}

// sin(pi a), cos(pi a) in the working precision.
__device__ __forceinline__ void sincospi_t(float a, float *s, float *c) { sincospif(a, s, c); }
__device__ __forceinline__ void sincospi_t(double a, double *s, double *c) { sincospi(a, s, c); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree for a fixed block size). scratch: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? scratch[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;  // valid in thread 0
}

// Block sum of per-thread float terms: FP32 within each warp (5 pairwise levels), FP64 across
// the warps by one thread (FP64 issue is scarce on this part). Fixed order; valid in thread 0.
__device__ __forceinline__ double block_sum_warpf(float v, double *scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) s += scratch[w];
    return s;
}

// Block sum in the working precision's scheme: FP32 terms summed per warp in FP32 then in
// FP64 across warps; FP64 terms in FP64 throughout.
__device__ __forceinline__ double block_sum_t(float v, double *scratch) { return block_sum_warpf(v, scratch); }
__device__ __forceinline__ double block_sum_t(double v, double *scratch) { return block_sum(v, scratch); }

__device__ __forceinline__ void atomic_add_c(float2 *p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_add_c(double2 *p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

}  // namespace ivis
