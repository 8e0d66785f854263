// Accumulators and load helpers shared by the product kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbsp {

enum ValMode { VM_F64 = 0, VM_F32 = 1, VM_F32C = 2 };

__host__ __device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) {
    return (a + b - 1) / b;
}

template <int VM> struct ValT;
template <> struct ValT<VM_F64> { typedef double T; };
template <> struct ValT<VM_F32> { typedef float T; };
template <> struct ValT<VM_F32C> { typedef float T; };

// Streaming loads for the matrix arrays: each element is used once, so mark
// it evict-first (ld.global.cs) and keep L2 for the gathered vector.
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }

// Gathered vector loads through the read-only path.
__device__ __forceinline__ double ld_vec(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_vec(const float *p) { return __ldg(p); }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// Plain accumulator: fused multiply-add chain.
template <int VM> struct Acc {
    typedef typename ValT<VM>::T T;
    T s;
    __device__ __forceinline__ void init() { s = T(0); }
    __device__ __forceinline__ void add(T a, T x) { s = fma(a, x, s); }
    __device__ __forceinline__ void add_value(T v) { s = s + v; }
    __device__ __forceinline__ void merge(const Acc &o) { s = s + o.s; }
    __device__ __forceinline__ void shfl_xor_merge(int off) {
        Acc o;
        o.s = __shfl_xor_sync(0xffffffffu, s, off);
        merge(o);
    }
    // this += (the partner lane's `send`), partner = lane ^ off
    __device__ __forceinline__ void merge_shfl_xor(const Acc &send, int off) {
        Acc o;
        o.s = __shfl_xor_sync(0xffffffffu, send.s, off);
        merge(o);
    }
    __device__ __forceinline__ T result() const { return s; }
};

// Compensated FP32 accumulator (Dot2 of Ogita, Rump & Oishi 2005): exact
// product split by fmaf, running sum by TwoSum, all error terms collected
// in c; merging two accumulators TwoSums the sums and adds the errors.
template <> struct Acc<VM_F32C> {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float a, float x) {
        float p = a * x;
        float e = fmaf(a, x, -p);
        float t;
        two_sum(s, p, s, t);
        c += t + e;
    }
    __device__ __forceinline__ void add_value(float v) {
        float t;
        two_sum(s, v, s, t);
        c += t;
    }
    __device__ __forceinline__ void merge(const Acc &o) {
        float t;
        two_sum(s, o.s, s, t);
        c += o.c + t;
    }
    __device__ __forceinline__ void shfl_xor_merge(int off) {
        Acc o;
        o.s = __shfl_xor_sync(0xffffffffu, s, off);
        o.c = __shfl_xor_sync(0xffffffffu, c, off);
        merge(o);
    }
    __device__ __forceinline__ void merge_shfl_xor(const Acc &send, int off) {
        Acc o;
        o.s = __shfl_xor_sync(0xffffffffu, send.s, off);
        o.c = __shfl_xor_sync(0xffffffffu, send.c, off);
        merge(o);
    }
    __device__ __forceinline__ float result() const { return s + c; }
};

// Reduce an accumulator over aligned groups of L lanes (L divides 32);
// every lane of the warp must call it.  Fixed butterfly order.
template <int L, int VM>
__device__ __forceinline__ void group_reduce(Acc<VM> &a) {
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) a.shfl_xor_merge(off);
}

}  // namespace gbsp
