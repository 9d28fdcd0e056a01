// vtraits.cuh -- value storage types of an RgCSR matrix and the arithmetic
// they use.  double and float are the paper's precisions (Sec. 4); bfloat16
// and half (reduced storage, not in the paper) carry a per-row float scale:
// y_i = s_i * sum_j q_ij x_j with x, y and the sum in float.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace rgcsr {

// Storage type V -> arithmetic type A, streaming load (read once, evict
// first), per-row scale flag.
template <typename V> struct VT;
template <> struct VT<double> {
    using A = double;
    static constexpr bool scaled = false;
    static __device__ __forceinline__ double ld(const double *p) { return __ldcs(p); }
};
template <> struct VT<float> {
    using A = float;
    static constexpr bool scaled = false;
    static __device__ __forceinline__ float ld(const float *p) { return __ldcs(p); }
};
template <> struct VT<__nv_bfloat16> {
    using A = float;
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to_float(__nv_bfloat16 h) { return __bfloat162float(h); }
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldcs(p)); }
};
template <> struct VT<__half> {
    using A = float;
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to_float(__half h) { return __half2float(h); }
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldcs(p)); }
};

// A row's sum -> its result: times the row's scale for reduced storage.
template <typename V>
__device__ __forceinline__ typename VT<V>::A finish(typename VT<V>::A acc, const float *scale, int64_t row) {
    if constexpr (VT<V>::scaled) return acc * __ldg(scale + row);
    else return acc;
}

}  // namespace rgcsr
