// common.cuh -- shared device/host helpers of librgcsr (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "rgcsr.h"

#define RGCSR_API extern "C" __attribute__((visibility("default")))

namespace rgcsr {

constexpr unsigned kFull = 0xffffffffu;

#define RGCSR_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return RGCSR_ERR_CUDA;         \
    } while (0)

// A launch error is read back without synchronising.
inline int launch_status() {
    return cudaGetLastError() == cudaSuccess ? RGCSR_OK : RGCSR_ERR_CUDA;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// warp collectives
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// W consecutive elements moved as one access: 16 bytes for W = 16 / sizeof(T)
// (a vector load or store), or one element for W = 1.  The vector kernels
// use W > 1 when every pointer is 16-byte aligned, so that each thread keeps
// 16 bytes per operand in flight, and finish the last n mod W elements one
// by one.
template <typename T, int W>
struct alignas(sizeof(T) * W) Pack {
    T v[W];
};
template <typename T, int W>
__device__ __forceinline__ Pack<T, W> ld_pack(const T *p) { return *reinterpret_cast<const Pack<T, W> *>(p); }
template <typename T, int W>
__device__ __forceinline__ void st_pack(T *p, const Pack<T, W> &v) { *reinterpret_cast<Pack<T, W> *>(p) = v; }
inline bool all_aligned16() { return true; }
template <typename P, typename... R>
inline bool all_aligned16(P p, R... r) { return ((uintptr_t)p & 15) == 0 && all_aligned16(r...); }

// The SplitMix64 finalizer (Steele, Lea and Flood 2014; constants as
// published): a bijection of 64-bit words that scatters every input bit.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ int64_t shfl_i64(int64_t v, int src) {
    int lo = __shfl_sync(kFull, (int)(v & 0xffffffff), src);
    int hi = __shfl_sync(kFull, (int)(v >> 32), src);
    return (int64_t)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
}

// ---------------------------------------------------------------------------
// loads: matrix slabs are read once (streaming, evict-first), x through the
// read-only path so that it stays resident in L1/L2 for reuse.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }

template <typename T>
__device__ __forceinline__ T ld_x(const T *p) { return __ldg(p); }

// Split slot j0 for a warp whose rows differ a lot in length: every lane
// proposes its own row length as j0 and prices it as
//   4*j0 + w4 * sum_s ceil(max(0, len_s - j0) / 32)
// (thread-per-row steps plus weighted warp-cooperative steps); the warp
// takes the cheapest proposal, ties to the smaller j0.  Warp-uniform result.
__device__ __forceinline__ int choose_split(int len, int w4) {
    int cand = len;
    long long cost = 4LL * cand;
#pragma unroll 8
    for (int s = 0; s < 32; ++s) {
        const int d = __shfl_sync(kFull, len, s) - cand;
        if (d > 0) cost += (long long)w4 * ((d + 31) >> 5);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long oc = __shfl_xor_sync(kFull, cost, o);
        const int ocand = __shfl_xor_sync(kFull, cand, o);
        if (oc < cost || (oc == cost && ocand < cand)) { cost = oc; cand = ocand; }
    }
    return cand;
}

// KC consecutive entries of a row of X (read-only path); 16-byte vector
// loads when VEC (the caller checked the alignment of the row pieces).
template <typename A, int KC, bool VEC>
__device__ __forceinline__ void load_xrow(const A *__restrict__ p, A (&o)[KC]) {
    if constexpr (VEC && sizeof(A) == 4 && KC % 4 == 0) {
#pragma unroll
        for (int q = 0; q < KC / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + q);
            o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
        }
    } else if constexpr (VEC && sizeof(A) == 8 && KC % 2 == 0) {
#pragma unroll
        for (int q = 0; q < KC / 2; ++q) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(p) + q);
            o[2 * q] = t.x; o[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int w = 0; w < KC; ++w) o[w] = __ldg(p + w);
    }
}

// Output index of stored row `row`: the CSR row it holds under a row order
// (rgcsr_matrix::row_perm), or the row itself without one.
__device__ __forceinline__ int64_t out_row(const int32_t *perm, int64_t row) {
    return perm ? (int64_t)ld_stream(perm + row) : row;
}

// ---------------------------------------------------------------------------
// Row pointer access for int32 or int64 CSR row pointers.
// ---------------------------------------------------------------------------
struct RowPtr {
    const void *p;
    int wide;   // 1 = int64
    __device__ __forceinline__ int64_t operator[](int64_t i) const {
        return wide ? static_cast<const int64_t *>(p)[i]
                    : (int64_t) static_cast<const int32_t *>(p)[i];
    }
};

inline bool valid_value_type(int t) { return t == RGCSR_F64 || t == RGCSR_F32; }
inline size_t value_bytes(int t) {
    return t == RGCSR_F64 ? 8 : t == RGCSR_F32 ? 4 : (t == RGCSR_BF16 || t == RGCSR_F16) ? 2 : 0;
}

// Shared checks on a CSR descriptor (host side, no device access).
inline int check_csr(const rgcsr_csr *A) {
    if (!A) return RGCSR_ERR_INVALID_ARG;
    if (A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0) return RGCSR_ERR_INVALID_ARG;
    if (A->n_rows >= INT32_MAX || A->n_cols >= INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    if (A->row_ptr_type != RGCSR_I32 && A->row_ptr_type != RGCSR_I64) return RGCSR_ERR_INVALID_ARG;
    if (A->row_ptr_type == RGCSR_I32 && A->nnz >= INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    if (!valid_value_type(A->value_type)) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (A->n_rows > 0 && !A->row_ptr) return RGCSR_ERR_INVALID_ARG;
    if (A->nnz > 0 && (!A->col_idx || !A->values)) return RGCSR_ERR_INVALID_ARG;
    return RGCSR_OK;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of int64 counts, in place (scan.cu).
// data[0..count) are replaced by their exclusive prefix sums and
// data[count] receives the total.  Scratch: scan_partials_bytes(count).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
inline size_t scan_partials_bytes(int64_t count) {
    return align_up((size_t)(ceil_div(count + 1, kScanTile) + 1) * sizeof(int64_t), 256);
}
int exclusive_scan_i64(int64_t *data, int64_t count, int64_t *partials, cudaStream_t s);

// CSR validation (validate.cu): sets bits of *flags (device int) for a bad
// row pointer (1) or a column outside [0, n_cols) (2); also writes the
// longest row length to *max_len (device int64, must start at 0).
int launch_validate_csr(const rgcsr_csr *A, int *flags, int64_t *max_len, cudaStream_t s);
// row_lengths[k] = length of CSR row perm[k] (perm == nullptr: row k)
int launch_row_lengths(const rgcsr_csr *A, const int32_t *perm, int32_t *row_lengths, cudaStream_t s);
// sets bit 4 of *flags unless perm is a permutation of [0, n); seen: n ints of scratch
int launch_check_perm(const int32_t *perm, int64_t n, int32_t *seen, int *flags, cudaStream_t s);

// The kernel and variant RGCSR_KERNEL_AUTO runs for M (spmv.cu).
int auto_kernel(const rgcsr_matrix *M, int *variant);

// Checks mode (check.cu): RGCSR_OK when it is off, when `s` is being
// captured, or when M passes rgcsr_check_matrix; else RGCSR_ERR_CORRUPT
// (and RGCSR_STATUS_CORRUPT is raised).  Products call it before any launch.
int debug_check(const rgcsr_matrix *M, cudaStream_t s);
// Status bits raised on the host since the last call (rgcsr_get_status).
int take_host_status();

// Sum of v over the block (blockDim.x a multiple of 32, <= 1024); sh: 32
// doubles of shared memory.  Every thread returns the total.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

// Float vectors: the compensated dot product "Dot2" of Ogita, Rump and Oishi
// (Accurate sum and dot product, SIAM J. Sci. Comput. 26, 2005) in float,
// so that no FP64 instruction runs per element (GB300's FP64 pipe is
// narrow).  Each product is split exactly into p + e (TwoProduct: a rounded
// product and its FMA residual), the running sum s absorbs p with its exact
// rounding error q (TwoSum), and c collects q + e.  A thread's s + c is as
// accurate as a dot product in twice the working precision; it is widened to
// double and the block sums it in double.  The _rn intrinsics keep the
// compiler from contracting or reordering these steps.
__device__ __forceinline__ void dot2_step(float a, float b, float &s, float &c) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);                            // a b = p + e exactly
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // s + p = t + q exactly
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// The block's partial (every thread passes its own) goes to parts; true in
// the block that finishes last, whose threads then get the grand total.
__device__ __forceinline__ bool reduce_last(double v, double *parts, unsigned *ticket, double *sh, double &total) {
    __shared__ bool last;
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(parts + i);
    total = block_sum(t, sh);
    return true;
}

// Vector kernels (blas1.cu).  dot_device writes the dot product of x and y
// (deterministic; double vectors in double, float vectors by a compensated
// float dot per thread summed in double) to the device scalar *out, using
// kDotParts doubles of scratch.  With `count` (a device counter that is 0
// before the first call; each call leaves it at 0) the block partials are
// added by the last block to finish: one launch, the same result.
constexpr int kDotParts = 304;
int dot_device(int64_t n, const void *x, const void *y, double *out, double *partials, int value_type,
               cudaStream_t s, unsigned *count = nullptr);
int axpby_device(int64_t n, double a, const void *x, double b, void *y, int value_type, cudaStream_t s);
int convert_device(int64_t n, const void *src, int src_type, void *dst, int dst_type, cudaStream_t s);

// TMA-staged SpMV for G = 32 (spmv_tma.cu).
bool tma_eligible(const rgcsr_matrix *M);
// A texture object over x[0, n) (elements of elem_bytes = 4 or 8 bytes),
// created on first use and cached per device and buffer (xpath.cu).
int x_texture(const void *x, int64_t n, int elem_bytes, cudaTextureObject_t *out);
int launch_spmv_tma(const rgcsr_matrix *M, const void *x, void *y, int variant, uint32_t wait_limit,
                    cudaStream_t s);

}  // namespace rgcsr
