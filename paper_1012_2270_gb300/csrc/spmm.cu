// spmm.cu -- Y = A X for an RgCSR matrix and k right-hand sides (X row-major
// [n_cols x k] with row stride ldx, Y row-major [n_rows x k] with stride ldy).
// An extension of the paper's SpMV (Sec. 3.4) to several vectors: the
// matrix slabs are streamed once per chunk of up to KC columns.
//
// Mapping: one thread per row carrying KC accumulators (the columns of its
// row of Y); for every slot it reads one value and one column index
// (coalesced across the warp, as in SpMV) and one KC-wide piece of a row of
// X (16-byte vector loads when aligned).  Warps whose rows differ a lot in
// length split them like the SpMV split kernel: slots beyond the agreed j0
// are spread over the whole warp and the KC partial sums are combined with
// shuffles.
#include "common.cuh"
#include "vtraits.cuh"
#include <climits>

namespace rgcsr {
namespace {

constexpr int kThreads = 256;

// acc[0..KC) += v * X[c, 0..KC), vectorised when VEC (16-byte aligned rows).
template <typename A, int KC, bool VEC>
__device__ __forceinline__ void axpy_row(A (&acc)[KC], A v, const A *__restrict__ xr) {
    if constexpr (VEC && sizeof(A) == 4 && KC % 4 == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(xr);
#pragma unroll
        for (int q = 0; q < KC / 4; ++q) {
            const float4 t = __ldg(p + q);
            acc[4 * q + 0] = fma(v, t.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fma(v, t.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fma(v, t.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fma(v, t.w, acc[4 * q + 3]);
        }
    } else if constexpr (VEC && sizeof(A) == 8 && KC % 2 == 0) {
        const double2 *p = reinterpret_cast<const double2 *>(xr);
#pragma unroll
        for (int q = 0; q < KC / 2; ++q) {
            const double2 t = __ldg(p + q);
            acc[2 * q + 0] = fma(v, t.x, acc[2 * q + 0]);
            acc[2 * q + 1] = fma(v, t.y, acc[2 * q + 1]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < KC; ++q) acc[q] = fma(v, __ldg(xr + q), acc[q]);
    }
}

template <typename V, int KC, bool VEC>
__global__ void __launch_bounds__(kThreads)
rgcsr_spmm_kernel(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                  const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                  const float *__restrict__ scale, const typename VT<V>::A *__restrict__ X, int64_t ldx,
                  typename VT<V>::A *__restrict__ Y, int64_t ldy, const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = row < n;
    int len = 0, stride = 0;
    int64_t ptr = 0;
    if (valid) {
        const int64_t g = row / G;
        const int64_t first = g * G;
        stride = (int)min((int64_t)G, n - first);
        ptr = __ldg(gp + g) + (row - first);
        len = __ldg(rl + row);
    }
    const int lmax = warp_max_i(len);
    const int lmin = warp_min_i(valid ? len : INT_MAX);
    int j0 = lmax;
    if (lmax - lmin > 32) j0 = choose_split(len, 8);

    A acc[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) acc[q] = 0;
    const int jend = min(len, j0);
    constexpr int U = KC >= 8 ? 2 : 4;
    for (int j = 0; j < jend; j += U) {
        A v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < jend) {
                const int64_t p = ptr + (int64_t)(j + u) * stride;
                v[u] = VT<V>::ld(val + p);
                c[u] = ld_stream(col + p);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < jend) axpy_row<A, KC, VEC>(acc, v[u], X + (int64_t)c[u] * ldx);
    }

    unsigned long_rows = __ballot_sync(kFull, len > j0);
    while (long_rows) {
        const int r = __ffs(long_rows) - 1;
        long_rows &= long_rows - 1;
        const int Lr = __shfl_sync(kFull, len, r);
        const int sr = __shfl_sync(kFull, stride, r);
        const int64_t pr = shfl_i64(ptr, r);
        A part[KC];
#pragma unroll
        for (int q = 0; q < KC; ++q) part[q] = 0;
        for (int j = j0 + lane; j < Lr; j += 32) {
            const int64_t p = pr + (int64_t)j * sr;
            axpy_row<A, KC, VEC>(part, VT<V>::ld(val + p), X + (int64_t)ld_stream(col + p) * ldx);
        }
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            const A t = warp_sum(part[q]);
            if (lane == r) acc[q] += t;
        }
    }
    if (valid) {
        A *yr = Y + out_row(perm, row) * ldy;
        A s = 1;
        if constexpr (VT<V>::scaled) s = __ldg(scale + row);
#pragma unroll
        for (int q = 0; q < KC; ++q) yr[q] = VT<V>::scaled ? acc[q] * s : acc[q];
    }
}

template <typename V, int KC>
int launch_chunk(const rgcsr_matrix *M, const typename VT<V>::A *X, int64_t ldx,
                 typename VT<V>::A *Y, int64_t ldy, cudaStream_t s) {
    using A = typename VT<V>::A;
    const int64_t blocks = ceil_div(M->n_rows, kThreads);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    const bool vec = ((uintptr_t)X % 16 == 0) && ((ldx * (int64_t)sizeof(A)) % 16 == 0);
    const V *val = static_cast<const V *>(M->values);
    if (vec)
        rgcsr_spmm_kernel<V, KC, true><<<(unsigned)blocks, kThreads, 0, s>>>(
            M->n_rows, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, M->row_scale,
            X, ldx, Y, ldy, M->row_perm);
    else
        rgcsr_spmm_kernel<V, KC, false><<<(unsigned)blocks, kThreads, 0, s>>>(
            M->n_rows, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, M->row_scale,
            X, ldx, Y, ldy, M->row_perm);
    return launch_status();
}

// Columns in chunks of 32, 16, 8, 4, 2, 1 (FP64: at most 16) -- each chunk
// one launch that streams the matrix once.
template <typename V>
int spmm_t(const rgcsr_matrix *M, int k, const typename VT<V>::A *X, int64_t ldx,
           typename VT<V>::A *Y, int64_t ldy, cudaStream_t s) {
    constexpr int kmax = sizeof(typename VT<V>::A) == 8 ? 16 : 32;
    int c0 = 0;
    while (c0 < k) {
        const int left = k - c0;
        int st;
        if (left >= 32 && kmax >= 32) { st = launch_chunk<V, (kmax >= 32 ? 32 : 16)>(M, X + c0, ldx, Y + c0, ldy, s); c0 += kmax >= 32 ? 32 : 16; }
        else if (left >= 16) { st = launch_chunk<V, 16>(M, X + c0, ldx, Y + c0, ldy, s); c0 += 16; }
        else if (left >= 8) { st = launch_chunk<V, 8>(M, X + c0, ldx, Y + c0, ldy, s); c0 += 8; }
        else if (left >= 4) { st = launch_chunk<V, 4>(M, X + c0, ldx, Y + c0, ldy, s); c0 += 4; }
        else if (left >= 2) { st = launch_chunk<V, 2>(M, X + c0, ldx, Y + c0, ldy, s); c0 += 2; }
        else { st = launch_chunk<V, 1>(M, X + c0, ldx, Y + c0, ldy, s); c0 += 1; }
        if (st != RGCSR_OK) return st;
    }
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_spmm(const rgcsr_matrix *M, int32_t k, const void *X, int64_t ldx, void *Y,
                         int64_t ldy, rgcsr_stream_t stream) {
    if (!M || M->n_rows < 0 || M->group_size < 1 || k < 0) return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows == 0 || k == 0) return RGCSR_OK;
    if (ldx < k || ldy < k || !Y || (M->n_cols > 0 && !X)) return RGCSR_ERR_INVALID_ARG;
    if (!M->group_ptr || !M->row_lengths || (M->n_stored > 0 && (!M->values || !M->columns)))
        return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64:
            return spmm_t<double>(M, k, static_cast<const double *>(X), ldx, static_cast<double *>(Y), ldy, s);
        case RGCSR_F32:
            return spmm_t<float>(M, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy, s);
        case RGCSR_BF16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_t<__nv_bfloat16>(M, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy, s);
        case RGCSR_F16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_t<__half>(M, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy, s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}
