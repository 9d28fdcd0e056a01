// batched.cu -- y_m = A_m x_m for many RgCSR matrices of uneven sizes in one
// persistent launch (an extension of the paper's SpMV to batches; the paper
// measures one matrix at a time and notes that GPU formats lose on small
// matrices, Sec. 4.2 -- batching is the remedy).
//
// The members' RgCSR arrays are concatenated: values/columns (member m's
// slabs start at desc[m].val_off), row lengths and scales (desc[m].row_off),
// group pointers kept local to each member (desc[m].group_off, n_groups+1
// entries starting at 0), x and y concatenated.  A host-built task list
// cuts every member into blocks of 32 rows, so a warp never straddles two
// members; warps of a persistent grid take tasks in an interleaved order.
// Per task the warp runs the split SpMV: one thread per row for the common
// slots, the whole warp for the tail of any much longer row.  Each member
// may have its own group size.  No host synchronisation and no allocation:
// the call can be captured in a CUDA graph.
#include "common.cuh"
#include "vtraits.cuh"
#include <climits>

namespace rgcsr {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;

__device__ __forceinline__ int split_point(int len, bool valid) {
    const int lmax = warp_max_i(len);
    const int lmin = warp_min_i(valid ? len : INT_MAX);
    return lmax - lmin <= 32 ? lmax : choose_split(len, 8);
}

template <typename V>
__global__ void __launch_bounds__(kThreads)
spmv_batched_kernel(int64_t n_tasks, const int32_t *__restrict__ tasks, const rgcsr_batch_desc *__restrict__ desc,
                    const V *__restrict__ val, const int32_t *__restrict__ col, const int64_t *__restrict__ gp,
                    const int32_t *__restrict__ rl, const float *__restrict__ scale,
                    const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y) {
    using A = typename VT<V>::A;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t t = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; t < n_tasks; t += warps) {
        const int m = tasks[2 * t];
        const int64_t first = tasks[2 * t + 1];
        const rgcsr_batch_desc d = desc[m];
        const int64_t lrow = first + lane;          // row within member m
        const bool valid = lrow < d.n_rows;
        int len = 0, stride = 0;
        int64_t ptr = 0;
        if (valid) {
            const int64_t g = lrow / d.group_size;
            const int64_t g0 = g * d.group_size;
            stride = (int)min((int64_t)d.group_size, d.n_rows - g0);
            ptr = d.val_off + __ldg(gp + d.group_off + g) + (lrow - g0);
            len = __ldg(rl + d.row_off + lrow);
        }
        const int j0 = split_point(len, valid);
        const A *xm = x + d.x_off;
        A acc = 0;
        const int jend = min(len, j0);
        for (int j = 0; j < jend; j += kUnroll) {
            A v[kUnroll];
            int c[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (j + u < jend) {
                    const int64_t p = ptr + (int64_t)(j + u) * stride;
                    v[u] = VT<V>::ld(val + p);
                    c[u] = __ldcs(col + p);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (j + u < jend) acc = fma(v[u], __ldg(xm + c[u]), acc);
        }
        unsigned long_rows = __ballot_sync(kFull, len > j0);
        while (long_rows) {
            const int r = __ffs(long_rows) - 1;
            long_rows &= long_rows - 1;
            const int Lr = __shfl_sync(kFull, len, r);
            const int sr = __shfl_sync(kFull, stride, r);
            const int64_t pr = shfl_i64(ptr, r);
            A part = 0;
            for (int j = j0 + lane; j < Lr; j += 32) {
                const int64_t p = pr + (int64_t)j * sr;
                part = fma(VT<V>::ld(val + p), __ldg(xm + __ldcs(col + p)), part);
            }
            part = warp_sum(part);
            if (lane == r) acc += part;
        }
        if (valid) {
            if constexpr (VT<V>::scaled) acc *= __ldg(scale + d.row_off + lrow);
            y[d.row_off + lrow] = acc;
        }
    }
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_batch_tasks(const rgcsr_batch_desc *desc, int32_t n_matrices, int32_t *tasks,
                                int64_t capacity, int64_t *n_tasks) {
    if (!desc || n_matrices < 0 || !n_tasks) return RGCSR_ERR_INVALID_ARG;
    int64_t k = 0;
    for (int32_t m = 0; m < n_matrices; ++m) {
        if (desc[m].n_rows < 0 || desc[m].group_size < 1) return RGCSR_ERR_INVALID_ARG;
        for (int64_t r = 0; r < desc[m].n_rows; r += 32) {
            if (tasks) {
                if (k >= capacity) return RGCSR_ERR_WORKSPACE;
                tasks[2 * k] = m;
                tasks[2 * k + 1] = (int32_t)r;
            }
            ++k;
        }
    }
    *n_tasks = k;
    return RGCSR_OK;
}

RGCSR_API int rgcsr_spmv_batched(const rgcsr_batch *B, const void *x, void *y, rgcsr_stream_t stream) {
    if (!B || B->n_tasks < 0) return RGCSR_ERR_INVALID_ARG;
    if (B->n_tasks == 0) return RGCSR_OK;
    if (!B->desc || !B->tasks || !B->group_ptr || !B->row_lengths || !x || !y) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t blocks = ceil_div(B->n_tasks, kThreads / 32);
    if (blocks > 152 * 8) blocks = 152 * 8;                 // persistent: 8 CTAs per SM
    const unsigned g = (unsigned)blocks;
    switch (B->value_type) {
        case RGCSR_F64:
            spmv_batched_kernel<double><<<g, kThreads, 0, s>>>(
                B->n_tasks, B->tasks, B->desc, static_cast<const double *>(B->values), B->columns, B->group_ptr,
                B->row_lengths, B->row_scale, static_cast<const double *>(x), static_cast<double *>(y));
            break;
        case RGCSR_F32:
            spmv_batched_kernel<float><<<g, kThreads, 0, s>>>(
                B->n_tasks, B->tasks, B->desc, static_cast<const float *>(B->values), B->columns, B->group_ptr,
                B->row_lengths, B->row_scale, static_cast<const float *>(x), static_cast<float *>(y));
            break;
        case RGCSR_BF16:
            if (!B->row_scale) return RGCSR_ERR_INVALID_ARG;
            spmv_batched_kernel<__nv_bfloat16><<<g, kThreads, 0, s>>>(
                B->n_tasks, B->tasks, B->desc, static_cast<const __nv_bfloat16 *>(B->values), B->columns,
                B->group_ptr, B->row_lengths, B->row_scale, static_cast<const float *>(x), static_cast<float *>(y));
            break;
        case RGCSR_F16:
            if (!B->row_scale) return RGCSR_ERR_INVALID_ARG;
            spmv_batched_kernel<__half><<<g, kThreads, 0, s>>>(
                B->n_tasks, B->tasks, B->desc, static_cast<const __half *>(B->values), B->columns,
                B->group_ptr, B->row_lengths, B->row_scale, static_cast<const float *>(x), static_cast<float *>(y));
            break;
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
    return launch_status();
}
