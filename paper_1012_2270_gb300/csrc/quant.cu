// quant.cu -- reduced-precision value storage for RgCSR (not in the paper,
// which stores single or double precision values).
//
// Per row i:  s_i = 2^ceil(log2 max_j |a_ij|)  (1 for an empty or all-zero row;
// exponent kept in the binary32 normal range [-126, 127]), stored as float;
// q_ij = round-to-nearest-even of the exact quotient a_ij / s_i (exact because
// s_i is a power of two) in bfloat16 or binary16, subnormals kept.  The SpMV
// then computes y_i = s_i * sum_j q_ij x_j in float (spmv.cu).
//
// rgcsr_quantize reads an F64/F32 RgCSR matrix and writes the quantised
// values into another descriptor that shares its columns, group pointers and
// row lengths.  Padding slots become +0.
#include "common.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace rgcsr {
namespace {

// Binary exponent e of the power of two 2^e = 2^ceil(log2 m) for m > 0,
// read from the IEEE-754 bit fields of m, clamped to [-126, 127].
__device__ __forceinline__ int ceil_log2_exponent(double m) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(m);
    const int biased = (int)((b >> 52) & 0x7ff);
    const unsigned long long frac = b & ((1ull << 52) - 1);
    int e;
    if (biased == 0) e = -1022;                      // subnormal: far below the clamp
    else e = (biased - 1023) + (frac != 0 ? 1 : 0);  // m = 1.f * 2^(biased-1023)
    return max(-126, min(127, e));
}

// One thread per row: largest magnitude over the row's slots, then scale.
template <typename S>
__global__ void row_scale_kernel(int64_t n, int32_t G, const S *__restrict__ val,
                                 const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                                 float *__restrict__ scale) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int64_t g = row / G;
    const int64_t first = g * G;
    const int stride = (int)min((int64_t)G, n - first);
    int64_t p = gp[g] + (row - first);
    const int len = rl[row];
    double mx = 0.0;
    for (int j = 0; j < len; ++j, p += stride) mx = fmax(mx, fabs((double)val[p]));
    // a power of two in the normal range, built from its exponent field
    scale[row] = mx > 0.0 ? __int_as_float((ceil_log2_exponent(mx) + 127) << 23) : 1.0f;
}

template <typename Q> __device__ __forceinline__ Q to_q(double v);
template <> __device__ __forceinline__ __nv_bfloat16 to_q<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __half to_q<__half>(double v) { return __double2half(v); }

// One warp per group streams the group's slab: slot e = (j, t) -> row t.
template <typename S, typename Q>
__global__ void __launch_bounds__(256)
quantize_kernel(int64_t n, int32_t G, int64_t n_groups, const S *__restrict__ val,
                const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                const float *__restrict__ scale, uint16_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const int64_t base = gp[g];
        const int64_t size = gp[g + 1] - base;
        int64_t j = lane / R;
        int t = lane % R;
        for (int64_t e = lane; e < size; e += 32) {
            const int64_t row = first + t;
            uint16_t bits = 0;
            if (j < rl[row]) {
                const double q = (double)val[base + e] / (double)scale[row];   // exact
                const Q h = to_q<Q>(q);
                bits = *reinterpret_cast<const uint16_t *>(&h);
            }
            out[base + e] = bits;
            t += 32;
            while (t >= R) { t -= R; ++j; }
        }
    }
}

template <typename S>
int quantize_t(const rgcsr_matrix *src, rgcsr_matrix *dst, cudaStream_t s) {
    const S *val = static_cast<const S *>(src->values);
    row_scale_kernel<S><<<(unsigned)ceil_div(src->n_rows, 256), 256, 0, s>>>(
        src->n_rows, src->group_size, val, src->group_ptr, src->row_lengths, dst->row_scale);
    int st = launch_status();
    if (st != RGCSR_OK || src->n_stored == 0) return st;
    int64_t blocks = ceil_div(src->n_groups, 8);
    if (blocks > 152 * 64) blocks = 152 * 64;
    uint16_t *out = static_cast<uint16_t *>(dst->values);
    if (dst->value_type == RGCSR_BF16)
        quantize_kernel<S, __nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(
            src->n_rows, src->group_size, src->n_groups, val, src->group_ptr, src->row_lengths,
            dst->row_scale, out);
    else
        quantize_kernel<S, __half><<<(unsigned)blocks, 256, 0, s>>>(
            src->n_rows, src->group_size, src->n_groups, val, src->group_ptr, src->row_lengths,
            dst->row_scale, out);
    return launch_status();
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_quantize(const rgcsr_matrix *src, rgcsr_matrix *dst, rgcsr_stream_t stream) {
    if (!src || !dst || src->group_size < 1 || src->n_rows < 0) return RGCSR_ERR_INVALID_ARG;
    if (src->value_type != RGCSR_F64 && src->value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (dst->value_type != RGCSR_BF16 && dst->value_type != RGCSR_F16) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    dst->n_rows = src->n_rows;
    dst->n_cols = src->n_cols;
    dst->nnz = src->nnz;
    dst->group_size = src->group_size;
    dst->n_groups = src->n_groups;
    dst->n_stored = src->n_stored;
    dst->max_row_len = src->max_row_len;
    dst->row_perm = src->row_perm;        // the slabs keep src's stored row order
    if (src->n_rows == 0) return RGCSR_OK;
    if (!src->group_ptr || !src->row_lengths || !dst->row_scale) return RGCSR_ERR_INVALID_ARG;
    if (src->n_stored > 0 && (!src->values || !dst->values)) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (src->value_type == RGCSR_F64) return quantize_t<double>(src, dst, s);
    return quantize_t<float>(src, dst, s);
}
