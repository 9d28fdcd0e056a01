// hyb_spmm.cu -- Y = A X for the Hybrid ELL + COO format (Sec. 3.3 of the
// paper; several right-hand sides are an extension, as for RgCSR).
//
// ELL step: one thread per row over its K1 column-major slots (coalesced
// across rows), KC <= 8 columns of X per pass; it writes Y.  COO step: one
// warp per run of entries (row-sorted), lane q owning column q of a chunk of
// up to 32 columns; each entry's row, column and value are read by the
// whole warp (one broadcast load each) and its X row piece is one coalesced
// load; a row's sum goes to Y with one atomic add per column when the row
// changes or the run ends.
#include "common.cuh"

namespace rgcsr {
namespace {

constexpr int kCooRun = 256;           // COO entries per warp

template <typename T, int KC, bool VEC>
__global__ void __launch_bounds__(256)
hyb_ell_spmm_kernel(int64_t n, int32_t K1, const T *__restrict__ ev, const int32_t *__restrict__ ec,
                    const T *__restrict__ X, int64_t ldx, T *__restrict__ Y, int64_t ldy) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[KC];
#pragma unroll
    for (int w = 0; w < KC; ++w) acc[w] = 0;
    for (int j = 0; j < K1; ++j) {
        const int c = ld_stream(ec + (int64_t)j * n + i);
        if (c < 0) break;                          // rows are packed: padding ends the row
        const T v = ld_stream(ev + (int64_t)j * n + i);
        T xw[KC];
        load_xrow<T, KC, VEC>(X + (int64_t)c * ldx, xw);
#pragma unroll
        for (int w = 0; w < KC; ++w) acc[w] = fma(v, xw[w], acc[w]);
    }
#pragma unroll
    for (int w = 0; w < KC; ++w) Y[i * ldy + w] = acc[w];
}

template <typename T>
__global__ void __launch_bounds__(256)
hyb_coo_spmm_kernel(int64_t nnz, int kc, const int32_t *__restrict__ cr, const int32_t *__restrict__ cc,
                    const T *__restrict__ cv, const T *__restrict__ X, int64_t ldx, T *__restrict__ Y,
                    int64_t ldy) {
    const int q = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t e0 = warp * kCooRun;
    if (e0 >= nnz) return;                         // warp-uniform
    const int64_t e1 = min(e0 + kCooRun, nnz);
    const bool on = q < kc;
    T acc = 0;
    int row = __ldg(cr + e0);
    for (int64_t e = e0; e < e1; ++e) {
        const int r = __ldg(cr + e);
        if (r != row) {
            if (on) atomicAdd(Y + (int64_t)row * ldy + q, acc);
            acc = 0;
            row = r;
        }
        const T v = __ldg(cv + e);
        const int c = __ldg(cc + e);
        if (on) acc = fma(v, __ldg(X + (int64_t)c * ldx + q), acc);
    }
    if (on) atomicAdd(Y + (int64_t)row * ldy + q, acc);
}

template <typename T, int KC, bool VEC>
int launch_ell_spmm(const hyb_matrix *H, const T *X, int64_t ldx, T *Y, int64_t ldy, cudaStream_t s) {
    const int64_t blocks = ceil_div(H->n_rows, 256);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    hyb_ell_spmm_kernel<T, KC, VEC><<<(unsigned)blocks, 256, 0, s>>>(
        H->n_rows, H->ell_width, static_cast<const T *>(H->ell_val), H->ell_col, X, ldx, Y, ldy);
    return launch_status();
}

template <typename T>
int hyb_spmm_t(const hyb_matrix *H, int k, const T *X, int64_t ldx, T *Y, int64_t ldy, cudaStream_t s) {
    const bool vec = ((uintptr_t)X & 15) == 0 && (ldx * (int64_t)sizeof(T)) % 16 == 0;
    int st;
    // ELL: writes every row of Y (K1 = 0 writes zeros)
    for (int c0 = 0; c0 < k;) {
        const int left = k - c0;
        int w;
        if (left >= 8) {
            st = vec ? launch_ell_spmm<T, 8, true>(H, X + c0, ldx, Y + c0, ldy, s)
                     : launch_ell_spmm<T, 8, false>(H, X + c0, ldx, Y + c0, ldy, s);
            w = 8;
        } else if (left >= 4) {
            st = vec ? launch_ell_spmm<T, 4, true>(H, X + c0, ldx, Y + c0, ldy, s)
                     : launch_ell_spmm<T, 4, false>(H, X + c0, ldx, Y + c0, ldy, s);
            w = 4;
        } else {
            st = launch_ell_spmm<T, 1, false>(H, X + c0, ldx, Y + c0, ldy, s);
            w = 1;
        }
        if (st != RGCSR_OK) return st;
        c0 += w;
    }
    if (H->nnz_coo == 0) return RGCSR_OK;
    // COO: adds the overflow, up to 32 columns per pass
    const int64_t warps = ceil_div(H->nnz_coo, (int64_t)kCooRun);
    const int64_t blocks = ceil_div(warps, (int64_t)8);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    for (int c0 = 0; c0 < k; c0 += 32) {
        const int kc = k - c0 < 32 ? k - c0 : 32;
        hyb_coo_spmm_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(
            H->nnz_coo, kc, H->coo_row, H->coo_col, static_cast<const T *>(H->coo_val), X + c0, ldx, Y + c0, ldy);
        if ((st = launch_status()) != RGCSR_OK) return st;
    }
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int hyb_spmm(const hyb_matrix *H, int32_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       rgcsr_stream_t stream) {
    if (!H || H->n_rows < 0 || H->n_cols < 0 || H->ell_width < 0 || H->nnz_coo < 0 || k < 0)
        return RGCSR_ERR_INVALID_ARG;
    if (H->value_type != RGCSR_F64 && H->value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (H->n_rows == 0 || k == 0) return RGCSR_OK;
    if (ldx < k || ldy < k || !Y || (H->n_cols > 0 && !X)) return RGCSR_ERR_INVALID_ARG;
    if (H->ell_width > 0 && (!H->ell_val || !H->ell_col)) return RGCSR_ERR_INVALID_ARG;
    if (H->nnz_coo > 0 && (!H->coo_row || !H->coo_col || !H->coo_val)) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (H->value_type == RGCSR_F64)
        return hyb_spmm_t<double>(H, k, static_cast<const double *>(X), ldx, static_cast<double *>(Y), ldy, s);
    return hyb_spmm_t<float>(H, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy, s);
}
