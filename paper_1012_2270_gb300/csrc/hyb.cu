// hyb.cu -- Hybrid ELLPACK + COO format (Sec. 3.3 of the paper), the
// comparison format of the paper's experiments.
//
// hyb_plan:    validate CSR, histogram of row lengths, ELL width K1 (given, or
//              by the byte-cost rule, evaluated on the host from the
//              histogram), nnz_coo = sum_i max(0, len_i - K1).
// hyb_convert: per-row COO offsets (exclusive scan), then one thread per row
//              writes its ELL slots (column-major, coalesced across rows) and
//              its COO overflow.
// hyb_spmv:    ELL kernel (thread per row, stops at the first padding slot,
//              writes y), then a COO kernel: each warp owns a tile of
//              32*kCooItems entries, forms products, runs a segmented
//              inclusive scan across lanes and adds every finished row
//              segment to y with one atomic add.
#include "common.cuh"

#include <vector>

namespace rgcsr {
namespace {

constexpr size_t kHybStatusBytes = 256;
constexpr int kCooItems = 8;
constexpr int kEllUnroll = 4;

struct HybStatus {
    int flags;
    int pad;
    int64_t max_len;
};

__global__ void length_histogram_kernel(RowPtr rp, int64_t n, unsigned long long *hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(hist + (rp[i + 1] - rp[i]), 1ull);
}

__global__ void coo_counts_kernel(RowPtr rp, int64_t n, int32_t K1, int64_t *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = max((int64_t)0, rp[i + 1] - rp[i] - K1);
}

template <typename V>
__global__ void hyb_fill_kernel(RowPtr rp, const int32_t *__restrict__ col, const V *__restrict__ val,
                                int64_t n, int32_t K1, const int64_t *__restrict__ coo_off,
                                V *__restrict__ ell_val, int32_t *__restrict__ ell_col,
                                int32_t *__restrict__ coo_row, int32_t *__restrict__ coo_col,
                                V *__restrict__ coo_val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = rp[i];
    const int64_t len = rp[i + 1] - a;
    for (int j = 0; j < K1; ++j) {
        const int64_t s = (int64_t)j * n + i;
        if (j < len) {
            ell_val[s] = val[a + j];
            ell_col[s] = col[a + j];
        } else {
            ell_val[s] = 0;
            ell_col[s] = -1;
        }
    }
    int64_t o = coo_off[i];
    for (int64_t j = K1; j < len; ++j, ++o) {
        coo_row[o] = (int32_t)i;
        coo_col[o] = col[a + j];
        coo_val[o] = val[a + j];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
hyb_ell_kernel(int64_t n, int32_t K1, const T *__restrict__ ev, const int32_t *__restrict__ ec,
               const T *__restrict__ x, T *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc = 0;
    for (int j = 0; j < K1; j += kEllUnroll) {
        int c[kEllUnroll];
        T v[kEllUnroll];
#pragma unroll
        for (int u = 0; u < kEllUnroll; ++u)
            c[u] = (j + u < K1) ? ld_stream(ec + (int64_t)(j + u) * n + i) : -1;
#pragma unroll
        for (int u = 0; u < kEllUnroll; ++u)
            if (c[u] >= 0) v[u] = ld_stream(ev + (int64_t)(j + u) * n + i);
#pragma unroll
        for (int u = 0; u < kEllUnroll; ++u)
            if (c[u] >= 0) acc = fma(v[u], ld_x(x + c[u]), acc);
        if (c[kEllUnroll - 1] < 0) break;      // rows are packed: padding ends the row
    }
    y[i] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256)
hyb_coo_kernel(int64_t nnz, const int32_t *__restrict__ cr, const int32_t *__restrict__ cc,
               const T *__restrict__ cv, const T *__restrict__ x, T *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t base = warp * (32 * kCooItems);
    if (base >= nnz) return;                  // warp-uniform
    int carry_row = -1;
    T carry = 0;
    for (int k = 0; k < kCooItems; ++k) {
        const int64_t idx = base + k * 32 + lane;
        int r = -1;
        T v = 0;
        if (idx < nnz) {
            r = ld_stream(cr + idx);
            v = ld_stream(cv + idx) * ld_x(x + ld_stream(cc + idx));
        }
        if (lane == 0) {
            if (r == carry_row) v += carry;
            else if (carry_row >= 0) atomicAdd(y + carry_row, carry);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ov = __shfl_up_sync(kFull, v, o);
            int orow = __shfl_up_sync(kFull, r, o);
            if (lane >= o && orow == r) v += ov;
        }
        const int next = __shfl_down_sync(kFull, r, 1);
        if (lane < 31 && r >= 0 && next != r) atomicAdd(y + r, v);
        carry_row = __shfl_sync(kFull, r, 31);
        carry = __shfl_sync(kFull, v, 31);
    }
    if (lane == 0 && carry_row >= 0) atomicAdd(y + carry_row, carry);
}

int check_hyb(const hyb_matrix *H) {
    if (!H || H->n_rows < 0 || H->n_cols < 0 || H->ell_width < 0 || H->nnz_coo < 0) return RGCSR_ERR_INVALID_ARG;
    if (!valid_value_type(H->value_type)) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (H->n_rows > 0 && H->ell_width > 0 && (!H->ell_val || !H->ell_col)) return RGCSR_ERR_INVALID_ARG;
    if (H->nnz_coo > 0 && (!H->coo_row || !H->coo_col || !H->coo_val)) return RGCSR_ERR_INVALID_ARG;
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t hyb_workspace_bytes(int64_t n_rows, int64_t n_cols) {
    if (n_rows < 0 || n_cols < 0) return 0;
    size_t hist = (size_t)(n_cols + 2) * sizeof(int64_t);
    size_t offs = align_up((size_t)(n_rows + 1) * sizeof(int64_t), 256) + scan_partials_bytes(n_rows);
    return kHybStatusBytes + align_up(hist > offs ? hist : offs, 256);
}

RGCSR_API int hyb_plan(const rgcsr_csr *A, int32_t ell_width, hyb_matrix *H, void *workspace,
                       size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (!H) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < hyb_workspace_bytes(A->n_rows, A->n_cols)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    auto *status = static_cast<HybStatus *>(workspace);
    auto *hist = reinterpret_cast<unsigned long long *>(static_cast<char *>(workspace) + kHybStatusBytes);
    RGCSR_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(HybStatus), s));
    if ((st = launch_validate_csr(A, &status->flags, &status->max_len, s)) != RGCSR_OK) return st;
    HybStatus hs;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.flags & 1) return RGCSR_ERR_BAD_ROWPTR;
    if (hs.flags & 2) return RGCSR_ERR_COL_OOB;
    const int64_t maxlen = hs.max_len;
    if (maxlen > A->n_cols + 1) return RGCSR_ERR_INVALID_ARG;   // duplicates beyond the hist bound

    // histogram of row lengths -> host
    std::vector<unsigned long long> h((size_t)maxlen + 1, 0);
    RGCSR_CUDA_TRY(cudaMemsetAsync(hist, 0, h.size() * sizeof(unsigned long long), s));
    if (A->n_rows > 0) {
        RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
        length_histogram_kernel<<<(unsigned)ceil_div(A->n_rows, 256), 256, 0, s>>>(rp, A->n_rows, hist);
        if ((st = launch_status()) != RGCSR_OK) return st;
    }
    RGCSR_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));

    // coo(K) = sum_{L > K} (L - K) h[L] for every K, by one backward pass:
    // coo(K) = coo(K+1) + #rows longer than K.
    std::vector<int64_t> coo((size_t)maxlen + 2, 0);
    int64_t longer = 0;
    for (int64_t K = maxlen; K >= 0; --K) {
        coo[(size_t)K] = coo[(size_t)K + 1] + longer;
        longer += (int64_t)h[(size_t)K];
    }
    int64_t K1 = ell_width;
    if (ell_width < 0) {
        const int64_t sv = (int64_t)value_bytes(A->value_type), si = 4;
        int64_t best = -1;
        K1 = 0;
        for (int64_t K = 0; K <= maxlen; ++K) {
            // exact in 128 bits: n*K*(sv+si) + 2*coo(K)*(sv+2si)
            __int128 c = (__int128)A->n_rows * K * (sv + si) + (__int128)2 * coo[(size_t)K] * (sv + 2 * si);
            if (best < 0 || c < (__int128)best) { best = (int64_t)c; K1 = K; }
        }
    }
    if (K1 > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    H->n_rows = A->n_rows;
    H->n_cols = A->n_cols;
    H->nnz = A->nnz;
    H->value_type = A->value_type;
    H->ell_width = (int32_t)K1;
    H->nnz_coo = K1 <= maxlen ? coo[(size_t)K1] : 0;
    H->max_row_len = maxlen;
    return RGCSR_OK;
}

RGCSR_API int hyb_convert(const rgcsr_csr *A, const hyb_matrix *H, void *workspace,
                          size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if ((st = check_hyb(H)) != RGCSR_OK) return st;
    if (H->n_rows != A->n_rows || H->value_type != A->value_type) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < hyb_workspace_bytes(A->n_rows, A->n_cols)) return RGCSR_ERR_WORKSPACE;
    if (A->n_rows == 0) return RGCSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    auto *offs = reinterpret_cast<int64_t *>(static_cast<char *>(workspace) + kHybStatusBytes);
    auto *partials = reinterpret_cast<int64_t *>(
        reinterpret_cast<char *>(offs) + align_up((size_t)(A->n_rows + 1) * sizeof(int64_t), 256));
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    const unsigned blocks = (unsigned)ceil_div(A->n_rows, 256);
    coo_counts_kernel<<<blocks, 256, 0, s>>>(rp, A->n_rows, H->ell_width, offs);
    if ((st = launch_status()) != RGCSR_OK) return st;
    if ((st = exclusive_scan_i64(offs, A->n_rows, partials, s)) != RGCSR_OK) return st;
    if (A->value_type == RGCSR_F64)
        hyb_fill_kernel<uint64_t><<<blocks, 256, 0, s>>>(
            rp, A->col_idx, static_cast<const uint64_t *>(A->values), A->n_rows, H->ell_width, offs,
            static_cast<uint64_t *>(H->ell_val), H->ell_col, H->coo_row, H->coo_col,
            static_cast<uint64_t *>(H->coo_val));
    else
        hyb_fill_kernel<uint32_t><<<blocks, 256, 0, s>>>(
            rp, A->col_idx, static_cast<const uint32_t *>(A->values), A->n_rows, H->ell_width, offs,
            static_cast<uint32_t *>(H->ell_val), H->ell_col, H->coo_row, H->coo_col,
            static_cast<uint32_t *>(H->coo_val));
    return launch_status();
}

template <typename T>
static int hyb_spmv_t(const hyb_matrix *H, const T *x, T *y, cudaStream_t s) {
    const unsigned blocks = (unsigned)ceil_div(H->n_rows, 256);
    hyb_ell_kernel<T><<<blocks, 256, 0, s>>>(H->n_rows, H->ell_width, static_cast<const T *>(H->ell_val),
                                             H->ell_col, x, y);
    int st = launch_status();
    if (st != RGCSR_OK || H->nnz_coo == 0) return st;
    const int64_t tiles = ceil_div(H->nnz_coo, 32 * kCooItems);
    const int64_t cblocks = ceil_div(tiles, 8);
    if (cblocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    hyb_coo_kernel<T><<<(unsigned)cblocks, 256, 0, s>>>(H->nnz_coo, H->coo_row, H->coo_col,
                                                       static_cast<const T *>(H->coo_val), x, y);
    return launch_status();
}

RGCSR_API int hyb_spmv(const hyb_matrix *H, const void *x, void *y, rgcsr_stream_t stream) {
    int st = check_hyb(H);
    if (st != RGCSR_OK) return st;
    if (H->n_rows == 0) return RGCSR_OK;
    if (!y || (H->n_cols > 0 && !x)) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (H->value_type == RGCSR_F64)
        return hyb_spmv_t<double>(H, static_cast<const double *>(x), static_cast<double *>(y), s);
    return hyb_spmv_t<float>(H, static_cast<const float *>(x), static_cast<float *>(y), s);
}
