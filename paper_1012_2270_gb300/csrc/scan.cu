// scan.cu -- device-wide exclusive prefix sum of int64 counts and CSR
// validation, used by the RgCSR and HYB conversions.
#include "common.cuh"

namespace rgcsr {
namespace {

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nwarps ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nwarps) warp_sums[lane] = wi - w;     // exclusive warp offsets
        if (lane == 31) warp_sums[32] = wi;               // block total
    }
    __syncthreads();
    int64_t r = warp_sums[warp] + inc - v;
    total = warp_sums[32];
    __syncthreads();
    return r;
}

// Tile b covers scan positions [b*kScanTile, (b+1)*kScanTile) of the count+1
// positions; position `count` contributes 0.
__global__ void __launch_bounds__(kScanThreads)
scan_tile_sums(const int64_t *__restrict__ data, int64_t count, int64_t *__restrict__ partials) {
    __shared__ int64_t ws[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < count) s += data[i];
    }
    int64_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024)
scan_partials_kernel(int64_t *partials, int64_t ntiles) {
    __shared__ int64_t ws[33];
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? partials[i] : 0;
        int64_t total;
        int64_t ex = block_exclusive_scan(v, ws, total);
        if (i < ntiles) partials[i] = carry + ex;
        carry += total;
    }
}

// Each thread owns kScanItems consecutive positions of the tile.
__global__ void __launch_bounds__(kScanThreads)
scan_tiles(int64_t *__restrict__ data, int64_t count, const int64_t *__restrict__ partials) {
    __shared__ int64_t ws[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < count ? data[i] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, ws, total) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i <= count) data[i] = run;
        run += v[k];
    }
}

__global__ void validate_rows_kernel(RowPtr rp, int64_t n, int64_t nnz, int *flags,
                                     unsigned long long *max_len) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int len = 0;
    if (i < n) {
        int64_t a = rp[i], b = rp[i + 1];
        bool bad = (b < a) || (b - a > (int64_t)INT32_MAX) || (i == 0 && a != 0) || (i == n - 1 && b != nnz);
        if (bad) atomicOr(flags, 1);
        else len = (int)(b - a);
    }
    len = warp_max_i(len);
    if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(max_len, (unsigned long long)len);
}

__global__ void validate_cols_kernel(const int32_t *__restrict__ col, int64_t nnz, int64_t n_cols, int *flags) {
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        int c = col[p];
        bad |= (c < 0) || (c >= n_cols);
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, 2);
}

// rl[k] = length of CSR row perm[k] (row k without perm).
__global__ void row_lengths_kernel(RowPtr rp, int64_t n, const int32_t *__restrict__ perm, int32_t *rl) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm ? perm[k] : k;
    // an out-of-range entry is flagged by check_perm_kernel; never read past row_ptr
    rl[k] = (i >= 0 && i < n) ? (int32_t)(rp[i + 1] - rp[i]) : 0;
}

// perm is a permutation of [0, n) iff every entry is in range and no row is
// hit twice; seen[] (n counters, zeroed) counts the hits.
__global__ void check_perm_kernel(const int32_t *__restrict__ perm, int64_t n, int32_t *seen, int *flags) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t i = perm[k];
    if (i < 0 || (int64_t)i >= n || atomicAdd(seen + i, 1) != 0) atomicOr(flags, 4);
}

}  // namespace

int exclusive_scan_i64(int64_t *data, int64_t count, int64_t *partials, cudaStream_t s) {
    const int64_t ntiles = ceil_div(count + 1, kScanTile);
    if (ntiles > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, s>>>(data, count, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, ntiles);
    scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(data, count, partials);
    return launch_status();
}

int launch_validate_csr(const rgcsr_csr *A, int *flags, int64_t *max_len, cudaStream_t s) {
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    if (A->n_rows > 0) {
        validate_rows_kernel<<<(unsigned)ceil_div(A->n_rows, 256), 256, 0, s>>>(
            rp, A->n_rows, A->nnz, flags, reinterpret_cast<unsigned long long *>(max_len));
    }
    if (A->nnz > 0) {
        int64_t blocks = ceil_div(A->nnz, 256);
        if (blocks > 152 * 32) blocks = 152 * 32;
        validate_cols_kernel<<<(unsigned)blocks, 256, 0, s>>>(A->col_idx, A->nnz, A->n_cols, flags);
    }
    return launch_status();
}

int launch_row_lengths(const rgcsr_csr *A, const int32_t *perm, int32_t *row_lengths, cudaStream_t s) {
    if (A->n_rows == 0) return RGCSR_OK;
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    row_lengths_kernel<<<(unsigned)ceil_div(A->n_rows, 256), 256, 0, s>>>(rp, A->n_rows, perm, row_lengths);
    return launch_status();
}

int launch_check_perm(const int32_t *perm, int64_t n, int32_t *seen, int *flags, cudaStream_t s) {
    if (n == 0) return RGCSR_OK;
    RGCSR_CUDA_TRY(cudaMemsetAsync(seen, 0, (size_t)n * sizeof(int32_t), s));
    check_perm_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(perm, n, seen, flags);
    return launch_status();
}

}  // namespace rgcsr
