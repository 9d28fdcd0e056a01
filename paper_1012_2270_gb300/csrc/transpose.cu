// transpose.cu -- structure operations for the backward pass of y = A x:
//   * a stable LSD radix sort of (key, index) pairs, 8-bit digits;
//   * rgcsr_csr_transpose: CSR of A^T, its entries in increasing original
//     row (stable by construction), with the permutation to A's entries;
//   * rgcsr_csr_row_index: the row of every stored entry;
//   * rgcsr_gather_values / rgcsr_compose_index: refresh an RgCSR matrix's
//     values from CSR-ordered values through a slot -> source index map;
//   * rgcsr_sampled_dot: out[p] = sum_b G[row_p, b] X[col_p, b], the gradient
//     of sum(G .* (A X)) with respect to every stored value;
//   * rgcsr_descending_order: the rows sorted by length, longest first
//     (stable), the row order of Sec. 4.4.2 / Table 7 (the same radix sort).
// None of this is in the paper (which has no backward pass); the transposed
// matrix is an ordinary RgCSR matrix built with rgcsr_plan / rgcsr_convert.
#include "common.cuh"

#include <algorithm>

namespace rgcsr {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;   // items per tile
constexpr int kDigits = 256;
static_assert(kSortThreads == kDigits, "the scatter's prefix step uses one thread per digit");

// Per-tile digit histogram -> counts[d * n_tiles + tile].
__global__ void __launch_bounds__(kSortThreads)
radix_histogram(const uint32_t *__restrict__ keys, int64_t n, int shift, int64_t n_tiles,
                int64_t *__restrict__ counts) {
    __shared__ int hist[kDigits];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter.  Items of a tile are taken in index order, 256 per round;
// an item's destination is the digit's global offset for this tile, plus the
// items of that digit in earlier rounds, earlier warps, and earlier lanes.
// vals_in == nullptr means "the item's own index".
__global__ void __launch_bounds__(kSortThreads)
radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
              uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n, int shift,
              int64_t n_tiles, const int64_t *__restrict__ offsets) {
    __shared__ int wcnt[kSortThreads / 32][kDigits];
    __shared__ int run[kDigits];
    __shared__ int64_t base_off[kDigits];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = 0;
    base_off[tid] = offsets[(int64_t)tid * n_tiles + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
        for (int q = 0; q < kDigits / 32; ++q) wcnt[w][lane + 32 * q] = 0;
        __syncthreads();
        const int64_t i = base + r * kSortThreads + tid;
        const bool valid = i < n;
        const uint32_t key = valid ? keys_in[i] : 0u;
        const uint32_t val = valid ? (vals_in ? vals_in[i] : (uint32_t)i) : 0u;
        const int digit = (int)((key >> shift) & 0xff);
        const unsigned peers = __match_any_sync(kFull, valid ? digit : kDigits + lane);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][digit] = __popc(peers);
        __syncthreads();
        {   // exclusive prefix of digit tid over warps, continuing earlier rounds
            int s = run[tid];
#pragma unroll
            for (int ww = 0; ww < kSortThreads / 32; ++ww) {
                const int c = wcnt[ww][tid];
                wcnt[ww][tid] = s;
                s += c;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = base_off[digit] + wcnt[w][digit] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

struct SortBuffers {
    uint32_t *k0, *v0, *k1, *v1;
    int64_t *counts, *partials;
};

size_t sort_workspace_bytes(int64_t n) {
    const int64_t n_tiles = ceil_div(n > 0 ? n : 1, kSortTile);
    return 4 * align_up((size_t)n * 4, 256) + align_up((size_t)(kDigits * n_tiles + 1) * 8, 256) +
           scan_partials_bytes(kDigits * n_tiles);
}

SortBuffers carve_sort(void *ws, int64_t n) {
    const int64_t n_tiles = ceil_div(n > 0 ? n : 1, kSortTile);
    char *p = static_cast<char *>(ws);
    SortBuffers b;
    const size_t a = align_up((size_t)n * 4, 256);
    b.k0 = reinterpret_cast<uint32_t *>(p); p += a;
    b.v0 = reinterpret_cast<uint32_t *>(p); p += a;
    b.k1 = reinterpret_cast<uint32_t *>(p); p += a;
    b.v1 = reinterpret_cast<uint32_t *>(p); p += a;
    b.counts = reinterpret_cast<int64_t *>(p); p += align_up((size_t)(kDigits * n_tiles + 1) * 8, 256);
    b.partials = reinterpret_cast<int64_t *>(p);
    return b;
}

// Stable sort of keys (all < 2^key_bits) with their indices.  Result in
// (*keys_out, *idx_out), pointing into the buffers.
int radix_sort_indices(const uint32_t *keys, int64_t n, int key_bits, SortBuffers &b,
                       const uint32_t **keys_out, const uint32_t **idx_out, cudaStream_t s) {
    const int64_t n_tiles = ceil_div(n, kSortTile);
    if (n_tiles > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    const uint32_t *kin = keys, *vin = nullptr;
    uint32_t *kout = b.k0, *vout = b.v0;
    const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        radix_histogram<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, n, shift, n_tiles, b.counts);
        int st = exclusive_scan_i64(b.counts, kDigits * n_tiles, b.partials, s);
        if (st != RGCSR_OK) return st;
        radix_scatter<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, n_tiles,
                                                                 b.counts);
        if ((st = launch_status()) != RGCSR_OK) return st;
        kin = kout;
        vin = vout;
        if (kout == b.k0) { kout = b.k1; vout = b.v1; } else { kout = b.k0; vout = b.v0; }
    }
    *keys_out = kin;
    *idx_out = vin;
    return RGCSR_OK;
}

// One warp per row writes the row's index into its entries.
__global__ void row_index_kernel(RowPtr rp, int64_t n, int32_t *__restrict__ row_index) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t a = rp[i], e = rp[i + 1];
        for (int64_t p = a + lane; p < e; p += 32) row_index[p] = (int32_t)i;
    }
}

__global__ void column_counts_kernel(const int32_t *__restrict__ col, int64_t nnz,
                                     unsigned long long *__restrict__ cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[p], 1ull);
}

template <typename V>
__global__ void transpose_fill_kernel(const uint32_t *__restrict__ idx, int64_t nnz,
                                      const int32_t *__restrict__ row_index, int32_t *__restrict__ t_col,
                                      int64_t *__restrict__ perm, const V *__restrict__ val,
                                      V *__restrict__ t_val) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    const uint32_t p = idx[q];
    t_col[q] = row_index[p];
    if (perm) perm[q] = p;
    if (t_val) t_val[q] = val[p];
}

template <typename V>
__global__ void gather_kernel(const V *__restrict__ src, const int64_t *__restrict__ index, int64_t n,
                              V *__restrict__ dst) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = index[s];
        dst[s] = i >= 0 ? src[i] : V(0);
    }
}

// Only when the values changed: flags is the state record's word 1, whose
// bit 1 the hash kernel sets when the hash differs from the held one.
template <typename V>
__global__ void gather_if_kernel(const V *__restrict__ src, const int64_t *__restrict__ index, int64_t n,
                                 V *__restrict__ dst, const unsigned long long *__restrict__ flags) {
    if (!(*flags & 2ull)) return;
    constexpr int U = 4;                         // slots a thread has in flight
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
#pragma unroll 1
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s0 < n; s0 += U * S) {
        int64_t i[U];
#pragma unroll
        for (int u = 0; u < U; ++u) i[u] = s0 + u * S < n ? __ldcs(index + s0 + u * S) : -1;
        V w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = i[u] >= 0 ? __ldg(src + i[u]) : V(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (s0 + u * S < n) dst[s0 + u * S] = w[u];
    }
}

// Hash of n values of ES bytes (2, 4 or 8): one 64-bit sum over the 8-byte
// words w_j of their bytes (little-endian; the last word zero-filled past
// the end):
//     h = sum_j mix(w_j ^ ((j + 1) K))   (mod 2^64),   K = 0x9E3779B97F4A7C15
// with mix the SplitMix64 finalizer (Steele, Lea and Flood 2014; constants
// as published), a bijection of 64-bit words, so changing any one value
// always changes h; changes of several values leave h unchanged only by
// chance (about 2^-64), since each word goes through its own mix: a common
// change of bits (every value negated or scaled by one factor) reaches the
// sum as unrelated 64-bit terms.  (Combining a block's words linearly
// before one mix is cheaper but not safe: negating four FP64 values flips
// bit 63 of four words, and four multiples of 2^63 cancel.)  The sum is
// exact modular arithmetic, so it does not depend on the order of the
// additions.  The last block to finish (a ticket after a fence) adds the
// block sums and updates the state record: word 0 the hash, word 1 bit 0
// "holds values", bit 1 "changed by this call".
constexpr int kHashParts = 1216;         // 8 blocks per SM
constexpr int kHashThreads = 256;
constexpr unsigned long long kHashK = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int o) {
    const unsigned lo = __shfl_xor_sync(kFull, (unsigned)v, o), hi = __shfl_xor_sync(kFull, (unsigned)(v >> 32), o);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u64(v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < kHashThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Word j of the byte stream, assembled from its values (each loaded at its
// own alignment); 0 past the end.
template <int ES>
__device__ __forceinline__ unsigned long long hash_word(const void *v, int64_t n, int64_t j) {
    constexpr int PER = 8 / ES;
    unsigned long long w = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int64_t i = j * PER + e;
        if (i < n) {
            unsigned long long b;
            if constexpr (ES == 8) b = static_cast<const unsigned long long *>(v)[i];
            else if constexpr (ES == 4) b = static_cast<const unsigned *>(v)[i];
            else b = static_cast<const unsigned short *>(v)[i];
            w |= b << (8 * ES * e);
        }
    }
    return w;
}

// The terms of the four words of 32-byte block q, k = (4q + 1) K the salt of
// its first word.
__device__ __forceinline__ unsigned long long block_term(unsigned long long w0, unsigned long long w1,
                                                         unsigned long long w2, unsigned long long w3,
                                                         unsigned long long k) {
    return mix64(w0 ^ k) + mix64(w1 ^ (k + kHashK)) + mix64(w2 ^ (k + 2 * kHashK)) + mix64(w3 ^ (k + 3 * kHashK));
}

__device__ __forceinline__ unsigned long long block_term(const uint4 &a, const uint4 &b, unsigned long long k) {
    return block_term(((unsigned long long)a.y << 32) | a.x, ((unsigned long long)a.w << 32) | a.z,
                      ((unsigned long long)b.y << 32) | b.x, ((unsigned long long)b.w << 32) | b.z, k);
}

// Each thread takes one 32-byte block (two 16-byte loads, four words) per
// step of a grid-stride loop, on a full-occupancy grid (8 CTAs per SM, at
// most 32 registers): the many warps of an SM, not deep unrolling, keep the
// reads in flight while others mix.  Then the blocks past the last whole one;
// with a base that is not 16-byte aligned every block is assembled from
// its values.
template <int ES>
__global__ void __launch_bounds__(kHashThreads, 8)
values_hash_kernel(const void *__restrict__ v, int64_t n, unsigned long long *__restrict__ state) {
    __shared__ unsigned long long sh[kHashThreads / 32];
    __shared__ bool last;
    unsigned long long h = 0;
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t bytes = n * ES, blocks = (bytes + 31) / 32;
    const int64_t nq = ((uintptr_t)v & 15) == 0 ? bytes / 32 : 0;
    const uint4 *pv = static_cast<const uint4 *>(v);
    const unsigned long long kS = 4ull * (unsigned long long)S * kHashK;       // salt step of S blocks
    unsigned long long k = (4ull * (unsigned long long)tid + 1) * kHashK;       // salt of block tid's word 0
#pragma unroll 1
    for (int64_t q = tid; q < nq; q += S, k += kS) {
        const uint4 a = __ldcs(pv + 2 * q), b = __ldcs(pv + 2 * q + 1);
        h += block_term(a, b, k);
    }
    for (int64_t q = nq + tid; q < blocks; q += S)
        h += block_term(hash_word<ES>(v, n, 4 * q), hash_word<ES>(v, n, 4 * q + 1), hash_word<ES>(v, n, 4 * q + 2),
                        hash_word<ES>(v, n, 4 * q + 3), (4ull * (unsigned long long)q + 1) * kHashK);
    h = block_sum_u64(h, sh);
    unsigned long long *part = state + 8;               // [kHashParts] block sums
    unsigned *ticket = reinterpret_cast<unsigned *>(state + 2);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = h;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned long long t = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(part + b);
    t = block_sum_u64(t, sh);
    if (threadIdx.x != 0) return;
    const bool held = (state[1] & 1ull) != 0;
    const bool changed = !held || state[0] != t;
    state[0] = t;
    state[1] = 1ull | (changed ? 2ull : 0ull);
    *ticket = 0u;
}

__global__ void compose_kernel(const int64_t *__restrict__ outer, const int64_t *__restrict__ inner,
                               int64_t n, int64_t *__restrict__ out) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = outer[s];
        out[s] = i >= 0 ? inner[i] : -1;
    }
}

// out[p] = sum_b G[row_p, b] * X[col_p, b], b ascending.
template <typename T>
__global__ void sampled_dot_kernel(int64_t nnz, int k, const int32_t *__restrict__ row_index,
                                   const int32_t *__restrict__ col, const T *__restrict__ G, int64_t ldg,
                                   const T *__restrict__ X, int64_t ldx, T *__restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const T *g = G + (int64_t)row_index[p] * ldg;
        const T *x = X + (int64_t)col[p] * ldx;
        T s = 0;
        for (int b = 0; b < k; ++b) s = fma(__ldg(g + b), __ldg(x + b), s);
        out[p] = s;
    }
}

// The same for k == KC with 16-byte aligned rows of G and X: each row is
// read with KC * sizeof(T) / 16 vector loads (load_xrow), and the products
// are added in increasing b as above.
template <typename T, int KC>
__global__ void sampled_dot_vec_kernel(int64_t nnz, const int32_t *__restrict__ row_index,
                                       const int32_t *__restrict__ col, const T *__restrict__ G, int64_t ldg,
                                       const T *__restrict__ X, int64_t ldx, T *__restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        T g[KC], x[KC];
        load_xrow<T, KC, true>(G + (int64_t)row_index[p] * ldg, g);
        load_xrow<T, KC, true>(X + (int64_t)col[p] * ldx, x);
        T s = 0;
#pragma unroll
        for (int b = 0; b < KC; ++b) s = fma(g[b], x[b], s);
        out[p] = s;
    }
}

// Sort key of stored position k for the descending order: larger rows get
// smaller keys; lengths are clamped to [0, mask] so that any row_ptr gives
// keys within the sorted bits.
__global__ void descending_keys_kernel(RowPtr rp, int64_t n, uint32_t mask, uint32_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t len = rp[i + 1] - rp[i];
    len = len < 0 ? 0 : (len > (int64_t)mask ? (int64_t)mask : len);
    keys[i] = mask - (uint32_t)len;
}

// dval[slot_to_csr[e]] = sum_b G[row(e), b] X[col[e], b] over a group's slab
// (one warp per group, slab elements e = (slot j, row t) as in the layout).
template <typename T>
__global__ void bwd_values_kernel(int64_t n, int32_t G, int64_t n_groups, const int64_t *__restrict__ gp,
                                  const int32_t *__restrict__ col, const int64_t *__restrict__ s2c,
                                  const int32_t *__restrict__ perm, int k, const T *__restrict__ Gy, int64_t ldg,
                                  const T *__restrict__ X, int64_t ldx, T *__restrict__ dval) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const int64_t base = gp[g];
        const int64_t size = gp[g + 1] - base;
        for (int64_t e = lane; e < size; e += 32) {
            const int64_t p = s2c[base + e];
            if (p < 0) continue;                              // padding
            const int64_t row = first + (int)(e % R);
            const T *gr = Gy + out_row(perm, row) * ldg;
            const T *xr = X + (int64_t)col[base + e] * ldx;
            T acc = 0;
            for (int b = 0; b < k; ++b) acc = fma(__ldg(gr + b), __ldg(xr + b), acc);
            dval[p] = acc;
        }
    }
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = ceil_div(n, threads);
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b > 0 ? b : 1);
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t rgcsr_transpose_workspace_bytes(int64_t nnz, int64_t n_rows, int64_t n_cols) {
    if (nnz < 0 || n_rows < 0 || n_cols < 0) return 0;
    return sort_workspace_bytes(nnz) + align_up((size_t)nnz * 4, 256) + scan_partials_bytes(n_cols) + 256;
}

RGCSR_API int rgcsr_csr_row_index(const rgcsr_csr *A, int32_t *row_index, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (A->nnz == 0 || A->n_rows == 0) return RGCSR_OK;
    if (!row_index) return RGCSR_ERR_INVALID_ARG;
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    row_index_kernel<<<grid_for(A->n_rows * 32, 256), 256, 0, (cudaStream_t)stream>>>(rp, A->n_rows, row_index);
    return launch_status();
}

RGCSR_API int rgcsr_csr_transpose(const rgcsr_csr *A, int64_t *t_row_ptr, int32_t *t_col_idx,
                                  int64_t *perm, void *t_values, void *workspace, size_t workspace_bytes,
                                  rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (A->nnz >= (int64_t)UINT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    if (!t_row_ptr || (A->nnz > 0 && !t_col_idx)) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_transpose_workspace_bytes(A->nnz, A->n_rows, A->n_cols))
        return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nnz = A->nnz;
    SortBuffers b = carve_sort(workspace, nnz);
    char *after = static_cast<char *>(workspace) + sort_workspace_bytes(nnz);
    int32_t *row_index = reinterpret_cast<int32_t *>(after);
    int64_t *tpart = reinterpret_cast<int64_t *>(after + align_up((size_t)nnz * 4, 256));

    // column counts -> t_row_ptr (exclusive scan, last = nnz)
    RGCSR_CUDA_TRY(cudaMemsetAsync(t_row_ptr, 0, (size_t)(A->n_cols + 1) * sizeof(int64_t), s));
    if (nnz > 0) {
        column_counts_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(A->col_idx, nnz,
                                                                reinterpret_cast<unsigned long long *>(t_row_ptr));
        if ((st = launch_status()) != RGCSR_OK) return st;
    }
    if ((st = exclusive_scan_i64(t_row_ptr, A->n_cols, tpart, s)) != RGCSR_OK) return st;
    if (nnz == 0) return RGCSR_OK;

    if ((st = rgcsr_csr_row_index(A, row_index, stream)) != RGCSR_OK) return st;
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < A->n_cols) ++bits;
    const uint32_t *skeys = nullptr, *sidx = nullptr;
    if ((st = radix_sort_indices(reinterpret_cast<const uint32_t *>(A->col_idx), nnz, bits, b, &skeys, &sidx, s)) != RGCSR_OK)
        return st;
    const unsigned blocks = (unsigned)ceil_div(nnz, 256);
    if (A->value_type == RGCSR_F64)
        transpose_fill_kernel<double><<<blocks, 256, 0, s>>>(sidx, nnz, row_index, t_col_idx, perm,
                                                             static_cast<const double *>(A->values),
                                                             static_cast<double *>(t_values));
    else
        transpose_fill_kernel<float><<<blocks, 256, 0, s>>>(sidx, nnz, row_index, t_col_idx, perm,
                                                            static_cast<const float *>(A->values),
                                                            static_cast<float *>(t_values));
    return launch_status();
}

RGCSR_API int rgcsr_gather_values(const rgcsr_matrix *M, const void *src, const int64_t *src_index,
                                  rgcsr_stream_t stream) {
    if (!M || M->n_stored < 0) return RGCSR_ERR_INVALID_ARG;
    if (M->n_stored == 0) return RGCSR_OK;
    if (!M->values || !src || !src_index) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = grid_for(M->n_stored, 256);
    if (M->value_type == RGCSR_F64)
        gather_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(src), src_index, M->n_stored,
                                                static_cast<double *>(M->values));
    else if (M->value_type == RGCSR_F32)
        gather_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(src), src_index, M->n_stored,
                                               static_cast<float *>(M->values));
    else
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    return launch_status();
}

RGCSR_API int rgcsr_gather_values_if_changed(const rgcsr_matrix *M, const void *src, int64_t n_src,
                                             const int64_t *src_index, void *state, rgcsr_stream_t stream) {
    static_assert(8 * (8 + kHashParts) <= RGCSR_VALUES_STATE_BYTES, "state record too small");
    if (!M || M->n_stored < 0 || n_src < 0 || !state) return RGCSR_ERR_INVALID_ARG;
    if (M->value_type != RGCSR_F64 && M->value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if ((n_src > 0 && !src) || (M->n_stored > 0 && (!M->values || !src_index))) return RGCSR_ERR_INVALID_ARG;
    if (((uintptr_t)state & 7) != 0) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    auto *st = static_cast<unsigned long long *>(state);
    // a grid-stride gather on a bounded grid: when nothing changed, each of
    // its blocks only reads the flag and exits
    const unsigned g = std::min<unsigned>(grid_for(M->n_stored, 256), 152u * 8u);
    if (M->value_type == RGCSR_F64) {
        values_hash_kernel<8><<<kHashParts, kHashThreads, 0, s>>>(src, n_src, st);
        if (M->n_stored > 0)
            gather_if_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(src), src_index, M->n_stored,
                                                       static_cast<double *>(M->values), st + 1);
    } else {
        values_hash_kernel<4><<<kHashParts, kHashThreads, 0, s>>>(src, n_src, st);
        if (M->n_stored > 0)
            gather_if_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(src), src_index, M->n_stored,
                                                      static_cast<float *>(M->values), st + 1);
    }
    return launch_status();
}

RGCSR_API int rgcsr_compose_index(const int64_t *outer, const int64_t *inner, int64_t n, int64_t *out,
                                  rgcsr_stream_t stream) {
    if (n < 0) return RGCSR_ERR_INVALID_ARG;
    if (n == 0) return RGCSR_OK;
    if (!outer || !inner || !out) return RGCSR_ERR_INVALID_ARG;
    compose_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(outer, inner, n, out);
    return launch_status();
}

RGCSR_API int rgcsr_sampled_dot(int64_t nnz, int32_t k, const int32_t *row_index, const int32_t *col_idx,
                                const void *G, int64_t ldg, const void *X, int64_t ldx, void *out,
                                int32_t value_type, rgcsr_stream_t stream) {
    if (nnz < 0 || k < 0 || ldg < k || ldx < k) return RGCSR_ERR_INVALID_ARG;
    if (nnz == 0) return RGCSR_OK;
    if (!row_index || !col_idx || !out || (k > 0 && (!G || !X))) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = grid_for(nnz, 256);
    const size_t es = value_type == RGCSR_F64 ? 8 : 4;
    const bool vec = all_aligned16(G, X) && (ldg * es) % 16 == 0 && (ldx * es) % 16 == 0 &&
                     (k == 8 || k == 4 || (k == 2 && es == 8));
    if (vec && value_type == RGCSR_F32) {
        const float *Gf = static_cast<const float *>(G), *Xf = static_cast<const float *>(X);
        float *of = static_cast<float *>(out);
        if (k == 8) sampled_dot_vec_kernel<float, 8><<<g, 256, 0, s>>>(nnz, row_index, col_idx, Gf, ldg, Xf, ldx, of);
        else sampled_dot_vec_kernel<float, 4><<<g, 256, 0, s>>>(nnz, row_index, col_idx, Gf, ldg, Xf, ldx, of);
        return launch_status();
    }
    if (vec && value_type == RGCSR_F64) {
        const double *Gd = static_cast<const double *>(G), *Xd = static_cast<const double *>(X);
        double *od = static_cast<double *>(out);
        if (k == 8) sampled_dot_vec_kernel<double, 8><<<g, 256, 0, s>>>(nnz, row_index, col_idx, Gd, ldg, Xd, ldx, od);
        else if (k == 4) sampled_dot_vec_kernel<double, 4><<<g, 256, 0, s>>>(nnz, row_index, col_idx, Gd, ldg, Xd, ldx, od);
        else sampled_dot_vec_kernel<double, 2><<<g, 256, 0, s>>>(nnz, row_index, col_idx, Gd, ldg, Xd, ldx, od);
        return launch_status();
    }
    if (value_type == RGCSR_F64)
        sampled_dot_kernel<double><<<g, 256, 0, s>>>(nnz, k, row_index, col_idx, static_cast<const double *>(G),
                                                     ldg, static_cast<const double *>(X), ldx,
                                                     static_cast<double *>(out));
    else if (value_type == RGCSR_F32)
        sampled_dot_kernel<float><<<g, 256, 0, s>>>(nnz, k, row_index, col_idx, static_cast<const float *>(G),
                                                    ldg, static_cast<const float *>(X), ldx,
                                                    static_cast<float *>(out));
    else
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    return launch_status();
}

RGCSR_API size_t rgcsr_row_order_workspace_bytes(int64_t n_rows) {
    if (n_rows < 0) return 0;
    return sort_workspace_bytes(n_rows) + align_up((size_t)n_rows * 4, 256);
}

RGCSR_API int rgcsr_descending_order(const rgcsr_csr *A, int32_t *row_perm, void *workspace,
                                     size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    const int64_t n = A->n_rows;
    if (n == 0) return RGCSR_OK;
    if (n > (int64_t)INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    if (!row_perm) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_row_order_workspace_bytes(n)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    SortBuffers b = carve_sort(workspace, n);
    uint32_t *keys = reinterpret_cast<uint32_t *>(static_cast<char *>(workspace) + sort_workspace_bytes(n));
    // a valid row has at most nnz entries: sort on just enough bits for that
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= A->nnz) ++bits;
    const uint32_t mask = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    descending_keys_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(rp, n, mask, keys);
    if ((st = launch_status()) != RGCSR_OK) return st;
    const uint32_t *skeys = nullptr, *sidx = nullptr;
    if ((st = radix_sort_indices(keys, n, bits, b, &skeys, &sidx, s)) != RGCSR_OK) return st;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(row_perm, sidx, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return RGCSR_OK;
}

RGCSR_API int rgcsr_spmv_bwd_values(const rgcsr_matrix *M, int32_t k, const void *G, int64_t ldg, const void *X,
                                    int64_t ldx, void *dval, rgcsr_stream_t stream) {
    if (!M || M->n_rows < 0 || M->group_size < 1 || k < 0 || ldg < k || ldx < k) return RGCSR_ERR_INVALID_ARG;
    if (M->value_type != RGCSR_F64 && M->value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_stored == 0 || M->nnz == 0) return RGCSR_OK;
    if (!M->group_ptr || !M->columns || !M->slot_to_csr || !dval || (k > 0 && (!G || !X)))
        return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    const unsigned g = grid_for(M->n_groups * 32, 256);
    if (M->value_type == RGCSR_F64)
        bwd_values_kernel<double><<<g, 256, 0, s>>>(M->n_rows, M->group_size, M->n_groups, M->group_ptr, M->columns,
                                                    M->slot_to_csr, M->row_perm, k, static_cast<const double *>(G),
                                                    ldg, static_cast<const double *>(X), ldx,
                                                    static_cast<double *>(dval));
    else
        bwd_values_kernel<float><<<g, 256, 0, s>>>(M->n_rows, M->group_size, M->n_groups, M->group_ptr, M->columns,
                                                   M->slot_to_csr, M->row_perm, k, static_cast<const float *>(G),
                                                   ldg, static_cast<const float *>(X), ldx, static_cast<float *>(dval));
    return launch_status();
}
