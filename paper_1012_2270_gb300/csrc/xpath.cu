// xpath.cu -- where the x gathers of an RgCSR SpMV are served from: the
// x read-path study of the paper (Sec. 4.3 measures SpMV with and without
// binding x to the texture cache) redone with the read paths of this GPU.
//
//  * x_texture: texture objects over x for RGCSR_XLOAD_TEX (the kernels are
//    in spmv.cu), cached per device and buffer.
//  * x-window staging: for blocks of RGCSR_XWINDOW_ROWS consecutive stored
//    rows, a plan finds the column ranges the block's entries touch -- at
//    most RGCSR_XWINDOW_MAX_RANGES ranges, cut where two consecutive used
//    columns are more than RGCSR_XWINDOW_GAP apart -- and the SpMV stages
//    those pieces of x in shared memory once per block, so the gathers of
//    all the block's rows read shared memory.  A 3D 7-point stencil's block
//    of 256 rows touches three bands (the rows below, at and above in z),
//    1,024 elements in all; a banded matrix one range.  Blocks whose ranges
//    are too many or too wide gather from global memory as before.
#include "common.cuh"
#include "vtraits.cuh"

#include <climits>
#include <mutex>
#include <vector>

namespace rgcsr {

// ---------------------------------------------------------------------------
// texture objects over x
// ---------------------------------------------------------------------------
namespace {
struct TexEntry {
    int dev;
    const void *ptr;
    int64_t n;
    int elem_bytes;
    cudaTextureObject_t tex;
};
constexpr size_t kTexCacheMax = 64;
std::mutex g_tex_mutex;
std::vector<TexEntry> g_tex_cache;
}  // namespace

int x_texture(const void *x, int64_t n, int elem_bytes, cudaTextureObject_t *out) {
    if (!x || n <= 0 || !out || (elem_bytes != 4 && elem_bytes != 8)) return RGCSR_ERR_INVALID_ARG;
    int dev = 0;
    RGCSR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tex_mutex);
    for (const TexEntry &e : g_tex_cache)
        if (e.dev == dev && e.ptr == x && e.n == n && e.elem_bytes == elem_bytes) {
            *out = e.tex;
            return RGCSR_OK;
        }
    int max_width = 0;
    RGCSR_CUDA_TRY(cudaDeviceGetAttribute(&max_width, cudaDevAttrMaxTexture1DLinearWidth, dev));
    if (n > (int64_t)max_width) return RGCSR_ERR_INVALID_ARG;
    if (g_tex_cache.size() >= kTexCacheMax) {
        // kernels launched earlier may still read through these objects
        RGCSR_CUDA_TRY(cudaDeviceSynchronize());
        for (const TexEntry &e : g_tex_cache) {
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(e.dev);
            cudaDestroyTextureObject(e.tex);
            cudaSetDevice(cur);
        }
        g_tex_cache.clear();
    }
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = const_cast<void *>(x);
    rd.res.linear.desc = elem_bytes == 8 ? cudaCreateChannelDesc<int2>() : cudaCreateChannelDesc<float>();
    rd.res.linear.sizeInBytes = (size_t)n * elem_bytes;
    cudaTextureDesc td = {};
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t tex = 0;
    RGCSR_CUDA_TRY(cudaCreateTextureObject(&tex, &rd, &td, nullptr));
    g_tex_cache.push_back({dev, x, n, elem_bytes, tex});
    *out = tex;
    return RGCSR_OK;
}

// ---------------------------------------------------------------------------
// x-window plan
// ---------------------------------------------------------------------------
namespace {

constexpr int kRows = RGCSR_XWINDOW_ROWS;        // one thread per row
constexpr int kSortCap = 8192;                   // entries of a block the plan sorts at most
constexpr int kMaxRanges = RGCSR_XWINDOW_MAX_RANGES;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < kRows / 32; ++i) {
            const int t = warp_tot[i];
            warp_tot[i] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return warp_tot[w] + incl - v;
}

// One CTA per block of kRows stored rows: gathers the columns of the
// block's stored entries (padding excluded), sorts them (bitonic, in shared
// memory), cuts the sorted list where consecutive columns are more than
// `gap` apart, and keeps the ranges if there are at most kMaxRanges of them
// spanning at most `cap` elements; otherwise (or with more than kSortCap
// entries, or none) the block's record says "not staged" (n_ranges = 0).
__global__ void __launch_bounds__(kRows)
xwindow_plan_kernel(int64_t n, int32_t G, const int32_t *__restrict__ col, const int64_t *__restrict__ gp,
                    const int32_t *__restrict__ rl, int32_t gap, int32_t cap, rgcsr_xwindow *__restrict__ out) {
    __shared__ int s[kSortCap];
    __shared__ int warp_tot[kRows / 32];
    __shared__ int total, n_breaks, fail;
    __shared__ int brk[kMaxRanges];
    const int64_t row = (int64_t)blockIdx.x * kRows + threadIdx.x;
    int len = 0, stride = 0;
    int64_t ptr = 0;
    if (row < n) {
        const int64_t g = row / G, first = g * G;
        stride = (int)min((int64_t)G, n - first);
        ptr = gp[g] + (row - first);
        len = rl[row];
    }
    if (threadIdx.x == 0) { n_breaks = 0; fail = 0; }
    const int off = block_exclusive_scan(len, warp_tot, &total);
    rgcsr_xwindow rec = {};
    const int T = total;
    if (T == 0 || T > kSortCap) {
        if (threadIdx.x == 0) out[blockIdx.x] = rec;
        return;
    }
    for (int j = 0; j < len; ++j) s[off + j] = col[ptr + (int64_t)j * stride];
    int P = 1;
    while (P < T) P <<= 1;
    for (int i = T + threadIdx.x; i < P; i += kRows) s[i] = INT_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kRows) {
                const int ij = i ^ j;
                if (ij > i) {
                    const int a = s[i], b = s[ij];
                    if ((a > b) == ((i & k) == 0)) { s[i] = b; s[ij] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i + 1 < T; i += kRows)
        if (s[i + 1] - s[i] > gap) {
            const int q = atomicAdd(&n_breaks, 1);
            if (q < kMaxRanges - 1) brk[q] = i;
            else fail = 1;
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nb = n_breaks;
        if (!fail) {
            for (int a = 1; a < nb; ++a)                   // at most three breaks: insertion sort
                for (int b = a; b > 0 && brk[b - 1] > brk[b]; --b) { const int t = brk[b]; brk[b] = brk[b - 1]; brk[b - 1] = t; }
            int start = s[0], sum = 0;
            for (int r = 0; r <= nb; ++r) {
                const int end = (r < nb ? s[brk[r]] : s[T - 1]) + 1;
                rec.lo[r] = start;
                rec.len[r] = end - start;
                sum += end - start;
                if (r < nb) start = s[brk[r] + 1];
            }
            rec.n_ranges = nb + 1;
            rec.total = sum;
            if (sum > cap) rec = rgcsr_xwindow{};
        }
        out[blockIdx.x] = rec;
    }
}

// ---------------------------------------------------------------------------
// SpMV with the x-window staged in shared memory: one thread per stored row
// (kRows rows per CTA, the plan's blocks), U slots in flight per thread.
// ---------------------------------------------------------------------------
template <typename V, int U>
__global__ void __launch_bounds__(kRows)
rgcsr_spmv_xwindow_kernel(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                          const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                          const float *__restrict__ scale, const typename VT<V>::A *__restrict__ x,
                          typename VT<V>::A *__restrict__ y, const int32_t *__restrict__ perm,
                          const rgcsr_xwindow *__restrict__ win) {
    using A = typename VT<V>::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *sx = reinterpret_cast<A *>(smem_raw);
    const rgcsr_xwindow w = win[blockIdx.x];
    int lo[kMaxRanges], len[kMaxRanges], base[kMaxRanges];
    int b = 0;
#pragma unroll
    for (int r = 0; r < kMaxRanges; ++r) {
        lo[r] = w.lo[r];
        len[r] = r < w.n_ranges ? w.len[r] : 0;
        base[r] = b;
        b += len[r];
    }
    const bool staged = w.n_ranges > 0;
    if (staged) {
#pragma unroll
        for (int r = 0; r < kMaxRanges; ++r)
            for (int i = threadIdx.x; i < len[r]; i += kRows) sx[base[r] + i] = __ldg(x + lo[r] + i);
        __syncthreads();
    }
    const int64_t row = (int64_t)blockIdx.x * kRows + threadIdx.x;
    if (row >= n) return;
    const int64_t g = row / G, first = g * G;
    const int stride = (int)min((int64_t)G, n - first);
    const int64_t off = __ldg(gp + g) + (row - first);
    const V *vp = val + off;
    const int32_t *cp = col + off;
    const int L = __ldg(rl + row);
    A acc = 0;
    for (int j = 0; j < L; j += U) {
        A v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < L) {
                v[u] = VT<V>::ld(vp + (int64_t)u * stride);
                c[u] = ld_stream(cp + (int64_t)u * stride);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < L) {
                // shared memory if the column lies in a staged range, else
                // the read-only path (a block not staged, or a column outside
                // the planned ranges)
                int sidx = -1;
#pragma unroll
                for (int r = 0; r < kMaxRanges; ++r)
                    if ((unsigned)(c[u] - lo[r]) < (unsigned)len[r]) sidx = base[r] + c[u] - lo[r];
                acc = fma(v[u], sidx >= 0 ? sx[sidx] : __ldg(x + c[u]), acc);
            }
        vp += (int64_t)U * stride;
        cp += (int64_t)U * stride;
    }
    y[out_row(perm, row)] = finish<V>(acc, scale, row);
}

int x_elem_bytes(const rgcsr_matrix *M) { return M->value_type == RGCSR_F64 ? 8 : 4; }

int check_xwindow_matrix(const rgcsr_matrix *M) {
    if (!M || M->n_rows < 0 || M->n_cols < 0 || M->group_size < 1) return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!M->group_ptr || !M->row_lengths || (M->n_stored > 0 && (!M->values || !M->columns)))
        return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (M->value_type < RGCSR_F64 || M->value_type > RGCSR_F16) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    return RGCSR_OK;
}

template <typename V>
int launch_xwindow(const rgcsr_matrix *M, const rgcsr_xwindow *win, const void *x, void *y, cudaStream_t s) {
    using A = typename VT<V>::A;
    if (VT<V>::scaled && !M->row_scale) return RGCSR_ERR_INVALID_ARG;
    const int64_t blocks = ceil_div(M->n_rows, kRows);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    rgcsr_spmv_xwindow_kernel<V, 4><<<(unsigned)blocks, kRows, RGCSR_XWINDOW_CAP_BYTES, s>>>(
        M->n_rows, M->group_size, static_cast<const V *>(M->values), M->columns, M->group_ptr,
        M->row_lengths, M->row_scale, static_cast<const A *>(x), static_cast<A *>(y), M->row_perm, win);
    return launch_status();
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int64_t rgcsr_xwindow_count(int64_t n_rows) {
    return n_rows > 0 ? ceil_div(n_rows, RGCSR_XWINDOW_ROWS) : 0;
}

RGCSR_API int rgcsr_xwindow_plan(const rgcsr_matrix *M, rgcsr_xwindow *windows, rgcsr_stream_t stream) {
    int st = check_xwindow_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!windows) return RGCSR_ERR_INVALID_ARG;
    const int64_t blocks = rgcsr_xwindow_count(M->n_rows);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    const int cap = RGCSR_XWINDOW_CAP_BYTES / x_elem_bytes(M);
    xwindow_plan_kernel<<<(unsigned)blocks, kRows, 0, (cudaStream_t)stream>>>(
        M->n_rows, M->group_size, M->columns, M->group_ptr, M->row_lengths, RGCSR_XWINDOW_GAP, cap, windows);
    return launch_status();
}

RGCSR_API int rgcsr_spmv_xwindow(const rgcsr_matrix *M, const rgcsr_xwindow *windows, const void *x, void *y,
                                 rgcsr_stream_t stream) {
    int st = check_xwindow_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!windows || !y || (M->n_cols > 0 && !x)) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64: return launch_xwindow<double>(M, windows, x, y, s);
        case RGCSR_F32: return launch_xwindow<float>(M, windows, x, y, s);
        case RGCSR_BF16: return launch_xwindow<__nv_bfloat16>(M, windows, x, y, s);
        case RGCSR_F16: return launch_xwindow<__half>(M, windows, x, y, s);
        default: return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}
