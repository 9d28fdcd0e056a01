// spmm_rows.cu -- Y = A X (row-major X [n_cols x k], Y [n_rows x k]) with a
// few lanes per row and the long-row segment schedule of spmv.cu.
//
// A sub-warp of S lanes owns one row (or one segment of a long row); lane q
// holds W consecutive columns of the row's result.  The sub-warp loads S
// slots of the row at a time (value and column of slot jj+q on lane q) and
// broadcasts each slot with a shuffle; every lane then reads W consecutive
// entries of row col of X.  With W = 4 the S lanes of a sub-warp read one
// contiguous 16*S-byte piece of X per non-zero, so a gather of the full
// 32-column piece costs one L1 request instead of eight per-thread vector
// loads.  Rows longer than the schedule's threshold T are cut: slots < T
// here, the rest in segments of `segment` slots whose partial sums are added
// in order by a last pass (deterministic).  Not in the paper: an extension
// of its SpMV (Sec. 3.4) to several right-hand sides.
#include "common.cuh"
#include "vtraits.cuh"

namespace rgcsr {
namespace {

constexpr int kRowThreads = 256;
// Blocks of the row kernel (rows up to the long-row threshold): two warps,
// so that an SM slot is freed as soon as its few rows are done -- rows of
// very different lengths end at very different times.
constexpr int kShortThreads = 64;

template <typename A, int W, bool VEC>
__device__ __forceinline__ void load_w(const A *__restrict__ p, A (&o)[W]) {
    if constexpr (VEC && W == 4 && sizeof(A) == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (VEC && W == 4 && sizeof(A) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] = __ldg(p + w);
    }
}

template <typename A, int W, bool VEC>
__device__ __forceinline__ void store_w(A *__restrict__ p, const A (&v)[W]) {
    if constexpr (VEC && W == 4 && sizeof(A) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (VEC && W == 4 && sizeof(A) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    } else {
#pragma unroll
        for (int w = 0; w < W; ++w) p[w] = v[w];
    }
}

// SEG = false: task t is row t, slots [0, min(len, cap)), result (times the
// row scale) to Y.  SEG = true: task t is segment t -- row seg_row[t], slots
// [seg_start[t], min(seg_start[t] + seg_len, len)) -- unscaled partial sums
// to part[t * ldp + ...].  U slots per lane are loaded per step.
template <typename V, int S, int W, int U, bool VEC, bool SEG>
__global__ void __launch_bounds__(kRowThreads)
spmm_rows_kernel(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                 const int64_t *__restrict__ gp, const int32_t *__restrict__ rl, const float *__restrict__ scale,
                 int cap, int64_t n_tasks, const int32_t *__restrict__ seg_row,
                 const int32_t *__restrict__ seg_start, int seg_len, const typename VT<V>::A *__restrict__ X,
                 int64_t ldx, typename VT<V>::A *__restrict__ Y, int64_t ldy, const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    constexpr int kRowsPerWarp = 32 / S;
    const int lane = threadIdx.x & 31;
    const int q = lane % S;
    const int64_t task = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kRowsPerWarp + lane / S;
    const bool valid = task < n_tasks;
    int64_t row = 0, base = 0;
    int R = 0, ja = 0, jb = 0;
    if (valid) {
        row = SEG ? (int64_t)seg_row[task] : task;
        const int64_t g = row / G;
        const int64_t first = g * G;
        R = (int)min((int64_t)G, n - first);
        base = __ldg(gp + g) + (row - first);
        const int len = __ldg(rl + row);
        if (SEG) {
            ja = seg_start[task];
            jb = min(ja + seg_len, len);
        } else {
            jb = min(len, cap);
        }
    }
    const int span = jb - ja;
    const int smax = warp_max_i(span);
    A acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0;
    for (int jj = 0; jj < smax; jj += S * U) {
        A v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int my = jj + u * S + q;
            v[u] = 0;
            c[u] = 0;
            if (my < span) {
                const int64_t p = base + (int64_t)(ja + my) * R;
                v[u] = VT<V>::ld(val + p);
                c[u] = ld_stream(col + p);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const A vs = __shfl_sync(kFull, v[u], s, S);
                const int cs = __shfl_sync(kFull, c[u], s, S);
                if (jj + u * S + s < span) {
                    A xw[W];
                    load_w<A, W, VEC>(X + (int64_t)cs * ldx + W * q, xw);
#pragma unroll
                    for (int w = 0; w < W; ++w) acc[w] = fma(vs, xw[w], acc[w]);
                }
            }
        }
    }
    if (!valid) return;
    if (SEG) {
        store_w<A, W, VEC>(Y + task * ldy + W * q, acc);
    } else {
        if constexpr (VT<V>::scaled) {
            const float sc = __ldg(scale + row);
#pragma unroll
            for (int w = 0; w < W; ++w) acc[w] *= sc;
        }
        store_w<A, W, VEC>(Y + out_row(perm, row) * ldy + W * q, acc);
    }
}

// Y[row, c] += s_row * sum_q part[(first + q) * ldp + c], one thread per
// (long row, column of the chunk).
template <typename V>
__global__ void spmm_combine_kernel(int64_t n_long, int kc, const int32_t *__restrict__ long_row,
                                    const int32_t *__restrict__ long_first, const int32_t *__restrict__ long_count,
                                    const typename VT<V>::A *__restrict__ part, int64_t ldp,
                                    const float *__restrict__ scale, typename VT<V>::A *__restrict__ Y,
                                    int64_t ldy, const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_long * kc) return;
    const int64_t k = i / kc;
    const int c = (int)(i - k * kc);
    const int64_t row = long_row[k];
    const int64_t f = long_first[k];
    A s = 0;
    for (int q = 0; q < long_count[k]; ++q) s += part[(f + q) * ldp + c];
    Y[out_row(perm, row) * ldy + c] += finish<V>(s, scale, row);
}

template <typename V, int S, int W, int U, bool VEC>
int launch_chunk_rows(const rgcsr_matrix *M, const rgcsr_long_rows *L, const typename VT<V>::A *X, int64_t ldx,
                      typename VT<V>::A *Y, int64_t ldy, typename VT<V>::A *part, cudaStream_t s) {
    constexpr int kc = S * W;
    constexpr int rows_per_block = (kRowThreads / 32) * (32 / S);
    constexpr int rows_per_short_block = (kShortThreads / 32) * (32 / S);
    const V *val = static_cast<const V *>(M->values);
    const int cap = L ? L->threshold : INT_MAX;
    int64_t blocks = ceil_div(M->n_rows, rows_per_short_block);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    spmm_rows_kernel<V, S, W, U, VEC, false><<<(unsigned)blocks, kShortThreads, 0, s>>>(
        M->n_rows, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, M->row_scale, cap, M->n_rows,
        nullptr, nullptr, 0, X, ldx, Y, ldy, M->row_perm);
    int st = launch_status();
    if (st != RGCSR_OK || !L || L->n_segments == 0) return st;
    blocks = ceil_div(L->n_segments, rows_per_block);
    spmm_rows_kernel<V, S, W, U, VEC, true><<<(unsigned)blocks, kRowThreads, 0, s>>>(
        M->n_rows, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, M->row_scale, cap,
        L->n_segments, L->seg_row, L->seg_start, L->segment, X, ldx, part, kc, M->row_perm);
    if ((st = launch_status()) != RGCSR_OK) return st;
    const int64_t threads = L->n_long_rows * kc;
    spmm_combine_kernel<V><<<(unsigned)ceil_div(threads, 256), 256, 0, s>>>(
        L->n_long_rows, kc, L->long_row, L->long_first, L->long_count, part, kc, M->row_scale, Y, ldy,
        M->row_perm);
    return launch_status();
}

// Column chunks: 4*S columns with S = 8, 4, 2, 1 lanes per row, then single
// columns.  Vector loads of X and Y when both are 16-byte aligned at every
// chunk start.
template <typename V>
int spmm_rows_t(const rgcsr_matrix *M, const rgcsr_long_rows *L, int k, const typename VT<V>::A *X, int64_t ldx,
                typename VT<V>::A *Y, int64_t ldy, typename VT<V>::A *part, cudaStream_t s) {
    using A = typename VT<V>::A;
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    const bool vec = al(X) && al(Y) && (ldx * (int64_t)sizeof(A)) % 16 == 0 && (ldy * (int64_t)sizeof(A)) % 16 == 0;
    int c0 = 0;
    while (c0 < k) {
        const int left = k - c0;
        const A *Xc = X + c0;
        A *Yc = Y + c0;
        int st, w;
        if (left >= 32) {
            st = vec ? launch_chunk_rows<V, 8, 4, 2, true>(M, L, Xc, ldx, Yc, ldy, part, s)
                     : launch_chunk_rows<V, 8, 4, 2, false>(M, L, Xc, ldx, Yc, ldy, part, s);
            w = 32;
        } else if (left >= 16) {
            st = vec ? launch_chunk_rows<V, 4, 4, 2, true>(M, L, Xc, ldx, Yc, ldy, part, s)
                     : launch_chunk_rows<V, 4, 4, 2, false>(M, L, Xc, ldx, Yc, ldy, part, s);
            w = 16;
        } else if (left >= 8) {
            st = vec ? launch_chunk_rows<V, 2, 4, 4, true>(M, L, Xc, ldx, Yc, ldy, part, s)
                     : launch_chunk_rows<V, 2, 4, 4, false>(M, L, Xc, ldx, Yc, ldy, part, s);
            w = 8;
        } else if (left >= 4) {
            st = vec ? launch_chunk_rows<V, 1, 4, 8, true>(M, L, Xc, ldx, Yc, ldy, part, s)
                     : launch_chunk_rows<V, 1, 4, 8, false>(M, L, Xc, ldx, Yc, ldy, part, s);
            w = 4;
        } else {
            st = launch_chunk_rows<V, 1, 1, 8, false>(M, L, Xc, ldx, Yc, ldy, part, s);
            w = 1;
        }
        if (st != RGCSR_OK) return st;
        c0 += w;
    }
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_spmm_long_rows(const rgcsr_matrix *M, const rgcsr_long_rows *L, int32_t k, const void *X,
                                   int64_t ldx, void *Y, int64_t ldy, void *partials, int64_t partials_count,
                                   rgcsr_stream_t stream) {
    if (!M || M->n_rows < 0 || M->group_size < 1 || k < 0) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows == 0 || k == 0) return RGCSR_OK;
    if (ldx < k || ldy < k || !Y || (M->n_cols > 0 && !X)) return RGCSR_ERR_INVALID_ARG;
    if (!M->group_ptr || !M->row_lengths || (M->n_stored > 0 && (!M->values || !M->columns)))
        return RGCSR_ERR_INVALID_ARG;
    if (L) {
        if (L->threshold < 0 || L->segment < 1) return RGCSR_ERR_INVALID_ARG;
        if (L->n_segments > 0) {
            if (!L->seg_row || !L->seg_start || !L->long_row || !L->long_first || !L->long_count)
                return RGCSR_ERR_INVALID_ARG;
            if (!partials || partials_count < L->n_segments * (int64_t)(k < 32 ? k : 32)) return RGCSR_ERR_WORKSPACE;
        }
    }
    if (k == 1 && ldx == 1 && ldy == 1)      // one right-hand side: the SpMV path
        return L ? rgcsr_spmv_long_rows(M, L, X, Y, stream) : rgcsr_spmv(M, X, Y, stream);
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64:
            return spmm_rows_t<double>(M, L, k, static_cast<const double *>(X), ldx, static_cast<double *>(Y), ldy,
                                       static_cast<double *>(partials), s);
        case RGCSR_F32:
            return spmm_rows_t<float>(M, L, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy,
                                      static_cast<float *>(partials), s);
        case RGCSR_BF16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_rows_t<__nv_bfloat16>(M, L, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y),
                                              ldy, static_cast<float *>(partials), s);
        case RGCSR_F16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_rows_t<__half>(M, L, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy,
                                       static_cast<float *>(partials), s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}
