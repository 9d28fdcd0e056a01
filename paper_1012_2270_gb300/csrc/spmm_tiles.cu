// spmm_tiles.cu -- Y = A X on the group-tile schedule of tiles.cu (G <= 32).
//
// As in the tiled SpMV, a warp takes a tile of at most C slot-rows of one
// row group, lane t owns row t, and every value/column load of the warp is
// one coalesced slot-row.  Here lane t also owns KC consecutive columns of
// its row of Y, reading KC entries of row col of X per non-zero (16-byte
// vector loads when aligned).  Tiles of a split group publish KC partial
// sums per row; the last tile to arrive adds them in tile order.  Suited to
// few right-hand sides (the per-lane X piece is one or two sectors);
// rgcsr_spmm_long_rows covers wide X.  Not in the paper: an extension of its
// SpMV (Sec. 3.4) to several right-hand sides.
#include "common.cuh"
#include "vtraits.cuh"

namespace rgcsr {
namespace {

constexpr int kThreadsT = 256;

template <typename V, int KC, bool VEC>
__global__ void __launch_bounds__(kThreadsT, 4)
rgcsr_spmm_tiles_kernel(int64_t n, int32_t G, int32_t C, int64_t n_groups, int64_t n_tasks,
                        const V *__restrict__ val, const int32_t *__restrict__ col,
                        const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                        const float *__restrict__ scale, const int64_t *__restrict__ first_extra,
                        const int64_t *__restrict__ part_base, const int32_t *__restrict__ extra_group,
                        int32_t *__restrict__ arrivals, typename VT<V>::A *partials,
                        const typename VT<V>::A *__restrict__ X, int64_t ldx, typename VT<V>::A *__restrict__ Y,
                        int64_t ldy, const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tasks; t += warps) {
        int64_t g, k;
        if (t < n_groups) {
            g = t;
            k = 0;
        } else {
            g = __ldg(extra_group + (t - n_groups));
            k = 1 + (t - n_groups) - __ldg(first_extra + g);
        }
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const bool active = lane < R;
        const int64_t base = __ldg(gp + g);
        const int len = active ? __ldg(rl + first + lane) : 0;
        const int64_t nt = first_extra ? 1 + __ldg(first_extra + g + 1) - __ldg(first_extra + g) : 1;
        const int j0 = (int)(k * C);
        const int jend = min(len, j0 + C);
        A acc[KC];
#pragma unroll
        for (int w = 0; w < KC; ++w) acc[w] = 0;
        for (int j = j0; j < jend; j += U) {
            A v[U];
            int c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = 0;
                c[u] = 0;
                if (j + u < jend) {
                    const int64_t p = base + (int64_t)(j + u) * R + lane;
                    v[u] = VT<V>::ld(val + p);
                    c[u] = ld_stream(col + p);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j + u < jend) {
                    A xw[KC];
                    load_xrow<A, KC, VEC>(X + (int64_t)c[u] * ldx, xw);
#pragma unroll
                    for (int w = 0; w < KC; ++w) acc[w] = fma(v[u], xw[w], acc[w]);
                }
            }
        }
        const int64_t row = first + lane;
        if (nt == 1) {
            if (active) {
                A *yr = Y + out_row(perm, row) * ldy;
#pragma unroll
                for (int w = 0; w < KC; ++w) yr[w] = finish<V>(acc[w], scale, row);
            }
            continue;
        }
        const int64_t pb = __ldg(part_base + g);
        if (active) {
            A *pr = partials + ((pb + k) * 32 + lane) * KC;
#pragma unroll
            for (int w = 0; w < KC; ++w) pr[w] = acc[w];
        }
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(arrivals + g, 1) == (int)(nt - 1);
        }
        last = __shfl_sync(kFull, last, 0);
        if (!last) continue;
        __threadfence();
        if (active) {
            A s[KC];
#pragma unroll
            for (int w = 0; w < KC; ++w) s[w] = 0;
            for (int64_t q = 0; q < nt; ++q) {
                const A *pr = partials + ((pb + q) * 32 + lane) * KC;
#pragma unroll
                for (int w = 0; w < KC; ++w) s[w] += __ldcg(pr + w);
            }
            A *yr = Y + out_row(perm, row) * ldy;
#pragma unroll
            for (int w = 0; w < KC; ++w) yr[w] = finish<V>(s[w], scale, row);
        }
        if (lane == 0) arrivals[g] = 0;
    }
}

template <typename V, int KC, bool VEC>
int launch_spmm_tiles(const rgcsr_matrix *M, const rgcsr_tiles *T, const typename VT<V>::A *X, int64_t ldx,
                      typename VT<V>::A *Y, int64_t ldy, typename VT<V>::A *part, cudaStream_t s) {
    auto kern = rgcsr_spmm_tiles_kernel<V, KC, VEC>;
    int dev = 0, sms = 152, occ = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreadsT, 0) != cudaSuccess || occ < 1) occ = 1;
    const int64_t n_tasks = M->n_groups + T->n_extra;
    int64_t grid = (int64_t)sms * occ;
    const int64_t need = ceil_div(n_tasks, kThreadsT / 32);
    if (need < grid) grid = need;
    kern<<<(unsigned)grid, kThreadsT, 0, s>>>(
        M->n_rows, M->group_size, T->tile, M->n_groups, n_tasks, static_cast<const V *>(M->values), M->columns,
        M->group_ptr, M->row_lengths, M->row_scale, T->n_extra > 0 ? T->first_extra : nullptr, T->part_base,
        T->extra_group, T->arrivals, part, X, ldx, Y, ldy, M->row_perm);
    return launch_status();
}

// Column chunks of 8, 4, then single columns; vector loads of X when its
// base and row stride are 16-byte aligned.
template <typename V>
int spmm_tiles_t(const rgcsr_matrix *M, const rgcsr_tiles *T, int k, const typename VT<V>::A *X, int64_t ldx,
                 typename VT<V>::A *Y, int64_t ldy, typename VT<V>::A *part, cudaStream_t s) {
    using A = typename VT<V>::A;
    const bool vec = ((uintptr_t)X & 15) == 0 && (ldx * (int64_t)sizeof(A)) % 16 == 0;
    int c0 = 0;
    while (c0 < k) {
        const int left = k - c0;
        int st, w;
        if (left >= 8) {
            st = vec ? launch_spmm_tiles<V, 8, true>(M, T, X + c0, ldx, Y + c0, ldy, part, s)
                     : launch_spmm_tiles<V, 8, false>(M, T, X + c0, ldx, Y + c0, ldy, part, s);
            w = 8;
        } else if (left >= 4) {
            st = vec ? launch_spmm_tiles<V, 4, true>(M, T, X + c0, ldx, Y + c0, ldy, part, s)
                     : launch_spmm_tiles<V, 4, false>(M, T, X + c0, ldx, Y + c0, ldy, part, s);
            w = 4;
        } else {
            st = launch_spmm_tiles<V, 1, false>(M, T, X + c0, ldx, Y + c0, ldy, part, s);
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

RGCSR_API int rgcsr_spmm_tiles(const rgcsr_matrix *M, const rgcsr_tiles *T, int32_t k, const void *X,
                               int64_t ldx, void *Y, int64_t ldy, void *partials, int64_t partials_count,
                               rgcsr_stream_t stream) {
    if (!M || M->n_rows < 0 || M->group_size < 1 || M->group_size > 32 || k < 0) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups > (int64_t)INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    if (M->n_rows == 0 || k == 0) return RGCSR_OK;
    if (!T || T->tile < 1 || T->n_groups != M->n_groups) return RGCSR_ERR_INVALID_ARG;
    if (ldx < k || ldy < k || !Y || (M->n_cols > 0 && !X)) return RGCSR_ERR_INVALID_ARG;
    if (!M->group_ptr || !M->row_lengths || (M->n_stored > 0 && (!M->values || !M->columns)))
        return RGCSR_ERR_INVALID_ARG;
    if (T->n_extra > 0) {
        if (!T->first_extra || !T->part_base || !T->extra_group || !T->arrivals) return RGCSR_ERR_INVALID_ARG;
        if (!partials || partials_count < T->n_partials * 32 * (int64_t)(k < 8 ? k : 8)) return RGCSR_ERR_WORKSPACE;
    }
    if (k == 1 && ldx == 1 && ldy == 1) return rgcsr_spmv_tiles(M, T, X, Y, stream);   // the SpMV
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64:
            return spmm_tiles_t<double>(M, T, k, static_cast<const double *>(X), ldx, static_cast<double *>(Y), ldy,
                                        static_cast<double *>(partials), s);
        case RGCSR_F32:
            return spmm_tiles_t<float>(M, T, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy,
                                       static_cast<float *>(partials), s);
        case RGCSR_BF16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_tiles_t<__nv_bfloat16>(M, T, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y),
                                               ldy, static_cast<float *>(partials), s);
        case RGCSR_F16:
            if (!M->row_scale) return RGCSR_ERR_INVALID_ARG;
            return spmm_tiles_t<__half>(M, T, k, static_cast<const float *>(X), ldx, static_cast<float *>(Y), ldy,
                                        static_cast<float *>(partials), s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}
