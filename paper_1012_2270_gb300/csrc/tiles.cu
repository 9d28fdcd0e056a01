// tiles.cu -- group-tile schedule for the RgCSR SpMV (G <= 32).
//
// The paper maps one thread to each row of a group (Sec. 3.4), so a group
// takes as long as its longest row, and a group holding a very long row
// holds up its warp (Sec. 4.4.2, Table 6).  Here a warp takes a tile of a
// group: lane t owns row t, and a tile covers at most `tile` slot-rows
// [j0, j0 + tile) of the group's slab.  Slot-row j of a group is R_g
// consecutive words (the format's column-major slab), so each load of the
// warp is one coalesced segment.  A group longer than one tile is cut into
// several tasks; they write per-row partial sums and the last task of the
// group to arrive (an atomic counter, no waiting) sums them in a fixed order
// (eight interleaved sums over the tasks for FP32 storage, four otherwise,
// then a fixed tree).
//
// Task numbering: task g < n_groups is the first tile of group g (no lookup
// needed); task n_groups + e is extra tile e, of group extra_group[e], and
// tile index 1 + e - first_extra[g] within it.
#include "common.cuh"
#include "vtraits.cuh"

namespace rgcsr {
namespace {

constexpr int kTileThreads = 256;

// Per group: extra tasks (ceil(K_g / C) - 1, at least 0) and partial slots
// (all its tasks if it is split, else none).
__global__ void tile_count_kernel(int64_t n, int32_t G, int64_t n_groups, const int64_t *__restrict__ gp,
                                  int32_t C, int64_t *__restrict__ n_extra, int64_t *__restrict__ n_part) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const int64_t R = min((int64_t)G, n - g * G);
    const int64_t K = (gp[g + 1] - gp[g]) / R;
    const int64_t tasks = K > C ? (K + C - 1) / C : 1;
    n_extra[g] = tasks - 1;
    n_part[g] = tasks > 1 ? tasks : 0;
}

__global__ void tile_fill_kernel(int64_t n_groups, const int64_t *__restrict__ first_extra,
                                 int32_t *__restrict__ extra_group) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    for (int64_t e = first_extra[g]; e < first_extra[g + 1]; ++e) extra_group[e] = (int32_t)g;
}

template <typename A>
__device__ __forceinline__ A ld_coherent(const A *p) { return __ldcg(p); }

// Sum of a row's nt tile partials (stride 32 between consecutive tiles):
// NS interleaved sums -- tile q goes to sum q mod NS, so NS loads are in
// flight at once -- added in a fixed tree.  Deterministic for a given nt.
// Every index is static, so the sums stay in registers.  NS = 8 for FP32
// storage, 4 otherwise (more would spill in the tighter FP64 and BF16/FP16
// variants).
template <typename V, typename A>
__device__ __forceinline__ A sum_partials(const A *p, int64_t nt) {
    constexpr int NS = (sizeof(A) == 8 || VT<V>::scaled) ? 4 : 8;
    A s[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = 0;
    int64_t q = 0;
    for (; q + NS <= nt; q += NS) {
#pragma unroll
        for (int k = 0; k < NS; ++k) s[k] += ld_coherent(p + (q + k) * 32);
    }
#pragma unroll
    for (int k = 0; k < NS - 1; ++k)
        if (q + k < nt) s[k] += ld_coherent(p + (q + k) * 32);
#pragma unroll
    for (int w = NS / 2; w > 0; w /= 2)                 // pairwise tree: (s0+s1)+(s2+s3)...
#pragma unroll
        for (int k = 0; k < w; ++k) s[k] = s[2 * k] + s[2 * k + 1];
    return s[0];
}

// CP: the columns of a tile's next step are loaded before the current
// step's gathers (its values after them), so the DRAM latency of the
// columns overlaps the gathers of the step before; the same sums in the
// same order as without.
template <typename V, int U, int MIN_BLOCKS, bool CP = false>
__global__ void __launch_bounds__(kTileThreads, MIN_BLOCKS)
rgcsr_spmv_tiles_kernel(int64_t n, int32_t G, int32_t C, int64_t n_groups, int64_t n_tasks,
                        const V *__restrict__ val, const int32_t *__restrict__ col,
                        const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                        const float *__restrict__ scale, const int64_t *__restrict__ first_extra,
                        const int64_t *__restrict__ part_base, const int32_t *__restrict__ extra_group,
                        int32_t *__restrict__ arrivals, typename VT<V>::A *partials,
                        const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
                        const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
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
        // issued now so that the result's store does not wait on them later
        const int64_t orow = active ? out_row(perm, first + lane) : 0;
        const float sc = (VT<V>::scaled && active) ? __ldg(scale + first + lane) : 1.0f;
        const int64_t nt = first_extra ? 1 + __ldg(first_extra + g + 1) - __ldg(first_extra + g) : 1;
        const int j0 = (int)(k * C);
        const int jend = min(len, j0 + C);
        const V *vp = val + base + (int64_t)j0 * R + lane;
        const int32_t *cp = col + base + (int64_t)j0 * R + lane;
        A acc = 0;
        if constexpr (CP) {
            int c[U], cn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) c[u] = j0 + u < jend ? ld_stream(cp + (int64_t)u * R) : 0;
            for (int j = j0; j < jend; j += U) {
#pragma unroll
                for (int u = 0; u < U; ++u) cn[u] = j + U + u < jend ? ld_stream(cp + (int64_t)(U + u) * R) : 0;
                A xv[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < jend) xv[u] = __ldg(x + c[u]);
                A v[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < jend) v[u] = VT<V>::ld(vp + (int64_t)u * R);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < jend) acc = fma(v[u], xv[u], acc);
#pragma unroll
                for (int u = 0; u < U; ++u) c[u] = cn[u];
                vp += (int64_t)U * R;
                cp += (int64_t)U * R;
            }
        } else {
            for (int j = j0; j < jend; j += U) {
                A v[U];
                int c[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (j + u < jend) {
                        v[u] = VT<V>::ld(vp + (int64_t)u * R);
                        c[u] = ld_stream(cp + (int64_t)u * R);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < jend) acc = fma(v[u], __ldg(x + c[u]), acc);
                vp += (int64_t)U * R;
                cp += (int64_t)U * R;
            }
        }
        if (nt == 1) {
            if (active) y[orow] = VT<V>::scaled ? acc * sc : acc;
            continue;
        }
        // split group: publish this tile's partials; the last tile to
        // arrive adds them in a fixed order (deterministic) and resets the
        // group's counter for the next launch.
        const int64_t pb = __ldg(part_base + g);
        if (active) partials[(pb + k) * 32 + lane] = acc;
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
            const A s = sum_partials<V>(partials + pb * 32 + lane, nt);
            y[orow] = VT<V>::scaled ? s * sc : s;
        }
        if (lane == 0) arrivals[g] = 0;
    }
}

// The same tiles, software-pipelined across a warp's tasks: while the x
// gathers of one step run, the value/column loads of the next step (the
// next slot-rows of this tile, or the first ones of the warp's next tile)
// are already in flight, and the next tile's metadata is fetched one tile
// ahead.  Results and their summation order are those of the plain kernel.
template <typename V>
struct TileMeta {
    int64_t base, orow, pb;
    int g, k, R, len, nt;       // group indices fit int32 (checked at plan)
    float sc;
};

template <typename V>
__device__ __forceinline__ void tile_meta(int64_t t, int64_t n, int32_t G, int64_t n_groups, int64_t n_tasks,
                                          const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                                          const float *__restrict__ scale, const int64_t *__restrict__ first_extra,
                                          const int64_t *__restrict__ part_base,
                                          const int32_t *__restrict__ extra_group,
                                          const int32_t *__restrict__ perm, int lane, TileMeta<V> &m) {
    m.len = 0;
    m.nt = 1;
    m.R = 0;
    m.base = m.orow = m.pb = m.g = m.k = 0;
    m.sc = 1.0f;
    if (t >= n_tasks) return;
    if (t < n_groups) {
        m.g = (int)t;
    } else {
        m.g = __ldg(extra_group + (t - n_groups));
        m.k = (int)(1 + (t - n_groups) - __ldg(first_extra + m.g));
    }
    const int64_t first = (int64_t)m.g * G;
    m.R = (int)min((int64_t)G, n - first);
    m.base = __ldg(gp + m.g);
    if (lane < m.R) {
        m.len = __ldg(rl + first + lane);
        m.orow = out_row(perm, first + lane);
        if (VT<V>::scaled) m.sc = __ldg(scale + first + lane);
    }
    if (first_extra) {
        m.nt = (int)(1 + __ldg(first_extra + m.g + 1) - __ldg(first_extra + m.g));
        if (m.nt > 1) m.pb = __ldg(part_base + m.g);
    }
}

template <typename V, int U>
__device__ __forceinline__ void tile_loads(const TileMeta<V> &m, int j, int jend, const V *__restrict__ val,
                                           const int32_t *__restrict__ col, int lane,
                                           typename VT<V>::A (&v)[U], int (&c)[U]) {
    const int64_t p0 = m.base + (int64_t)j * m.R + lane;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        v[u] = 0;
        c[u] = 0;
        if (j + u < jend) {
            v[u] = VT<V>::ld(val + p0 + (int64_t)u * m.R);
            c[u] = ld_stream(col + p0 + (int64_t)u * m.R);
        }
    }
}

template <typename V, int U, int MIN_BLOCKS>
__global__ void __launch_bounds__(kTileThreads, MIN_BLOCKS)
rgcsr_spmv_tiles_pipe_kernel(int64_t n, int32_t G, int32_t C, int64_t n_groups, int64_t n_tasks,
                             const V *__restrict__ val, const int32_t *__restrict__ col,
                             const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                             const float *__restrict__ scale, const int64_t *__restrict__ first_extra,
                             const int64_t *__restrict__ part_base, const int32_t *__restrict__ extra_group,
                             int32_t *__restrict__ arrivals, typename VT<V>::A *partials,
                             const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
                             const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    TileMeta<V> cur, nxt;
    tile_meta<V>(t, n, G, n_groups, n_tasks, gp, rl, scale, first_extra, part_base, extra_group, perm, lane, cur);
    tile_meta<V>(t + warps, n, G, n_groups, n_tasks, gp, rl, scale, first_extra, part_base, extra_group, perm,
                 lane, nxt);
    A v[U], vn[U];
    int c[U], cn[U];
    {
        const int j0 = cur.k * C;
        tile_loads<V, U>(cur, j0, min(cur.len, j0 + C), val, col, lane, v, c);
    }
    while (t < n_tasks) {
        const int j0 = cur.k * C;
        const int jend = min(cur.len, j0 + C);
        const int steps = (warp_max_i(jend - j0) + U - 1) / U;      // uniform over the warp
        const int nj0 = nxt.k * C;
        const int njend = min(nxt.len, nj0 + C);
        A acc = 0;
        for (int st = 0; st < steps; ++st) {
            const int j = j0 + st * U;
            if (st + 1 < steps) tile_loads<V, U>(cur, j + U, jend, val, col, lane, vn, cn);
            else tile_loads<V, U>(nxt, nj0, njend, val, col, lane, vn, cn);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u < jend) acc = fma(v[u], __ldg(x + c[u]), acc);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = vn[u];
                c[u] = cn[u];
            }
        }
        if (steps == 0) tile_loads<V, U>(nxt, nj0, njend, val, col, lane, v, c);
        const bool active = lane < cur.R;
        if (cur.nt == 1) {
            if (active) y[cur.orow] = VT<V>::scaled ? acc * cur.sc : acc;
        } else {
            if (active) partials[(cur.pb + cur.k) * 32 + lane] = acc;
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) {
                __threadfence();
                last = atomicAdd(arrivals + cur.g, 1) == cur.nt - 1;
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                if (active) {
                    const A s = sum_partials<V>(partials + cur.pb * 32 + lane, (int64_t)cur.nt);
                    y[cur.orow] = VT<V>::scaled ? s * cur.sc : s;
                }
                if (lane == 0) arrivals[cur.g] = 0;
            }
        }
        t += warps;
        cur = nxt;
        tile_meta<V>(t + warps, n, G, n_groups, n_tasks, gp, rl, scale, first_extra, part_base, extra_group,
                     perm, lane, nxt);
    }
}

// Resident CTAs of `kern` on the whole current device (queried once per
// device and kernel).
template <typename K>
int resident_ctas(K kern, int *cache) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] > 0) return cache[dev];
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTileThreads, 0) != cudaSuccess || occ <= 0)
        occ = 1;
    cache[dev] = sms * occ;
    return cache[dev];
}

template <typename V>
int launch_tiles(const rgcsr_matrix *M, const rgcsr_tiles *T, const typename VT<V>::A *x,
                 typename VT<V>::A *y, cudaStream_t s) {
    using A = typename VT<V>::A;
    const V *val = static_cast<const V *>(M->values);
    if (VT<V>::scaled && !M->row_scale) return RGCSR_ERR_INVALID_ARG;
    const int64_t n_tasks = M->n_groups + T->n_extra;
    // slot-rows in flight per lane (U) and CTAs per SM by variant:
    // 0: U = 8 (FP64: 4), 5 CTAs;  1: U = 4 (FP64: 2), 6 CTAs;  2: U = 16 (FP64: 8), 4 CTAs;
    // 3, 4: software-pipelined, U = 4 (FP64: 2) with 4 CTAs, U = 8 (FP64: 4) with 3 CTAs;
    // 5: software-pipelined, U = 16 (FP64: 8) with 2 CTAs;
    // 6, 7: each step's columns loaded one step ahead, U = 8 with 3 CTAs, U = 8 (FP64: 4) with 4
    constexpr int U0 = sizeof(A) == 8 ? 4 : 8;
    void (*kern)(int64_t, int32_t, int32_t, int64_t, int64_t, const V *, const int32_t *, const int64_t *,
                 const int32_t *, const float *, const int64_t *, const int64_t *, const int32_t *, int32_t *,
                 A *, const A *, A *, const int32_t *);
    static int cache[8][64];
    int *cc;
    switch (T->variant) {
        case 0: kern = rgcsr_spmv_tiles_kernel<V, U0, 5>; cc = cache[0]; break;
        case 1: kern = rgcsr_spmv_tiles_kernel<V, U0 / 2, 6>; cc = cache[1]; break;
        case 2: kern = rgcsr_spmv_tiles_kernel<V, 2 * U0, 4>; cc = cache[2]; break;
        case 3: kern = rgcsr_spmv_tiles_pipe_kernel<V, U0 / 2, 4>; cc = cache[3]; break;
        case 4: kern = rgcsr_spmv_tiles_pipe_kernel<V, U0, 3>; cc = cache[4]; break;
        case 5: kern = rgcsr_spmv_tiles_pipe_kernel<V, 2 * U0, 2>; cc = cache[5]; break;
        case 6: kern = rgcsr_spmv_tiles_kernel<V, 8, 3, true>; cc = cache[6]; break;
        case 7: kern = rgcsr_spmv_tiles_kernel<V, U0, 4, true>; cc = cache[7]; break;
        default: return RGCSR_ERR_INVALID_ARG;
    }
    int64_t grid = resident_ctas(kern, cc);                                 // persistent
    const int64_t need = ceil_div(n_tasks, kTileThreads / 32);
    if (need < grid) grid = need;
    kern<<<(unsigned)grid, kTileThreads, 0, s>>>(
        M->n_rows, M->group_size, T->tile, M->n_groups, n_tasks, val, M->columns, M->group_ptr,
        M->row_lengths, M->row_scale, T->n_extra > 0 ? T->first_extra : nullptr, T->part_base,
        T->extra_group, T->arrivals, static_cast<A *>(T->partials), x, y, M->row_perm);
    return launch_status();
}

int check_tiles_matrix(const rgcsr_matrix *M) {
    if (!M || M->n_rows < 0 || M->group_size < 1 || M->group_size > 32) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows > 0 && (!M->group_ptr || !M->row_lengths)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_stored > 0 && (!M->values || !M->columns)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups > (int64_t)INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t rgcsr_tiles_workspace_bytes(int64_t n_groups) {
    if (n_groups < 0) return 0;
    return scan_partials_bytes(n_groups);
}

RGCSR_API int rgcsr_tiles_plan(const rgcsr_matrix *M, rgcsr_tiles *T, void *workspace,
                               size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_tiles_matrix(M);
    if (st != RGCSR_OK) return st;
    if (!T || T->tile < 1) return RGCSR_ERR_INVALID_ARG;
    const int64_t ng = M->n_groups;
    T->n_groups = ng;
    T->n_extra = T->n_split = T->n_partials = 0;
    if (ng == 0) return RGCSR_OK;
    if (!T->first_extra || !T->part_base) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_tiles_workspace_bytes(ng)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *scratch = static_cast<int64_t *>(workspace);
    tile_count_kernel<<<(unsigned)ceil_div(ng, 256), 256, 0, s>>>(M->n_rows, M->group_size, ng, M->group_ptr,
                                                                  T->tile, T->first_extra, T->part_base);
    if ((st = launch_status()) != RGCSR_OK) return st;
    if ((st = exclusive_scan_i64(T->first_extra, ng, scratch, s)) != RGCSR_OK) return st;
    if ((st = exclusive_scan_i64(T->part_base, ng, scratch, s)) != RGCSR_OK) return st;
    int64_t tot[2] = {0, 0};
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&tot[0], T->first_extra + ng, 8, cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&tot[1], T->part_base + ng, 8, cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    T->n_extra = tot[0];
    T->n_partials = tot[1];
    T->n_split = tot[1] - tot[0];            // each split group has one task besides its extras
    if (ng + tot[0] > (int64_t)INT32_MAX * 32) return RGCSR_ERR_INDEX_OVERFLOW;
    return RGCSR_OK;
}

RGCSR_API int rgcsr_tiles_build(const rgcsr_matrix *M, const rgcsr_tiles *T, rgcsr_stream_t stream) {
    int st = check_tiles_matrix(M);
    if (st != RGCSR_OK) return st;
    if (!T || T->tile < 1 || T->n_groups != M->n_groups) return RGCSR_ERR_INVALID_ARG;
    if (T->n_extra == 0 || M->n_groups == 0) return RGCSR_OK;
    if (!T->first_extra || !T->part_base || !T->extra_group || !T->arrivals) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    RGCSR_CUDA_TRY(cudaMemsetAsync(T->arrivals, 0, (size_t)M->n_groups * sizeof(int32_t), s));
    tile_fill_kernel<<<(unsigned)ceil_div(M->n_groups, 256), 256, 0, s>>>(M->n_groups, T->first_extra,
                                                                         T->extra_group);
    return launch_status();
}

RGCSR_API int rgcsr_spmv_tiles(const rgcsr_matrix *M, const rgcsr_tiles *T, const void *x, void *y,
                               rgcsr_stream_t stream) {
    int st = check_tiles_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!T || T->tile < 1 || T->n_groups != M->n_groups || !y || (M->n_cols > 0 && !x))
        return RGCSR_ERR_INVALID_ARG;
    if (T->n_extra > 0 && (!T->first_extra || !T->part_base || !T->extra_group || !T->arrivals || !T->partials))
        return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64:
            return launch_tiles<double>(M, T, static_cast<const double *>(x), static_cast<double *>(y), s);
        case RGCSR_F32:
            return launch_tiles<float>(M, T, static_cast<const float *>(x), static_cast<float *>(y), s);
        case RGCSR_BF16:
            return launch_tiles<__nv_bfloat16>(M, T, static_cast<const float *>(x), static_cast<float *>(y), s);
        case RGCSR_F16:
            return launch_tiles<__half>(M, T, static_cast<const float *>(x), static_cast<float *>(y), s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}
