// spmv_tma.cu -- RgCSR SpMV for group size 32 with the group slabs staged in
// shared memory by the bulk-copy engine (TMA, cp.async.bulk).
//
// With G = 32 a group's j-th slot-row (the j-th entries of its 32 rows,
// Sec. 3.4) is one 128 B line of `values` (256 B for FP64) and one of
// `columns`, and the whole slab [group_ptr[g], group_ptr[g+1]) is contiguous
// and 128 B aligned.  So a warp fetches a group -- or a chunk of up to CAP
// slot-rows of it -- with three bulk copies (values, columns, the 32 row
// lengths) and no per-thread address arithmetic.
//
// Persistent grid: every CTA that fits on an SM (by shared memory and
// registers) is resident; each warp owns a contiguous range of full 32-row
// groups and runs a private ring of STAGES shared-memory stages that lane 0
// keeps filled, each stage guarded by an mbarrier with a transaction count.
// The warp waits for its oldest chunk, reads values and columns from shared
// memory, gathers x[col] through the read-only path for the valid slots only
// (j < rowLength: padding is never touched), refills the stage with the next
// chunk, sums, and stores y after a group's last chunk.  Every wait is
// bounded; on timeout the kernel records RGCSR_STATUS_TIMEOUT, drains its own
// copies (again bounded) and returns.
#include "common.cuh"
#include "ptx.cuh"
#include "vtraits.cuh"

#include <mutex>

namespace rgcsr {
namespace {

__device__ int g_spmv_status;     // sticky error bits, read by rgcsr_get_status

constexpr int kTmaWarps = 8;
constexpr uint32_t kSpinLimit = 1u << 26;   // non-blocking probes per wait (~1 s at most)

// CAP slot-rows per chunk, STAGES chunks in each warp's ring.
template <typename T, int CAP, int STAGES>
struct TmaCfg {
    static constexpr int VAL_BYTES = CAP * 32 * (int)sizeof(T);
    static constexpr int COL_BYTES = CAP * 32 * 4;
    static constexpr int STAGE_BYTES = VAL_BYTES + COL_BYTES + 128;  // + 32 row lengths
    static constexpr int WARP_BYTES = STAGES * STAGE_BYTES;
    static constexpr int SMEM = kTmaWarps * WARP_BYTES;
};

// One warp's producer side: walks the warp's groups [pb, b1) chunk by chunk
// (warp-uniform state) and issues the bulk copies from lane 0.
template <typename T, int CAP, int STAGES>
struct SlabRing {
    using C = TmaCfg<T, CAP, STAGES>;
    const T *val;
    const int32_t *col;
    const int64_t *gp;
    const int32_t *rl;
    int64_t nb_full;
    unsigned char *ring;
    uint64_t *bars;
    int4 *meta;            // per stage: (group, first slot-row, rows, last)
    int lane;
    uint64_t pol;
    int64_t pb, b1;        // next group to issue, end of range
    int pj;                // next slot-row within pb
    int64_t win, gpw, gpw_end;   // group_ptr window: lane i holds gp[win + i]
    int issued;

    __device__ void load_window(int64_t base) {
        win = base;
        gpw = gp[min(base + lane, nb_full)];
        gpw_end = gp[min(base + 32, nb_full)];
    }
    __device__ int64_t gp_at(int64_t b) const {
        const int64_t v = shfl_i64(gpw, (int)min(b - win, (int64_t)31));
        return (b - win < 32) ? v : gpw_end;
    }
    // Issues the next chunk into stage s; warp-uniform; false when done.
    __device__ bool issue(int s) {
        if (pb >= b1) return false;
        if (pb + 1 > win + 32) load_window(pb);
        const int64_t g0 = gp_at(pb), g1 = gp_at(pb + 1);
        const int K = (int)((g1 - g0) >> 5);
        const int rows = min(CAP, K - pj);
        const bool last = pj + rows >= K;
        if (lane == 0) {
            unsigned char *st = ring + (size_t)s * C::STAGE_BYTES;
            const uint32_t vb = (uint32_t)rows * 32 * sizeof(T), cb = (uint32_t)rows * 128;
            meta[s] = make_int4((int)pb, pj, rows, last ? 1 : 0);
            ptx::mbar_arrive_expect_tx(&bars[s], vb + cb + 128);
            const int64_t off = g0 + (int64_t)pj * 32;
            if (rows > 0) {
                ptx::bulk_g2s(st, val + off, vb, &bars[s], pol);
                ptx::bulk_g2s(st + C::VAL_BYTES, col + off, cb, &bars[s], pol);
            }
            ptx::bulk_g2s(st + C::VAL_BYTES + C::COL_BYTES, rl + pb * 32, 128, &bars[s], pol);
        }
        pj += rows;
        if (last) { ++pb; pj = 0; }
        ++issued;
        return true;
    }
    // Probes chunk k's stage (its (k / STAGES)-th completion: the warp never
    // waits more than one phase ahead, since it consumes its own chunks in
    // order) at most `limit` times; the whole warp takes the same decision.
    __device__ bool probe(int k, uint32_t limit) const {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)(k / STAGES) & 1u;
        for (uint32_t t = 0; t < limit; ++t)
            if (__all_sync(0xffffffffu, ptx::mbar_test_wait(&bars[s], parity))) return true;
        return false;
    }
    // Bounded wait for chunk k; false after `limit` probes, with the error
    // recorded and every copy of this warp still in flight -- chunk k's own
    // and the ones issued after it -- waited for (default bound) before the
    // warp ends, so none lands in shared memory after the warp has gone.
    __device__ bool wait(int k, uint32_t limit) {
        if (probe(k, limit)) return true;
        if (lane == 0) atomicOr(&g_spmv_status, RGCSR_STATUS_TIMEOUT);
        for (int k2 = k; k2 < issued; ++k2) (void)probe(k2, kSpinLimit);
        return false;
    }
    __device__ const unsigned char *stage(int k) const { return ring + (size_t)(k % STAGES) * C::STAGE_BYTES; }
    // After the warp has read stage k: order the reads before the async
    // proxy's refill, then refill it with the next chunk.
    __device__ void release(int k) {
        __syncwarp();
        if (lane == 0) ptx::fence_proxy_async_smem();
        issue(k % STAGES);
    }
};

// The partial last group (n not a multiple of 32) by plain loads.
template <typename T>
__device__ void tail_group(int64_t n, int64_t nb_full, const T *val, const int32_t *col,
                           const int64_t *gp, const int32_t *rl, const T *x, T *y, const int32_t *perm,
                           int lane) {
    const int64_t row = nb_full * 32 + lane;
    const int R = (int)(n - nb_full * 32);
    if (row < n) {
        int64_t p = gp[nb_full] + lane;
        const int L = rl[row];
        T a = 0;
        for (int j = 0; j < L; ++j, p += R) a = fma(val[p], __ldg(x + col[p]), a);
        y[out_row(perm, row)] = a;
    }
}

template <typename T, int CAP, int STAGES>
__global__ void __launch_bounds__(kTmaWarps * 32)
rgcsr_spmv_tma(int64_t n, int64_t nb_full, const T *__restrict__ val, const int32_t *__restrict__ col,
               const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
               const T *__restrict__ x, T *__restrict__ y, const int32_t *__restrict__ perm,
               uint32_t wait_limit) {
    using C = TmaCfg<T, CAP, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kTmaWarps][STAGES];
    __shared__ int4 meta[kTmaWarps][STAGES];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kTmaWarps + w;
    const int64_t tw = (int64_t)gridDim.x * kTmaWarps;

    if (lane == 0)
        for (int s = 0; s < STAGES; ++s) ptx::mbar_init(&bars[w][s], 1);
    ptx::fence_mbar_init();
    __syncwarp();

    SlabRing<T, CAP, STAGES> R;
    R.val = val; R.col = col; R.gp = gp; R.rl = rl; R.nb_full = nb_full;
    R.ring = smem + (size_t)w * C::WARP_BYTES; R.bars = bars[w]; R.meta = meta[w]; R.lane = lane;
    R.pol = ptx::policy_evict_first();
    R.pb = nb_full * gw / tw;
    R.b1 = nb_full * (gw + 1) / tw;
    R.pj = 0;
    R.win = R.pb; R.gpw = 0; R.gpw_end = 0;
    R.issued = 0;
    if (R.pb < R.b1) R.load_window(R.pb);
    for (int s = 0; s < STAGES; ++s)
        if (!R.issue(s)) break;

    T acc = 0;
    for (int it = 0; it < R.issued; ++it) {
        if (!R.wait(it, wait_limit)) return;
        __syncwarp();
        const int4 m = R.meta[it % STAGES];
        const unsigned char *st = R.stage(it);
        const T *sv = reinterpret_cast<const T *>(st);
        const int32_t *sc = reinterpret_cast<const int32_t *>(st + C::VAL_BYTES);
        const int len = reinterpret_cast<const int32_t *>(st + C::VAL_BYTES + C::COL_BYTES)[lane];
        const int cnt = max(0, min(m.z, len - m.y));      // valid slot-rows of this lane's row
        T v[CAP], xv[CAP];
#pragma unroll
        for (int u = 0; u < CAP; ++u) {
            if (u < cnt) {
                v[u] = sv[u * 32 + lane];
                xv[u] = __ldg(x + sc[u * 32 + lane]);
            }
        }
        R.release(it);
#pragma unroll
        for (int u = 0; u < CAP; ++u)
            if (u < cnt) acc = fma(v[u], xv[u], acc);
        if (m.w) {
            y[out_row(perm, (int64_t)m.x * 32 + lane)] = acc;
            acc = 0;
        }
    }
    if (gw == tw - 1 && nb_full * 32 < n) tail_group(n, nb_full, val, col, gp, rl, x, y, perm, lane);
}

// ---------------------------------------------------------------------------
// Multi-group chunks.  A full group's slab is contiguous and so are
// consecutive groups' slabs, so one bulk copy (per array) can carry several
// whole groups: a chunk packs consecutive groups while their slot-rows fit
// in CAP (and there are at most MAXG of them); a group longer than CAP is
// copied in pieces of CAP slot-rows as above.  Short-row matrices (a 7-point
// stencil has 7 slot-rows per group) then move 4 KB and more per copy, and
// the STAGES-deep ring keeps that many bytes in flight per warp whatever the
// registers allow.  Any value type: reduced storage (BF16/FP16) multiplies by
// the row's scale at the end.  The consumer takes a group's slot-row count
// as the warp maximum of its row lengths (that is K_g by definition).
// ---------------------------------------------------------------------------
template <typename V, int CAP, int STAGES, int WARPS>
struct MultiCfg {
    static constexpr int MAXG = 16;
    static constexpr int VAL_BYTES = CAP * 32 * (int)sizeof(V);
    static constexpr int COL_BYTES = CAP * 32 * 4;
    static constexpr int RL_BYTES = MAXG * 32 * 4;
    static constexpr int KS_BYTES = 128;            // the packed groups' slot-row counts
    static constexpr int STAGE_BYTES = VAL_BYTES + COL_BYTES + RL_BYTES + KS_BYTES;
    static constexpr int WARP_BYTES = STAGES * STAGE_BYTES;
    static constexpr int SMEM = WARPS * WARP_BYTES;
    static_assert(VAL_BYTES % 128 == 0 && MAXG < 32 && MAXG * 4 <= KS_BYTES, "stage layout");
};

template <typename V, int CAP, int STAGES, int WARPS>
struct MultiRing {
    using C = MultiCfg<V, CAP, STAGES, WARPS>;
    const V *val;
    const int32_t *col;
    const int64_t *gp;
    const int32_t *rl;
    int64_t nb_full;
    unsigned char *ring;
    uint64_t *bars;
    int4 *meta;            // per stage: (first group, first slot-row, slot-rows, groups << 1 | last)
    int lane;
    uint64_t pol;
    int64_t pb, b1;
    int pj;
    int64_t win, gpw, gpw_end;
    int issued;

    __device__ void load_window(int64_t base) {
        win = base;
        gpw = gp[min(base + lane, nb_full)];
        gpw_end = gp[min(base + 32, nb_full)];
    }
    __device__ int64_t gp_at(int64_t b) const {      // b in [win, win + 32]
        const int64_t v = shfl_i64(gpw, (int)min(b - win, (int64_t)31));
        return (b - win < 32) ? v : gpw_end;
    }
    __device__ bool issue(int s) {
        if (pb >= b1) return false;
        if (pb + C::MAXG > win + 32) load_window(pb);
        const int64_t g0 = gp_at(pb);
        const int K0 = (int)((gp_at(pb + 1) - g0) >> 5);
        int rows, ng = 1;
        bool last;
        unsigned char *st = ring + (size_t)s * C::STAGE_BYTES;
        int *ks = reinterpret_cast<int *>(st + C::VAL_BYTES + C::COL_BYTES + C::RL_BYTES);
        if (pj > 0 || K0 > CAP) {
            rows = min(CAP, K0 - pj);
            last = pj + rows >= K0;
        } else {
            rows = K0;
            if (lane == 0) ks[0] = K0;
            while (ng < C::MAXG && pb + ng < b1) {
                const int Kn = (int)((gp_at(pb + ng + 1) - gp_at(pb + ng)) >> 5);
                if (rows + Kn > CAP) break;
                if (lane == 0) ks[ng] = Kn;
                rows += Kn;
                ++ng;
            }
            last = true;
        }
        if (lane == 0) {
            const uint32_t vb = (uint32_t)rows * 32 * sizeof(V), cb = (uint32_t)rows * 128, rb = (uint32_t)ng * 128;
            meta[s] = make_int4((int)pb, pj, rows, (ng << 1) | (last ? 1 : 0));
            ptx::mbar_arrive_expect_tx(&bars[s], vb + cb + rb);
            const int64_t off = g0 + (int64_t)pj * 32;
            if (rows > 0) {
                ptx::bulk_g2s(st, val + off, vb, &bars[s], pol);
                ptx::bulk_g2s(st + C::VAL_BYTES, col + off, cb, &bars[s], pol);
            }
            ptx::bulk_g2s(st + C::VAL_BYTES + C::COL_BYTES, rl + pb * 32, rb, &bars[s], pol);
        }
        if (ng == 1 && !last) {
            pj += rows;
        } else {
            pb += ng;
            pj = 0;
        }
        ++issued;
        return true;
    }
    __device__ bool probe(int k, uint32_t limit) const {
        const int s = k % STAGES;
        const uint32_t parity = (uint32_t)(k / STAGES) & 1u;
        for (uint32_t t = 0; t < limit; ++t)
            if (__all_sync(0xffffffffu, ptx::mbar_test_wait(&bars[s], parity))) return true;
        return false;
    }
    // As SlabRing::wait: bounded, and on timeout every copy of this warp
    // still in flight (chunk k's included) is waited for before the warp ends.
    __device__ bool wait(int k, uint32_t limit) {
        if (probe(k, limit)) return true;
        if (lane == 0) atomicOr(&g_spmv_status, RGCSR_STATUS_TIMEOUT);
        for (int k2 = k; k2 < issued; ++k2) (void)probe(k2, kSpinLimit);
        return false;
    }
    __device__ const unsigned char *stage(int k) const { return ring + (size_t)(k % STAGES) * C::STAGE_BYTES; }
    __device__ void release(int k) {
        __syncwarp();
        if (lane == 0) ptx::fence_proxy_async_smem();
        issue(k % STAGES);
    }
};

// Slot-rows [0, K) of one group from a stage (values sv, columns sc, both
// with 32-element slot-rows), this lane's row of length len: eight gathers
// in flight per step.
template <typename V>
__device__ __forceinline__ typename VT<V>::A stage_rows(const V *sv, const int32_t *sc, int K, int len, int lane,
                                                       const typename VT<V>::A *__restrict__ x,
                                                       typename VT<V>::A acc) {
    using A = typename VT<V>::A;
    for (int u0 = 0; u0 < K; u0 += 8) {
        A v[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u0 + u < len) {
                const V e = sv[(u0 + u) * 32 + lane];
                if constexpr (VT<V>::scaled) v[u] = VT<V>::to_float(e);
                else v[u] = e;
                xv[u] = __ldg(x + sc[(u0 + u) * 32 + lane]);
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u0 + u < len) acc = fma(v[u], xv[u], acc);
    }
    return acc;
}

// The partial last group (R_g < 32 rows, slot stride R_g) by plain loads.
template <typename V>
__device__ void tail_group_v(int64_t n, int64_t nb_full, const V *val, const int32_t *col, const int64_t *gp,
                             const int32_t *rl, const float *scale, const typename VT<V>::A *x,
                             typename VT<V>::A *y, const int32_t *perm, int lane) {
    using A = typename VT<V>::A;
    const int64_t row = nb_full * 32 + lane;
    const int R = (int)(n - nb_full * 32);
    if (row < n) {
        int64_t p = gp[nb_full] + lane;
        const int L = rl[row];
        A a = 0;
        for (int j = 0; j < L; ++j, p += R) a = fma(VT<V>::ld(val + p), __ldg(x + col[p]), a);
        y[out_row(perm, row)] = finish<V>(a, scale, row);
    }
}

template <typename V, int CAP, int STAGES, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
rgcsr_spmv_tma_multi(int64_t n, int64_t nb_full, const V *__restrict__ val, const int32_t *__restrict__ col,
                     const int64_t *__restrict__ gp, const int32_t *__restrict__ rl, const float *__restrict__ scale,
                     const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
                     const int32_t *__restrict__ perm, uint32_t wait_limit) {
    using A = typename VT<V>::A;
    using C = MultiCfg<V, CAP, STAGES, WARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[WARPS][STAGES];
    __shared__ int4 meta[WARPS][STAGES];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + w;
    const int64_t tw = (int64_t)gridDim.x * WARPS;

    if (lane == 0)
        for (int s = 0; s < STAGES; ++s) ptx::mbar_init(&bars[w][s], 1);
    ptx::fence_mbar_init();
    __syncwarp();

    MultiRing<V, CAP, STAGES, WARPS> R;
    R.val = val; R.col = col; R.gp = gp; R.rl = rl; R.nb_full = nb_full;
    R.ring = smem + (size_t)w * C::WARP_BYTES; R.bars = bars[w]; R.meta = meta[w]; R.lane = lane;
    R.pol = ptx::policy_evict_first();
    R.pb = nb_full * gw / tw;
    R.b1 = nb_full * (gw + 1) / tw;
    R.pj = 0;
    R.win = R.pb; R.gpw = 0; R.gpw_end = 0;
    R.issued = 0;
    if (R.pb < R.b1) R.load_window(R.pb);
    for (int s = 0; s < STAGES; ++s)
        if (!R.issue(s)) break;

    A acc = 0;
    for (int it = 0; it < R.issued; ++it) {
        if (!R.wait(it, wait_limit)) return;
        __syncwarp();
        const int4 m = R.meta[it % STAGES];
        const int ng = m.w >> 1;
        const unsigned char *st = R.stage(it);
        const V *sv = reinterpret_cast<const V *>(st);
        const int32_t *sc = reinterpret_cast<const int32_t *>(st + C::VAL_BYTES);
        const int32_t *srl = reinterpret_cast<const int32_t *>(st + C::VAL_BYTES + C::COL_BYTES);
        if (ng == 1) {                        // one group, or a piece of a long one
            const int len = srl[lane];
            const int cnt = max(0, min(m.z, len - m.y));
            acc = stage_rows<V>(sv, sc, m.z, cnt, lane, x, acc);
            if (m.w & 1) {
                const int64_t row = (int64_t)m.x * 32 + lane;
                y[out_row(perm, row)] = finish<V>(acc, scale, row);
                acc = 0;
            }
        } else {                              // several whole groups, walked slot-row by slot-row
            const int *ks = reinterpret_cast<const int *>(st + C::VAL_BYTES + C::COL_BYTES + C::RL_BYTES);
            for (int q = 0; q < ng; ++q)      // groups with no entries at all: y = 0
                if (ks[q] == 0) {
                    const int64_t row = ((int64_t)m.x + q) * 32 + lane;
                    y[out_row(perm, row)] = finish<V>(A(0), scale, row);
                }
            int q = 0, j = 0, K = ks[0], len = srl[lane];
            int q2 = 0, j2 = 0, K2 = ks[0];
            A sum = 0;
            // halves of H slot-rows: every gather of a half is issued before
            // any of its products, then the products are added in slot order
            // and a group's result is stored where its last slot-row ends
            constexpr int H = 16;
            for (int u0 = 0; u0 < m.z; u0 += H) {
                A v[H], xv[H];
                unsigned valid = 0;
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    if (u0 + u < m.z) {
                        while (j == K) { ++q; j = 0; K = ks[q]; len = srl[q * 32 + lane]; }
                        if (j < len) {
                            const V e = sv[(u0 + u) * 32 + lane];
                            if constexpr (VT<V>::scaled) v[u] = VT<V>::to_float(e);
                            else v[u] = e;
                            xv[u] = __ldg(x + sc[(u0 + u) * 32 + lane]);
                            valid |= 1u << u;
                        }
                        ++j;
                    }
                }
#pragma unroll
                for (int u = 0; u < H; ++u) {
                    if (u0 + u < m.z) {
                        while (j2 == K2) { ++q2; j2 = 0; K2 = ks[q2]; }
                        if (valid >> u & 1u) sum = fma(v[u], xv[u], sum);
                        if (++j2 == K2) {
                            const int64_t row = ((int64_t)m.x + q2) * 32 + lane;
                            y[out_row(perm, row)] = finish<V>(sum, scale, row);
                            sum = 0;
                        }
                    }
                }
            }
        }
        R.release(it);
    }
    if (gw == tw - 1 && nb_full * 32 < n) tail_group_v<V>(n, nb_full, val, col, gp, rl, scale, x, y, perm, lane);
}

int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

template <typename T, int CAP, int STAGES>
int launch_tma_cfg(const rgcsr_matrix *M, const T *x, T *y, uint32_t wait_limit, cudaStream_t s) {
    using C = TmaCfg<T, CAP, STAGES>;
    auto kern = rgcsr_spmv_tma<T, CAP, STAGES>;
    static std::once_flag once[64];
    static int ctas_per_sm[64];
    static cudaError_t setup_err[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RGCSR_ERR_CUDA;
    std::call_once(once[dev], [&] {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        int occ = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaWarps * 32, C::SMEM);
        ctas_per_sm[dev] = occ > 0 ? occ : 1;
        setup_err[dev] = e;
    });
    if (setup_err[dev] != cudaSuccess) return RGCSR_ERR_CUDA;
    const int64_t nb_full = M->n_rows / 32;
    int64_t grid = (int64_t)sm_count() * ctas_per_sm[dev];      // persistent: all CTAs resident
    const int64_t need = ceil_div(nb_full, kTmaWarps);
    if (need < grid) grid = need > 0 ? need : 1;
    kern<<<(unsigned)grid, kTmaWarps * 32, C::SMEM, s>>>(
        M->n_rows, nb_full, static_cast<const T *>(M->values), M->columns, M->group_ptr,
        M->row_lengths, x, y, M->row_perm, wait_limit ? wait_limit : kSpinLimit);
    return launch_status();
}

template <typename V, int CAP, int STAGES, int WARPS>
int launch_tma_multi(const rgcsr_matrix *M, const void *x, void *y, uint32_t wait_limit, cudaStream_t s) {
    using C = MultiCfg<V, CAP, STAGES, WARPS>;
    using A = typename VT<V>::A;
    if (VT<V>::scaled && !M->row_scale) return RGCSR_ERR_INVALID_ARG;
    auto kern = rgcsr_spmv_tma_multi<V, CAP, STAGES, WARPS>;
    static std::once_flag once[64];
    static int ctas_per_sm[64];
    static cudaError_t setup_err[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RGCSR_ERR_CUDA;
    std::call_once(once[dev], [&] {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        int occ = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WARPS * 32, C::SMEM);
        ctas_per_sm[dev] = occ > 0 ? occ : 1;
        setup_err[dev] = e;
    });
    if (setup_err[dev] != cudaSuccess) return RGCSR_ERR_CUDA;
    const int64_t nb_full = M->n_rows / 32;
    int64_t grid = (int64_t)sm_count() * ctas_per_sm[dev];
    const int64_t need = ceil_div(nb_full, WARPS);
    if (need < grid) grid = need > 0 ? need : 1;
    kern<<<(unsigned)grid, WARPS * 32, C::SMEM, s>>>(
        M->n_rows, nb_full, static_cast<const V *>(M->values), M->columns, M->group_ptr, M->row_lengths,
        M->row_scale, static_cast<const A *>(x), static_cast<A *>(y), M->row_perm,
        wait_limit ? wait_limit : kSpinLimit);
    return launch_status();
}

// Multi-group rings (slot-rows per chunk, stages, warps per CTA): variant 4
// = (32, 2, 4), 5 = (32, 3, 4), 6 = (16, 4, 4); every value type (FP64 at
// most 172 KB of shared memory per CTA).
template <typename V>
int launch_tma_multi_t(const rgcsr_matrix *M, const void *x, void *y, int variant, uint32_t wl, cudaStream_t s) {
    switch (variant) {
        case 4: return launch_tma_multi<V, 32, 2, 4>(M, x, y, wl, s);
        case 5: return launch_tma_multi<V, 32, 3, 4>(M, x, y, wl, s);
        case 6: return launch_tma_multi<V, 16, 4, 4>(M, x, y, wl, s);
        default: return RGCSR_ERR_INVALID_ARG;
    }
}

// Ring configurations (slot-rows per chunk, stages), selectable for tuning.
template <typename T>
int launch_tma_t(const rgcsr_matrix *M, const T *x, T *y, int variant, uint32_t wl, cudaStream_t s) {
    switch (variant) {
        case 0: return launch_tma_cfg<T, 8, 2>(M, x, y, wl, s);
        case 1: return launch_tma_cfg<T, 8, 4>(M, x, y, wl, s);
        case 2: return launch_tma_cfg<T, 16, 2>(M, x, y, wl, s);
        case 3: return launch_tma_cfg<T, 4, 4>(M, x, y, wl, s);
        default: return RGCSR_ERR_INVALID_ARG;
    }
}

}  // namespace

bool tma_eligible(const rgcsr_matrix *M) {
    auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    // (the ring's stage records hold group indices as int)
    return M->group_size == 32 && M->value_type >= RGCSR_F64 && M->value_type <= RGCSR_F16 &&
           M->n_rows >= 32 && M->n_groups <= (int64_t)INT32_MAX && aligned(M->values) &&
           aligned(M->columns) && aligned(M->row_lengths);
}

int launch_spmv_tma(const rgcsr_matrix *M, const void *x, void *y, int variant, uint32_t wait_limit,
                    cudaStream_t s) {
    if (!tma_eligible(M)) return RGCSR_ERR_INVALID_ARG;
    if (variant >= 4) {
        switch (M->value_type) {
            case RGCSR_F64: return launch_tma_multi_t<double>(M, x, y, variant, wait_limit, s);
            case RGCSR_F32: return launch_tma_multi_t<float>(M, x, y, variant, wait_limit, s);
            case RGCSR_BF16: return launch_tma_multi_t<__nv_bfloat16>(M, x, y, variant, wait_limit, s);
            default: return launch_tma_multi_t<__half>(M, x, y, variant, wait_limit, s);
        }
    }
    if (M->value_type == RGCSR_BF16 || M->value_type == RGCSR_F16) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (M->value_type == RGCSR_F64)
        return launch_tma_t<double>(M, static_cast<const double *>(x), static_cast<double *>(y), variant,
                                    wait_limit, s);
    return launch_tma_t<float>(M, static_cast<const float *>(x), static_cast<float *>(y), variant, wait_limit,
                               s);
}

}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_get_status(int *status_out, rgcsr_stream_t stream) {
    if (!status_out) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int zero = 0;
    RGCSR_CUDA_TRY(cudaMemcpyFromSymbolAsync(status_out, g_spmv_status, sizeof(int), 0,
                                             cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    RGCSR_CUDA_TRY(cudaMemcpyToSymbolAsync(g_spmv_status, &zero, sizeof(int), 0,
                                           cudaMemcpyHostToDevice, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    *status_out |= take_host_status();
    return RGCSR_OK;
}
