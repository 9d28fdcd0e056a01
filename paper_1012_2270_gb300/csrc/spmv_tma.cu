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
    return M->group_size == 32 && (M->value_type == RGCSR_F32 || M->value_type == RGCSR_F64) &&
           M->n_rows >= 32 && M->n_groups <= (int64_t)INT32_MAX && aligned(M->values) &&
           aligned(M->columns) && aligned(M->row_lengths);
}

int launch_spmv_tma(const rgcsr_matrix *M, const void *x, void *y, int variant, uint32_t wait_limit,
                    cudaStream_t s) {
    if (!tma_eligible(M)) return RGCSR_ERR_INVALID_ARG;
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
    return RGCSR_OK;
}
