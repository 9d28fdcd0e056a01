// spmv.cu -- y = A x for a matrix in Row-grouped CSR (Sec. 3.4 of the paper).
//
// Kernels here (the TMA-staged kernel for G = 32 is in spmv_tma.cu):
//  * rgcsr_spmv_paper: the paper's mapping -- one block per group, one thread
//    per row, the row's slots visited with stride R_g (currentGroupSize).
//  * rgcsr_spmv_split: one thread per row, but a warp first agrees on a
//    split slot j0.  Every row runs its slots [0, j0) on its own thread
//    (coalesced: the j-th slots of a group's rows are adjacent), and the
//    slots [j0, len) of the few rows longer than j0 are then finished by the
//    whole warp, one row at a time, with a shuffle reduction.  A warp whose
//    rows have similar lengths skips the split logic (j0 = its longest row).
//    This removes the paper's weak point, where one very long row in a
//    group serialises its warp (Sec. 4.4.2, Table 6: trans4 and Raj1).
//  * rgcsr_spmv_lean: one thread per row, no split, sized for full
//    occupancy; for matrices whose rows in a warp have similar lengths.
//  * sliced_ell_spmv: the sliced ELLPACK comparator on the same slabs.
//
// Value storage V is double, float, or (reduced storage, not in the paper)
// bfloat16 / half with a per-row float scale: y_i = s_i * sum_j q_ij x_j
// with x, y and the sum in float.
//
// Loads: value and column slabs are streamed once (evict-first); x is read
// through the read-only path so it stays cached for reuse (the paper's
// texture binding of x, Sec. 3.4 and Sec. 4.3).
#include "common.cuh"
#include "vtraits.cuh"
#include <climits>
#include <type_traits>

namespace rgcsr {
namespace {

constexpr int kDefaultThreads = 256;
constexpr int kUnroll = 8;          // slots in flight per thread

// x[c] through the chosen read path XL: the read-only (non-coherent) path
// (RGCSR_XLOAD_NC), an ordinary load (RGCSR_XLOAD_PLAIN), or a texture fetch
// from a texture object bound to x (RGCSR_XLOAD_TEX) -- the read paths of
// the paper's texture study (Sec. 4.3) on this architecture.
template <typename A, int XL>
__device__ __forceinline__ A gather(const A *x, cudaTextureObject_t tex, int c) {
    if constexpr (XL == RGCSR_XLOAD_NC) {
        return __ldg(x + c);
    } else if constexpr (XL == RGCSR_XLOAD_PLAIN) {
        return x[c];
    } else if constexpr (sizeof(A) == 8) {
        const int2 v = tex1Dfetch<int2>(tex, c);
        return __hiloint2double(v.y, v.x);
    } else {
        return tex1Dfetch<float>(tex, c);
    }
}

template <typename T, int XL>
__global__ void rgcsr_spmv_paper(int64_t n, int32_t G, const T *__restrict__ val,
                                 const int32_t *__restrict__ col, const int64_t *__restrict__ gp,
                                 const int32_t *__restrict__ rl, const T *__restrict__ x,
                                 T *__restrict__ y, const int32_t *__restrict__ perm, cudaTextureObject_t tex) {
    const int64_t g = blockIdx.x;
    const int64_t row = g * G + threadIdx.x;
    if (row >= n) return;
    const int R = (int)min((int64_t)G, n - g * G);     // the last group may be smaller
    int64_t ptr = gp[g] + threadIdx.x;
    const int len = rl[row];
    T acc = 0;
    for (int j = 0; j < len; ++j) {
        acc += val[ptr] * gather<T, XL>(x, tex, col[ptr]);
        ptr += R;
    }
    y[out_row(perm, row)] = acc;
}

template <typename V, int XL>
__global__ void __launch_bounds__(kDefaultThreads)
rgcsr_spmv_split(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                 const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                 const float *__restrict__ scale, const typename VT<V>::A *__restrict__ x,
                 typename VT<V>::A *__restrict__ y, const int32_t *__restrict__ perm, int w4, int cap,
                 cudaTextureObject_t tex) {
    using A = typename VT<V>::A;
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = row < n;
    int len = 0, stride = 0;
    int64_t ptr = 0;
    if (valid) {
        const int64_t g = row / G;
        const int64_t first = g * G;
        stride = (int)min((int64_t)G, n - first);
        ptr = __ldg(gp + g) + (row - first);
        len = min(__ldg(rl + row), cap);      // slots >= cap are left to the long-row segments
    }
    const int lmax = warp_max_i(len);
    const int lmin = warp_min_i(valid ? len : INT_MAX);
    int j0 = lmax;
    if (lmax - lmin > 32) j0 = choose_split(len, w4);

    // Phase 1: thread per row over slots [0, min(len, j0)).
    A acc = 0;
    const int jend = min(len, j0);
    for (int j = 0; j < jend; j += kUnroll) {
        A v[kUnroll];
        int c[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (j + u < jend) {
                const int64_t p = ptr + (int64_t)(j + u) * stride;
                v[u] = VT<V>::ld(val + p);
                c[u] = ld_stream(col + p);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (j + u < jend) acc = fma(v[u], gather<A, XL>(x, tex, c[u]), acc);
    }

    // Phase 2: the whole warp finishes each row longer than j0.
    unsigned long_rows = __ballot_sync(kFull, len > j0);
    while (long_rows) {
        const int r = __ffs(long_rows) - 1;
        long_rows &= long_rows - 1;
        const int Lr = __shfl_sync(kFull, len, r);
        const int sr = __shfl_sync(kFull, stride, r);
        const int64_t pr = shfl_i64(ptr, r);
        A part = 0;
        for (int j = j0 + lane; j < Lr; j += 32 * kUnroll) {
            A v[kUnroll];
            int c[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int jj = j + 32 * u;
                if (jj < Lr) {
                    const int64_t p = pr + (int64_t)jj * sr;
                    v[u] = VT<V>::ld(val + p);
                    c[u] = ld_stream(col + p);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (j + 32 * u < Lr) part = fma(v[u], gather<A, XL>(x, tex, c[u]), part);
        }
        part = warp_sum(part);
        if (lane == r) acc += part;
    }
    if (valid) y[out_row(perm, row)] = finish<V>(acc, scale, row);
}

// One thread per row and no long-row split, sized for full occupancy
// (FP32: <= 32 registers, 64 warps per SM; FP64: 48 warps per SM) so that
// enough loads stay in flight.  For matrices whose rows within a warp have
// similar lengths.
template <typename V, int U, int MIN_BLOCKS, int XL>
__global__ void __launch_bounds__(kDefaultThreads, MIN_BLOCKS)
rgcsr_spmv_lean(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                const float *__restrict__ scale, const typename VT<V>::A *__restrict__ x,
                typename VT<V>::A *__restrict__ y, const int32_t *__restrict__ perm, cudaTextureObject_t tex) {
    using A = typename VT<V>::A;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int64_t g = row / G;
    const int64_t first = g * G;
    const int stride = (int)min((int64_t)G, n - first);
    const int64_t off = __ldg(gp + g) + (row - first);
    const V *vp = val + off;
    const int32_t *cp = col + off;
    const int len = __ldg(rl + row);
    A acc = 0;
    for (int j = 0; j < len; j += U) {
        A v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < len) {
                v[u] = VT<V>::ld(vp + (int64_t)u * stride);
                c[u] = ld_stream(cp + (int64_t)u * stride);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < len) acc = fma(v[u], gather<A, XL>(x, tex, c[u]), acc);
        vp += (int64_t)U * stride;
        cp += (int64_t)U * stride;
    }
    y[out_row(perm, row)] = finish<V>(acc, scale, row);
}

// Vector loads for G = 32: lane q of a warp owns RPL consecutive rows of a
// group (4; FP64: 2), so one 8- or 16-byte load brings RPL values of a
// slot-row and one 8- or 16-byte load their columns; a warp covers 32 * RPL
// rows.  Fewer, wider requests than one thread per row, with the same
// per-row summation order.  The partial last group (R_g < 32, slot stride
// R_g) goes through scalar loads.
// RPL consecutive values and their columns with one load each.
template <int BYTES> struct RawVec;
template <> struct RawVec<4> { using T = uint32_t; };
template <> struct RawVec<8> { using T = uint2; };
template <> struct RawVec<16> { using T = uint4; };
template <int RPL> struct ColVec;
template <> struct ColVec<2> { using T = int2; };
template <> struct ColVec<4> { using T = int4; };

template <typename V, int RPL>
__device__ __forceinline__ void vec_get(const V *p, const int32_t *c, typename VT<V>::A (&v)[RPL], int (&k)[RPL]) {
    using R = typename RawVec<RPL * sizeof(V)>::T;
    using CV = typename ColVec<RPL>::T;
    const R a = __ldcs(reinterpret_cast<const R *>(p));
    const CV b = __ldcs(reinterpret_cast<const CV *>(c));
    const V *e = reinterpret_cast<const V *>(&a);
    const int *q = reinterpret_cast<const int *>(&b);
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        if constexpr (VT<V>::scaled) v[r] = VT<V>::to_float(e[r]);
        else v[r] = e[r];
        k[r] = q[r];
    }
}

// The row sums of thread `tid` under that mapping: acc[r] for row
// first + t0 + r of group g = tid / (32 / RPL).  Returns R_g, or 0 when the
// thread is past the last group (nothing loaded).
template <typename V, int RPL, int U>
__device__ __forceinline__ int vec_rows(int64_t n, const V *__restrict__ val, const int32_t *__restrict__ col,
                                        const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                                        const typename VT<V>::A *__restrict__ x, int64_t tid, int64_t &first,
                                        int &t0, typename VT<V>::A (&acc)[RPL]) {
    using A = typename VT<V>::A;
    constexpr int LPG = 32 / RPL;                                   // lanes per group
    const int64_t g = tid / LPG;
    t0 = (int)(tid % LPG) * RPL;                                    // first row within the group
    first = g * 32;
    if (first >= n) return 0;
    const int R = (int)min((int64_t)32, n - first);
    const int64_t base = __ldg(gp + g);
    int len[RPL];
    int lmax = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        len[r] = (t0 + r < R) ? __ldg(rl + first + t0 + r) : 0;
        lmax = max(lmax, len[r]);
    }
#pragma unroll
    for (int r = 0; r < RPL; ++r) acc[r] = 0;
    if (R == 32) {
        for (int j = 0; j < lmax; j += U) {
            A v[U][RPL];
            int c[U][RPL];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u < lmax) vec_get<V, RPL>(val + base + (int64_t)(j + u) * 32 + t0,
                                                  col + base + (int64_t)(j + u) * 32 + t0, v[u], c[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (j + u < len[r]) acc[r] = fma(v[u][r], __ldg(x + c[u][r]), acc[r]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
            for (int j = 0; j < len[r]; ++j) {
                const int64_t p = base + (int64_t)j * R + t0 + r;
                acc[r] = fma(VT<V>::ld(val + p), __ldg(x + __ldcs(col + p)), acc[r]);
            }
    }
    return R;
}

template <typename V, int RPL, int U, int MIN_BLOCKS>
__global__ void __launch_bounds__(kDefaultThreads, MIN_BLOCKS)
rgcsr_spmv_vec(int64_t n, const V *__restrict__ val, const int32_t *__restrict__ col,
               const int64_t *__restrict__ gp, const int32_t *__restrict__ rl, const float *__restrict__ scale,
               const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
               const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    int64_t first;
    int t0;
    A acc[RPL];
    const int R = vec_rows<V, RPL, U>(n, val, col, gp, rl, x, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                      first, t0, acc);
#pragma unroll
    for (int r = 0; r < RPL; ++r)
        if (t0 + r < R) y[out_row(perm, first + t0 + r)] = finish<V>(acc[r], scale, first + t0 + r);
}

// The same mapping software-pipelined, with every value load 16 bytes wide:
// a lane owns RPL = 16 / sizeof(V) consecutive rows of a group (FP64 2,
// FP32 4, BF16/FP16 8) and keeps two stages of U slot-rows in registers.
// The loads of the next stage (values, and RPL columns in 8- or 16-byte
// pieces) are issued before the x gathers of the current one, so every
// warp has streamed bytes in flight while it gathers; without that, the
// dependent load -> gather -> FMA chain of each step leaves the memory
// system idle between steps and the kernel's time stops falling with its
// bytes (reduced storage then runs no faster than FP32).
template <typename V, int RPL>
struct VecStage {
    using R = typename RawVec<RPL * sizeof(V)>::T;
    R v;
    int c[RPL];
    __device__ __forceinline__ void load(const V *p, const int32_t *q) {
        v = __ldcs(reinterpret_cast<const R *>(p));
        if constexpr (RPL == 2) {
            const int2 a = __ldcs(reinterpret_cast<const int2 *>(q));
            c[0] = a.x; c[1] = a.y;
        } else {
#pragma unroll
            for (int h = 0; h < RPL / 4; ++h) {
                const int4 a = __ldcs(reinterpret_cast<const int4 *>(q) + h);
                c[4 * h] = a.x; c[4 * h + 1] = a.y; c[4 * h + 2] = a.z; c[4 * h + 3] = a.w;
            }
        }
    }
    // 32-bit word i of the 16 bytes (i known at compile time after unrolling)
    __device__ __forceinline__ uint32_t word(int i) const {
        return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
    }
    __device__ __forceinline__ typename VT<V>::A value(int r) const {
        if constexpr (sizeof(V) == 8) {
            return __hiloint2double((int)word(2 * r + 1), (int)word(2 * r));
        } else if constexpr (sizeof(V) == 4) {
            return __uint_as_float(word(r));
        } else {
            const unsigned short h = (unsigned short)(word(r >> 1) >> (16 * (r & 1)));
            if constexpr (std::is_same<V, __nv_bfloat16>::value) return __bfloat162float(__ushort_as_bfloat16(h));
            else return __half2float(__ushort_as_half(h));
        }
    }
};

template <typename V, int U, int MIN_BLOCKS>
__global__ void __launch_bounds__(kDefaultThreads, MIN_BLOCKS)
rgcsr_spmv_vecp(int64_t n, const V *__restrict__ val, const int32_t *__restrict__ col,
                const int64_t *__restrict__ gp, const int32_t *__restrict__ rl, const float *__restrict__ scale,
                const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
                const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    constexpr int RPL = 16 / (int)sizeof(V);
    constexpr int LPG = 32 / RPL;                                   // lanes per group
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = tid / LPG;
    const int t0 = (int)(tid % LPG) * RPL;                          // first row within the group
    const int64_t first = g * 32;
    if (first >= n) return;
    const int R = (int)min((int64_t)32, n - first);
    const int64_t base = __ldg(gp + g);
    int len[RPL];
    int lmax = 0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        len[r] = (t0 + r < R) ? __ldg(rl + first + t0 + r) : 0;
        lmax = max(lmax, len[r]);
    }
    A acc[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) acc[r] = 0;
    if (R == 32) {
        const V *vp = val + base + t0;
        const int32_t *cp = col + base + t0;
        VecStage<V, RPL> cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (u < lmax) cur[u].load(vp + u * 32, cp + u * 32);
        for (int j = 0; j < lmax; j += U) {
            VecStage<V, RPL> nxt[U];
            const int jn = j + U;
#pragma unroll
            for (int u = 0; u < U; ++u)                             // next stage first
                if (jn + u < lmax) nxt[u].load(vp + (int64_t)(jn + u) * 32, cp + (int64_t)(jn + u) * 32);
            A xv[U][RPL];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (j + u < len[r]) xv[u][r] = __ldg(x + cur[u].c[r]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (j + u < len[r]) acc[r] = fma(cur[u].value(r), xv[u][r], acc[r]);
#pragma unroll
            for (int u = 0; u < U; ++u) cur[u] = nxt[u];
        }
    } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
            for (int j = 0; j < len[r]; ++j) {
                const int64_t p = base + (int64_t)j * R + t0 + r;
                acc[r] = fma(VT<V>::ld(val + p), __ldg(x + __ldcs(col + p)), acc[r]);
            }
    }
#pragma unroll
    for (int r = 0; r < RPL; ++r)
        if (t0 + r < R) y[out_row(perm, first + t0 + r)] = finish<V>(acc[r], scale, first + t0 + r);
}

// Sliced ELLPACK on the same slabs (the related format discussed in
// Sec. 3.4): one thread per row, but every row of group g runs all
// K_g = (gp[g+1] - gp[g]) / R_g slots -- no rowLengths -- so the padding is
// multiplied too (value 0 times x[column 0]).  A comparator, not the method.
template <typename V>
__global__ void __launch_bounds__(kDefaultThreads)
sliced_ell_spmv(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                const int64_t *__restrict__ gp, const float *__restrict__ scale,
                const typename VT<V>::A *__restrict__ x, typename VT<V>::A *__restrict__ y,
                const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    constexpr int U = 4;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int64_t g = row / G;
    const int64_t first = g * G;
    const int stride = (int)min((int64_t)G, n - first);
    const int64_t g0 = __ldg(gp + g);
    const int64_t K = (__ldg(gp + g + 1) - g0) / stride;
    const V *vp = val + g0 + (row - first);
    const int32_t *cp = col + g0 + (row - first);
    A acc = 0;
    for (int64_t j = 0; j < K; j += U) {
        A v[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u < K) {
                v[u] = VT<V>::ld(vp + (int64_t)u * stride);
                c[u] = ld_stream(cp + (int64_t)u * stride);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < K) acc = fma(v[u], __ldg(x + c[u]), acc);
        vp += (int64_t)U * stride;
        cp += (int64_t)U * stride;
    }
    y[out_row(perm, row)] = finish<V>(acc, scale, row);
}

template <typename V>
int launch_spmv(const rgcsr_matrix *M, const typename VT<V>::A *x, typename VT<V>::A *y,
                const rgcsr_launch *L, cudaStream_t s) {
    const int kernel = L ? L->kernel : RGCSR_KERNEL_AUTO;
    const int xl = L ? L->x_load : RGCSR_XLOAD_NC;
    if (xl != RGCSR_XLOAD_NC && xl != RGCSR_XLOAD_PLAIN && xl != RGCSR_XLOAD_TEX) return RGCSR_ERR_INVALID_ARG;
    if (xl != RGCSR_XLOAD_NC && kernel != RGCSR_KERNEL_PAPER && kernel != RGCSR_KERNEL_SPLIT &&
        !(kernel == RGCSR_KERNEL_LEAN && (!L || L->variant == 0)))
        return RGCSR_ERR_INVALID_ARG;          // the other kernels read x through the read-only path only
    cudaTextureObject_t tex = 0;
    if (xl == RGCSR_XLOAD_TEX && M->n_cols > 0) {
        const int st = x_texture(x, M->n_cols, (int)sizeof(typename VT<V>::A), &tex);
        if (st != RGCSR_OK) return st;
    }
    const V *val = static_cast<const V *>(M->values);
    const int64_t n = M->n_rows;
    const int32_t G = M->group_size;
    const float *scale = M->row_scale;
    if (VT<V>::scaled && !scale) return RGCSR_ERR_INVALID_ARG;
    if (kernel == RGCSR_KERNEL_LEAN && L && L->variant >= 5 && L->variant <= 7) {
        auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
        if (G != 32 || !aligned(val) || !aligned(M->columns)) return RGCSR_ERR_INVALID_ARG;
        // variants 5, 6, 7: software-pipelined, 16-byte value loads, U = 2, 1, 4
        constexpr int lpg = 32 / (16 / (int)sizeof(V));
        const int64_t blocks = ceil_div(M->n_groups * lpg, (int64_t)kDefaultThreads);
        if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
        // resident blocks per SM: as many as the registers allow without
        // spills (8 rows per lane for 2-byte values need more registers)
        constexpr bool two = sizeof(V) == 2;
        if (L->variant == 5)
            rgcsr_spmv_vecp<V, 2, two ? 2 : 3><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        else if (L->variant == 6)
            rgcsr_spmv_vecp<V, 1, two ? 3 : 4><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        else
            rgcsr_spmv_vecp<V, 4, 2><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        return launch_status();
    }
    if (kernel == RGCSR_KERNEL_LEAN && L && (L->variant == 1 || L->variant == 2 || L->variant == 4 ||
                                             L->variant == 8 || L->variant == 9)) {
        auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
        if (G != 32 || !aligned(val) || !aligned(M->columns)) return RGCSR_ERR_INVALID_ARG;
        // variant 1: 4 rows per lane (FP64: 2), 2 slot-rows in flight;
        // variant 2: 2 rows per lane, 4 slot-rows in flight;
        // variant 4: 4 rows per lane (FP64: 2), 4 slot-rows in flight
        constexpr int rpl1 = sizeof(V) == 8 ? 2 : 4;
        const int lpg = L->variant == 2 ? 16 : 32 / rpl1;
        const int64_t blocks = ceil_div(M->n_groups * lpg, (int64_t)kDefaultThreads);
        if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
        if (L->variant == 8)          // every slot-row of a short row in flight at once
            rgcsr_spmv_vec<V, rpl1, 8, 2><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        else if (L->variant == 9) {   // BF16/FP16: as 1 at 6 blocks per SM (40 registers, no spills)
            if constexpr (sizeof(V) == 2)
                rgcsr_spmv_vec<V, rpl1, 2, 6><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                    n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
            else
                return RGCSR_ERR_INVALID_ARG;
        }
        else if (L->variant == 1)
            rgcsr_spmv_vec<V, rpl1, 2, 5><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        else if (L->variant == 2)
            rgcsr_spmv_vec<V, 2, 4, 5><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        else
            rgcsr_spmv_vec<V, rpl1, 4, 4><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
                n, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm);
        return launch_status();
    }
    if (kernel == RGCSR_KERNEL_LEAN) {
        const int64_t blocks = ceil_div(n, kDefaultThreads);
        if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
        if (L && L->variant != 0) return RGCSR_ERR_INVALID_ARG;
        // 8 blocks (32 registers) fit plain FP32; FP64 and scaled storage need 6
        constexpr int min_blocks = (std::is_same<V, float>::value) ? 8 : 6;
#define RGCSR_LEAN(XL_)                                                                             \
    rgcsr_spmv_lean<V, 4, min_blocks, XL_><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(             \
        n, G, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm, tex)
        if (xl == RGCSR_XLOAD_NC) RGCSR_LEAN(RGCSR_XLOAD_NC);
        else if (xl == RGCSR_XLOAD_PLAIN) RGCSR_LEAN(RGCSR_XLOAD_PLAIN);
        else RGCSR_LEAN(RGCSR_XLOAD_TEX);
#undef RGCSR_LEAN
        return launch_status();
    }
    if (kernel == RGCSR_KERNEL_SELL) {
        const int64_t blocks = ceil_div(n, kDefaultThreads);
        if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
        if (L && L->variant != 0) return RGCSR_ERR_INVALID_ARG;
        sliced_ell_spmv<V><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(n, G, val, M->columns, M->group_ptr,
                                                                       scale, x, y, M->row_perm);
        return launch_status();
    }
    if (kernel == RGCSR_KERNEL_PAPER) {
        if constexpr (VT<V>::scaled) {
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
        } else {
            if (G > 1024) return RGCSR_ERR_INVALID_ARG;
#define RGCSR_PAPER(XL_)                                                                            \
    rgcsr_spmv_paper<V, XL_><<<(unsigned)M->n_groups, G, 0, s>>>(n, G, val, M->columns, M->group_ptr, \
                                                              M->row_lengths, x, y, M->row_perm, tex)
            if (xl == RGCSR_XLOAD_NC) RGCSR_PAPER(RGCSR_XLOAD_NC);
            else if (xl == RGCSR_XLOAD_PLAIN) RGCSR_PAPER(RGCSR_XLOAD_PLAIN);
            else RGCSR_PAPER(RGCSR_XLOAD_TEX);
#undef RGCSR_PAPER
            return launch_status();
        }
    }
    if (kernel != RGCSR_KERNEL_SPLIT) return RGCSR_ERR_INVALID_ARG;
    int threads = (L && L->block_threads) ? L->block_threads : kDefaultThreads;
    if (threads % 32 || threads < 32 || threads > kDefaultThreads) return RGCSR_ERR_INVALID_ARG;
    const int w4 = (L && L->split_weight > 0) ? L->split_weight : 8;
    const int64_t blocks = ceil_div(n, threads);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
#define RGCSR_SPLIT(XL_)                                                                            \
    rgcsr_spmv_split<V, XL_><<<(unsigned)blocks, threads, 0, s>>>(                                   \
        n, G, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm, w4, INT_MAX, tex)
    if (xl == RGCSR_XLOAD_NC) RGCSR_SPLIT(RGCSR_XLOAD_NC);
    else if (xl == RGCSR_XLOAD_PLAIN) RGCSR_SPLIT(RGCSR_XLOAD_PLAIN);
    else RGCSR_SPLIT(RGCSR_XLOAD_TEX);
#undef RGCSR_SPLIT
    return launch_status();
}

// ---------------------------------------------------------------------------
// Long-row segments.  The slots j >= T of every row longer than T are cut
// into segments of S slots; each segment is one warp's work (its slots are
// read with the row's group stride), giving one partial sum per segment.
// The last segment of a row to finish (an arrival counter at the row's first
// segment, no waiting) adds the row's partials with its whole warp -- lane l
// sums partials l, l + 32, ..., then a fixed shuffle tree -- and adds that to
// y.  The rest of every row (slots < T) goes through the split kernel with
// its length capped at T, one launch earlier.
// Work per warp is bounded by S slots whatever the row lengths are, so no
// warp is held up by a very long row; the result is deterministic.
// ---------------------------------------------------------------------------
__global__ void seg_count_kernel(int64_t n, const int32_t *__restrict__ rl, int32_t T, int32_t S,
                                 int64_t *__restrict__ nseg, int64_t *__restrict__ nlong) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = rl[i];
    const int64_t c = L > T ? ((int64_t)L - T + S - 1) / S : 0;
    nseg[i] = c;
    nlong[i] = c > 0 ? 1 : 0;
}

__global__ void seg_fill_kernel(int64_t n, const int32_t *__restrict__ rl, int32_t T, int32_t S,
                                const int64_t *__restrict__ seg_off, const int64_t *__restrict__ long_off,
                                int32_t *__restrict__ seg_row, int32_t *__restrict__ seg_start,
                                int32_t *__restrict__ long_row, int32_t *__restrict__ long_first,
                                int32_t *__restrict__ long_count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = rl[i];
    if (L <= T) return;
    const int c = (L - T + S - 1) / S;
    const int64_t base = seg_off[i];
    for (int s = 0; s < c; ++s) {
        seg_row[base + s] = (int32_t)i;
        seg_start[base + s] = T + s * S;
    }
    const int64_t k = long_off[i];
    long_row[k] = (int32_t)i;
    long_first[k] = (int32_t)base;
    long_count[k] = c;
}

template <typename V>
__global__ void __launch_bounds__(kDefaultThreads)
seg_spmv_kernel(int64_t n, int32_t G, const V *__restrict__ val, const int32_t *__restrict__ col,
                const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                const int32_t *__restrict__ seg_row, const int32_t *__restrict__ seg_start, int32_t T, int32_t S,
                int64_t n_seg, const typename VT<V>::A *__restrict__ x, typename VT<V>::A *partials,
                int32_t *__restrict__ arrivals, const float *__restrict__ scale, typename VT<V>::A *__restrict__ y,
                const int32_t *__restrict__ perm) {
    using A = typename VT<V>::A;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_seg; s += warps) {
        const int64_t row = seg_row[s];
        const int ja = seg_start[s];
        const int jb = min(ja + S, __ldg(rl + row));
        const int64_t g = row / G;
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const int64_t ptr = __ldg(gp + g) + (row - first);
        A part = 0;
        for (int j = ja + lane; j < jb; j += 32 * kUnroll) {
            A v[kUnroll];
            int c[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int jj = j + 32 * u;
                if (jj < jb) {
                    const int64_t p = ptr + (int64_t)jj * R;
                    v[u] = VT<V>::ld(val + p);
                    c[u] = ld_stream(col + p);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (j + 32 * u < jb) part = fma(v[u], __ldg(x + c[u]), part);
        }
        part = warp_sum(part);
        if (lane == 0) partials[s] = part;
        // the row's segments are s - q .. s - q + c - 1
        const int64_t f = s - (ja - T) / S;
        const int c = (__ldg(rl + row) - T + S - 1) / S;
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence();
            last = atomicAdd(arrivals + f, 1) == c - 1;
        }
        last = __shfl_sync(kFull, last, 0);
        if (!last) continue;
        __threadfence();
        A sum = 0;
        for (int i = lane; i < c; i += 32) sum += __ldcg(partials + f + i);
        sum = warp_sum(sum);
        if (lane == 0) {
            y[out_row(perm, row)] += finish<V>(sum, scale, row);
            arrivals[f] = 0;
        }
    }
}

template <typename V>
int launch_long_rows(const rgcsr_matrix *M, const rgcsr_long_rows *S, const typename VT<V>::A *x,
                     typename VT<V>::A *y, cudaStream_t s) {
    using A = typename VT<V>::A;
    const V *val = static_cast<const V *>(M->values);
    const int64_t n = M->n_rows;
    const float *scale = M->row_scale;
    if (VT<V>::scaled && !scale) return RGCSR_ERR_INVALID_ARG;
    const int64_t blocks = ceil_div(n, kDefaultThreads);
    if (blocks > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    rgcsr_spmv_split<V, RGCSR_XLOAD_NC><<<(unsigned)blocks, kDefaultThreads, 0, s>>>(
        n, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, scale, x, y, M->row_perm, 8,
        S->threshold, 0);
    if (S->n_segments == 0) return launch_status();
    int64_t sb = ceil_div(S->n_segments, kDefaultThreads / 32);
    if (sb > 152 * 16) sb = 152 * 16;
    A *part = static_cast<A *>(S->partials);
    seg_spmv_kernel<V><<<(unsigned)sb, kDefaultThreads, 0, s>>>(
        n, M->group_size, val, M->columns, M->group_ptr, M->row_lengths, S->seg_row, S->seg_start,
        S->threshold, S->segment, S->n_segments, x, part, S->arrivals, scale, y, M->row_perm);
    return launch_status();
}

}  // namespace

// The kernel RGCSR_KERNEL_AUTO runs, as timed on GB300.  Dense groups
// (padding <= 25% of the stored slots, no row far longer than the average)
// with short rows (<= 8 per row) at G = 32 take the vector-load kernel (4
// rows per lane with 2 slot-rows per step; FP64: 2 rows with 4); longer
// FP32 rows the TMA-staged kernel (16 slot-rows per stage); the rest the
// full-occupancy thread-per-row kernel.  Uneven or long rows take the
// warp-split kernel.
int auto_kernel(const rgcsr_matrix *M, int *variant) {
    const bool dense = M->n_stored * 4 <= M->nnz * 5 &&
                       !(M->max_row_len > 64 && M->max_row_len * M->n_rows > 8 * M->nnz);
    const bool short_rows = M->nnz <= 8 * M->n_rows;
    auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    *variant = 0;
    if (dense && short_rows && M->group_size == 32 && aligned(M->values) && aligned(M->columns)) {
        *variant = M->value_type == RGCSR_F64 ? 4 : 1;
        return RGCSR_KERNEL_LEAN;
    }
    if (dense && M->value_type == RGCSR_F32 && tma_eligible(M)) {
        *variant = 2;
        return RGCSR_KERNEL_TMA;
    }
    return dense ? RGCSR_KERNEL_LEAN : RGCSR_KERNEL_SPLIT;
}

namespace {
int check_matrix(const rgcsr_matrix *M) {
    if (!M || M->n_rows < 0 || M->n_cols < 0 || M->group_size < 1) return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!M->group_ptr || !M->row_lengths) return RGCSR_ERR_INVALID_ARG;
    if (M->n_stored > 0 && (!M->values || !M->columns)) return RGCSR_ERR_INVALID_ARG;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    return RGCSR_OK;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_spmv_ex(const rgcsr_matrix *M, const void *x, void *y,
                            const rgcsr_launch *launch, rgcsr_stream_t stream) {
    int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!y || (M->n_cols > 0 && !x)) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    int kernel = launch ? launch->kernel : RGCSR_KERNEL_AUTO;
    int variant = launch ? launch->variant : 0;
    // x read paths other than the read-only one are an ablation of the
    // paper's, scalar, x gathers: they need an explicit PAPER, SPLIT or LEAN
    // (variant 0) kernel
    if (launch && launch->x_load != RGCSR_XLOAD_NC &&
        !(kernel == RGCSR_KERNEL_PAPER || kernel == RGCSR_KERNEL_SPLIT ||
          (kernel == RGCSR_KERNEL_LEAN && variant == 0)))
        return RGCSR_ERR_INVALID_ARG;
    if (kernel == RGCSR_KERNEL_AUTO) kernel = auto_kernel(M, &variant);
    if (kernel == RGCSR_KERNEL_TMA) {
        if (!tma_eligible(M)) return RGCSR_ERR_INVALID_ARG;
        if (launch && launch->wait_limit < 0) return RGCSR_ERR_INVALID_ARG;
        return launch_spmv_tma(M, x, y, variant, launch ? (uint32_t)launch->wait_limit : 0u, s);
    }
    rgcsr_launch resolved = launch ? *launch : rgcsr_launch{};
    resolved.kernel = kernel;
    resolved.variant = variant;
    switch (M->value_type) {
        case RGCSR_F64:
            return launch_spmv<double>(M, static_cast<const double *>(x), static_cast<double *>(y), &resolved, s);
        case RGCSR_F32:
            return launch_spmv<float>(M, static_cast<const float *>(x), static_cast<float *>(y), &resolved, s);
        case RGCSR_BF16:
            return launch_spmv<__nv_bfloat16>(M, static_cast<const float *>(x), static_cast<float *>(y), &resolved, s);
        case RGCSR_F16:
            return launch_spmv<__half>(M, static_cast<const float *>(x), static_cast<float *>(y), &resolved, s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}

RGCSR_API int rgcsr_auto_kernel(const rgcsr_matrix *M, int32_t *kernel, int32_t *variant) {
    if (!kernel || !variant) return RGCSR_ERR_INVALID_ARG;
    const int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    int v = 0;
    *kernel = auto_kernel(M, &v);
    *variant = v;
    return RGCSR_OK;
}

RGCSR_API int rgcsr_spmv(const rgcsr_matrix *M, const void *x, void *y, rgcsr_stream_t stream) {
    return rgcsr_spmv_ex(M, x, y, nullptr, stream);
}

namespace {
struct SegScratch {
    int64_t *seg_off, *long_off, *partials;
};
SegScratch carve_seg(void *ws, int64_t n) {
    char *p = static_cast<char *>(ws);
    const size_t a = align_up((size_t)(n + 1) * 8, 256);
    SegScratch c;
    c.seg_off = reinterpret_cast<int64_t *>(p);
    c.long_off = reinterpret_cast<int64_t *>(p + a);
    c.partials = reinterpret_cast<int64_t *>(p + 2 * a);
    return c;
}
// counts per row, then exclusive scans: seg_off[n] / long_off[n] = totals
int seg_scan(const rgcsr_matrix *M, const rgcsr_long_rows *S, SegScratch &c, cudaStream_t s) {
    const int64_t n = M->n_rows;
    if (n > 0) {
        seg_count_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, M->row_lengths, S->threshold, S->segment,
                                                                    c.seg_off, c.long_off);
        int st = launch_status();
        if (st != RGCSR_OK) return st;
    }
    int st = exclusive_scan_i64(c.seg_off, n, c.partials, s);
    if (st != RGCSR_OK) return st;
    return exclusive_scan_i64(c.long_off, n, c.partials, s);
}
}  // namespace

RGCSR_API size_t rgcsr_long_rows_workspace_bytes(int64_t n_rows) {
    if (n_rows < 0) return 0;
    return 2 * align_up((size_t)(n_rows + 1) * 8, 256) + scan_partials_bytes(n_rows);
}

RGCSR_API int rgcsr_long_rows_plan(const rgcsr_matrix *M, rgcsr_long_rows *S, void *workspace,
                                   size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    if (!S || S->threshold < 0 || S->segment < 1) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_long_rows_workspace_bytes(M->n_rows)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    SegScratch c = carve_seg(workspace, M->n_rows);
    if ((st = seg_scan(M, S, c, s)) != RGCSR_OK) return st;
    int64_t tot[2] = {0, 0};
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&tot[0], c.seg_off + M->n_rows, 8, cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&tot[1], c.long_off + M->n_rows, 8, cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    if (tot[0] > INT32_MAX) return RGCSR_ERR_INDEX_OVERFLOW;
    S->n_segments = tot[0];
    S->n_long_rows = tot[1];
    return RGCSR_OK;
}

RGCSR_API int rgcsr_long_rows_build(const rgcsr_matrix *M, const rgcsr_long_rows *S, void *workspace,
                                    size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    if (!S || S->threshold < 0 || S->segment < 1) return RGCSR_ERR_INVALID_ARG;
    if (S->n_segments == 0 || M->n_rows == 0) return RGCSR_OK;
    if (!S->seg_row || !S->seg_start || !S->long_row || !S->long_first || !S->long_count || !S->arrivals)
        return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_long_rows_workspace_bytes(M->n_rows)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    SegScratch c = carve_seg(workspace, M->n_rows);
    if ((st = seg_scan(M, S, c, s)) != RGCSR_OK) return st;
    RGCSR_CUDA_TRY(cudaMemsetAsync(S->arrivals, 0, (size_t)S->n_segments * sizeof(int32_t), s));
    seg_fill_kernel<<<(unsigned)ceil_div(M->n_rows, 256), 256, 0, s>>>(
        M->n_rows, M->row_lengths, S->threshold, S->segment, c.seg_off, c.long_off, S->seg_row, S->seg_start,
        S->long_row, S->long_first, S->long_count);
    return launch_status();
}

RGCSR_API int rgcsr_spmv_long_rows(const rgcsr_matrix *M, const rgcsr_long_rows *S, const void *x, void *y,
                                   rgcsr_stream_t stream) {
    int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!S || S->threshold < 0 || S->segment < 1 || !y || (M->n_cols > 0 && !x)) return RGCSR_ERR_INVALID_ARG;
    if (S->n_segments > 0 && (!S->seg_row || !S->seg_start || !S->long_row || !S->long_first ||
                              !S->long_count || !S->partials || !S->arrivals))
        return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(M, s)) return cst;   // checks mode
    switch (M->value_type) {
        case RGCSR_F64:
            return launch_long_rows<double>(M, S, static_cast<const double *>(x), static_cast<double *>(y), s);
        case RGCSR_F32:
            return launch_long_rows<float>(M, S, static_cast<const float *>(x), static_cast<float *>(y), s);
        case RGCSR_BF16:
            return launch_long_rows<__nv_bfloat16>(M, S, static_cast<const float *>(x), static_cast<float *>(y), s);
        case RGCSR_F16:
            return launch_long_rows<__half>(M, S, static_cast<const float *>(x), static_cast<float *>(y), s);
        default:
            return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
}

RGCSR_API int rgcsr_spmv_host(const rgcsr_matrix *M, const void *x_host, void *y_host,
                              void *x_dev, void *y_dev, const rgcsr_launch *launch,
                              const rgcsr_long_rows *long_rows, const rgcsr_tiles *tiles,
                              rgcsr_stream_t stream) {
    int st = check_matrix(M);
    if (st != RGCSR_OK) return st;
    if (M->n_rows == 0) return RGCSR_OK;
    if (!x_host || !y_host || !x_dev || !y_dev) return RGCSR_ERR_INVALID_ARG;
    const size_t xb = M->value_type == RGCSR_F64 ? 8 : 4;
    cudaStream_t s = (cudaStream_t)stream;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(x_dev, x_host, (size_t)M->n_cols * xb, cudaMemcpyHostToDevice, s));
    st = tiles       ? rgcsr_spmv_tiles(M, tiles, x_dev, y_dev, stream)
         : long_rows ? rgcsr_spmv_long_rows(M, long_rows, x_dev, y_dev, stream)
                     : rgcsr_spmv_ex(M, x_dev, y_dev, launch, stream);
    if (st != RGCSR_OK) return st;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(y_host, y_dev, (size_t)M->n_rows * xb, cudaMemcpyDeviceToHost, s));
    return RGCSR_OK;
}
