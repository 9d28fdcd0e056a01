// cg.cu -- conjugate gradients on an RgCSR operator and mixed-precision
// iterative refinement (the Krylov setting of the paper's introduction:
// a CG iteration is one SpMV plus SAXPY and SDOT operations).
//
// rgcsr_cg:    textbook CG from x0 = 0; the step lengths live in device
//              scalars, so an iteration is four kernels (the SpMV and the
//              three below) and no host round trip; the host reads the
//              residual norm every `check_every` iterations to test
//              convergence.
// rgcsr_ir_cg: outer loop in FP64 -- r = b - A x with the FP64 matrix,
//              stop when ||r|| <= tol ||b||; inner CG in float on a
//              lower-precision copy of A (float, bfloat16 or half values)
//              solves A d = r to a loose tolerance; x += d in FP64.
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>

namespace rgcsr {
namespace {

constexpr int kThreads = 256;

// One CG iteration after the SpMV q = A d is three kernels, each moving 16
// bytes per access:
//   cg_dq:    dq = d . q; the last block to finish sets alpha = rr / dq;
//   cg_xr_rr: x += alpha d, r -= alpha q, and rr' = r . r from the new r in
//             the same pass; the last block sets beta = rr' / rr;
//   cg_d:     d = r + beta d.
// The step lengths are computed once, in double, by the last block of a
// reduction and read by every thread as scalars (a division per thread
// would run on the narrow FP64 pipe).  Dots are deterministic: a fixed grid
// for a given n, a fixed order within each thread (float vectors by the
// compensated Dot2 step, double vectors by FMAs), a block tree, then the
// block sums in block order.  Scalar block (doubles): [0], [1] rr (the slot
// `cur` holds the current one), [2] dq, [3] alpha, [4] beta; the ticket of
// the last-block reductions is the unsigned at byte 64.
constexpr int kCgParts = 1216;          // blocks of the fused kernels at most (8 per SM)
constexpr int kU = 4;                   // packs a reducing thread loads before it uses them

template <typename T>
__device__ __forceinline__ void acc_dot(T a, T b, float &s, float &c, double &sd) {
    if constexpr (sizeof(T) == 4) dot2_step(a, b, s, c);
    else sd = fma((double)a, (double)b, sd);
}

template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
cg_dq_kernel(int64_t n, const T *__restrict__ d, const T *__restrict__ q, double *scal, int cur, double *parts,
             unsigned *ticket) {
    __shared__ double sh[32];
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    float s = 0.0f, c = 0.0f;
    double sd = 0.0;
    // packs tid, tid + S, tid + 2S, ... in that order; kU of them loaded
    // before any is used, so each thread keeps kU * 32 bytes in flight
#pragma unroll 1
    for (int64_t i0 = tid; i0 < nw; i0 += kU * S) {
        Pack<T, W> dv[kU], qv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                dv[u] = ld_pack<T, W>(d + (i0 + u * S) * W);
                qv[u] = ld_pack<T, W>(q + (i0 + u * S) * W);
            }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
#pragma unroll
                for (int k = 0; k < W; ++k) acc_dot(dv[u].v[k], qv[u].v[k], s, c, sd);
            }
    }
    for (int64_t i = nw * W + tid; i < n; i += S) acc_dot(d[i], q[i], s, c, sd);
    double total;
    if (!reduce_last(sizeof(T) == 4 ? (double)s + (double)c : sd, parts, ticket, sh, total)) return;
    if (threadIdx.x == 0) {
        scal[2] = total;
        scal[3] = scal[cur] / total;
        *ticket = 0u;
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
cg_xr_rr_kernel(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ d,
                const T *__restrict__ q, double *scal, int cur, double *parts, unsigned *ticket) {
    __shared__ double sh[32];
    const T alpha = (T)scal[3];
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    float s = 0.0f, c = 0.0f;
    double sd = 0.0;
#pragma unroll 1
    for (int64_t i0 = tid; i0 < nw; i0 += kU * S) {
        Pack<T, W> xv[kU], rv[kU], dv[kU], qv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                const int64_t i = i0 + u * S;
                xv[u] = ld_pack<T, W>(x + i * W);
                rv[u] = ld_pack<T, W>(r + i * W);
                dv[u] = ld_pack<T, W>(d + i * W);
                qv[u] = ld_pack<T, W>(q + i * W);
            }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                const int64_t i = i0 + u * S;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    xv[u].v[k] = fma(alpha, dv[u].v[k], xv[u].v[k]);
                    rv[u].v[k] = fma(-alpha, qv[u].v[k], rv[u].v[k]);
                    acc_dot(rv[u].v[k], rv[u].v[k], s, c, sd);
                }
                st_pack<T, W>(x + i * W, xv[u]);
                st_pack<T, W>(r + i * W, rv[u]);
            }
    }
    for (int64_t i = nw * W + tid; i < n; i += S) {
        x[i] = fma(alpha, d[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc_dot(ri, ri, s, c, sd);
    }
    double total;
    if (!reduce_last(sizeof(T) == 4 ? (double)s + (double)c : sd, parts, ticket, sh, total)) return;
    if (threadIdx.x == 0) {
        scal[1 - cur] = total;
        scal[4] = total / scal[cur];
        *ticket = 0u;
    }
}

template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
cg_d_kernel(int64_t n, const double *__restrict__ scal, const T *__restrict__ r, T *__restrict__ d) {
    const T beta = (T)scal[4];
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
#pragma unroll 1
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<T, W> rv = ld_pack<T, W>(r + i * W), dv = ld_pack<T, W>(d + i * W);
        Pack<T, W> o;
#pragma unroll
        for (int k = 0; k < W; ++k) o.v[k] = fma(beta, dv.v[k], rv.v[k]);
        st_pack<T, W>(d + i * W, o);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) d[i] = fma(beta, d[i], r[i]);
}

// The same three steps as one cooperative kernel (every block resident),
// with two grid barriers in place of the kernel boundaries:
//   1. dq = d . q, block sums to parts[0, G);  barrier;  every block adds
//      parts[0, G) in block order with the same tree, so all blocks hold the
//      same dq, and alpha = rr / dq;
//   2. x += alpha d, r -= alpha q, rr' = r . r, block sums to parts[G, 2G);
//      barrier;  rr' and beta = rr' / rr likewise;
//   3. d = r + beta d.
// Each thread visits the same elements in every step (a grid-stride loop
// over 16-byte packs), so what step 2 writes, step 3 reads back from its own
// thread; the vectors are re-read from L2 rather than held.  Block 0 records
// dq, alpha, rr' and beta in the scalar block as the three kernels do.  A
// barrier is a counter in the scalar block: each block adds one and polls
// (acquire loads, a short sleep between polls) until all have; a wait gives
// up after wait_limit polls, sets the error word and its block returns, so
// the caller sees RGCSR_ERR_TIMEOUT instead of a hang.  The last block to
// leave resets the counters for the next launch.
struct CoopWords {                  // in the scalar block at byte 72
    unsigned arrive, leave;
    int error;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// false (in every thread of the block) when the wait ran out
__device__ __forceinline__ bool grid_barrier(CoopWords *w, unsigned target, unsigned limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&w->arrive, 1u);
        int done = 0;
        for (unsigned p = 0; p < limit; ++p) {
            if (ld_acquire_gpu(&w->arrive) >= target) { done = 1; break; }
            __nanosleep(32);
        }
        if (!done) atomicExch(&w->error, 1);
        ok = done;
    }
    __syncthreads();
    return ok != 0;
}

// the sum of parts[0, G) in block order, the same in every block
__device__ __forceinline__ double sum_parts(const double *parts, double *sh) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(parts + b);
    return block_sum(t, sh);
}

template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
cg_update_coop_kernel(int64_t n, T *__restrict__ x, T *__restrict__ r, T *__restrict__ d, const T *__restrict__ q,
                      double *scal, int cur, double *parts, CoopWords *w, unsigned limit) {
    __shared__ double sh[32];
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    const unsigned G = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // 1. dq
    float s = 0.0f, c = 0.0f;
    double sd = 0.0;
#pragma unroll 1
    for (int64_t i0 = tid; i0 < nw; i0 += kU * S) {
        Pack<T, W> dv[kU], qv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                dv[u] = ld_pack<T, W>(d + (i0 + u * S) * W);
                qv[u] = ld_pack<T, W>(q + (i0 + u * S) * W);
            }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
#pragma unroll
                for (int k = 0; k < W; ++k) acc_dot(dv[u].v[k], qv[u].v[k], s, c, sd);
            }
    }
    for (int64_t i = nw * W + tid; i < n; i += S) acc_dot(d[i], q[i], s, c, sd);
    double b = block_sum(sizeof(T) == 4 ? (double)s + (double)c : sd, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = b;
    if (!grid_barrier(w, G, limit)) return;
    const double dq = sum_parts(parts, sh);
    const double rr = scal[cur];
    const T alpha = (T)(rr / dq);
    if (lead) {
        scal[2] = dq;
        scal[3] = rr / dq;
    }
    // 2. x, r and rr'
    s = c = 0.0f;
    sd = 0.0;
#pragma unroll 1
    for (int64_t i0 = tid; i0 < nw; i0 += kU * S) {
        Pack<T, W> xv[kU], rv[kU], dv[kU], qv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                const int64_t i = i0 + u * S;
                xv[u] = ld_pack<T, W>(x + i * W);
                rv[u] = ld_pack<T, W>(r + i * W);
                dv[u] = ld_pack<T, W>(d + i * W);
                qv[u] = ld_pack<T, W>(q + i * W);
            }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                const int64_t i = i0 + u * S;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    xv[u].v[k] = fma(alpha, dv[u].v[k], xv[u].v[k]);
                    rv[u].v[k] = fma(-alpha, qv[u].v[k], rv[u].v[k]);
                    acc_dot(rv[u].v[k], rv[u].v[k], s, c, sd);
                }
                st_pack<T, W>(x + i * W, xv[u]);
                st_pack<T, W>(r + i * W, rv[u]);
            }
    }
    for (int64_t i = nw * W + tid; i < n; i += S) {
        x[i] = fma(alpha, d[i], x[i]);
        const T ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc_dot(ri, ri, s, c, sd);
    }
    b = block_sum(sizeof(T) == 4 ? (double)s + (double)c : sd, sh);
    if (threadIdx.x == 0) parts[G + blockIdx.x] = b;
    if (!grid_barrier(w, 2 * G, limit)) return;
    const double rr1 = sum_parts(parts + G, sh);
    const T beta = (T)(rr1 / rr);
    if (lead) {
        scal[1 - cur] = rr1;
        scal[4] = rr1 / rr;
    }
    // 3. d
#pragma unroll 1
    for (int64_t i0 = tid; i0 < nw; i0 += kU * S) {
        Pack<T, W> rv[kU], dv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
                rv[u] = ld_pack<T, W>(r + (i0 + u * S) * W);
                dv[u] = ld_pack<T, W>(d + (i0 + u * S) * W);
            }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (i0 + u * S < nw) {
#pragma unroll
                for (int k = 0; k < W; ++k) dv[u].v[k] = fma(beta, dv[u].v[k], rv[u].v[k]);
                st_pack<T, W>(d + (i0 + u * S) * W, dv[u]);
            }
    }
    for (int64_t i = nw * W + tid; i < n; i += S) d[i] = fma(beta, d[i], r[i]);
    // the last block to leave resets the counters (all others are past both barriers)
    if (threadIdx.x == 0 && atomicAdd(&w->leave, 1u) == G - 1) {
        w->arrive = 0u;
        w->leave = 0u;
        __threadfence();
    }
}

// Polls before a grid barrier of the cooperative update gives up (each poll
// is an L2 round trip plus a short sleep: the default is on the order of a
// second); rgcsr_set_wait_limit changes it, for tests of the timeout path.
constexpr unsigned kDefaultWaitLimit = 1u << 21;
std::atomic<unsigned> g_wait_limit{0};
unsigned cg_wait_limit() {
    const unsigned v = g_wait_limit.load(std::memory_order_relaxed);
    return v ? v : kDefaultWaitLimit;
}

// Blocks of the fused kernels: one 16-byte pack per thread where possible,
// at most `per_sm` blocks per SM and kCgParts in all.  The reducing kernels
// take 2 per SM (fewer same-address tickets, kU packs in flight per
// thread), the plain update 8.
unsigned cg_grid(int64_t units, int per_sm) {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                      cudaSuccess && v > 0)
            sms = v;
        else
            sms = 152;
    }
    int64_t b = ceil_div(units, kThreads);
    const int64_t cap = std::min<int64_t>((int64_t)sms * per_sm, kCgParts);
    if (b > cap) b = cap;
    return (unsigned)(b > 0 ? b : 1);
}

// The recorded round of CG iterations, destroyed when the solve returns.
struct GraphExec {
    cudaGraphExec_t h = nullptr;
    GraphExec() = default;
    GraphExec(const GraphExec &) = delete;
    GraphExec &operator=(const GraphExec &) = delete;
    ~GraphExec() {
        if (h) cudaGraphExecDestroy(h);
    }
};

struct CgScratch {
    void *r, *d, *q;
    double *scal;       // [rr0, rr1, dq, alpha, beta]
    unsigned *count;    // the one-pass dot's block ticket (in the scalar block)
    double *partials;
};

size_t cg_bytes(int64_t n, int vt) {
    const size_t es = vt == RGCSR_F64 ? 8 : 4;
    return 3 * align_up((size_t)n * es, 256) + 256 + align_up((size_t)std::max(kDotParts, 2 * kCgParts) * 8, 256);
}

CgScratch carve_cg(void *ws, int64_t n, int vt) {
    const size_t es = vt == RGCSR_F64 ? 8 : 4;
    const size_t a = align_up((size_t)n * es, 256);
    char *p = static_cast<char *>(ws);
    CgScratch c;
    c.r = p; p += a;
    c.d = p; p += a;
    c.q = p; p += a;
    c.scal = reinterpret_cast<double *>(p);
    c.count = reinterpret_cast<unsigned *>(p + 64);
    p += 256;
    c.partials = reinterpret_cast<double *>(p);
    return c;
}

int vector_type(const rgcsr_matrix *A) { return A->value_type == RGCSR_F64 ? RGCSR_F64 : RGCSR_F32; }

template <typename T>
int cg_run(const rgcsr_matrix *A, const void *b, void *x, double rel_tol, int max_iter, int check_every,
           CgScratch &c, int *iterations, double *rel_residual, cudaStream_t s) {
    const int64_t n = A->n_rows;
    const int vt = vector_type(A);
    const size_t bytes = (size_t)n * sizeof(T);
    int st;
    RGCSR_CUDA_TRY(cudaMemsetAsync(x, 0, bytes, s));
    RGCSR_CUDA_TRY(cudaMemcpyAsync(c.r, b, bytes, cudaMemcpyDeviceToDevice, s));
    RGCSR_CUDA_TRY(cudaMemcpyAsync(c.d, b, bytes, cudaMemcpyDeviceToDevice, s));
    RGCSR_CUDA_TRY(cudaMemsetAsync(c.count, 0, 32, s));            // the ticket and the barrier words
    if ((st = dot_device(n, c.r, c.r, &c.scal[0], c.partials, vt, s, c.count)) != RGCSR_OK) return st;
    double bb = 0.0;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&bb, &c.scal[0], sizeof(double), cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    *iterations = 0;
    *rel_residual = 0.0;
    if (!(bb > 0.0)) return RGCSR_OK;                 // b = 0: x = 0 is exact
    double rr = bb;
    int cur = 0, it = 0;
    // One CG iteration: q = A d; alpha = rr / (d.q); x += alpha d; r -= alpha q;
    // rr' = r.r; d = r + (rr' / rr) d.  `cur` selects which scalar slot holds rr.
    constexpr int kW = 16 / (int)sizeof(T);                 // 16-byte accesses when x is aligned
    const bool vec = all_aligned16(x, c.r, c.d, c.q);
    CoopWords *words = reinterpret_cast<CoopWords *>(reinterpret_cast<char *>(c.scal) + 72);
    // the update as one cooperative kernel when every block of its grid can
    // be resident (up to 4 per SM); else, or if the launch is refused, the
    // three kernels
    auto coop_kernel = vec ? cg_update_coop_kernel<T, kW> : cg_update_coop_kernel<T, 1>;
    unsigned coop_grid = 0;
    {
        int per_sm = 0, sms = 0, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coop_kernel, kThreads, 0) == cudaSuccess &&
            per_sm > 0 && sms > 0) {
            const int64_t want = ceil_div(ceil_div(n, vec ? kW : 1), kThreads);
            coop_grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)std::min(per_sm, 4) * sms,
                                                                           (int64_t)kCgParts}));
        }
        cudaGetLastError();
    }
    const unsigned limit = cg_wait_limit();
    auto iteration = [&](cudaStream_t st_, int cur_) -> int {
        int e;
        if ((e = rgcsr_spmv(A, c.d, c.q, (rgcsr_stream_t)st_)) != RGCSR_OK) return e;
        T *xt = static_cast<T *>(x), *rt = static_cast<T *>(c.r), *dt = static_cast<T *>(c.d);
        const T *qt = static_cast<const T *>(c.q);
        if (coop_grid) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(coop_grid);
            cfg.blockDim = dim3(kThreads);
            cfg.stream = st_;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, coop_kernel, n, xt, rt, dt, qt, c.scal, cur_, c.partials, words, limit) ==
                cudaSuccess)
                return RGCSR_OK;
            cudaGetLastError();
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st_, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                return RGCSR_ERR_CUDA;                  // not recordable: the round runs without a graph
            coop_grid = 0;                              // refused: the three kernels from now on
        }
        if (vec) {
            const unsigned gr = cg_grid(ceil_div(n, kW), 2), gu = cg_grid(ceil_div(n, kW), 8);
            cg_dq_kernel<T, kW><<<gr, kThreads, 0, st_>>>(n, dt, qt, c.scal, cur_, c.partials, c.count);
            cg_xr_rr_kernel<T, kW><<<gr, kThreads, 0, st_>>>(n, xt, rt, dt, qt, c.scal, cur_, c.partials, c.count);
            cg_d_kernel<T, kW><<<gu, kThreads, 0, st_>>>(n, c.scal, rt, dt);
        } else {
            const unsigned gr = cg_grid(n, 2), gu = cg_grid(n, 8);
            cg_dq_kernel<T, 1><<<gr, kThreads, 0, st_>>>(n, dt, qt, c.scal, cur_, c.partials, c.count);
            cg_xr_rr_kernel<T, 1><<<gr, kThreads, 0, st_>>>(n, xt, rt, dt, qt, c.scal, cur_, c.partials, c.count);
            cg_d_kernel<T, 1><<<gu, kThreads, 0, st_>>>(n, c.scal, rt, dt);
        }
        return launch_status();
    };
    // After the first round of iterations (which also runs any one-off kernel
    // setup), the check_every iterations between two convergence checks are
    // recorded once into a CUDA graph (on a private stream: the caller's may
    // be the legacy default stream, which cannot be captured) and replayed on
    // the caller's stream.  check_every is even, so a round leaves `cur` as
    // it found it.  If recording fails the iterations are launched directly.
    GraphExec round;                                 // destroyed on every return
    bool tried = false;
    while (it < max_iter) {
        const int chunk = check_every < max_iter - it ? check_every : max_iter - it;
        if (round.h && chunk == check_every) {
            RGCSR_CUDA_TRY(cudaGraphLaunch(round.h, s));
        } else {
            for (int i = 0; i < chunk; ++i) {
                if ((st = iteration(s, cur)) != RGCSR_OK) return st;
                cur = 1 - cur;
            }
        }
        it += chunk;
        CoopWords cw;
        RGCSR_CUDA_TRY(cudaMemcpyAsync(&rr, &c.scal[cur], sizeof(double), cudaMemcpyDeviceToHost, s));
        RGCSR_CUDA_TRY(cudaMemcpyAsync(&cw, words, sizeof(cw), cudaMemcpyDeviceToHost, s));
        RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
        if (cw.error) return RGCSR_ERR_TIMEOUT;
        if (!(rr == rr) || std::sqrt(rr) <= rel_tol * std::sqrt(bb)) break;   // converged (or NaN)
        if (!tried && check_every % 2 == 0 && max_iter - it >= 2 * check_every) {
            tried = true;
            cudaStream_t cap = nullptr;
            cudaGraph_t g = nullptr;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess) {
                if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    int e = RGCSR_OK;
                    for (int i = 0; i < check_every && e == RGCSR_OK; ++i) e = iteration(cap, (cur + i) & 1);
                    if (cudaStreamEndCapture(cap, &g) == cudaSuccess && g && e == RGCSR_OK &&
                        cudaGraphInstantiate(&round.h, g, 0) != cudaSuccess)
                        round.h = nullptr;
                    if (g) cudaGraphDestroy(g);
                }
                cudaStreamDestroy(cap);
            }
            cudaGetLastError();                      // a failed recording leaves no sticky error
        }
    }
    *iterations = it;
    *rel_residual = std::sqrt(rr / bb);
    return (rr == rr) ? RGCSR_OK : RGCSR_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t rgcsr_cg_workspace_bytes(int64_t n, int32_t value_type) {
    if (n < 0) return 0;
    return cg_bytes(n, value_type == RGCSR_F64 ? RGCSR_F64 : RGCSR_F32);
}

RGCSR_API int rgcsr_cg(const rgcsr_matrix *A, const void *b, void *x, double rel_tol, int32_t max_iter,
                       int32_t check_every, void *workspace, size_t workspace_bytes, int32_t *iterations,
                       double *rel_residual, rgcsr_stream_t stream) {
    if (!A || A->n_rows != A->n_cols || A->n_rows < 0 || max_iter < 0 || check_every < 1 || !iterations ||
        !rel_residual)
        return RGCSR_ERR_INVALID_ARG;
    if (A->n_rows == 0) { *iterations = 0; *rel_residual = 0.0; return RGCSR_OK; }
    if (!b || !x) return RGCSR_ERR_INVALID_ARG;
    const int vt = vector_type(A);
    if (!workspace || workspace_bytes < cg_bytes(A->n_rows, vt)) return RGCSR_ERR_WORKSPACE;
    CgScratch c = carve_cg(workspace, A->n_rows, vt);
    if (const int cst = debug_check(A, (cudaStream_t)stream)) return cst;   // checks mode
    int its = 0;
    double rel = 0.0;
    const int st = vt == RGCSR_F64
        ? cg_run<double>(A, b, x, rel_tol, max_iter, check_every, c, &its, &rel, (cudaStream_t)stream)
        : cg_run<float>(A, b, x, rel_tol, max_iter, check_every, c, &its, &rel, (cudaStream_t)stream);
    *iterations = its;
    *rel_residual = rel;
    return st;
}

RGCSR_API size_t rgcsr_ir_cg_workspace_bytes(int64_t n) {
    if (n < 0) return 0;
    return 2 * align_up((size_t)n * 8, 256) + 2 * align_up((size_t)n * 4, 256) + 256 +
           align_up((size_t)kDotParts * 8, 256) + cg_bytes(n, RGCSR_F32);
}

RGCSR_API int rgcsr_ir_cg(const rgcsr_matrix *A_hi, const rgcsr_matrix *A_lo, const double *b, double *x,
                          double outer_tol, int32_t max_outer, double inner_tol, int32_t max_inner,
                          void *workspace, size_t workspace_bytes, int32_t *outer_iters,
                          int32_t *inner_iters, double *rel_residual, rgcsr_stream_t stream) {
    if (!A_hi || !A_lo || A_hi->value_type != RGCSR_F64 || A_lo->value_type == RGCSR_F64)
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    const int64_t n = A_hi->n_rows;
    if (n != A_hi->n_cols || A_lo->n_rows != n || A_lo->n_cols != n || max_outer < 0 || max_inner < 0 ||
        !outer_iters || !inner_iters || !rel_residual)
        return RGCSR_ERR_INVALID_ARG;
    *outer_iters = 0;
    *inner_iters = 0;
    *rel_residual = 0.0;
    if (n == 0) return RGCSR_OK;
    if (!b || !x) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_ir_cg_workspace_bytes(n)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int cst = debug_check(A_hi, s)) return cst;   // checks mode
    if (const int cst = debug_check(A_lo, s)) return cst;
    char *p = static_cast<char *>(workspace);
    double *r64 = reinterpret_cast<double *>(p); p += align_up((size_t)n * 8, 256);
    double *d64 = reinterpret_cast<double *>(p); p += align_up((size_t)n * 8, 256);
    float *r32 = reinterpret_cast<float *>(p); p += align_up((size_t)n * 4, 256);
    float *d32 = reinterpret_cast<float *>(p); p += align_up((size_t)n * 4, 256);
    double *scal = reinterpret_cast<double *>(p); p += 256;
    double *partials = reinterpret_cast<double *>(p); p += align_up((size_t)kDotParts * 8, 256);
    CgScratch inner = carve_cg(p, n, RGCSR_F32);

    int st;
    RGCSR_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * 8, s));
    if ((st = dot_device(n, b, b, &scal[0], partials, RGCSR_F64, s)) != RGCSR_OK) return st;
    double bb = 0.0;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&bb, &scal[0], sizeof(double), cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(bb > 0.0)) return RGCSR_OK;
    int total_inner = 0;
    double rel = 1.0;
    for (int k = 0; k <= max_outer; ++k) {
        // r = b - A x in FP64
        if ((st = rgcsr_spmv(A_hi, x, r64, stream)) != RGCSR_OK) return st;
        if ((st = axpby_device(n, 1.0, b, -1.0, r64, RGCSR_F64, s)) != RGCSR_OK) return st;
        if ((st = dot_device(n, r64, r64, &scal[1], partials, RGCSR_F64, s)) != RGCSR_OK) return st;
        double rr = 0.0;
        RGCSR_CUDA_TRY(cudaMemcpyAsync(&rr, &scal[1], sizeof(double), cudaMemcpyDeviceToHost, s));
        RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
        rel = std::sqrt(rr / bb);
        *outer_iters = k;
        if (rel <= outer_tol || k == max_outer || !(rel == rel)) break;
        // inner: A_lo d = r in float, to the inner tolerance or, when the outer
        // goal is nearer, only as far as it needs: a correction that cuts the
        // residual by outer_tol / rel (halved for safety) ends the solve
        if ((st = convert_device(n, r64, RGCSR_F64, r32, RGCSR_F32, s)) != RGCSR_OK) return st;
        int its = 0;
        double irel = 0.0;
        const double tol_k = std::max(inner_tol, 0.5 * outer_tol / rel);
        if ((st = cg_run<float>(A_lo, r32, d32, tol_k, max_inner, 10, inner, &its, &irel, s)) != RGCSR_OK)
            return st;
        total_inner += its;
        if ((st = convert_device(n, d32, RGCSR_F32, d64, RGCSR_F64, s)) != RGCSR_OK) return st;
        if ((st = axpby_device(n, 1.0, d64, 1.0, x, RGCSR_F64, s)) != RGCSR_OK) return st;
    }
    *inner_iters = total_inner;
    *rel_residual = rel;
    return RGCSR_OK;
}

RGCSR_API int rgcsr_set_wait_limit(int32_t polls) {
    if (polls < 0) return RGCSR_ERR_INVALID_ARG;
    g_wait_limit.store((unsigned)polls);
    return RGCSR_OK;
}
