// cg.cu -- conjugate gradients on an RgCSR operator and mixed-precision
// iterative refinement (the Krylov setting of the paper's introduction:
// a CG iteration is one SpMV plus SAXPY and SDOT operations).
//
// rgcsr_cg:    textbook CG from x0 = 0; the step lengths live in device
//              scalars, so an iteration is five kernels and no host
//              round trip; the host reads the residual norm every
//              `check_every` iterations to test convergence.
// rgcsr_ir_cg: outer loop in FP64 -- r = b - A x with the FP64 matrix,
//              stop when ||r|| <= tol ||b||; inner CG in float on a
//              lower-precision copy of A (float, bfloat16 or half values)
//              solves A d = r to a loose tolerance; x += d in FP64.
#include "common.cuh"

#include <cmath>

namespace rgcsr {
namespace {

constexpr int kThreads = 256;

unsigned grid(int64_t n) {
    int64_t b = ceil_div(n, kThreads);
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b > 0 ? b : 1);
}

// alpha = rr / dq;  x += alpha d;  r -= alpha q   (W elements per access)
template <typename T, int W>
__global__ void cg_xr_kernel(int64_t n, const double *__restrict__ rr, const double *__restrict__ dq,
                             T *__restrict__ x, T *__restrict__ r, const T *__restrict__ d,
                             const T *__restrict__ q) {
    const T alpha = (T)(*rr / *dq);
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        Pack<T, W> xv = ld_pack<T, W>(x + i * W), rv = ld_pack<T, W>(r + i * W);
        const Pack<T, W> dv = ld_pack<T, W>(d + i * W), qv = ld_pack<T, W>(q + i * W);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            xv.v[k] = fma(alpha, dv.v[k], xv.v[k]);
            rv.v[k] = fma(-alpha, qv.v[k], rv.v[k]);
        }
        st_pack<T, W>(x + i * W, xv);
        st_pack<T, W>(r + i * W, rv);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) {
        x[i] = fma(alpha, d[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// beta = rr_new / rr_old;  d = r + beta d
template <typename T, int W>
__global__ void cg_d_kernel(int64_t n, const double *__restrict__ rr_new, const double *__restrict__ rr_old,
                            const T *__restrict__ r, T *__restrict__ d) {
    const T beta = (T)(*rr_new / *rr_old);
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<T, W> rv = ld_pack<T, W>(r + i * W);
        Pack<T, W> dv = ld_pack<T, W>(d + i * W);
#pragma unroll
        for (int k = 0; k < W; ++k) dv.v[k] = fma(beta, dv.v[k], rv.v[k]);
        st_pack<T, W>(d + i * W, dv);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) d[i] = fma(beta, d[i], r[i]);
}

struct CgScratch {
    void *r, *d, *q;
    double *scal;       // [rr0, rr1, dq, spare]
    unsigned *count;    // the one-pass dot's block ticket (in the scalar block)
    double *partials;
};

size_t cg_bytes(int64_t n, int vt) {
    const size_t es = vt == RGCSR_F64 ? 8 : 4;
    return 3 * align_up((size_t)n * es, 256) + 256 + align_up((size_t)kDotParts * 8, 256);
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
    RGCSR_CUDA_TRY(cudaMemsetAsync(c.count, 0, sizeof(unsigned), s));
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
    auto iteration = [&](cudaStream_t st_, int cur_) -> int {
        int e;
        if ((e = rgcsr_spmv(A, c.d, c.q, (rgcsr_stream_t)st_)) != RGCSR_OK) return e;
        if ((e = dot_device(n, c.d, c.q, &c.scal[2], c.partials, vt, st_, c.count)) != RGCSR_OK) return e;
        T *xt = static_cast<T *>(x), *rt = static_cast<T *>(c.r), *dt = static_cast<T *>(c.d);
        const T *qt = static_cast<const T *>(c.q);
        if (vec)
            cg_xr_kernel<T, kW><<<grid(ceil_div(n, kW)), kThreads, 0, st_>>>(n, &c.scal[cur_], &c.scal[2], xt, rt,
                                                                            dt, qt);
        else
            cg_xr_kernel<T, 1><<<grid(n), kThreads, 0, st_>>>(n, &c.scal[cur_], &c.scal[2], xt, rt, dt, qt);
        if ((e = dot_device(n, c.r, c.r, &c.scal[1 - cur_], c.partials, vt, st_, c.count)) != RGCSR_OK) return e;
        if (vec)
            cg_d_kernel<T, kW><<<grid(ceil_div(n, kW)), kThreads, 0, st_>>>(n, &c.scal[1 - cur_], &c.scal[cur_],
                                                                           rt, dt);
        else
            cg_d_kernel<T, 1><<<grid(n), kThreads, 0, st_>>>(n, &c.scal[1 - cur_], &c.scal[cur_], rt, dt);
        return launch_status();
    };
    // After the first round of iterations (which also runs any one-off kernel
    // setup), the check_every iterations between two convergence checks are
    // recorded once into a CUDA graph (on a private stream: the caller's may
    // be the legacy default stream, which cannot be captured) and replayed on
    // the caller's stream.  check_every is even, so a round leaves `cur` as
    // it found it.  If recording fails the iterations are launched directly.
    cudaGraphExec_t round = nullptr;
    bool tried = false;
    while (it < max_iter) {
        const int chunk = check_every < max_iter - it ? check_every : max_iter - it;
        if (round && chunk == check_every) {
            RGCSR_CUDA_TRY(cudaGraphLaunch(round, s));
        } else {
            for (int i = 0; i < chunk; ++i) {
                if ((st = iteration(s, cur)) != RGCSR_OK) { if (round) cudaGraphExecDestroy(round); return st; }
                cur = 1 - cur;
            }
        }
        it += chunk;
        RGCSR_CUDA_TRY(cudaMemcpyAsync(&rr, &c.scal[cur], sizeof(double), cudaMemcpyDeviceToHost, s));
        RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
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
                        cudaGraphInstantiate(&round, g, 0) != cudaSuccess)
                        round = nullptr;
                    if (g) cudaGraphDestroy(g);
                }
                cudaStreamDestroy(cap);
            }
            cudaGetLastError();                      // a failed recording leaves no sticky error
        }
    }
    if (round) cudaGraphExecDestroy(round);
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
        // inner: A_lo d = r in float
        if ((st = convert_device(n, r64, RGCSR_F64, r32, RGCSR_F32, s)) != RGCSR_OK) return st;
        int its = 0;
        double irel = 0.0;
        if ((st = cg_run<float>(A_lo, r32, d32, inner_tol, max_inner, 10, inner, &its, &irel, s)) != RGCSR_OK)
            return st;
        total_inner += its;
        if ((st = convert_device(n, d32, RGCSR_F32, d64, RGCSR_F64, s)) != RGCSR_OK) return st;
        if ((st = axpby_device(n, 1.0, d64, 1.0, x, RGCSR_F64, s)) != RGCSR_OK) return st;
    }
    *inner_iters = total_inner;
    *rel_residual = rel;
    return RGCSR_OK;
}
