// blas1.cu -- vector kernels for the Krylov and fixed-point solvers built on
// the SpMV (the paper's introduction: CG and GMRES need SpMV, SAXPY and
// SDOT).  Dot products are deterministic: fixed grid, fixed per-thread
// order, per-block tree, then one block sums the block results in order.
#include "common.cuh"

namespace rgcsr {
namespace {

constexpr int kDotThreads = 256;


// One thread's share of x . y over its grid-stride packs of W elements (in
// element order within a pack), then the last n mod W elements.
// Double vectors: one FP64 FMA per element.
template <int W>
__device__ __forceinline__ double dot_share(int64_t n, const double *__restrict__ x, const double *__restrict__ y) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    double s = 0.0;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<double, W> a = ld_pack<double, W>(x + i * W), b = ld_pack<double, W>(y + i * W);
#pragma unroll
        for (int k = 0; k < W; ++k) s = fma(a.v[k], b.v[k], s);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) s = fma(x[i], y[i], s);
    return s;
}


template <int W>
__device__ __forceinline__ double dot_share(int64_t n, const float *__restrict__ x, const float *__restrict__ y) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    float s = 0.0f, c = 0.0f;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<float, W> a = ld_pack<float, W>(x + i * W), b = ld_pack<float, W>(y + i * W);
#pragma unroll
        for (int k = 0; k < W; ++k) dot2_step(a.v[k], b.v[k], s, c);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) dot2_step(x[i], y[i], s, c);
    return (double)s + (double)c;
}

template <typename T, int W>
__global__ void __launch_bounds__(kDotThreads)
dot_partial(int64_t n, const T *__restrict__ x, const T *__restrict__ y, double *__restrict__ part) {
    __shared__ double sh[32];
    const double t = block_sum(dot_share<W>(n, x, y), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// The same partials, and the last block to finish (a ticket on *count after
// a fence) adds them in block order -- the sum dot_final forms -- and resets
// *count for the next call: one launch instead of two.
template <typename T, int W>
__global__ void __launch_bounds__(kDotThreads)
dot_onepass(int64_t n, const T *__restrict__ x, const T *__restrict__ y, double *__restrict__ part,
            unsigned *__restrict__ count, double *__restrict__ out) {
    __shared__ double sh[32];
    __shared__ bool last;
    const double t = block_sum(dot_share<W>(n, x, y), sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(part + i);
    const double total = block_sum(s, sh);
    if (threadIdx.x == 0) {
        *out = total;
        *count = 0u;
    }
}

__global__ void __launch_bounds__(kDotThreads)
dot_final(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) *out = t;
}

template <typename T, int W>
__global__ void axpby_kernel(int64_t n, double a, const T *__restrict__ x, double b, T *__restrict__ y) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<T, W> xv = ld_pack<T, W>(x + i * W);
        Pack<T, W> yv = ld_pack<T, W>(y + i * W);
#pragma unroll
        for (int k = 0; k < W; ++k) yv.v[k] = (T)(a * (double)xv.v[k] + b * (double)yv.v[k]);
        st_pack<T, W>(y + i * W, yv);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}

template <typename T, int W>
__global__ void jacobi_kernel(int64_t n, T omega, const T *__restrict__ dinv, const T *__restrict__ b,
                              const T *__restrict__ ax, const T *__restrict__ x, T *__restrict__ out) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<T, W> dv = ld_pack<T, W>(dinv + i * W), bv = ld_pack<T, W>(b + i * W),
                         av = ld_pack<T, W>(ax + i * W), xv = ld_pack<T, W>(x + i * W);
        Pack<T, W> o;
#pragma unroll
        for (int k = 0; k < W; ++k) o.v[k] = xv.v[k] + omega * dv.v[k] * (bv.v[k] - av.v[k]);
        st_pack<T, W>(out + i * W, o);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) out[i] = x[i] + omega * dinv[i] * (b[i] - ax[i]);
}

template <typename T, int W>
__global__ void diag_scale_kernel(int64_t n, T alpha, const T *__restrict__ d, const T *__restrict__ x,
                                  T *__restrict__ out) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<T, W> dv = ld_pack<T, W>(d + i * W), xv = ld_pack<T, W>(x + i * W);
        Pack<T, W> o;
#pragma unroll
        for (int k = 0; k < W; ++k) o.v[k] = alpha * dv.v[k] * xv.v[k];
        st_pack<T, W>(out + i * W, o);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) out[i] = alpha * d[i] * x[i];
}

// W = 2: 16 bytes on the double side, 8 on the float side.
template <typename S_, typename D, int W>
__global__ void convert_kernel(int64_t n, const S_ *__restrict__ src, D *__restrict__ dst) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x, tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = n / W;
    for (int64_t i = tid; i < nw; i += S) {
        const Pack<S_, W> a = ld_pack<S_, W>(src + i * W);
        Pack<D, W> o;
#pragma unroll
        for (int k = 0; k < W; ++k) o.v[k] = (D)a.v[k];
        st_pack<D, W>(dst + i * W, o);
    }
    for (int64_t i = nw * W + tid; i < n; i += S) dst[i] = (D)src[i];
}

unsigned vec_grid(int64_t n) {
    int64_t b = ceil_div(n, 256);
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b > 0 ? b : 1);
}

// A plain streaming read (16-byte loads, evict-first, grid-stride): the
// bandwidth reference for a kernel that moves the same bytes.  The sum is
// stored only if it equals a value the caller's data will not produce, so
// the loads cannot be dropped.
__global__ void __launch_bounds__(256)
stream_read_kernel(const float4 *__restrict__ p, int64_t n16, float *__restrict__ sink) {
    float s = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const float4 v = __ldcs(p + i);
        s += (v.x + v.y) + (v.z + v.w);
    }
    if (s == -1234567.0f) *sink = s;
}

// FP64 FMA throughput: eight independent chains a = a * m + c per thread,
// `iters` steps each.  m < 1 keeps every chain bounded; the sums are stored
// only if they equal a value the chains never reach, so no FMA is dropped.
__global__ void __launch_bounds__(256)
fp64_fma_kernel(int32_t iters, double m, double c, double *__restrict__ sink) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (double)(threadIdx.x + k);
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1234567.0) *sink = s;
}

// Random 8-byte loads of x[0, n) (n a power of two): each thread draws
// indices with a xorshift generator (Marsaglia 2003) and keeps four loads
// in flight per step; nothing is written unless the sum is exactly
// -1234567.  The gather pattern of an SpMV with random columns, without the
// matrix: its rate is the ceiling such an SpMV's x gathers can reach.
__global__ void __launch_bounds__(256)
gather_probe_kernel(const double *__restrict__ x, uint32_t mask, int32_t iters, double *__restrict__ sink) {
    uint32_t s = 0x9E3779B9u ^ ((uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u);
    auto next = [&s]() { s ^= s << 13; s ^= s >> 17; s ^= s << 5; return s; };
    double acc = 0.0;
    for (int32_t i = 0; i < iters; ++i) {
        const uint32_t a = next() & mask, b = next() & mask, c = next() & mask, d = next() & mask;
        acc += __ldg(x + a) + __ldg(x + b) + __ldg(x + c) + __ldg(x + d);
    }
    if (acc == -1234567.0) *sink = acc;
}

}  // namespace

int dot_device(int64_t n, const void *x, const void *y, double *out, double *partials, int value_type,
               cudaStream_t s, unsigned *count) {
    const unsigned g = (unsigned)kDotParts;
    const bool v = all_aligned16(x, y);
    const double *xd = static_cast<const double *>(x), *yd = static_cast<const double *>(y);
    const float *xf = static_cast<const float *>(x), *yf = static_cast<const float *>(y);
    if (count) {
        if (value_type == RGCSR_F64)
            v ? dot_onepass<double, 2><<<g, kDotThreads, 0, s>>>(n, xd, yd, partials, count, out)
              : dot_onepass<double, 1><<<g, kDotThreads, 0, s>>>(n, xd, yd, partials, count, out);
        else
            v ? dot_onepass<float, 4><<<g, kDotThreads, 0, s>>>(n, xf, yf, partials, count, out)
              : dot_onepass<float, 1><<<g, kDotThreads, 0, s>>>(n, xf, yf, partials, count, out);
        return launch_status();
    }
    if (value_type == RGCSR_F64)
        v ? dot_partial<double, 2><<<g, kDotThreads, 0, s>>>(n, xd, yd, partials)
          : dot_partial<double, 1><<<g, kDotThreads, 0, s>>>(n, xd, yd, partials);
    else
        v ? dot_partial<float, 4><<<g, kDotThreads, 0, s>>>(n, xf, yf, partials)
          : dot_partial<float, 1><<<g, kDotThreads, 0, s>>>(n, xf, yf, partials);
    dot_final<<<1, kDotThreads, 0, s>>>((int)g, partials, out);
    return launch_status();
}

int axpby_device(int64_t n, double a, const void *x, double b, void *y, int value_type, cudaStream_t s) {
    if (n <= 0) return RGCSR_OK;
    const bool v = all_aligned16(x, y);
    if (value_type == RGCSR_F64) {
        const double *xd = static_cast<const double *>(x);
        double *yd = static_cast<double *>(y);
        v ? axpby_kernel<double, 2><<<vec_grid(ceil_div(n, 2)), 256, 0, s>>>(n, a, xd, b, yd)
          : axpby_kernel<double, 1><<<vec_grid(n), 256, 0, s>>>(n, a, xd, b, yd);
    } else {
        const float *xf = static_cast<const float *>(x);
        float *yf = static_cast<float *>(y);
        v ? axpby_kernel<float, 4><<<vec_grid(ceil_div(n, 4)), 256, 0, s>>>(n, a, xf, b, yf)
          : axpby_kernel<float, 1><<<vec_grid(n), 256, 0, s>>>(n, a, xf, b, yf);
    }
    return launch_status();
}

int convert_device(int64_t n, const void *src, int src_type, void *dst, int dst_type, cudaStream_t s) {
    if (n <= 0) return RGCSR_OK;
    const bool v = all_aligned16(src, dst);
    if (src_type == RGCSR_F64 && dst_type == RGCSR_F32) {
        const double *a = static_cast<const double *>(src);
        float *o = static_cast<float *>(dst);
        v ? convert_kernel<double, float, 2><<<vec_grid(ceil_div(n, 2)), 256, 0, s>>>(n, a, o)
          : convert_kernel<double, float, 1><<<vec_grid(n), 256, 0, s>>>(n, a, o);
    } else if (src_type == RGCSR_F32 && dst_type == RGCSR_F64) {
        const float *a = static_cast<const float *>(src);
        double *o = static_cast<double *>(dst);
        v ? convert_kernel<float, double, 2><<<vec_grid(ceil_div(n, 2)), 256, 0, s>>>(n, a, o)
          : convert_kernel<float, double, 1><<<vec_grid(n), 256, 0, s>>>(n, a, o);
    } else {
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
    return launch_status();
}

}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t rgcsr_dot_workspace_bytes(void) { return (size_t)kDotParts * sizeof(double); }

RGCSR_API int rgcsr_dot(int64_t n, const void *x, const void *y, double *result, void *workspace,
                        size_t workspace_bytes, int32_t value_type, rgcsr_stream_t stream) {
    if (n < 0 || !result || (n > 0 && (!x || !y))) return RGCSR_ERR_INVALID_ARG;
    if (value_type != RGCSR_F64 && value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (!workspace || workspace_bytes < rgcsr_dot_workspace_bytes()) return RGCSR_ERR_WORKSPACE;
    return dot_device(n, x, y, result, static_cast<double *>(workspace), value_type, (cudaStream_t)stream);
}

RGCSR_API int rgcsr_axpby(int64_t n, double alpha, const void *x, double beta, void *y, int32_t value_type,
                          rgcsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return RGCSR_ERR_INVALID_ARG;
    if (value_type != RGCSR_F64 && value_type != RGCSR_F32) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    return axpby_device(n, alpha, x, beta, y, value_type, (cudaStream_t)stream);
}

RGCSR_API int rgcsr_jacobi_step(int64_t n, double omega, const void *dinv, const void *b, const void *Ax,
                                const void *x, void *x_out, int32_t value_type, rgcsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!dinv || !b || !Ax || !x || !x_out))) return RGCSR_ERR_INVALID_ARG;
    if (n == 0) return RGCSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool v = all_aligned16(dinv, b, Ax, x, x_out);
    if (value_type == RGCSR_F64) {
        auto p = [](const void *q) { return static_cast<const double *>(q); };
        double *o = static_cast<double *>(x_out);
        v ? jacobi_kernel<double, 2><<<vec_grid(ceil_div(n, 2)), 256, 0, s>>>(n, omega, p(dinv), p(b), p(Ax), p(x), o)
          : jacobi_kernel<double, 1><<<vec_grid(n), 256, 0, s>>>(n, omega, p(dinv), p(b), p(Ax), p(x), o);
    } else if (value_type == RGCSR_F32) {
        auto p = [](const void *q) { return static_cast<const float *>(q); };
        float *o = static_cast<float *>(x_out);
        const float w = (float)omega;
        v ? jacobi_kernel<float, 4><<<vec_grid(ceil_div(n, 4)), 256, 0, s>>>(n, w, p(dinv), p(b), p(Ax), p(x), o)
          : jacobi_kernel<float, 1><<<vec_grid(n), 256, 0, s>>>(n, w, p(dinv), p(b), p(Ax), p(x), o);
    } else {
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
    return launch_status();
}

RGCSR_API int rgcsr_diag_scale(int64_t n, double alpha, const void *d, const void *x, void *out,
                               int32_t value_type, rgcsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!d || !x || !out))) return RGCSR_ERR_INVALID_ARG;
    if (n == 0) return RGCSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool v = all_aligned16(d, x, out);
    if (value_type == RGCSR_F64) {
        const double *dd = static_cast<const double *>(d), *xd = static_cast<const double *>(x);
        double *o = static_cast<double *>(out);
        v ? diag_scale_kernel<double, 2><<<vec_grid(ceil_div(n, 2)), 256, 0, s>>>(n, alpha, dd, xd, o)
          : diag_scale_kernel<double, 1><<<vec_grid(n), 256, 0, s>>>(n, alpha, dd, xd, o);
    } else if (value_type == RGCSR_F32) {
        const float *df = static_cast<const float *>(d), *xf = static_cast<const float *>(x);
        float *o = static_cast<float *>(out);
        v ? diag_scale_kernel<float, 4><<<vec_grid(ceil_div(n, 4)), 256, 0, s>>>(n, (float)alpha, df, xf, o)
          : diag_scale_kernel<float, 1><<<vec_grid(n), 256, 0, s>>>(n, (float)alpha, df, xf, o);
    } else {
        return RGCSR_ERR_UNSUPPORTED_DTYPE;
    }
    return launch_status();
}

RGCSR_API int rgcsr_convert_vector(int64_t n, const void *src, int32_t src_type, void *dst, int32_t dst_type,
                                   rgcsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!src || !dst))) return RGCSR_ERR_INVALID_ARG;
    return convert_device(n, src, src_type, dst, dst_type, (cudaStream_t)stream);
}

RGCSR_API int rgcsr_stream_read(const void *data, int64_t bytes, void *sink, rgcsr_stream_t stream) {
    if (bytes < 0 || bytes % 16 != 0 || (bytes > 0 && (!data || !sink)) || ((uintptr_t)data & 15) != 0)
        return RGCSR_ERR_INVALID_ARG;
    if (bytes == 0) return RGCSR_OK;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n16 = bytes / 16;
    int64_t grid = (int64_t)sms * 8;                     // 8 CTAs of 256 threads per SM
    if (ceil_div(n16, (int64_t)256) < grid) grid = ceil_div(n16, (int64_t)256);
    stream_read_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(static_cast<const float4 *>(data), n16,
                                                                         static_cast<float *>(sink));
    return launch_status();
}

RGCSR_API int rgcsr_gather_probe(const void *x, int64_t n, int32_t iters, void *sink, int64_t *loads,
                                 rgcsr_stream_t stream) {
    if (!x || !sink || !loads || iters < 1 || n < 32 || n > ((int64_t)1 << 32) || (n & (n - 1)) != 0)
        return RGCSR_ERR_INVALID_ARG;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 4;                            // 4 CTAs of 256 threads per SM
    *loads = (int64_t)grid * 256 * 4 * iters;
    gather_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(static_cast<const double *>(x),
                                                                (uint32_t)(n - 1), iters,
                                                                static_cast<double *>(sink));
    return launch_status();
}

RGCSR_API int rgcsr_fp64_fma_probe(int32_t iters, void *sink, int64_t *fmas, rgcsr_stream_t stream) {
    if (iters < 1 || !sink || !fmas) return RGCSR_ERR_INVALID_ARG;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8;                            // 8 CTAs of 256 threads per SM
    *fmas = (int64_t)grid * 256 * 8 * iters;
    fp64_fma_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(iters, 0.9999999, 1e-7, static_cast<double *>(sink));
    return launch_status();
}
