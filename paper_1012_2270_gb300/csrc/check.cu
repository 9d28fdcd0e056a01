// check.cu -- structural checks of an RgCSR matrix on the device (a stand-in
// for a memory checker), and the checks mode in which every product checks
// its matrix before any kernel of it runs.
//
// The layout checked is that of Sec. 3.4: group g holds R_g = min(G, n - gG)
// rows whose j-th entries are contiguous, K_g = its longest row, so its slab
// is R_g * K_g slots starting at group_ptr[g]; the slots past a row's length
// are the artificial zeros (value bits 0, column 0 here).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <cstdlib>
#include <mutex>

#include "common.cuh"

namespace rgcsr {
namespace {

constexpr int kCheckThreads = 256;

struct CheckRecord {
    unsigned int flags;
    unsigned int reserved;
    unsigned long long first_group, first_row, first_slot;
    unsigned long long length_sum;   // sum of the non-negative row lengths
    unsigned long long perm_sum;     // sum over k of mix(k + 1) - mix(perm[k] + 1)
};

__device__ CheckRecord g_check;

__device__ __forceinline__ void fail(unsigned flag, unsigned long long *first, long long index) {
    atomicOr(&g_check.flags, flag);
    if (first) atomicMin(first, (unsigned long long)index);
}

__device__ __forceinline__ unsigned long long value_bits(const void *values, int bytes, int64_t s) {
    if (bytes == 8) return static_cast<const unsigned long long *>(values)[s];
    if (bytes == 4) return static_cast<const unsigned int *>(values)[s];
    return static_cast<const unsigned short *>(values)[s];
}

// One warp per group (grid-stride).  Every load is inside the sizes the
// matrix declares: group_ptr[0, n_groups], row_lengths / row_perm /
// row_scale [0, n_rows), the slabs [0, n_stored) -- whatever they hold.
__global__ void __launch_bounds__(kCheckThreads)
check_groups_kernel(int64_t n_rows, int64_t n_cols, int64_t nnz, int32_t G, int64_t n_groups,
                    int64_t n_stored, int64_t max_row_len, const void *__restrict__ values, int value_bytes,
                    const int32_t *__restrict__ columns, const int64_t *__restrict__ group_ptr,
                    const int32_t *__restrict__ row_lengths, const float *__restrict__ row_scale,
                    const int64_t *__restrict__ slot_to_csr, const int32_t *__restrict__ perm) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kCheckThreads / 32);
    for (int64_t g = (int64_t)blockIdx.x * (kCheckThreads / 32) + (threadIdx.x >> 5); g < n_groups; g += warps) {
        const int64_t base = g * G;
        const int R = (int)min((int64_t)G, n_rows - base);
        // rows: lengths, scale, permutation entries
        int K = 0;
        unsigned long long lsum = 0, psum = 0;
        for (int t = lane; t < R; t += 32) {
            const int64_t r = base + t;
            const int len = row_lengths[r];
            if (len < 0 || len > max_row_len) fail(RGCSR_CHECK_ROW_LENGTHS, &g_check.first_row, r);
            if (len > 0) { K = max(K, len); lsum += (unsigned long long)len; }
            if (row_scale) {
                const float sc = row_scale[r];
                if (!(sc > 0.0f) || !isfinite(sc)) fail(RGCSR_CHECK_SCALE, &g_check.first_row, r);
            }
            if (perm) {
                const int32_t p = perm[r];
                if (p < 0 || p >= n_rows) fail(RGCSR_CHECK_PERM, &g_check.first_row, r);
                psum += mix64((unsigned long long)r + 1) - mix64((unsigned long long)(int64_t)p + 1);
            }
        }
        K = warp_max_i(K);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lsum += __shfl_xor_sync(kFull, lsum, o);
            psum += __shfl_xor_sync(kFull, psum, o);
        }
        if (lane == 0) {
            atomicAdd(&g_check.length_sum, lsum);
            if (perm) atomicAdd(&g_check.perm_sum, psum);
        }
        // the group's slab
        const int64_t lo = group_ptr[g], hi = group_ptr[g + 1];
        const bool bad = lo < 0 || hi < lo || hi > n_stored || hi - lo != (int64_t)R * K ||
                         (g == 0 && lo != 0) || (g == n_groups - 1 && hi != n_stored);
        if (bad && lane == 0) fail(RGCSR_CHECK_GROUP_PTR, &g_check.first_group, g);
        const int64_t a = min(max(lo, (int64_t)0), n_stored);
        const int64_t b = min(max(hi, a), n_stored);
        for (int64_t s = a + lane; s < b; s += 32) {
            const int64_t off = s - lo;                 // >= 0: s >= a >= lo, or lo < 0
            const int t = (int)(off % R);
            const int64_t j = off / R;
            const bool valid = j < (int64_t)row_lengths[base + t];
            const int32_t c = columns[s];
            if (valid) {
                if (c < 0 || c >= n_cols) fail(RGCSR_CHECK_COLUMN, &g_check.first_slot, s);
            } else if (c != 0 || value_bits(values, value_bytes, s) != 0) {
                fail(RGCSR_CHECK_PADDING, &g_check.first_slot, s);
            }
            if (slot_to_csr) {
                const int64_t m = slot_to_csr[s];
                if (valid ? (m < 0 || m >= nnz) : m != -1) fail(RGCSR_CHECK_SLOT_MAP, &g_check.first_slot, s);
            }
        }
    }
}

std::mutex g_check_mutex;                  // one device record: one check at a time
std::atomic<int> g_checks_on{0};
std::atomic<int> g_host_status{0};

// RGCSR_CHECKS=1 in the environment turns checks mode on when the library loads.
const bool g_checks_env = [] {
    const char *e = std::getenv("RGCSR_CHECKS");
    if (e && e[0] == '1' && e[1] == '\0') g_checks_on.store(1);
    return true;
}();

int check_matrix_fields(const rgcsr_matrix *M) {
    if (!M || M->n_rows < 0 || M->n_cols < 0 || M->nnz < 0 || M->group_size < 1 || M->n_stored < 0)
        return RGCSR_ERR_INVALID_ARG;
    if (M->n_rows == 0) return RGCSR_OK;
    if (M->n_groups != ceil_div(M->n_rows, M->group_size)) return RGCSR_ERR_INVALID_ARG;
    if (value_bytes(M->value_type) == 0) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (!M->group_ptr || !M->row_lengths) return RGCSR_ERR_INVALID_ARG;
    if (M->n_stored > 0 && (!M->values || !M->columns)) return RGCSR_ERR_INVALID_ARG;
    return RGCSR_OK;
}

}  // namespace

int take_host_status() { return g_host_status.exchange(0); }

int run_check(const rgcsr_matrix *M, rgcsr_check_report *report, cudaStream_t s) {
    report->flags = 0;
    report->reserved = 0;
    report->group = report->row = report->slot = -1;
    if (M->n_rows == 0) return RGCSR_OK;
    const bool quantized = M->value_type == RGCSR_BF16 || M->value_type == RGCSR_F16;
    int flags = 0;
    if (quantized && !M->row_scale) flags |= RGCSR_CHECK_SCALE;
    CheckRecord rec;
    {
        std::lock_guard<std::mutex> lock(g_check_mutex);
        CheckRecord init{};
        init.first_group = init.first_row = init.first_slot = ULLONG_MAX;
        RGCSR_CUDA_TRY(cudaMemcpyToSymbolAsync(g_check, &init, sizeof(init), 0, cudaMemcpyHostToDevice, s));
        const int64_t blocks = std::min<int64_t>(ceil_div(M->n_groups, kCheckThreads / 32), 152 * 16);
        check_groups_kernel<<<(unsigned)blocks, kCheckThreads, 0, s>>>(
            M->n_rows, M->n_cols, M->nnz, M->group_size, M->n_groups, M->n_stored, M->max_row_len, M->values,
            (int)value_bytes(M->value_type), M->columns, M->group_ptr, M->row_lengths,
            quantized ? M->row_scale : nullptr, M->slot_to_csr, M->row_perm);
        RGCSR_CUDA_TRY(cudaGetLastError());
        RGCSR_CUDA_TRY(cudaMemcpyFromSymbolAsync(&rec, g_check, sizeof(rec), 0, cudaMemcpyDeviceToHost, s));
        RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    }
    flags |= (int)rec.flags;
    if (rec.length_sum != (unsigned long long)M->nnz) flags |= RGCSR_CHECK_ROW_LENGTHS;
    if (M->row_perm && rec.perm_sum != 0) flags |= RGCSR_CHECK_PERM;
    report->flags = flags;
    if (rec.first_group != ULLONG_MAX) report->group = (int64_t)rec.first_group;
    if (rec.first_row != ULLONG_MAX) report->row = (int64_t)rec.first_row;
    if (rec.first_slot != ULLONG_MAX) report->slot = (int64_t)rec.first_slot;
    return flags ? RGCSR_ERR_CORRUPT : RGCSR_OK;
}

int debug_check(const rgcsr_matrix *M, cudaStream_t s) {
    if (!g_checks_on.load(std::memory_order_relaxed) || !M) return RGCSR_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return RGCSR_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return RGCSR_OK;      // a graph being captured: unchecked
    if (check_matrix_fields(M) != RGCSR_OK) return RGCSR_OK;    // the product's own argument checks report it
    rgcsr_check_report rep;
    const int st = run_check(M, &rep, s);
    if (st == RGCSR_ERR_CORRUPT) g_host_status.fetch_or(RGCSR_STATUS_CORRUPT);
    return st;
}

}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API int rgcsr_check_matrix(const rgcsr_matrix *M, rgcsr_check_report *report, rgcsr_stream_t stream) {
    if (!report) return RGCSR_ERR_INVALID_ARG;
    const int st = check_matrix_fields(M);
    if (st != RGCSR_OK) return st;
    return run_check(M, report, (cudaStream_t)stream);
}

RGCSR_API int rgcsr_set_checks(int on) { return g_checks_on.exchange(on ? 1 : 0); }
