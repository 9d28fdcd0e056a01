// convert.cu -- CSR -> RgCSR conversion (Sec. 3.4 of the paper: row groups,
// padding to the group's longest row, groupPointers, rowLengths).
//
// rgcsr_plan:    validate CSR (and the row order, if given), row lengths,
//                per-group slab size R_g*K_g, exclusive scan -> group_ptr;
//                returns n_stored to the host.
// rgcsr_convert: one warp per group streams the group's slab
//                [group_ptr[g], group_ptr[g+1]) with coalesced writes; slot
//                e of the slab is (slot j, row t) = (e / R_g, e % R_g).
//                Slabs over kBigSlab slots (groups holding very long rows)
//                are written one warp per row instead.
#include "common.cuh"

namespace rgcsr {
namespace {

struct PlanStatus {          // lives at the start of the plan workspace
    int flags;
    int pad;
    int64_t max_len;
};
constexpr size_t kStatusBytes = 256;

// One thread per group: slab size R_g * K_g into gp[g].
__global__ void group_sizes_kernel(const int32_t *__restrict__ rl, int64_t n, int32_t G,
                                   int64_t n_groups, int64_t *__restrict__ gp) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const int64_t first = g * G;
    const int64_t rows = min((int64_t)G, n - first);
    int kmax = 0;
    for (int64_t t = 0; t < rows; ++t) kmax = max(kmax, rl[first + t]);
    gp[g] = rows * (int64_t)kmax;
}

// Slabs larger than this go to scatter_big_kernel (one warp per row), so
// that a group holding very long rows does not serialise one warp.
constexpr int64_t kBigSlab = 32 * 256;

// Raw element copy: V = uint64_t (f64) or uint32_t (f32) keeps bits exact.
template <typename V>
__global__ void __launch_bounds__(256)
scatter_kernel(RowPtr rp, const int32_t *__restrict__ col, const V *__restrict__ val,
               int64_t n, int32_t G, int64_t n_groups, const int64_t *__restrict__ gp,
               const int32_t *__restrict__ rl, const int32_t *__restrict__ perm, V *__restrict__ out_val,
               int32_t *__restrict__ out_col, int64_t *__restrict__ s2c) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += warps) {
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const int64_t base = gp[g];
        const int64_t size = gp[g + 1] - base;
        if (size > kBigSlab) continue;              // scatter_big_kernel's work
        // (j, t) of slab element e = lane, then advanced by 32 each step
        int64_t j = lane / R;
        int t = lane % R;
        for (int64_t e = lane; e < size; e += 32) {
            const int64_t row = first + t;          // stored row
            const int len = rl[row];
            V v = 0;
            int c = 0;
            int64_t src = -1;
            const int64_t src_row = perm ? (int64_t)perm[row] : row;   // checked by rgcsr_plan
            if (j < len && src_row >= 0 && src_row < n) {
                src = rp[src_row] + j;
                v = val[src];
                c = col[src];
            }
            out_val[base + e] = v;
            out_col[base + e] = c;
            if (s2c) s2c[base + e] = src;
            t += 32;
            while (t >= R) { t -= R; ++j; }
        }
    }
}

// The slabs of big groups: one warp per stored row writes the row's K_g
// slots j (lane j mod 32) -- its entries, then padding.
template <typename V>
__global__ void __launch_bounds__(256)
scatter_big_kernel(RowPtr rp, const int32_t *__restrict__ col, const V *__restrict__ val,
                   int64_t n, int32_t G, const int64_t *__restrict__ gp, const int32_t *__restrict__ rl,
                   const int32_t *__restrict__ perm, V *__restrict__ out_val, int32_t *__restrict__ out_col,
                   int64_t *__restrict__ s2c) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += warps) {
        const int64_t g = row / G;
        const int64_t base = gp[g];
        const int64_t size = gp[g + 1] - base;
        if (size <= kBigSlab) continue;
        const int64_t first = g * G;
        const int R = (int)min((int64_t)G, n - first);
        const int64_t K = size / R;
        const int t = (int)(row - first);
        const int len = rl[row];
        const int64_t src_row = perm ? (int64_t)perm[row] : row;   // checked by rgcsr_plan
        const bool ok = src_row >= 0 && src_row < n;
        const int64_t r0 = ok ? rp[src_row] : 0;
        for (int64_t j = lane; j < K; j += 32) {
            V v = 0;
            int c = 0;
            int64_t src = -1;
            if (j < len && ok) {
                src = r0 + j;
                v = val[src];
                c = col[src];
            }
            const int64_t e = base + j * R + t;
            out_val[e] = v;
            out_col[e] = c;
            if (s2c) s2c[e] = src;
        }
    }
}

}  // namespace
}  // namespace rgcsr

using namespace rgcsr;

RGCSR_API size_t rgcsr_plan_workspace_bytes(int64_t n_rows, int32_t group_size) {
    if (n_rows < 0 || group_size < 1) return 0;
    int64_t n_groups = ceil_div(n_rows, group_size);
    return kStatusBytes + scan_partials_bytes(n_groups);
}

RGCSR_API int rgcsr_plan(const rgcsr_csr *A, rgcsr_matrix *M, void *workspace,
                         size_t workspace_bytes, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (!M || M->group_size < 1) return RGCSR_ERR_INVALID_ARG;
    const int64_t n = A->n_rows;
    const int32_t G = M->group_size;
    const int64_t n_groups = ceil_div(n, G);
    if (!M->group_ptr || (n > 0 && !M->row_lengths)) return RGCSR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < rgcsr_plan_workspace_bytes(n, G)) return RGCSR_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;

    auto *status = static_cast<PlanStatus *>(workspace);
    auto *partials = reinterpret_cast<int64_t *>(static_cast<char *>(workspace) + kStatusBytes);
    RGCSR_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(PlanStatus), s));
    if ((st = launch_validate_csr(A, &status->flags, &status->max_len, s)) != RGCSR_OK) return st;
    if (M->row_perm && n > 0) {
        // row_lengths doubles as the permutation check's hit counters
        if ((st = launch_check_perm(M->row_perm, n, M->row_lengths, &status->flags, s)) != RGCSR_OK) return st;
    }
    if ((st = launch_row_lengths(A, M->row_perm, M->row_lengths, s)) != RGCSR_OK) return st;
    if (n_groups > 0) {
        group_sizes_kernel<<<(unsigned)ceil_div(n_groups, 256), 256, 0, s>>>(
            M->row_lengths, n, G, n_groups, M->group_ptr);
        if ((st = launch_status()) != RGCSR_OK) return st;
    }
    if ((st = exclusive_scan_i64(M->group_ptr, n_groups, partials, s)) != RGCSR_OK) return st;

    PlanStatus host_status;
    int64_t n_stored = 0;
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&host_status, status, sizeof(PlanStatus), cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaMemcpyAsync(&n_stored, M->group_ptr + n_groups, sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, s));
    RGCSR_CUDA_TRY(cudaStreamSynchronize(s));
    if (host_status.flags & 1) return RGCSR_ERR_BAD_ROWPTR;
    if (host_status.flags & 2) return RGCSR_ERR_COL_OOB;
    if (host_status.flags & 4) return RGCSR_ERR_BAD_PERM;

    M->n_rows = n;
    M->n_cols = A->n_cols;
    M->nnz = A->nnz;
    M->n_groups = n_groups;
    M->n_stored = n_stored;
    M->max_row_len = host_status.max_len;
    return RGCSR_OK;
}

RGCSR_API int rgcsr_convert(const rgcsr_csr *A, const rgcsr_matrix *M, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (!M || M->group_size < 1 || M->n_rows != A->n_rows || M->nnz != A->nnz) return RGCSR_ERR_INVALID_ARG;
    if (M->value_type != A->value_type) return RGCSR_ERR_UNSUPPORTED_DTYPE;
    if (M->n_groups == 0 || M->n_stored == 0) return RGCSR_OK;
    if (!M->values || !M->columns || !M->group_ptr || !M->row_lengths) return RGCSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    RowPtr rp{A->row_ptr, A->row_ptr_type == RGCSR_I64};
    int64_t blocks = ceil_div(M->n_groups, 8);
    if (blocks > 152 * 64) blocks = 152 * 64;
    // big groups exist only if some row is longer than kBigSlab / G slots
    const bool big = M->max_row_len * M->group_size > kBigSlab || M->max_row_len > kBigSlab;
    int64_t big_blocks = ceil_div(M->n_rows, 8);
    if (big_blocks > 152 * 64) big_blocks = 152 * 64;
    if (A->value_type == RGCSR_F64) {
        scatter_kernel<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(
            rp, A->col_idx, static_cast<const uint64_t *>(A->values), M->n_rows, M->group_size,
            M->n_groups, M->group_ptr, M->row_lengths, M->row_perm, static_cast<uint64_t *>(M->values),
            M->columns, M->slot_to_csr);
        if (big)
            scatter_big_kernel<uint64_t><<<(unsigned)big_blocks, 256, 0, s>>>(
                rp, A->col_idx, static_cast<const uint64_t *>(A->values), M->n_rows, M->group_size,
                M->group_ptr, M->row_lengths, M->row_perm, static_cast<uint64_t *>(M->values), M->columns,
                M->slot_to_csr);
    } else {
        scatter_kernel<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(
            rp, A->col_idx, static_cast<const uint32_t *>(A->values), M->n_rows, M->group_size,
            M->n_groups, M->group_ptr, M->row_lengths, M->row_perm, static_cast<uint32_t *>(M->values),
            M->columns, M->slot_to_csr);
        if (big)
            scatter_big_kernel<uint32_t><<<(unsigned)big_blocks, 256, 0, s>>>(
                rp, A->col_idx, static_cast<const uint32_t *>(A->values), M->n_rows, M->group_size,
                M->group_ptr, M->row_lengths, M->row_perm, static_cast<uint32_t *>(M->values), M->columns,
                M->slot_to_csr);
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// rgcsr_plan_noalloc: rgcsr_plan for callers that cannot allocate device
// memory.  Its scratch (the plan's status block and scan partials) is one
// fixed array of this library, resident on every GPU that loads it until
// the process exits.  Host code must not hand the array's name to a kernel:
// on the host that symbol is only a stand-in, so every call looks up the
// array's device address on the current device with cudaGetSymbolAddress.
// The lookup is not cached: after a device reset or a new primary context
// the address may change, and the plan synchronises its stream anyway.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_plan_scratch[RGCSR_PLAN_NOALLOC_SCRATCH_BYTES];

RGCSR_API int rgcsr_plan_noalloc(const rgcsr_csr *A, rgcsr_matrix *M, rgcsr_stream_t stream) {
    int st = check_csr(A);
    if (st != RGCSR_OK) return st;
    if (!M || M->group_size < 1) return RGCSR_ERR_INVALID_ARG;
    const size_t need = rgcsr_plan_workspace_bytes(A->n_rows, M->group_size);
    if (need > sizeof(g_plan_scratch)) return RGCSR_ERR_WORKSPACE;   // beyond the fixed maximum
    void *scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_plan_scratch) != cudaSuccess || !scratch) return RGCSR_ERR_CUDA;
    // rgcsr_plan clears the status block itself and overwrites every scan
    // partial it reads, so stale contents of the shared array do not matter.
    return rgcsr_plan(A, M, scratch, sizeof(g_plan_scratch), stream);
}
