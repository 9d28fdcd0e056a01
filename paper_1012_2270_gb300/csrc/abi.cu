// abi.cu -- status strings and version of librgcsr.
#include "common.cuh"

RGCSR_API const char *rgcsr_status_string(int status) {
    switch (status) {
        case RGCSR_OK: return "ok";
        case RGCSR_ERR_INVALID_ARG: return "invalid argument";
        case RGCSR_ERR_BAD_ROWPTR: return "bad CSR row pointer (must start at 0, not decrease, end at nnz)";
        case RGCSR_ERR_COL_OOB: return "column index outside [0, n_cols)";
        case RGCSR_ERR_INDEX_OVERFLOW: return "size exceeds its index type";
        case RGCSR_ERR_UNSUPPORTED_DTYPE: return "unsupported value type for this call";
        case RGCSR_ERR_CUDA: return "CUDA runtime error";
        case RGCSR_ERR_WORKSPACE: return "workspace missing or too small";
        case RGCSR_ERR_BAD_PERM: return "row_perm is not a permutation of the rows";
        case RGCSR_ERR_CORRUPT: return "RgCSR matrix failed its structural checks";
        case RGCSR_ERR_TIMEOUT: return "a bounded device wait gave up";
        default: return "unknown status";
    }
}

RGCSR_API int rgcsr_version(void) { return 100; }
