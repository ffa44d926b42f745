// cuSPARSE SpSV wrapper used ONLY as the benchmark's comparison column
// (the paper compares against cuSPARSE csrsv/csrsv2, Sec. 5; SpSV is the
// current API).  Built into its own library; the solver never links it.
#include <cuda_runtime.h>
#include <cusparse.h>

#include <cstdio>

namespace {
struct CusRef {
    cusparseHandle_t handle = nullptr;
    cusparseSpMatDescr_t A = nullptr;
    cusparseDnVecDescr_t x = nullptr, y = nullptr;
    cusparseSpSVDescr_t sv = nullptr;
    void* buffer = nullptr;
    cudaDataType dt = CUDA_R_64F;
};
}  // namespace

#define CS(expr)                                   \
    do {                                           \
        cusparseStatus_t _s = (expr);              \
        if (_s != CUSPARSE_STATUS_SUCCESS) return 100 + (int)_s; \
    } while (0)
#define CC(expr)                                   \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return 200 + (int)_e; \
    } while (0)

#define CUSREF_API __attribute__((visibility("default")))

extern "C" {

// Builds the cuSPARSE matrix/vector descriptors and runs SpSV analysis on
// `stream`.  Returns 0 on success; *out receives an opaque handle.
CUSREF_API int cusref_create(int n, int nnz, const int* rowptr, const int* colidx, const void* vals, int f64,
                  int upper, int unit, const void* x, void* y, void* stream, void** out) {
    if (!out) return 1;
    *out = nullptr;
    CusRef* h = new CusRef();
    h->dt = f64 ? CUDA_R_64F : CUDA_R_32F;
    CS(cusparseCreate(&h->handle));
    CS(cusparseSetStream(h->handle, (cudaStream_t)stream));
    CS(cusparseCreateCsr(&h->A, n, n, nnz, (void*)rowptr, (void*)colidx, (void*)vals,
                         CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, h->dt));
    cusparseFillMode_t fill = upper ? CUSPARSE_FILL_MODE_UPPER : CUSPARSE_FILL_MODE_LOWER;
    cusparseDiagType_t dg = unit ? CUSPARSE_DIAG_TYPE_UNIT : CUSPARSE_DIAG_TYPE_NON_UNIT;
    CS(cusparseSpMatSetAttribute(h->A, CUSPARSE_SPMAT_FILL_MODE, &fill, sizeof(fill)));
    CS(cusparseSpMatSetAttribute(h->A, CUSPARSE_SPMAT_DIAG_TYPE, &dg, sizeof(dg)));
    CS(cusparseCreateDnVec(&h->x, n, (void*)x, h->dt));
    CS(cusparseCreateDnVec(&h->y, n, y, h->dt));
    CS(cusparseSpSV_createDescr(&h->sv));
    double one64 = 1.0;
    float one32 = 1.0f;
    const void* alpha = f64 ? (const void*)&one64 : (const void*)&one32;
    size_t bytes = 0;
    CS(cusparseSpSV_bufferSize(h->handle, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, h->A, h->x, h->y,
                               h->dt, CUSPARSE_SPSV_ALG_DEFAULT, h->sv, &bytes));
    CC(cudaMalloc(&h->buffer, bytes > 0 ? bytes : 16));
    CS(cusparseSpSV_analysis(h->handle, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, h->A, h->x, h->y,
                             h->dt, CUSPARSE_SPSV_ALG_DEFAULT, h->sv, h->buffer));
    *out = h;
    return 0;
}

// y = op(A)^{-1} x with the analysed matrix; x and y may be new pointers.
CUSREF_API int cusref_solve(void* handle, const void* x, void* y, void* stream) {
    CusRef* h = (CusRef*)handle;
    if (!h) return 1;
    CS(cusparseSetStream(h->handle, (cudaStream_t)stream));
    CS(cusparseDnVecSetValues(h->x, (void*)x));
    CS(cusparseDnVecSetValues(h->y, y));
    double one64 = 1.0;
    float one32 = 1.0f;
    const void* alpha = h->dt == CUDA_R_64F ? (const void*)&one64 : (const void*)&one32;
    CS(cusparseSpSV_solve(h->handle, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, h->A, h->x, h->y,
                          h->dt, CUSPARSE_SPSV_ALG_DEFAULT, h->sv));
    return 0;
}

CUSREF_API int cusref_destroy(void* handle) {
    CusRef* h = (CusRef*)handle;
    if (!h) return 0;
    cudaDeviceSynchronize();
    if (h->sv) cusparseSpSV_destroyDescr(h->sv);
    if (h->x) cusparseDestroyDnVec(h->x);
    if (h->y) cusparseDestroyDnVec(h->y);
    if (h->A) cusparseDestroySpMat(h->A);
    if (h->handle) cusparseDestroy(h->handle);
    cudaFree(h->buffer);
    delete h;
    return 0;
}

}  // extern "C"
