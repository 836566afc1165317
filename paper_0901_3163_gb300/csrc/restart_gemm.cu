// Restart GEMM through cuBLAS (a plain dense product, V_new = V P), FP32 basis.
#include <cublas_v2.h>

#include <vector>

#include "dlz_internal.cuh"

namespace dlz {

namespace {
int handle(Op &op, cublasHandle_t &h) {
    if (!op.blas) {
        cublasHandle_t c = nullptr;
        if (cublasCreate(&c) != CUBLAS_STATUS_SUCCESS) return fail(DLZ_ERR_CUDA, "cublasCreate failed");
        cublasSetMathMode(c, CUBLAS_DEFAULT_MATH);
        op.blas = c;
    }
    h = (cublasHandle_t)op.blas;
    if (cublasSetStream(h, op.stream) != CUBLAS_STATUS_SUCCESS) return fail(DLZ_ERR_CUDA, "cublasSetStream failed");
    return DLZ_OK;
}
}  // namespace

// Column-major view: the nin input vectors are the columns of A (ld = reals per
// vector); the row-major (nin x nout) P is, read column-major, the (nout x nin)
// matrix P^T, so C = A op(B) with op = transpose.
// dev_scratch: at least nin * nout doubles, alive until the GEMM has run (the host
// copy is staged by cudaMemcpyAsync before it returns).
int restart_gemm32(Op &op, float4 *out, const float4 *in, long n, int nin, int nout, const double *P_host,
                   void *dev_scratch) {
    cublasHandle_t h;
    DLZ_TRY(handle(op, h));
    std::vector<float> pf((size_t)nin * nout);
    for (size_t i = 0; i < pf.size(); ++i) pf[i] = (float)P_host[i];
    float *d = (float *)dev_scratch;
    DLZ_CUDA_TRY(cudaMemcpyAsync(d, pf.data(), pf.size() * sizeof(float), cudaMemcpyHostToDevice, op.stream));
    const int rows = (int)(4 * n);
    const float one = 1.f, zero = 0.f;
    if (cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, rows, nout, nin, &one, (const float *)in, rows, d, nout,
                    &zero, (float *)out, rows) != CUBLAS_STATUS_SUCCESS)
        return fail(DLZ_ERR_CUDA, "cublasSgemm failed");
    return DLZ_OK;      // cuBLAS's kernels are not counted among this library's launches
}

void blas_destroy(Op &op) {
    if (op.blas) cublasDestroy((cublasHandle_t)op.blas);
    op.blas = nullptr;
}

}  // namespace dlz
