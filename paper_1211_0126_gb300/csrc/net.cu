// net.cu -- tensor-core GEMM entry (tcgen05) used by the learned preconditioner.
#include "context.h"
#include "umma.cuh"

namespace tsm {

// C (FP32, M x N, leading dim ldc) = A (BF16, M x K) * B (BF16, N x K)^T (+ C if beta)
int launch_umma_gemm(cudaStream_t stream, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                     int K, int ldc, int beta, int* error) {
  if (M <= 0 || N <= 0) return TSM_OK;
  if (K <= 0 || (K % 8) != 0) {
    set_error("umma gemm needs K > 0 and K %% 8 == 0 (got %d)", K);
    return TSM_ERR_ARG;
  }
  const int gm = (M + UMMA_BM - 1) / UMMA_BM;
#define TSM_UMMA_CASE(BN)                                                                              \
  if (N <= BN) {                                                                                       \
    umma_gemm_kernel<BN><<<dim3(gm, 1), UMMA_THREADS, 0, stream>>>(A, B, C, M, N, K, ldc, beta, error); \
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_CUDA;                                  \
  }
  TSM_UMMA_CASE(16)
  TSM_UMMA_CASE(32)
  TSM_UMMA_CASE(64)
  TSM_UMMA_CASE(96)
  TSM_UMMA_CASE(128)
  TSM_UMMA_CASE(192)
#undef TSM_UMMA_CASE
  umma_gemm_kernel<128><<<dim3(gm, (N + 127) / 128), UMMA_THREADS, 0, stream>>>(A, B, C, M, N, K, ldc, beta, error);
  return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_CUDA;
}

}  // namespace tsm

extern "C" int tsm_umma_gemm(const void* A, const void* B, float* C, int M, int N, int K, int beta,
                             void* cuda_stream) {
  using namespace tsm;
  if (A == nullptr || B == nullptr || C == nullptr) {
    set_error("tsm_umma_gemm: null argument");
    return TSM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* err = nullptr;
  TSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(int), s));
  TSM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  int rc = launch_umma_gemm(s, static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), C, M, N, K,
                            N, beta, err);
  int herr = 0;
  if (rc == TSM_OK) {
    TSM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TSM_CUDA(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(err, s);
  if (rc != TSM_OK) {
    set_error("tsm_umma_gemm: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  if (herr) {
    set_error("tsm_umma_gemm: a tensor-core wait timed out");
    return TSM_ERR_TIMEOUT;
  }
  return TSM_OK;
}
