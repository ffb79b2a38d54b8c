// peaks.cu -- measured arithmetic peaks of the device (instrumentation: the
// denominators of the FP32 and FP64 rooflines the benchmark reports).
//
// A register-resident FMA loop: every thread runs CHAINS independent
// dependency chains a = a * b + c for `iters` rounds (no memory traffic
// inside the loop), the grid is a multiple of the SM count with full
// occupancy, and the kernel is timed with CUDA events after a warm-up launch.
// 2 flop per FMA.
#include <cuda_runtime.h>

#include "context.h"

namespace tsm {

namespace {

constexpr int PEAK_NT = 256;
constexpr int PEAK_CHAINS = 8;

template <class T>
__global__ void __launch_bounds__(PEAK_NT) fma_loop_kernel(int iters, T b, T c, T* __restrict__ sink) {
  T a[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
  // b = 1 and c = 0 keep the values bounded; the store happens only for a
  // value that never occurs, but the compiler cannot know it
  if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int measure_on(int device, double* tflops) {
  int sms = 0, per_sm = 0;
  TSM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  TSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_loop_kernel<T>, PEAK_NT, 0));
  if (sms <= 0 || per_sm <= 0) {
    set_error("tsm_measure_fma_peak: no resident blocks");
    return TSM_ERR_CUDA;
  }
  const int blocks = sms * per_sm;
  const int iters = sizeof(T) == 4 ? 1 << 10 : 1 << 11;   // tens of milliseconds per launch
  T* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  (void)cudaGetLastError();   // errors below are this routine's own
  cudaError_t e = cudaMalloc(&sink, (size_t)blocks * PEAK_NT * sizeof(T));
  const char* what = "cudaMalloc";
  if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    what = "cudaStreamCreateWithFlags";
  }
  if (e == cudaSuccess) {
    e = cudaEventCreate(&e0);
    what = "cudaEventCreate";
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {   // rep 0 is the warm-up
    what = "timed launch";
    e = cudaEventRecord(e0, s);
    if (e != cudaSuccess) break;
    fma_loop_kernel<T><<<blocks, PEAK_NT, 0, s>>>(iters, (T)1, (T)0, sink);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  int rc = TSM_OK;
  if (e == cudaSuccess && best > 0.f) {
    const double flop = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_NT;
    *tflops = flop / (best * 1e-3) / 1e12;
  } else {
    set_error("tsm_measure_fma_peak: %s: %s", what, cudaGetErrorString(e));
    rc = TSM_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  return rc;
}

// on `device`, leaving the calling thread's current device as it was
template <class T>
int measure(int device, double* tflops) {
  int prev = 0;
  TSM_CUDA(cudaGetDevice(&prev));
  TSM_CUDA(cudaSetDevice(device));
  const int rc = measure_on<T>(device, tflops);
  cudaSetDevice(prev);
  return rc;
}

}  // namespace

}  // namespace tsm

extern "C" int tsm_measure_fma_peak(int device, int prec, double* tflops) {
  if (tflops == nullptr) {
    tsm::set_error("tsm_measure_fma_peak: null output");
    return TSM_ERR_ARG;
  }
  if (prec == TSM_F32) return tsm::measure<float>(device, tflops);
  if (prec == TSM_F64) return tsm::measure<double>(device, tflops);
  tsm::set_error("tsm_measure_fma_peak: tier must be TSM_F32 or TSM_F64");
  return TSM_ERR_ARG;
}
