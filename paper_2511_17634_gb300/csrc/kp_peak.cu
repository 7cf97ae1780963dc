// kp_peak.cu -- measured FMA throughput of the FP64 and FP32 pipes, the
// denominators of the solvers' ALU roofline (the FP64 Krylov path is bound by
// its FP64 pipe on this part, not by HBM).
//
// Every thread runs eight independent FMA chains (enough to cover the pipe
// latency), all SMs are filled, and the kernel is timed with CUDA events on
// the context's stream after a warm-up launch.  The chains' results feed a
// guarded store, so the compiler cannot drop them.
#include <cuda_runtime.h>

#include "kp.h"
#include "kp_ctx.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345e-7) sink[blockIdx.x] = s;   // never true for these inputs
}

template <typename T>
cudaError_t time_chains(kp_ctx* c, int blocks, int iters, double* tflops) {
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&sink, (size_t)blocks * sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, 256, 0, c->stream>>>(sink, iters / 8, (T)0.999, (T)1e-4);   // warm-up
    e = cudaEventRecord(e0, c->stream);
  }
  if (e == cudaSuccess) {
    fma_chains_kernel<T><<<blocks, 256, 0, c->stream>>>(sink, iters, (T)0.999, (T)1e-4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *tflops = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return e;
}

}  // namespace

extern "C" kp_status kp_measure_alu_peaks(kp_ctx* c, double* fp64_tflops, double* fp32_tflops) {
  if (!c || !fp64_tflops || !fp32_tflops) return c ? kp::set_error(c, KP_ERR_ARG, "peaks: NULL output") : KP_ERR_ARG;
  const int blocks = 8 * c->sms;                  // 2048 threads per SM
  cudaError_t e = time_chains<double>(c, blocks, 1 << 12, fp64_tflops);
  if (e == cudaSuccess) e = time_chains<float>(c, blocks, 1 << 16, fp32_tflops);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "ALU peak measurement");
}
