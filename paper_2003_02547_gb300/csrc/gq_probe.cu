// Arithmetic-rate probe of the GPU the library runs on: FP32 and FP64 FMA
// throughput measured with CUDA events, used as the denominators of the
// solver kernels' ALU roofline (the solver is neither a dense contraction
// nor bound by memory bandwidth, so its ceiling is the FMA rate of the
// precision it computes in).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gq.h"
#include "gq_batch.h"

namespace {

// eight independent FMA chains per thread, kIters rounds; the result is
// stored (conditionally) so that the chains are not removed
constexpr int kChains = 8;
constexpr int kIters = 4096;

__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe(T seed) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x * kChains + c);
  const T m = (T)0.999999, k = (T)1e-7;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (T)-1) g_probe_sink = (double)s;  // never true for these inputs (the chains tend to 0.1)
}

template <typename T>
int run_probe(double* flops, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return gq::set_error(GQ_ERR_CUDA, "probe: %s", cudaGetErrorString(e));
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return gq::set_error(GQ_ERR_CUDA, "probe: event creation failed");
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up clocks and caches
    cudaEventRecord(e0, stream);
    fma_probe<T><<<blocks, threads, 0, stream>>>((T)1);
    cudaEventRecord(e1, stream);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * kChains * kIters * (double)blocks * threads / (ms * 1e-3);
    if (rep > 0 && f > best) best = f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return gq::set_error(GQ_ERR_CUDA, "probe: %s", cudaGetErrorString(e));
  *flops = best;
  return GQ_OK;
}

}  // namespace

extern "C" int gq_probe_fma_rate(int fp64, void* stream, double* flops_per_s) {
  if (flops_per_s == nullptr) return gq::set_error(GQ_ERR_ARG, "flops_per_s is NULL");
  return fp64 ? run_probe<double>(flops_per_s, static_cast<cudaStream_t>(stream))
              : run_probe<float>(flops_per_s, static_cast<cudaStream_t>(stream));
}
