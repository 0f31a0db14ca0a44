// Device probe: the FP64 rate that bounds the state-vector kernels on this GPU.
// Measures independent-DFMA throughput over the whole device and the latency of
// a dependent DFMA chain in one warp, and reports SM count, clock and memory
// limits. Every loop is bounded; timings use CUDA events around each launch.
#include <cuda_runtime.h>

#include <string>

#include "../../include/vqe.h"
#include "vqe_internal.h"

namespace {

__global__ void k_dfma_throughput(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_dfma_latency(double* out, long long* clk, int iters, double a, double b) {
  double x = threadIdx.x * 1e-9;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) x = fma(x, a, b);
  const long long t1 = clock64();
  out[threadIdx.x] = x;
  if (threadIdx.x == 0) *clk = t1 - t0;
}

}  // namespace

extern "C" int vqe_probe_fp64(double* dfma_per_sec, double* dfma_per_clock_per_sm, double* dependent_dfma_clocks,
                              int* sm_count, int* sm_clock_khz, size_t* smem_optin, int* l2_bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&p, dev);
  int clk = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return vqe::set_error(VQE_ERR_CUDA, (std::string("probe: ") + cudaGetErrorString(e)).c_str());
  const int blocks = p.multiProcessorCount * 4, threads = 256, iters = 1 << 13;
  double* d = nullptr;
  long long* c = nullptr;
  e = cudaMalloc(&d, size_t(blocks) * threads * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(long long));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  long long lat = 0;
  if (e == cudaSuccess) {
    k_dfma_throughput<<<blocks, threads>>>(d, iters, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0);
    k_dfma_throughput<<<blocks, threads>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) {
    k_dfma_latency<<<1, 32>>>(d, c, iters, 0.999999, 1e-7);
    e = cudaMemcpy(&lat, c, sizeof(long long), cudaMemcpyDeviceToHost);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  cudaFree(c);
  if (e != cudaSuccess) return vqe::set_error(VQE_ERR_CUDA, (std::string("probe: ") + cudaGetErrorString(e)).c_str());
  const double fmas = double(blocks) * threads * iters * 8.0;
  const double rate = fmas / (double(ms) * 1e-3);
  if (dfma_per_sec) *dfma_per_sec = rate;
  if (dfma_per_clock_per_sm) *dfma_per_clock_per_sm = rate / (double(p.multiProcessorCount) * double(clk) * 1e3);
  if (dependent_dfma_clocks) *dependent_dfma_clocks = double(lat) / iters;
  if (sm_count) *sm_count = p.multiProcessorCount;
  if (sm_clock_khz) *sm_clock_khz = clk;
  if (smem_optin) *smem_optin = p.sharedMemPerBlockOptin;
  if (l2_bytes) *l2_bytes = p.l2CacheSize;
  return VQE_OK;
}
