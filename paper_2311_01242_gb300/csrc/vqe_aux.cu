// Small device helpers outside the state-vector path:
//   - refolding the Hamiltonian's group tables from new term coefficients
//     (same Pauli structure, new geometry r along a scan, Sec. 2.1.1);
//   - the sum of |table value| over all slots, which bounds every row sum of
//     |H| (the fixed-point H psi scales its tables by it);
//   - packing per-instance angle vectors given as an array of device pointers
//     into one row-major matrix, and unpacking gradients the same way.
//
// Every table slot of a group is a fixed linear combination of the kept terms'
// coefficients, with weights f * i^p, f in {+-1, +-2, +-4} and p in {0, 1}
// (the i^{|x&z|} phase of a Pauli term times the (-1)^{|u&z|} pattern sign and
// the 1 - 2n occupation factors). Each product w * c is exact in FP64, so the
// sum taken in the stored order gives the same bits on host and device.
#include <cuda_runtime.h>

#include "vqe_internal.h"

namespace vqe {
namespace {

__global__ void k_fold_coefs(int64_t n_slots, const int64_t* __restrict__ off, const int32_t* __restrict__ term,
                             const float* __restrict__ w, const double* __restrict__ coefs,
                             double* __restrict__ vals, double2* __restrict__ cvals) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  double re = 0.0, im = 0.0;
  for (int64_t j = off[s]; j < off[s + 1]; ++j) {
    const int32_t t = term[j];
    const double v = double(w[j]) * coefs[t & 0x7fffffff];
    if (t < 0)
      im += v;
    else
      re += v;
  }
  vals[s] = re;
  cvals[s] = make_double2(re, im);
}

__global__ void k_pack_rows(RowPtrs rp, double* __restrict__ dst, int64_t ld) {
  const int r = blockIdx.y;
  if (r >= rp.count) return;
  const double* src = rp.p[r];
  double* row = dst + int64_t(rp.base + r) * ld;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < rp.len[r]; k += gridDim.x * blockDim.x)
    row[k] = src[k];
}

__global__ void k_unpack_rows(RowPtrs rp, const double* __restrict__ src, int64_t ld) {
  const int r = blockIdx.y;
  if (r >= rp.count) return;
  double* dst = const_cast<double*>(rp.p[r]);
  const double* row = src + int64_t(rp.base + r) * ld;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < rp.len[r]; k += gridDim.x * blockDim.x)
    dst[k] = row[k];
}

// sum of |v| over n values, one block of 256 threads, fixed order
__global__ void k_abs_sum(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += fabs(v[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

cudaError_t abs_sum(const double* v, int64_t n, double* out, cudaStream_t stream) {
  k_abs_sum<<<1, 256, 0, stream>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t fold_coefs(int64_t n_slots, const int64_t* off, const int32_t* term, const float* w,
                       const double* coefs, double* vals, double2* cvals, cudaStream_t stream) {
  if (n_slots <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_slots + threads - 1) / threads;
  k_fold_coefs<<<unsigned(blocks), threads, 0, stream>>>(n_slots, off, term, w, coefs, vals, cvals);
  return cudaGetLastError();
}

cudaError_t pack_rows(const RowPtrs& rp, double* dst, int64_t ld, int max_len, cudaStream_t stream) {
  if (rp.count <= 0 || max_len <= 0) return cudaSuccess;
  const int threads = 128;
  dim3 grid(unsigned((max_len + threads - 1) / threads), unsigned(rp.count));
  k_pack_rows<<<grid, threads, 0, stream>>>(rp, dst, ld);
  return cudaGetLastError();
}

cudaError_t unpack_rows(const RowPtrs& rp, const double* src, int64_t ld, int max_len, cudaStream_t stream) {
  if (rp.count <= 0 || max_len <= 0) return cudaSuccess;
  const int threads = 128;
  dim3 grid(unsigned((max_len + threads - 1) / threads), unsigned(rp.count));
  k_unpack_rows<<<grid, threads, 0, stream>>>(rp, src, ld);
  return cudaGetLastError();
}

}  // namespace vqe
