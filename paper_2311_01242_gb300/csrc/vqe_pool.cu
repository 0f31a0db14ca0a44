// ADAPT-VQE operator screening (Sec. 2.1.1, ADAPT-VQE): after the forward sweep
// and H psi, the energy gradient of every pool operator appended at angle 0,
//   g_j = 2 Re <lambda| T_j - T_j^dagger |psi>,   lambda = H psi,
// in one launch over the pool's amplitude pairs plus one finalising launch.
//
// For a pair (k, k') of operator j with T_j|k> = s|k'>, the generator maps
// |k> -> s|k'> and |k'> -> -s|k>, so the pair adds s (lambda[k'] psi[k] -
// lambda[k] psi[k']) (real parts of conj(lambda) psi for complex amplitudes).
// Pairs come from the pool handle's rank-pair list (sector ranks of k and k',
// the sign in bit 31), so psi and lambda are read in the compressed sector
// layout the streaming kernels leave them in.
//
// psi and lambda are first copied side by side (entry r = {psi[r], lambda[r]}),
// so each rank of a pair costs one 16-byte (real) or 32-byte (complex) gather
// from one L2 sector instead of two gathers from two sectors. The pair records
// are read once, with the streaming (evict-first) cache hint, so that they do
// not push the gathered entries out of L2.
//
// Work split: operator j's pairs are cut into chunks of kPoolChunk; a block
// sums one chunk (thread-strided, then a fixed shuffle/shared-memory tree) and
// writes one partial; the finaliser adds operator j's partials in chunk order.
// The result does not depend on the grid size or on scheduling.
#include <cuda_runtime.h>

#include "vqe_internal.h"

namespace vqe {
namespace {

constexpr int kPoolThreads = 256;
constexpr int kPoolUnroll = 4;
static_assert(kPoolChunk % (kPoolThreads * kPoolUnroll) == 0, "chunk must be whole unrolled sweeps");

// v with its sign bit flipped when s == 1
__device__ __forceinline__ double flip_sign(double v, uint32_t s) {
  return __hiloint2double(__double2hiint(v) ^ int(s << 31), __double2loint(v));
}

// lb pa - la pb (real), Re(conj(lb) pa) - Re(conj(la) pb) (complex)
__device__ __forceinline__ double pair_term(double lb, double pa, double la, double pb) {
  return fma(lb, pa, -(la * pb));
}
__device__ __forceinline__ double pair_term(double2 lb, double2 pa, double2 la, double2 pb) {
  return fma(lb.x, pa.x, fma(lb.y, pa.y, -fma(la.x, pb.x, la.y * pb.y)));
}

// index m with chunk_off[m] <= c < chunk_off[m + 1] (chunk_off nondecreasing)
__device__ __forceinline__ int owner_of(const int64_t* __restrict__ chunk_off, int M, int64_t c) {
  int lo = 0, hi = M;  // invariant: chunk_off[lo] <= c < chunk_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(chunk_off + mid) <= c)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// psi and lambda of one sector entry, side by side
template <typename T> struct alignas(2 * sizeof(T)) PsiLam {
  T p, l;
};

__device__ __forceinline__ PsiLam<double> load_pl(const PsiLam<double>* v) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(v));
  return {t.x, t.y};
}
__device__ __forceinline__ PsiLam<double2> load_pl(const PsiLam<double2>* v) {
  const double2* q = reinterpret_cast<const double2*>(v);
  return {__ldg(q), __ldg(q + 1)};
}

template <typename T>
__global__ void k_interleave(const T* __restrict__ psi, const T* __restrict__ lam, int64_t D,
                             PsiLam<T>* __restrict__ out) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D; r += int64_t(gridDim.x) * blockDim.x)
    out[r] = PsiLam<T>{psi[r], lam[r]};
}

template <typename T>
__global__ void __launch_bounds__(kPoolThreads) k_pool_grad(const uint2* __restrict__ rp,
                                                            const int64_t* __restrict__ pair_off,
                                                            const int64_t* __restrict__ chunk_off, int M,
                                                            const PsiLam<T>* __restrict__ pl,
                                                            double* __restrict__ part) {
  __shared__ double red[kPoolThreads / 32];
  const int64_t n_chunks = __ldg(chunk_off + M);
  for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const int m = owner_of(chunk_off, M, c);
    const int64_t p0 = __ldg(pair_off + m) + (c - __ldg(chunk_off + m)) * int64_t(kPoolChunk);
    const int64_t p_end = __ldg(pair_off + m + 1);
    const int64_t p1 = p0 + kPoolChunk < p_end ? p0 + kPoolChunk : p_end;
    double acc = 0.0;
    for (int64_t base = p0 + threadIdx.x; base < p1; base += int64_t(kPoolThreads) * kPoolUnroll) {
      uint2 pr[kPoolUnroll];
#pragma unroll
      for (int u = 0; u < kPoolUnroll; ++u) {
        const int64_t p = base + int64_t(u) * kPoolThreads;
        pr[u] = p < p1 ? __ldcs(rp + p) : make_uint2(0u, 0u);  // read once: evict first from L2
      }
      PsiLam<T> a[kPoolUnroll], b[kPoolUnroll];
#pragma unroll
      for (int u = 0; u < kPoolUnroll; ++u) {
        a[u] = load_pl(pl + (pr[u].x & 0x7fffffffu));
        b[u] = load_pl(pl + pr[u].y);
      }
#pragma unroll
      for (int u = 0; u < kPoolUnroll; ++u) {
        const int64_t p = base + int64_t(u) * kPoolThreads;
        if (p < p1) acc += flip_sign(pair_term(b[u].l, a[u].p, a[u].l, b[u].p), pr[u].x >> 31);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kPoolThreads / 32; ++w) s += red[w];
      part[c] = s;
    }
    __syncthreads();
  }
}

// g[m] = 2 * (sum of operator m's chunk partials in chunk order); one warp per operator
__global__ void k_pool_finalize(const double* __restrict__ part, const int64_t* __restrict__ chunk_off, int M,
                                double* __restrict__ g) {
  const int m = blockIdx.x;
  if (m >= M) return;
  const int64_t c0 = __ldg(chunk_off + m), c1 = __ldg(chunk_off + m + 1);
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += 32) s += part[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) g[m] = 2.0 * s;
}

}  // namespace

cudaError_t pool_gradients(const uint2* rpairs, const int64_t* pair_off, const int64_t* chunk_off, int M,
                           int64_t n_chunks, bool real, const void* psi, const void* lam, int64_t D, void* pl,
                           double* part, double* grad, cudaStream_t stream) {
  if (M <= 0) return cudaSuccess;
  if (n_chunks > 0) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t cap = int64_t(sms) * 8;  // 8 resident blocks of 256 threads per SM
    const unsigned grid = unsigned(n_chunks < cap ? n_chunks : cap);
    const int64_t ib = (D + 255) / 256;
    const unsigned igrid = unsigned(ib < cap ? ib : cap);
    if (real) {
      auto* v = static_cast<PsiLam<double>*>(pl);
      k_interleave<double><<<igrid, 256, 0, stream>>>(static_cast<const double*>(psi),
                                                      static_cast<const double*>(lam), D, v);
      k_pool_grad<double><<<grid, kPoolThreads, 0, stream>>>(rpairs, pair_off, chunk_off, M, v, part);
    } else {
      auto* v = static_cast<PsiLam<double2>*>(pl);
      k_interleave<double2><<<igrid, 256, 0, stream>>>(static_cast<const double2*>(psi),
                                                       static_cast<const double2*>(lam), D, v);
      k_pool_grad<double2><<<grid, kPoolThreads, 0, stream>>>(rpairs, pair_off, chunk_off, M, v, part);
    }
  }
  k_pool_finalize<<<unsigned(M), 32, 0, stream>>>(part, chunk_off, M, grad);
  return cudaGetLastError();
}

}  // namespace vqe
