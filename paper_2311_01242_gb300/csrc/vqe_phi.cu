// Streaming energy + adjoint gradient of one large real instance with the forward
// sweep's outputs kept (Sec. 2.1.2's rotations, Eq. 1's energy, and the adjoint
// gradient g_k = 2 Re <lambda|A_k|phi_k>).
//
// The plain streaming path (vqe_kernels.cu) recovers phi_k in the reverse sweep
// by un-applying each gate to the final psi, so its reverse step gathers psi and
// lambda at both ranks of every pair. When psi and lambda together exceed the L2
// (30 qubits: 2 x 72 MB against 126 MB) those scattered gathers miss it. Here the
// forward gate also writes its two outputs of each pair, phi_k at (k, k ^ flip),
// to a per-pair stream (16 bytes per pair, in the gate's pair order, stored and
// later read with the evict-first cache hint), and the reverse step reads that
// stream and gathers only lambda, which then stays in L2. phi_k comes from the
// forward values themselves rather than from un-rotation, so the gradient agrees
// with the plain path to rounding, not bit for bit; psi, lambda and the energy are
// the same bits. Pair-to-thread mapping, grid and partial sums are those of the
// plain path's reverse step.
#include <cuda_runtime.h>

#include "vqe_internal.h"
#include "vqe_device.cuh"

namespace vqe {
namespace {

// Waits for the previous kernel on the stream (programmatic dependent launch),
// then lets the next launch begin.
__device__ __forceinline__ void pdl_wait_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__global__ void k_phi_trig(const double* __restrict__ theta, int M, double2* __restrict__ cs) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) {
    double s, c;
    sincos(theta[m], &s, &c);
    cs[m] = make_double2(c, s);
  }
}

// psi = |HF> on the sector (entry r is sector state sector[r])
__global__ void k_phi_init(const uint32_t* __restrict__ sector, int64_t D, uint32_t hf, double* __restrict__ psi) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D; r += int64_t(gridDim.x) * blockDim.x)
    psi[r] = __ldg(sector + r) == hf ? 1.0 : 0.0;
}

// One gate: (a, b) <- (c a - s' b, s' a + c b) on each pair (s' = +-s by the
// pair's JW sign), and phi[p] = the pair's outputs.
__global__ void k_gate_fwd_keep(const uint2* __restrict__ rp, int64_t P, const double2* __restrict__ cs,
                                double* __restrict__ psi, double2* __restrict__ phi) {
  typedef Amp<true> A;
  pdl_wait_release();
  const double2 c_s = __ldg(cs);
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P; p += int64_t(gridDim.x) * blockDim.x) {
    const uint2 pr = __ldg(rp + p);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    double a = psi[ra], b = psi[rb];
    A::rot(a, b, c_s.x, sflip(c_s.y, sb), sflip(c_s.y, sb ^ 1));
    psi[ra] = a;
    psi[rb] = b;
    __stcs(phi + p, make_double2(a, b));
  }
}

// One reverse step: the pair's contribution s' (lambda_b phi_a - lambda_a phi_b)
// with phi read from the forward stream, then lambda <- U_k^dagger lambda; one
// partial sum per block (the plain path's layout).
__global__ void __launch_bounds__(kStreamThreads, 5)
k_gate_adj_kept(const uint2* __restrict__ rp, int64_t P, const double2* __restrict__ cs,
                const double2* __restrict__ phi, double* __restrict__ lam, double* __restrict__ gpart) {
  typedef Amp<true> A;
  __shared__ double red[32];
  pdl_wait_release();
  const double2 c_s = __ldg(cs);
  double acc = 0.0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P; p += int64_t(gridDim.x) * blockDim.x) {
    const uint2 pr = __ldg(rp + p);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    const double2 f = __ldcs(phi + p);
    double la = lam[ra], lb = lam[rb];
    acc += sflip(A::cross(lb, f.x, la, f.y), sb);
    A::rot(la, lb, c_s.x, sflip(c_s.y, sb ^ 1), sflip(c_s.y, sb));
    lam[ra] = la;
    lam[rb] = lb;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) gpart[blockIdx.x] = s;
}

// out[row] = scale * (sum of the row's nb_rows[row] partials), in a fixed order
// (lane-strided sums, then a fixed shuffle tree).
__global__ void k_phi_finalize(const double* __restrict__ part, const int32_t* __restrict__ nb_rows, int rows,
                               double scale, double* __restrict__ out) {
  const int row = blockIdx.x;
  if (row >= rows) return;
  const int nb = nb_rows[row];
  const double* p = part + int64_t(row) * kMaxPartials;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += p[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[row] = scale * s;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), int grid, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(kStreamThreads));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
}  // namespace

cudaError_t stream_energy_grad_kept(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                                    const double* theta, double* energy, double* grad, cudaStream_t stream) {
  double* psi = static_cast<double*>(b.psi);
  double* lam = static_cast<double*>(b.lam);
  if (d.M > 0) k_phi_trig<<<(d.M + 255) / 256, 256, 0, stream>>>(theta, d.M, b.cs);
  k_phi_init<<<stream_grid(d.D), kStreamThreads, 0, stream>>>(d.sector, d.D, d.hf, psi);
  for (int m = 0; m < d.M; ++m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    if (p1 > p0) {
      const cudaError_t e = launch_dependent(k_gate_fwd_keep, stream_grid(p1 - p0), stream, d.rpairs + p0, p1 - p0,
                                             static_cast<const double2*>(b.cs + m), psi, b.phi + p0);
      if (e != cudaSuccess) return e;
    }
  }
  cudaError_t e = stream_apply_h_real(d, sp, b, energy, stream);
  if (e != cudaSuccess) return e;
  for (int m = d.M - 1; m >= 0; --m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    e = launch_dependent(k_gate_adj_kept, stream_grid(p1 - p0), stream, d.rpairs + p0, p1 - p0,
                         static_cast<const double2*>(b.cs + m), static_cast<const double2*>(b.phi + p0), lam,
                         b.gpart + int64_t(m) * kMaxPartials);
    if (e != cudaSuccess) return e;
  }
  if (d.M > 0) k_phi_finalize<<<d.M, 32, 0, stream>>>(b.gpart, sp.d_nb_rows, d.M, 2.0, grad);
  return cudaGetLastError();
}

}  // namespace vqe
