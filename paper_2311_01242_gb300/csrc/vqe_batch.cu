// Persistent batched evaluation of many independent instances (the paper runs
// hundreds of independent simulation jobs over geometries and molecules,
// abstract and Sec. 4): one launch evaluates E(theta) of Eq. 1 and its adjoint
// gradient for every streamed instance of a batch, whatever their qubit counts,
// excitation counts and Hamiltonians.
//
// The work is a device queue of tasks in a fixed order (built on the host by a
// list-scheduling pass over cost estimates). Each instance is a chain of
// levels whose tasks may run in parallel:
//   INIT      psi = e_hf and the cos/sin table of its angles
//   FWD m     gate m's rotation on a range of its amplitude pairs (a2)
//   GATHER    psi to alpha-major order (string-driven H psi only)
//   HPSI      lambda = H psi for a range of output alpha strings (string form) or
//             output rows (connectivity rows / group scan) (a3)
//   SCATTER   lambda back to sector order (string form only)
//   DOT       per-256-entry partial sums of <psi|lambda>
//   ADJ m     gate m's gradient contributions and its un-rotation of phi and
//             lambda on a range of pairs, one partial sum per 256 pairs (a4)
// A CTA takes the next task from an atomic counter and waits until its
// instance's progress counter shows every task of the earlier levels done
// (acquire load by one thread, a bounded wait with backoff), runs it, and adds
// one to the counter (release). Every task is taken only by a running CTA and
// every task it waits for comes earlier in the queue, so the earliest
// unfinished task can always run: the queue cannot deadlock, whatever the
// grid size. Waits are bounded in time: on expiry the CTA writes the task's
// index + 1 into the status word and returns, every other CTA stops at its
// next task or wait, and the finalising launch writes NaN to every output.
//
// Arithmetic and reduction order are those of the single-instance streaming
// kernels (same rotation per pair, same H psi device code, same 256-element
// block sums, same partial sums in the finalising launch), so a batch gives
// the same bits as vqe_energy_grad on each instance.
#include <climits>
#include <cuda_runtime.h>

#include "vqe_internal.h"
#include "vqe_device.cuh"

namespace vqe {
namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 only: wait until *ctr >= need, for at most budget_ns nanoseconds (and
// a matching cap on the number of polls). Returns false when the wait ran out
// (code recorded in the status word) or another CTA recorded a failure.
__device__ bool wait_progress(const int* ctr, int need, int* status, long long budget_ns, int code) {
  if (ld_acquire(ctr) >= need) return true;
  const unsigned long long t0 = global_ns();
  const long long max_polls = budget_ns / 64 + 1024;
  unsigned ns = 32;
  for (long long it = 0; it < max_polls; ++it) {
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
    if (ld_acquire(ctr) >= need) return true;
    if (ld_acquire(status) != 0) return false;
    if ((long long)(global_ns() - t0) > budget_ns) break;
  }
  atomicCAS(status, 0, code);
  return false;
}

// Pairs per thread in flight in the gate tasks: forward rotations (4 x 256 =
// 1024 pairs per round) and adjoint steps (2 x 256, four amplitudes each).
constexpr int kPairsInFlight = 4;
constexpr int kAdjInFlight = 2;
static_assert(kAdjInFlight * 8 <= 32, "red[] holds 8 warp sums per block");

template <typename T>
__device__ __forceinline__ T* at(char* ws, int64_t off) {
  return reinterpret_cast<T*>(ws + off);
}

__global__ void __launch_bounds__(kPersistThreads, 2)
k_batch_persistent(const PersistDev p, const double* __restrict__ theta, int64_t ld_theta) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ int s_task, s_ok;
  const int tid = threadIdx.x;
  int* progress = p.counters;
  int* next = p.counters + p.n;
  int* status = p.counters + p.n + 1;
  for (;;) {
    if (tid == 0) {
      int t = ld_acquire(status) != 0 ? INT_MAX : atomicAdd(next, 1);
      int ok = 0;
      if (t < p.n_tasks) {
        const PTask& tk = p.tasks[t];
        const int need = t == p.probe_task ? INT_MAX : tk.need;  // the probe waits for a count nothing reaches
        ok = wait_progress(progress + tk.slot, need, status, p.budget_ns, t + 1) ? 1 : 0;
        if (ok) __threadfence();
      }
      s_task = t;
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const PTask tk = p.tasks[s_task];
    const InstDesc& d = p.desc[tk.slot];
    const PSlot& so = p.slots[tk.slot];
    char* ws = p.ws;
    double* psi = at<double>(ws, so.psi);
    double* lam = at<double>(ws, so.lam);
    double2* cs = at<double2>(ws, so.cs);
    switch (tk.kind) {
      case PT_INIT: {
        for (int64_t r = tid; r < d.D; r += kPersistThreads) psi[r] = (__ldg(d.sector + r) == d.hf) ? 1.0 : 0.0;
        for (int m = tid; m < d.M; m += kPersistThreads) {
          double sn, c;
          sincos(theta[d.inst * ld_theta + m], &sn, &c);
          cs[m] = make_double2(c, sn);
        }
        break;
      }
      case PT_FWD: {
        // kPairsInFlight pairs per thread: every pair record and amplitude load of
        // a round is issued before the first rotation (a gate's pairs are disjoint)
        const double2 c_s = __ldcg(cs + tk.m);
        const uint2* rp = d.rpairs + __ldg(d.pair_off + tk.m);
        for (int64_t q0 = tk.lo; q0 < tk.hi; q0 += kPairsInFlight * kPersistThreads) {
          uint2 pr[kPairsInFlight];
          double a[kPairsInFlight], b[kPairsInFlight];
#pragma unroll
          for (int k = 0; k < kPairsInFlight; ++k) {
            const int64_t q = q0 + k * kPersistThreads + tid;
            pr[k] = q < tk.hi ? __ldg(rp + q) : make_uint2(0u, 0u);
          }
#pragma unroll
          for (int k = 0; k < kPairsInFlight; ++k) {
            const int64_t q = q0 + k * kPersistThreads + tid;
            if (q < tk.hi) {
              a[k] = __ldcg(psi + (pr[k].x & 0x7fffffffu));
              b[k] = __ldcg(psi + pr[k].y);
            }
          }
#pragma unroll
          for (int k = 0; k < kPairsInFlight; ++k) {
            const int64_t q = q0 + k * kPersistThreads + tid;
            if (q < tk.hi) {
              const int sb = int(pr[k].x >> 31);
              const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
              Amp<true>::rot(a[k], b[k], c_s.x, ss, nss);
              psi[pr[k].x & 0x7fffffffu] = a[k];
              psi[pr[k].y] = b[k];
            }
          }
        }
        break;
      }
      case PT_GATHER: {
        double* psi_am = at<double>(ws, so.psi_am);
        const uint32_t* perm = d.str->perm;
        for (int64_t i = tk.lo + tid; i < tk.hi; i += kPersistThreads) psi_am[i] = __ldcg(psi + __ldg(perm + i));
        break;
      }
      case PT_HPSI: {
        if (d.str) {
          const StrPlan sp = *d.str;
          const double* psi_am = at<double>(ws, so.psi_am);
          double* lam_am = at<double>(ws, so.lam_am);
          if (sp.Db < kStrMinDb)
            hpsi_str_warps<true, true>(sp, int(tk.lo), d.groups, d.emask, d.vals, psi_am, lam_am, smem);
          else if (sp.Db < kStrWideDb)
            hpsi_str_row<true, false, true>(sp, int(tk.lo), d.groups, d.emask, d.vals, psi_am, lam_am, smem);
          else
            hpsi_str_row<true, true, true, 4>(sp, int(tk.lo), d.groups, d.emask, d.vals, psi_am, lam_am, smem);
        } else {
          for (int64_t r = tk.lo + tid; r < tk.hi; r += kPersistThreads) {
            const uint32_t k = __ldg(d.sector + r);
            double acc = 0.0;
            if (d.W > 0) {
              acc = hpsi_row<true, 4, true>(d.ell, d.ell16, d.W, d.D, r, k, d.groups, d.emask, d.vals, psi, d.rank_hi,
                                            d.rank_lo, d.lo_bits);
            } else {
              for (int gi = 0; gi < d.G; ++gi) {
                const GroupRec g = load_group(d.groups + gi);
                const uint32_t src = k ^ g.x;
                if (!in_sector(src, d.n_elec, d.n_alpha)) continue;
                acc = fma(group_coef<true>(g, d.emask, d.vals, src), __ldcg(psi + sector_rank(d, src)), acc);
              }
            }
            lam[r] = acc;
          }
        }
        break;
      }
      case PT_SCATTER: {
        const double* lam_am = at<double>(ws, so.lam_am);
        const uint32_t* perm = d.str->perm;
        for (int64_t i = tk.lo + tid; i < tk.hi; i += kPersistThreads) lam[__ldg(perm + i)] = __ldcg(lam_am + i);
        break;
      }
      case PT_DOT: {
        double* ep = at<double>(ws, so.ep);
        for (int64_t b = tk.lo; b < tk.hi; ++b) {
          const int64_t r = b * kPersistThreads + tid;
          double v = 0.0;
          if (r < d.D) v += __ldcg(psi + r) * __ldcg(lam + r);
          const double s = block_sum(v, red);
          if (tid == 0) ep[b] = s;
        }
        break;
      }
      case PT_ADJ: {
        // kAdjInFlight 256-pair blocks per round, one pair of each per thread;
        // each block's contributions are summed exactly as block_sum does (warp
        // shuffle tree, then the eight warp sums in order by one thread)
        double* gp = at<double>(ws, so.gp) + tk.aux;
        const double2 c_s = __ldcg(cs + tk.m);
        const uint2* rp = d.rpairs + __ldg(d.pair_off + tk.m);
        const int lane = tid & 31, w = tid >> 5;
        for (int64_t b0 = tk.lo; b0 < tk.hi; b0 += kAdjInFlight * kPersistThreads) {
          uint2 pr[kAdjInFlight];
          double pa[kAdjInFlight], pb[kAdjInFlight], la[kAdjInFlight], lb[kAdjInFlight];
          double acc[kAdjInFlight];
#pragma unroll
          for (int k = 0; k < kAdjInFlight; ++k) {
            const int64_t q = b0 + k * kPersistThreads + tid;
            pr[k] = q < tk.hi ? __ldg(rp + q) : make_uint2(0u, 0u);
          }
#pragma unroll
          for (int k = 0; k < kAdjInFlight; ++k) {
            const int64_t q = b0 + k * kPersistThreads + tid;
            if (q < tk.hi) {
              const uint32_t ra = pr[k].x & 0x7fffffffu, rb = pr[k].y;
              pa[k] = __ldcg(psi + ra);
              pb[k] = __ldcg(psi + rb);
              la[k] = __ldcg(lam + ra);
              lb[k] = __ldcg(lam + rb);
            }
          }
#pragma unroll
          for (int k = 0; k < kAdjInFlight; ++k) {
            const int64_t q = b0 + k * kPersistThreads + tid;
            acc[k] = 0.0;
            if (q < tk.hi) {
              const uint32_t ra = pr[k].x & 0x7fffffffu, rb = pr[k].y;
              const int sb = int(pr[k].x >> 31);
              const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
              acc[k] += sflip(Amp<true>::cross(lb[k], pa[k], la[k], pb[k]), sb);
              Amp<true>::rot(pa[k], pb[k], c_s.x, nss, ss);
              Amp<true>::rot(la[k], lb[k], c_s.x, nss, ss);
              psi[ra] = pa[k];
              psi[rb] = pb[k];
              lam[ra] = la[k];
              lam[rb] = lb[k];
            }
          }
#pragma unroll
          for (int k = 0; k < kAdjInFlight; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
          }
          __syncthreads();  // red[] from the previous round is read
          if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kAdjInFlight; ++k) red[k * 8 + w] = acc[k];
          }
          __syncthreads();
          if (tid < kAdjInFlight) {
            const int64_t blk = b0 + int64_t(tid) * kPersistThreads;
            if (blk < tk.hi) {
              double s = 0.0;
              for (int i = 0; i < kPersistThreads / 32; ++i) s += red[tid * 8 + i];
              gp[blk / kPersistThreads] = s;
            }
          }
        }
        break;
      }
      case PT_ADJS: {
        // partials b in [lo, hi) of a gate with more than 2^18 pairs: partial b sums
        // pairs b * 256 + t + j * (nb * 256), j = 0, 1, ..., in that order, exactly
        // as k_gate_adj's block b does with nb = 1024 blocks
        double* gp = at<double>(ws, so.gp) + tk.aux;
        const double2 c_s = __ldcg(cs + tk.m);
        const int64_t p0 = __ldg(d.pair_off + tk.m), P = __ldg(d.pair_off + tk.m + 1) - p0;
        const uint2* rp = d.rpairs + p0;
        const int64_t stride = int64_t(kMaxPartials) * kPersistThreads;
        for (int64_t b = tk.lo; b < tk.hi; ++b) {
          double acc = 0.0;
          for (int64_t q = b * kPersistThreads + tid; q < P; q += stride) {
            const uint2 pr = __ldg(rp + q);
            const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
            const int sb = int(pr.x >> 31);
            const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
            double pa = __ldcg(psi + ra), pb = __ldcg(psi + rb), la = __ldcg(lam + ra), lb = __ldcg(lam + rb);
            acc += sflip(Amp<true>::cross(lb, pa, la, pb), sb);
            Amp<true>::rot(pa, pb, c_s.x, nss, ss);
            Amp<true>::rot(la, lb, c_s.x, nss, ss);
            psi[ra] = pa;
            psi[rb] = pb;
            lam[ra] = la;
            lam[rb] = lb;
          }
          const double s = block_sum(acc, red);
          if (tid == 0) gp[b] = s;
        }
        break;
      }
      default:
        break;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      red_release_add(progress + tk.slot, 1);
    }
  }
}

// One warp per output: the fixed-order sum of its partials (lane-strided
// sequential sums, then a fixed shuffle tree), times its scale; NaN when the
// persistent launch recorded a failure.
__global__ void k_batch_finalize(const PFinal* __restrict__ rows, int n_rows, const char* __restrict__ ws,
                                 const int* __restrict__ status, double* __restrict__ energy,
                                 double* __restrict__ grad, int64_t ld_grad) {
  const int w = int((blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= n_rows) return;
  const PFinal f = rows[w];
  const double* part = reinterpret_cast<const double*>(ws + f.off);
  double s = 0.0;
  for (int i = lane; i < f.nb; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double v = *status != 0 ? __longlong_as_double(0x7ff8000000000000ll) : f.scale * s;
    if (f.m < 0)
      energy[f.inst] = v;
    else if (grad)
      grad[f.inst * ld_grad + f.m] = v;
  }
}

}  // namespace

cudaError_t set_persist_smem_limit(size_t smem) {
  return cudaFuncSetAttribute(k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

cudaError_t persist_occupancy(size_t smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_persistent, kPersistThreads, smem);
}

cudaError_t persistent_sweep_run(const PersistDev& p, int grid, const double* theta, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(p.counters, 0, size_t(p.n + 2) * sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k_batch_persistent<<<grid, kPersistThreads, 0, stream>>>(p, theta, 0);
  return cudaGetLastError();
}

cudaError_t batch_persistent_run(const PersistDev& p, int grid, size_t smem, const PFinal* rows, int n_rows,
                                 int n_grad_rows, const double* theta, int64_t ld_theta, double* energy, double* grad,
                                 int64_t ld_grad, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(p.counters, 0, size_t(p.n + 2) * sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k_batch_persistent<<<grid, kPersistThreads, smem, stream>>>(p, theta, ld_theta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // gradient rows come first; without a gradient only the energy rows run
  const PFinal* r0 = grad ? rows : rows + n_grad_rows;
  const int nr = grad ? n_rows : n_rows - n_grad_rows;
  if (nr > 0)
    k_batch_finalize<<<(nr + 7) / 8, 256, 0, stream>>>(r0, nr, p.ws, p.counters + p.n + 1, energy, grad, ld_grad);
  return cudaGetLastError();
}

}  // namespace vqe
