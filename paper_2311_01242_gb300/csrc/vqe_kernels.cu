// CUDA kernels of libvqe for sm_103a: the hot path of E(theta) (Eq. 1) and its
// adjoint gradient.
//
//   a1  |HF>                      : the reference bitstring of Eq. 1
//   a2  psi <- U_M ... U_1 psi     : UCCSD excitation rotations (Sec. 2.1.2)
//   a3  lambda = H psi, E = <psi|lambda> : Pauli sum grouped by X mask
//   a4  reverse sweep              : g_k = 2 Re <lambda|A_k|phi>, then
//                                    phi <- U_k^dagger phi, lambda <- U_k^dagger lambda
//
// psi(theta) is real for every theta (real rotations of a real bitstring), so
// the REAL instantiation stores amplitudes as doubles and folds only the real
// part of each Pauli coefficient c * i^{|x&z|}; the imaginary part of H psi
// does not enter E or g. The complex instantiation (double2) computes the same
// quantities with complex amplitudes and full complex coefficients.
//
// Every reduction is deterministic: fixed work assignment, fixed shuffle
// trees, fixed summation order of partials.
#include <cooperative_groups.h>
#include <type_traits>
#include <cuda_runtime.h>

#include "vqe_internal.h"
#include "vqe_device.cuh"

namespace vqe {
namespace {

// ---------------------------------------------------------------- resident kernel
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Loads in flight per thread when staging tables into shared memory.
constexpr int kStageLoads = 8;

__device__ __forceinline__ void sweep_barrier(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// A gate as the sweeps read it from shared memory: its pair range and the
// signs of cos and sin (bit 0, bit 1); cos and sin themselves sit in cs[m].
struct SweepRec {
  int32_t p0, cnt, unused, signs;
};

// The lane's pair entry at position q of a gate; past the gate's end, `pad`.
__device__ __forceinline__ uint32_t entry_or(const uint32_t* rp, const SweepRec& g, int q, uint32_t pad) {
  return q < g.cnt ? rp[g.p0 + q] : pad;
}

// One CTA evaluates one instance with its state in shared memory, compressed to
// the sector (entry r is the amplitude of sector[r]): HF init, forward sweep,
// H psi with the energy, and the reverse sweep with per-pair gradient
// contributions summed per gate in pair order at the end. Gate records,
// cos/sin, pair offsets and pair lists (two ranks and the JW sign per pair)
// are staged in shared memory first; H psi reads packed connectivity entries
// (source rank, source pattern, group), so a source needs no lookup. The sweeps run on the first `sweep_threads`
// threads (one warp per SM sub-partition or more) with a named barrier between
// gates; the instance's pairs are dealt round-robin over those warps.
//
// Real amplitudes: two lanes per pair. The forward sweep also keeps each lane's
// output in that lane's per-pair slot: it is phi at that gate, which the
// reverse sweep then reads instead of un-rotating phi, so the reverse sweep
// rotates lambda only and leaves the gradient contribution in the same slot.
//
// CL = 2 (real amplitudes only): a cluster of two CTAs per instance. Both run the
// sweeps identically; each computes lambda for half of the outputs and writes it
// into its own and its partner's shared memory, then one cluster barrier joins
// the halves. Rank 0 adds the two energy halves (rank 0's first) and writes the
// outputs. No distributed-shared-memory access follows the barrier.
template <bool REAL, int CL, bool FIX>
__global__ void __launch_bounds__(kResidentThreads, 1)
k_resident(const InstDesc* __restrict__ descs, const InstDesc one, const double* __restrict__ theta,
           int64_t ld_theta, double* __restrict__ energy, double* __restrict__ grad, int64_t ld_grad,
           int with_grad) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  typedef typename A::C C;
  static_assert(CL == 1 || (CL == 2 && REAL), "clusters of two need real amplitudes");
  static_assert(!FIX || REAL, "fixed-point sweeps need real amplitudes");
  extern __shared__ __align__(16) unsigned char smem[];
  const int inst_idx = int(blockIdx.x) / CL;
  const int crank = CL == 2 ? int(cooperative_groups::this_cluster().block_rank()) : 0;
  InstDesc d;
  if (descs) {
    d = descs[inst_idx];
  } else {
    d = one;
  }
  const int tid = threadIdx.x, bs = blockDim.x;
  const int n = d.n, M = d.M, G = d.G, W = d.W;
  const int D = int(d.D);
  const int P = int(d.pair_off[M]);
  const bool stage = d.stage_tables != 0;
  const int sw = d.sweep_threads;
  const ResidentLayout L = resident_layout(n, M, P, G, d.E, d.S, D, d.lo_bits, REAL, stage);
  T* psi = reinterpret_cast<T*>(smem + L.psi);
  T* lam = reinterpret_cast<T*>(smem + L.lam);
  // real amplitudes: psi and lambda in two arrays of D + 1 doubles (entry D is the
  // sweeps' scratch row), 8-byte strides for the scattered accesses
  double* pr = reinterpret_cast<double*>(smem + L.psi);
  double* lr = pr + (D + 1);
  double2* cs = reinterpret_cast<double2*>(smem + L.cs);
  SweepRec* gates = reinterpret_cast<SweepRec*>(smem + L.gates);
  int32_t* poff = reinterpret_cast<int32_t*>(smem + L.poff);
  uint32_t* rp = reinterpret_cast<uint32_t*>(smem + L.pairs);
  double* gbuf = reinterpret_cast<double*>(smem + L.gbuf);
  double* red = reinterpret_cast<double*>(smem + L.red);
  const int64_t row = d.inst;
  const double* th = theta + row * ld_theta;

  // pull the tables H psi reads later into L2 while the staging and the forward
  // sweep run (the precomputed entry coefficients, when used, are pulled in by
  // the warps outside the sweep once it has started, so that they do not
  // compete with the staging)
  const bool mat_h = FIX && d.hmat != nullptr;
  {
    const char* ell_b = reinterpret_cast<const char*>(d.ellp);
    const int64_t ell_bytes = int64_t(W) * D * 4;
    for (int64_t o = int64_t(tid) * 128; o < ell_bytes; o += int64_t(bs) * 128) prefetch_l2(ell_b + o);
    if (!mat_h) {
      const char* val_b = REAL ? reinterpret_cast<const char*>(d.vals) : reinterpret_cast<const char*>(d.cvals);
      const int64_t val_bytes = int64_t(d.S) * (REAL ? 8 : 16);
      for (int64_t o = int64_t(tid) * 128; o < val_bytes; o += int64_t(bs) * 128) prefetch_l2(val_b + o);
    }
    const char* sec_b = reinterpret_cast<const char*>(d.sector);
    for (int64_t o = int64_t(tid) * 128; o < int64_t(D) * 4; o += int64_t(bs) * 128) prefetch_l2(sec_b + o);
  }
  // stage ansatz tables, clear the state
  for (int m = tid; m < M; m += bs) {
    double s, c;
    sincos(th[m], &s, &c);
    const int64_t pa = __ldg(d.pair_off + m), pb = __ldg(d.pair_off + m + 1);
    SweepRec gr;
    gr.p0 = int32_t(pa);
    gr.cnt = int32_t(pb - pa);
    gr.unused = 0;
    gr.signs = 0;
    if constexpr (FIX) {
      // magnitudes in Q0.64 (bit patterns kept in the double2 slot), signs apart
      cs[m] = make_double2(llbits(static_cast<long long>(fix_mag(c))), llbits(static_cast<long long>(fix_mag(s))));
      gr.signs = (c < 0.0 ? 1 : 0) | (s < 0.0 ? 2 : 0);
    } else {
      cs[m] = make_double2(c, s);
    }
    gates[m] = gr;
  }
  for (int m = tid; m <= M; m += bs) poff[m] = int32_t(__ldg(d.pair_off + m));
  // pair list: kStageLoads loads in flight per thread
  for (int p0 = tid; p0 < P; p0 += kStageLoads * bs) {
    uint2 e[kStageLoads];
#pragma unroll
    for (int k = 0; k < kStageLoads; ++k) {
      const int p = p0 + k * bs;
      e[k] = p < P ? __ldg(d.rpairs + p) : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int k = 0; k < kStageLoads; ++k) {
      const int p = p0 + k * bs;
      if (p < P) rp[p] = (e[k].x & 0x7fffu) | ((e[k].x >> 31) << 15) | (e[k].y << 16);
    }
  }
  if constexpr (REAL) {
    for (int r = tid; r <= D; r += bs) {
      pr[r] = 0.0;
      lr[r] = 0.0;
    }
  } else {
    for (int r = tid; r < D; r += bs) {
      psi[r] = A::zero();
      lam[r] = A::zero();
    }
  }
  __syncthreads();
  if (tid == 0) {
    if constexpr (FIX)
      pr[d.hf_rank] = llbits(1ll << 62);
    else if constexpr (REAL)
      pr[d.hf_rank] = 1.0;
    else
      psi[d.hf_rank] = A::unit();
  }
  __syncthreads();

  // position of this thread in the sweep: warp w takes the pairs [16 w, 16 w + 16)
  // of each slice of a gate's pairs (real: two adjacent lanes per pair, role 0
  // and 1; complex: one lane per pair, [32 w, 32 w + 32)), so a warp's slot
  // stores are contiguous
  const int role = REAL ? (tid & 1) : 0;
  const int pstride = REAL ? (sw >> 1) : sw;
  const int spos = REAL ? ((tid >> 5) * 16 + ((tid & 31) >> 1)) : tid;

  // a2: forward sweep. A gate's record and cos/sin are loaded at its start (they
  // are first needed after the amplitude loads), the lane's first pair entry one
  // gate ahead. Lanes past a gate's end (real amplitudes) get a scratch entry:
  // state row D and slot 2P + role, so every lane loads and stores without a
  // predicate and the gate body is straight-line code; later slices of a gate
  // with more pairs than lanes run in a loop.
  const uint32_t pad_e = REAL ? (uint32_t(D) | (uint32_t(D) << 16)) : 0u;
  const int scratch = 2 * P + role;
  if (tid < sw && M > 0) {
    uint32_t ea = entry_or(rp, gates[0], spos, pad_e);
    for (int m = 0; m < M; ++m) {
      const SweepRec g0 = gates[m];
      const double2 c0 = cs[m];
      const uint32_t ean = entry_or(rp, gates[min(m + 1, M - 1)], spos, pad_e);
      if constexpr (REAL) {
        // two lanes per pair: role 0 writes c a - s b at ra, role 1 writes c b + s a
        // at rb; both lanes read before either writes
        auto slice = [&](uint32_t e, int q) {
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const uint32_t kd = role ? rb : ra, ko = role ? ra : rb;
          const int sg = int((e >> 15) & 1u) ^ role ^ 1;
          const double self = pr[kd], other = pr[ko];
          __syncwarp();
          double out;
          if constexpr (FIX) {
            out = llbits(neg_if(mulhi_su(dbits(self), static_cast<unsigned long long>(dbits(c0.x))), g0.signs & 1) +
                         neg_if(mulhi_su(dbits(other), static_cast<unsigned long long>(dbits(c0.y))),
                                sg ^ ((g0.signs >> 1) & 1)));
          } else {
            out = fma(sflip(c0.y, sg), other, c0.x * self);
          }
          pr[kd] = out;
          gbuf[q < g0.cnt ? 2 * (g0.p0 + q) + role : scratch] = out;
        };
        slice(ea, spos);
        for (int q0 = pstride; q0 < g0.cnt; q0 += pstride) slice(entry_or(rp, g0, q0 + spos, pad_e), q0 + spos);
      } else {
        for (int q = spos; q < g0.cnt; q += sw) {
          const uint32_t e = (q == spos) ? ea : rp[g0.p0 + q];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sb = int((e >> 15) & 1u);
          const double ss = sflip(c0.y, sb), nss = sflip(c0.y, sb ^ 1);
          T a = psi[ra], b = psi[rb];
          A::rot(a, b, c0.x, ss, nss);
          psi[ra] = a;
          psi[rb] = b;
        }
      }
      sweep_barrier(sw);
      ea = ean;
    }
  }
  // stage the H psi tables
  const GroupRec* tg = d.groups;
  const uint32_t* te = d.emask;
  const C* tv;
  if constexpr (REAL) tv = d.vals; else tv = d.cvals;
  if (mat_h) {
    const int st = (sw < bs && M > 0) ? tid - sw : tid, sbs = (sw < bs && M > 0) ? bs - sw : bs;
    const char* mat_b = reinterpret_cast<const char*>(d.hmat);
    const int64_t mat_bytes = int64_t(W) * D * 8;
    if (st >= 0)
      for (int64_t o = int64_t(st) * 128; o < mat_bytes; o += int64_t(sbs) * 128) prefetch_l2(mat_b + o);
  } else if (stage) {
    GroupRec* sg = reinterpret_cast<GroupRec*>(smem + L.tab);
    uint32_t* se = reinterpret_cast<uint32_t*>(smem + L.tab + uint32_t(G) * 32u);
    C* sv = reinterpret_cast<C*>(smem + L.tab + uint32_t(G) * 32u + align_up(uint32_t(d.E) * 4u, 16u));
    // the threads outside the sweep stage the tables while the sweep runs (its
    // shared-memory regions are disjoint from these); with no such threads, all
    // threads stage after the sweep
    const int st = (sw < bs && M > 0) ? tid - sw : tid, sbs = (sw < bs && M > 0) ? bs - sw : bs;
    if (st >= 0) {
      const int4* gsrc = reinterpret_cast<const int4*>(d.groups);
      int4* gdst = reinterpret_cast<int4*>(sg);
      for (int i = st; i < 2 * G; i += sbs) gdst[i] = __ldg(gsrc + i);
      for (int i = st; i < d.E; i += sbs) se[i] = __ldg(d.emask + i);
      if constexpr (FIX) {
        // fixed-point tables: v * 2^(62 - eh), where 2^eh bounds the sum of |v|
        // over every slot and so every row sum of |H|
        const int eh = bound_exp(*d.hbound);
        const double sc = pow2(62 - eh);
        for (int i0 = st; i0 < d.S; i0 += kStageLoads * sbs) {
          double v[kStageLoads];
#pragma unroll
          for (int k = 0; k < kStageLoads; ++k) {
            const int i = i0 + k * sbs;
            v[k] = i < d.S ? __ldg(d.vals + i) : 0.0;
          }
#pragma unroll
          for (int k = 0; k < kStageLoads; ++k) {
            const int i = i0 + k * sbs;
            if (i < d.S) sv[i] = llbits(__double2ll_rn(v[k] * sc));
          }
        }
      } else {
        for (int i = st; i < d.S; i += sbs) sv[i] = A::coef(d, i);
      }
    }
    tg = sg;
    te = se;
    tv = sv;
  }
  __syncthreads();
  // fixed-point H psi: staged integer tables times psi in Q1.62 (needs the
  // staged tables; otherwise psi goes to FP64 for the FP64 H psi)
  const bool int_h = FIX && (stage || mat_h);  // precomputed entry coefficients need no tables
  const int eh = int_h ? bound_exp(*d.hbound) : 0;
  if (FIX && !int_h) {
    for (int r = tid; r < D; r += bs) pr[r] = __ll2double_rn(dbits(pr[r])) * 0x1p-62;
    __syncthreads();
  }

  // a3: lambda = H psi on the sector, E = <psi|lambda>
  double e_part = 0.0;
  const int r_half = (D + CL - 1) / CL;
  const int r_lo = crank * r_half, r_hi = min(D, r_lo + r_half);
  double* lr_peer = lr;
  if constexpr (CL == 2) lr_peer = cooperative_groups::this_cluster().map_shared_rank(lr, crank ^ 1);
  // Real amplitudes: two threads per output row, one on the row's even slots and
  // one on its odd slots, added (even + odd) by a fixed shuffle; the split
  // depends on nothing but the row, so every launch form gives the same bits.
  constexpr int TPR = REAL ? 2 : 1;
  const int rows = r_hi - r_lo, per_pass = bs / TPR, half = tid % TPR;
  const bool fast = d.ellp_fast != 0;
  for (int base = 0; base < rows; base += per_pass) {  // same trip count in every thread
    const int lrow = base + tid / TPR;
    const bool live = lrow < rows;
    const int r = r_lo + (live ? lrow : 0);
    const uint32_t k = __ldg(d.sector + r);
    if constexpr (FIX) {
      if (int_h) {
        // lambda in units of 2^(eh - 60): the high word of (table value) x (psi)
        long long acc = 0;
        if (live && mat_h) {
          ell_row_mat<kEllChunk>(d.ellp, d.hmat, W, D, r, half, TPR, [&](uint32_t e, long long f) {
            acc += __mul64hi(f, dbits(pr[e & 0x7fffu]));
          });
        } else if (live) {
          const long long* tvi = reinterpret_cast<const long long*>(tv);
          ell_row(d.ellp, nullptr, W, D, r, half, TPR, [&](uint32_t e) {
            long long f;
            if (fast && (e >> 31)) {
              f = neg_if(tvi[(e >> 16) & 0x7fffu], int((e >> 15) & 1u));
            } else {
              const GroupRec g = load_group(tg + (e >> 19));
              f = group_coef_int(g, te, tvi, k ^ g.x, (e >> 15) & 15u);
            }
            acc += __mul64hi(f, dbits(pr[e & 0x7fffu]));
          });
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);  // even + odd slots (exact)
        if (live && half == 0) {
          lr[r] = llbits(acc);
          if constexpr (CL == 2) lr_peer[r] = llbits(acc);
          e_part += (__ll2double_rn(dbits(pr[r])) * 0x1p-62) * (__ll2double_rn(acc) * pow2(eh - 60));
        }
        continue;
      }
    }
    T acc = A::zero();
    if (live) {
      ell_row(d.ellp, nullptr, W, D, r, half, TPR, [&](uint32_t e) {
        C f;
        if (fast && (e >> 31)) {
          f = sflip(tv[(e >> 16) & 0x7fffu], int((e >> 15) & 1u));
        } else {
          const GroupRec g = load_group(tg + (e >> 19));
          f = group_coef_u<REAL>(g, te, tv, k ^ g.x, (e >> 15) & 15u);
        }
        if constexpr (REAL)
          A::mac(acc, f, pr[e & 0x7fffu]);
        else
          A::mac(acc, f, psi[e & 0x7fffu]);
      });
    }
    if constexpr (TPR == 2) {
      const double odd = __shfl_xor_sync(0xffffffffu, acc, 1);
      acc = acc + odd;  // used by the even-slot thread only
    }
    if (live && half == 0) {
      if constexpr (REAL) {
        lr[r] = acc;
        if constexpr (CL == 2) lr_peer[r] = acc;
        e_part += pr[r] * acc;
      } else {
        lam[r] = acc;
        e_part += A::redot(psi[r], acc);
      }
    }
  }
  const double e_tot = block_sum(e_part, red);
  if constexpr (CL == 2) {
    if (tid == 0 && crank == 1) *cooperative_groups::this_cluster().map_shared_rank(red + 48, 0) = e_tot;
    cooperative_groups::this_cluster().sync();
    if (tid == 0 && crank == 0) energy[row] = e_tot + red[48];
  } else {
    if (tid == 0) energy[row] = e_tot;
  }
  __syncthreads();

  if (!with_grad) return;

  // Fixed point for the reverse sweep: lambda scaled by 2^(61 - e), where 2^e
  // bounds ||lambda|| (so every entry stays below 2^61 in magnitude through the
  // rotations); phi comes from the forward sweep's per-pair slots in Q1.62.
  // Both CTAs of a cluster hold all of lambda here and derive the same e.
  int lam_e = 0;
  if (int_h) {
    // lambda is already fixed point in units of 2^(eh - 60) = 2^(61 - lam_e):
    // ||lambda|| <= ||H||_2 <= ||H||_inf < 2^eh keeps every entry below 2^61 of them
    lam_e = eh + 1;
  } else if constexpr (FIX) {
    double l2 = 0.0;
    for (int r = tid; r < D; r += bs) {
      const double v = lr[r];
      l2 = fma(v, v, l2);
    }
    const double tot = block_sum(l2, red);
    if (tid == 0) red[56] = tot;
    __syncthreads();
    const int ex = int((dbits(red[56]) >> 52) & 0x7ff);
    // ||lambda||^2 < 2^(ex - 1022) <= 2^(2 lam_e)
    lam_e = ex == 0 ? -500 : (ex - 1022 + 1) >> 1;
    const double sc = pow2(61 - lam_e);
    for (int r = tid; r < D; r += bs) lr[r] = llbits(__double2ll_rn(lr[r] * sc));
    __syncthreads();
  }

  // a4: reverse sweep (loads ahead as in the forward sweep; the lane's slot of the
  // next gate is also computed one gate ahead, since the slot is the address of a
  // load here)
  if (tid < sw && M > 0) {
    uint32_t ea;
    int slot0;
    {
      const SweepRec g = gates[M - 1];
      ea = entry_or(rp, g, spos, pad_e);
      slot0 = spos < g.cnt ? 2 * (g.p0 + spos) + role : scratch;
    }
    for (int m = M - 1; m >= 0; --m) {
      const SweepRec g0 = gates[m];
      const double2 c0 = cs[m];
      const SweepRec g1 = gates[max(m - 1, 0)];
      const uint32_t ean = entry_or(rp, g1, spos, pad_e);
      const int slotn = spos < g1.cnt ? 2 * (g1.p0 + spos) + role : scratch;
      if constexpr (REAL) {
        // two lanes per pair: the lane's slot holds phi at its own index (role 0
        // at ra, role 1 at rb); role 0 keeps s lambda_b phi_a, role 1 keeps
        // -s lambda_a phi_b, and each un-applies the gate to lambda at its index
        auto slice = [&](uint32_t e, int slot) {
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sr = int((e >> 15) & 1u) ^ role;
          const uint32_t ks = role ? rb : ra, ko = role ? ra : rb;
          const double ph = gbuf[slot], ls = lr[ks], lo = lr[ko];
          __syncwarp();
          double g_term, nl;
          if constexpr (FIX) {
            const unsigned long long cm = static_cast<unsigned long long>(dbits(c0.x));
            const unsigned long long sm = static_cast<unsigned long long>(dbits(c0.y));
            const int cneg = g0.signs & 1, sneg = ((g0.signs >> 1) & 1) ^ sr;
            g_term = llbits(neg_if(__mul64hi(dbits(ph), dbits(lo)), sr));
            nl = llbits(neg_if(mulhi_su(dbits(ls), cm), cneg) + neg_if(mulhi_su(dbits(lo), sm), sneg));
          } else {
            g_term = sflip(lo * ph, sr);
            nl = fma(sflip(c0.y, sr), lo, c0.x * ls);
          }
          gbuf[slot] = g_term;
          lr[ks] = nl;
        };
        slice(ea, slot0);
        for (int q0 = pstride; q0 < g0.cnt; q0 += pstride) {
          const int q = q0 + spos;
          slice(entry_or(rp, g0, q, pad_e), q < g0.cnt ? 2 * (g0.p0 + q) + role : scratch);
        }
      } else {
        for (int q = spos; q < g0.cnt; q += sw) {
          const uint32_t e = (q == spos) ? ea : rp[g0.p0 + q];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sb = int((e >> 15) & 1u);
          const double ss = sflip(c0.y, sb), nss = sflip(c0.y, sb ^ 1);
          T pa = psi[ra], pb = psi[rb], la = lam[ra], lb = lam[rb];
          gbuf[g0.p0 + q] = sflip(A::cross(lb, pa, la, pb), sb);
          A::rot(pa, pb, c0.x, nss, ss);
          A::rot(la, lb, c0.x, nss, ss);
          psi[ra] = pa;
          psi[rb] = pb;
          lam[ra] = la;
          lam[rb] = lb;
        }
      }
      sweep_barrier(sw);
      ea = ean;
      slot0 = slotn;
    }
  }
  __syncthreads();
  // per-gate sums of the pair contributions: four consecutive lanes split a
  // gate's pairs into four contiguous quarters, combined by a fixed shuffle tree
  double* g_out = grad + row * ld_grad;
  // fixed point: a contribution h stands for h * 2^(e - 59) (Q1.62 times lambda
  // scaled by 2^(61 - e), high word); its integer sums are exact
  const double g_scale = FIX ? pow2(lam_e - 58) : 2.0;
  for (int base = 0; base < 4 * M; base += bs) {
    const int t = base + tid;
    const int m = t >> 2, qtr = t & 3;
    typedef typename std::conditional<FIX, long long, double>::type Acc;
    Acc s = 0;
    if (m < M) {
      const int per = REAL ? 2 : 1;  // contributions per pair
      const int p0 = per * poff[m], p1 = per * poff[m + 1];
      const int len = p1 - p0, chunk = (len + 3) >> 2;
      const int a = p0 + qtr * chunk, b = min(p1, a + chunk);
      for (int p = a; p < b; ++p) {
        if constexpr (FIX)
          s += dbits(gbuf[p]);
        else
          s += gbuf[p];
      }
    }
    s += __shfl_down_sync(0xffffffffu, s, 2, 4);
    s += __shfl_down_sync(0xffffffffu, s, 1, 4);
    if (m < M && qtr == 0 && crank == 0) {
      if constexpr (FIX)
        g_out[m] = __ll2double_rn(s) * g_scale;
      else
        g_out[m] = g_scale * s;
    }
  }
}

// ---------------------------------------------------------------- streaming kernels
// Programmatic dependent launch of the per-gate kernels: each waits until the
// previous kernel on the stream has completed and its writes are visible
// (a no-op when launched without the attribute), then lets the next gate's
// launch begin, so that launch overlaps this kernel's execution instead of
// following its end.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__global__ void k_trig(const double* __restrict__ theta, int M, double2* __restrict__ cs) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) {
    double s, c;
    sincos(theta[m], &s, &c);
    cs[m] = make_double2(c, s);
  }
}

// The streaming kernels keep psi, phi and lambda compressed to the sector:
// entry r is the amplitude of basis state sector[r].
template <bool REAL>
__global__ void k_init_sector(const uint32_t* __restrict__ sector, int64_t D, uint32_t hf,
                              typename Amp<REAL>::T* __restrict__ psi) {
  typedef Amp<REAL> A;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D;
       r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(sector + r);
    psi[r] = (k == hf) ? A::unit() : A::zero();
  }
}

// rp[p] = (rank(k) | sign << 31, rank(k ^ flip)) of pair p; sign = (-1)-bit of T|k>
template <bool REAL>
__global__ void k_gate_fwd(const uint2* __restrict__ rp, int64_t P, const double2* __restrict__ cs,
                           typename Amp<REAL>::T* __restrict__ psi) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  pdl_wait_and_release();
  const double2 c_s = __ldg(cs);
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P;
       p += int64_t(gridDim.x) * blockDim.x) {
    const uint2 pr = __ldg(rp + p);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
    T a = psi[ra], b = psi[rb];
    A::rot(a, b, c_s.x, ss, nss);
    psi[ra] = a;
    psi[rb] = b;
  }
}

// lambda = H psi on the sector; per-block energy partials.
template <bool REAL, bool ELL>
__global__ void __launch_bounds__(kStreamThreads, 1)
k_hpsi(const InstDesc d, int n_elec, int n_alpha, const typename Amp<REAL>::T* __restrict__ psi,
       typename Amp<REAL>::T* __restrict__ lam, double* __restrict__ epart) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  typedef typename A::C C;
  __shared__ double red[32];
  const C* tv;
  if constexpr (REAL) tv = d.vals; else tv = d.cvals;
  double e_part = 0.0;
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < d.D;
       r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(d.sector + r);
    T acc = A::zero();
    if (ELL) {
      acc = hpsi_row<REAL, 4>(d.ell, d.ell16, d.W, d.D, r, k, d.groups, d.emask, tv, psi, d.rank_hi,
                                         d.rank_lo, d.lo_bits);
    } else {
      for (int gi = 0; gi < d.G; ++gi) {
        const GroupRec g = load_group(d.groups + gi);
        const uint32_t src = k ^ g.x;
        if (!in_sector(src, n_elec, n_alpha)) continue;
        A::mac(acc, group_coef<REAL>(g, d.emask, tv, src), psi[sector_rank(d, src)]);
      }
    }
    lam[r] = acc;
    e_part += A::redot(psi[r], acc);
  }
  const double s = block_sum(e_part, red);
  if (threadIdx.x == 0) epart[blockIdx.x] = s;
}

// (five blocks per SM: 48 registers, no spills; the 1,024-block grid that fixes the
// gradient's partial sums then runs in 1.3 waves instead of 2.2 at three blocks)
template <bool REAL>
__global__ void __launch_bounds__(kStreamThreads, 5)
k_gate_adj(const uint2* __restrict__ rp, int64_t P, const double2* __restrict__ cs,
           typename Amp<REAL>::T* __restrict__ phi, typename Amp<REAL>::T* __restrict__ lam,
           double* __restrict__ gpart) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  __shared__ double red[32];
  pdl_wait_and_release();
  const double2 c_s = __ldg(cs);
  double acc = 0.0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P;
       p += int64_t(gridDim.x) * blockDim.x) {
    const uint2 pr = __ldg(rp + p);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
    T pa = phi[ra], pb = phi[rb], la = lam[ra], lb = lam[rb];
    acc += sflip(A::cross(lb, pa, la, pb), sb);
    A::rot(pa, pb, c_s.x, nss, ss);
    A::rot(la, lb, c_s.x, nss, ss);
    phi[ra] = pa;
    phi[rb] = pb;
    lam[ra] = la;
    lam[rb] = lb;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) gpart[blockIdx.x] = s;
}

// WIDE: the block form for Db >= kStrWideDb (smaller shared-memory footprint,
// four blocks per SM); the other instance runs three.
template <bool REAL, bool WIDE>
__global__ void __launch_bounds__(kStrWarps * 32, WIDE ? 4 : 3)
k_hpsi_str(const StrPlan sp, const GroupRec* __restrict__ groups, const uint32_t* __restrict__ emask,
           const typename Amp<REAL>::C* __restrict__ vals, const typename Amp<REAL>::T* __restrict__ psi_am,
           typename Amp<REAL>::T* __restrict__ lam_am) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (sp.Db >= kStrMinDb)
    hpsi_str_row<REAL, WIDE>(sp, int(blockIdx.x), groups, emask, vals, psi_am, lam_am, smem);
  else
    hpsi_str_warps<REAL>(sp, int(blockIdx.x) * kStrWarps, groups, emask, vals, psi_am, lam_am, smem);
}

// dst[i] = src[perm[i]] (sector order -> alpha-major) and the reverse scatter
template <bool REAL>
__global__ void k_perm_gather(const uint32_t* __restrict__ perm, int64_t D,
                              const typename Amp<REAL>::T* __restrict__ src, typename Amp<REAL>::T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < D; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[__ldg(perm + i)];
}
template <bool REAL>
__global__ void k_perm_scatter(const uint32_t* __restrict__ perm, int64_t D,
                               const typename Amp<REAL>::T* __restrict__ src, typename Amp<REAL>::T* __restrict__ dst) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < D; i += int64_t(gridDim.x) * blockDim.x)
    dst[__ldg(perm + i)] = src[i];
}

// Per-block partials of Re <a|b> over D entries (fixed assignment and order).
template <bool REAL>
__global__ void __launch_bounds__(kStreamThreads) k_dot(const typename Amp<REAL>::T* __restrict__ a,
                                                        const typename Amp<REAL>::T* __restrict__ b, int64_t D,
                                                        double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < D; i += int64_t(gridDim.x) * blockDim.x)
    acc += Amp<REAL>::redot(a[i], b[i]);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Sums nb[i] partials of row i (row i at part + i*kMaxPartials) in a fixed
// order: lane-strided sequential sums, then a fixed shuffle tree.
__global__ void k_finalize(const double* __restrict__ part, const int32_t* __restrict__ nb_rows,
                           int rows, double scale, double* __restrict__ out) {
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

template <bool REAL>
__global__ void k_scatter_out(const uint32_t* __restrict__ sector, int64_t D,
                              const typename Amp<REAL>::T* __restrict__ v, double2* __restrict__ out) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D;
       r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(sector + r);
    out[k] = Amp<REAL>::to_c(v[r]);
  }
}

__global__ void k_gather_in(const uint32_t* __restrict__ sector, int64_t D, const double2* __restrict__ in,
                            double2* __restrict__ v) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D;
       r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(sector + r);
    v[r] = in[k];
  }
}

}  // namespace

// ---------------------------------------------------------------- device-built connectivity
__global__ void k_ell_count(const uint32_t* __restrict__ sector, int64_t D, const GroupRec* __restrict__ groups, int G,
                            int n_elec, int n_alpha, int32_t* __restrict__ len, int32_t* __restrict__ wmax) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D; r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(sector + r);
    int c = 0;
    for (int g = 0; g < G; ++g) c += in_sector(k ^ __ldg(&groups[g].x), n_elec, n_alpha);
    len[r] = c;
    atomicMax(wmax, c);
  }
}

__global__ void k_ell_fill(const uint32_t* __restrict__ sector, int64_t D, const GroupRec* __restrict__ groups, int G,
                           const int32_t* __restrict__ order, int n_elec, int n_alpha, int W,
                           uint16_t* __restrict__ ell) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < D; r += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t k = __ldg(sector + r);
    int j = 0;
    for (int oi = 0; oi < G && j < W; ++oi) {
      const int g = __ldg(order + oi);
      if (in_sector(k ^ __ldg(&groups[g].x), n_elec, n_alpha)) {
        ell[int64_t(j) * D + r] = uint16_t(g);
        ++j;
      }
    }
    for (; j < W; ++j) ell[int64_t(j) * D + r] = 0xFFFFu;
  }
}

// ---------------------------------------------------------------- fixed-point entry coefficients
// The staged tables of the resident kernel, v * 2^(62 - eh), and from them every
// packed entry's coefficient exactly as the kernel's H psi computes it.
__global__ void k_int_vals(const double* __restrict__ vals, int64_t S, const double* __restrict__ hbound,
                           long long* __restrict__ ivals) {
  const int eh = bound_exp(*hbound);
  const double sc = pow2(62 - eh);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < S; i += int64_t(gridDim.x) * blockDim.x)
    ivals[i] = __double2ll_rn(__ldg(vals + i) * sc);
}

__global__ void k_build_hmat(const uint32_t* __restrict__ ellp, int64_t n, int64_t D,
                             const uint32_t* __restrict__ sector, const GroupRec* __restrict__ groups,
                             const uint32_t* __restrict__ emask, const long long* __restrict__ ivals, int fast,
                             long long* __restrict__ hmat) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t e = __ldg(ellp + i);
    long long f = 0;
    if (e != kEllPad) {
      if (fast && (e >> 31)) {
        f = neg_if(__ldg(ivals + ((e >> 16) & 0x7fffu)), int((e >> 15) & 1u));
      } else {
        const uint32_t k = __ldg(sector + i % D);
        const GroupRec g = load_group(groups + (e >> 19));
        f = group_coef_int(g, emask, ivals, k ^ g.x, (e >> 15) & 15u);
      }
    }
    hmat[i] = f;
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t set_str_smem_limit(size_t smem) {
  const int b = int(smem);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_hpsi_str<true, false>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<false, false>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<true, true>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<false, true>, a, b);
  return e;
}

cudaError_t set_resident_smem_limit(size_t smem, bool real) {
  const int b = int(smem);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (!real) return cudaFuncSetAttribute(k_resident<false, 1, false>, a, b);
  cudaError_t e = cudaFuncSetAttribute(k_resident<true, 1, true>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resident<true, 2, true>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resident<true, 1, false>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resident<true, 2, false>, a, b);
  return e;
}

cudaError_t launch_resident(const InstDesc* d_descs, const InstDesc* one, int n_inst, size_t smem, bool real,
                            bool with_grad, const double* theta, int64_t ld_theta, double* energy, double* grad,
                            int64_t ld_grad, cudaStream_t stream, int ctas_per_instance, bool fixed_point) {
  InstDesc dummy = {};
  const InstDesc& o = one ? *one : dummy;
  const int wg = with_grad ? 1 : 0;
  if (real && ctas_per_instance == 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * n_inst);
    cfg.blockDim = dim3(kResidentThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (fixed_point)
      return cudaLaunchKernelEx(&cfg, k_resident<true, 2, true>, d_descs, o, theta, ld_theta, energy, grad,
                                ld_grad, wg);
    return cudaLaunchKernelEx(&cfg, k_resident<true, 2, false>, d_descs, o, theta, ld_theta, energy, grad,
                              ld_grad, wg);
  }
  const dim3 g(n_inst), b(kResidentThreads);
  if (real && fixed_point)
    k_resident<true, 1, true><<<g, b, smem, stream>>>(d_descs, o, theta, ld_theta, energy, grad, ld_grad, wg);
  else if (real)
    k_resident<true, 1, false><<<g, b, smem, stream>>>(d_descs, o, theta, ld_theta, energy, grad, ld_grad, wg);
  else
    k_resident<false, 1, false><<<g, b, smem, stream>>>(d_descs, o, theta, ld_theta, energy, grad, ld_grad, wg);
  return cudaGetLastError();
}

namespace {
// Launch with programmatic stream serialization allowed (see pdl_wait_and_release).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(block));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The gate sweeps of one instance as one persistent launch over its task queue
// (sp.sweep; real amplitudes): PSlot offsets are relative to b.psi, the start of
// the workspace layout.
cudaError_t sweep_launch(const StreamPlan& sp, const StreamBuffers& b, bool adjoint, const double* theta,
                         cudaStream_t stream) {
  PersistDev p;
  p.desc = sp.sweep->d_desc;
  p.slots = sp.sweep->d_slot;
  p.tasks = adjoint ? sp.sweep->d_adj : sp.sweep->d_fwd;
  p.n_tasks = adjoint ? sp.sweep->n_adj : sp.sweep->n_fwd;
  p.n = 1;
  p.ws = static_cast<char*>(b.psi);
  p.counters = reinterpret_cast<int*>(static_cast<char*>(b.psi) + sp.counters_off);
  p.budget_ns = 2000000000ll;
  p.probe_task = -1;
  p.pad = 0;
  return persistent_sweep_run(p, sp.sweep->grid, theta, stream);
}

template <bool REAL>
cudaError_t stream_forward(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                           const double* theta, cudaStream_t stream) {
  typedef typename Amp<REAL>::T T;
  if (REAL && sp.sweep) return sweep_launch(sp, b, false, theta, stream);
  T* psi = static_cast<T*>(b.psi);
  const int nt = kStreamThreads;
  if (d.M > 0) k_trig<<<(d.M + 255) / 256, 256, 0, stream>>>(theta, d.M, b.cs);
  k_init_sector<REAL><<<stream_grid(d.D), nt, 0, stream>>>(d.sector, d.D, d.hf, psi);
  for (int m = 0; m < d.M; ++m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    if (p1 > p0) {
      const cudaError_t e = launch_pdl(k_gate_fwd<REAL>, stream_grid(p1 - p0), nt, stream, d.rpairs + p0, p1 - p0,
                                       static_cast<const double2*>(b.cs + m), psi);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <bool REAL>
cudaError_t stream_hpsi(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                        double* energy, cudaStream_t stream) {
  typedef typename Amp<REAL>::T T;
  const T* psi = static_cast<const T*>(b.psi);
  T* lam = static_cast<T*>(b.lam);
  const int grid = stream_grid(d.D);
  if (sp.use_str) {
    typedef typename Amp<REAL>::C C;
    const C* tv;
    if constexpr (REAL) tv = d.vals; else tv = d.cvals;
    T* psi_am = static_cast<T*>(b.psi_am);
    T* lam_am = static_cast<T*>(b.lam_am);
    const size_t smem = str_smem_bytes(sp.str.Db, sizeof(T));
    k_perm_gather<REAL><<<grid, kStreamThreads, 0, stream>>>(sp.str.perm, d.D, psi, psi_am);
    if (sp.str.Db >= kStrWideDb)
      k_hpsi_str<REAL, true><<<str_blocks(sp.str.Da, sp.str.Db), kStrWarps * 32, smem, stream>>>(
          sp.str, d.groups, d.emask, tv, psi_am, lam_am);
    else
      k_hpsi_str<REAL, false><<<str_blocks(sp.str.Da, sp.str.Db), kStrWarps * 32, smem, stream>>>(
          sp.str, d.groups, d.emask, tv, psi_am, lam_am);
    k_perm_scatter<REAL><<<grid, kStreamThreads, 0, stream>>>(sp.str.perm, d.D, lam_am, lam);
    k_dot<REAL><<<grid, kStreamThreads, 0, stream>>>(psi, lam, d.D, b.epart);
  } else if (sp.use_ell) {
    k_hpsi<REAL, true><<<grid, kStreamThreads, 0, stream>>>(d, sp.n_elec, sp.n_alpha, psi, lam, b.epart);
  } else {
    k_hpsi<REAL, false><<<grid, kStreamThreads, 0, stream>>>(d, sp.n_elec, sp.n_alpha, psi, lam, b.epart);
  }
  k_finalize<<<1, 32, 0, stream>>>(b.epart, sp.d_nb_rows + d.M, 1, 1.0, energy);
  return cudaGetLastError();
}

template <bool REAL>
cudaError_t stream_adjoint(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                           double* grad, cudaStream_t stream) {
  typedef typename Amp<REAL>::T T;
  T* phi = static_cast<T*>(b.psi);
  T* lam = static_cast<T*>(b.lam);
  if (REAL && sp.sweep) {
    const cudaError_t e = sweep_launch(sp, b, true, nullptr, stream);
    if (e != cudaSuccess) return e;
    if (d.M > 0) k_finalize<<<d.M, 32, 0, stream>>>(b.gpart, sp.d_nb_rows, d.M, 2.0, grad);
    return cudaGetLastError();
  }
  for (int m = d.M - 1; m >= 0; --m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    double* gp = b.gpart + int64_t(m) * kMaxPartials;
    const cudaError_t e = launch_pdl(k_gate_adj<REAL>, stream_grid(p1 - p0), kStreamThreads, stream, d.rpairs + p0,
                                     p1 - p0, static_cast<const double2*>(b.cs + m), phi, lam, gp);
    if (e != cudaSuccess) return e;
  }
  if (d.M > 0) k_finalize<<<d.M, 32, 0, stream>>>(b.gpart, sp.d_nb_rows, d.M, 2.0, grad);
  return cudaGetLastError();
}
}  // namespace

cudaError_t stream_energy_grad(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                               bool real, bool with_grad, const double* theta, double* energy,
                               double* grad, cudaStream_t stream) {
  cudaError_t e;
  if (real) {
    if ((e = stream_forward<true>(d, sp, b, theta, stream)) != cudaSuccess) return e;
    if ((e = stream_hpsi<true>(d, sp, b, energy, stream)) != cudaSuccess) return e;
    if (with_grad) return stream_adjoint<true>(d, sp, b, grad, stream);
  } else {
    if ((e = stream_forward<false>(d, sp, b, theta, stream)) != cudaSuccess) return e;
    if ((e = stream_hpsi<false>(d, sp, b, energy, stream)) != cudaSuccess) return e;
    if (with_grad) return stream_adjoint<false>(d, sp, b, grad, stream);
  }
  return cudaGetLastError();
}

cudaError_t stream_state(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                         const double* theta, double* psi_out, cudaStream_t stream) {
  cudaError_t e = stream_forward<true>(d, sp, b, theta, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(psi_out, 0, (size_t(1) << d.n) * sizeof(double2), stream);
  if (e != cudaSuccess) return e;
  k_scatter_out<true><<<stream_grid(d.D), kStreamThreads, 0, stream>>>(
      d.sector, d.D, static_cast<const double*>(b.psi), reinterpret_cast<double2*>(psi_out));
  return cudaGetLastError();
}

cudaError_t stream_apply_h(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                           const double* psi_in, double* lam_out, double* energy,
                           cudaStream_t stream) {
  k_gather_in<<<stream_grid(d.D), kStreamThreads, 0, stream>>>(
      d.sector, d.D, reinterpret_cast<const double2*>(psi_in), static_cast<double2*>(b.psi));
  cudaError_t e = stream_hpsi<false>(d, sp, b, energy, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(lam_out, 0, (size_t(1) << d.n) * sizeof(double2), stream);
  if (e != cudaSuccess) return e;
  k_scatter_out<false><<<stream_grid(d.D), kStreamThreads, 0, stream>>>(
      d.sector, d.D, static_cast<const double2*>(b.lam), reinterpret_cast<double2*>(lam_out));
  return cudaGetLastError();
}

cudaError_t stream_apply_h_real(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b, double* energy,
                                cudaStream_t stream) {
  return stream_hpsi<true>(d, sp, b, energy, stream);
}

cudaError_t build_hmat(const uint32_t* ellp, int W, int64_t D, const uint32_t* sector, const GroupRec* groups,
                       const uint32_t* emask, const double* vals, int64_t S, const double* hbound, int fast,
                       long long* ivals, long long* hmat, cudaStream_t stream) {
  if (S > 0) k_int_vals<<<stream_grid(S), kStreamThreads, 0, stream>>>(vals, S, hbound, ivals);
  const int64_t n = int64_t(W) * D;
  if (n > 0) k_build_hmat<<<stream_grid(n), kStreamThreads, 0, stream>>>(ellp, n, D, sector, groups, emask, ivals, fast, hmat);
  return cudaGetLastError();
}

cudaError_t ell_device_count(const uint32_t* sector, int64_t D, const GroupRec* groups, int G, const int32_t* order,
                             int n_elec, int n_alpha, int32_t* len, int32_t* wmax, cudaStream_t stream) {
  (void)order;
  cudaError_t e = cudaMemsetAsync(wmax, 0, sizeof(int32_t), stream);
  if (e != cudaSuccess) return e;
  k_ell_count<<<stream_grid(D) * 4, kStreamThreads, 0, stream>>>(sector, D, groups, G, n_elec, n_alpha, len, wmax);
  return cudaGetLastError();
}

cudaError_t ell_device_fill(const uint32_t* sector, int64_t D, const GroupRec* groups, int G, const int32_t* order,
                            int n_elec, int n_alpha, int W, uint16_t* ell, cudaStream_t stream) {
  k_ell_fill<<<stream_grid(D) * 4, kStreamThreads, 0, stream>>>(sector, D, groups, G, order, n_elec, n_alpha, W, ell);
  return cudaGetLastError();
}

}  // namespace vqe
