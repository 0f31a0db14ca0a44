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

namespace vqe {
namespace {

__device__ __forceinline__ int parity32(uint32_t v) { return __popc(v) & 1; }

// v with its sign bit flipped when s == 1 (integer pipe, no FP64 op).
__device__ __forceinline__ double sflip(double v, int s) {
  return __hiloint2double(__double2hiint(v) ^ (s << 31), __double2loint(v));
}
__device__ __forceinline__ double2 sflip(double2 v, int s) {
  return make_double2(sflip(v.x, s), sflip(v.y, s));
}

// ---------------------------------------------------------------- fixed-point sweeps
// The resident kernel's real sweeps can run in 64-bit fixed point on the
// integer pipe: amplitudes of the unit-norm state as Q1.62 (value = v / 2^62),
// cos and sin magnitudes as unsigned Q0.64 with their signs kept apart, so a
// product is the high word of a 64 x 64 multiply. Rotations preserve the
// 2-norm, so |value| <= 1 holds for every entry at every gate.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ double llbits(long long v) { return __longlong_as_double(v); }
// floor(a * b / 2^64) for signed a, unsigned b
__device__ __forceinline__ long long mulhi_su(long long a, unsigned long long b) {
  const unsigned long long h = __umul64hi(static_cast<unsigned long long>(a), b);
  return static_cast<long long>(h - (a < 0 ? b : 0ull));
}
// v, negated when b == 1
__device__ __forceinline__ long long neg_if(long long v, int b) {
  const long long m = -static_cast<long long>(b);
  return (v ^ m) - m;
}
// |x| * 2^64 rounded, for |x| <= 1 (1 itself saturates to 2^64 - 1)
__device__ __forceinline__ unsigned long long fix_mag(double x) {
  const double a = fabs(x) * 18446744073709551616.0;
  return a >= 18446744073709551616.0 ? ~0ull : __double2ull_rn(a);
}
// 2^e as a double, for |e| < 1000
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double(static_cast<long long>(1023 + e) << 52); }
// smallest e with b < 2^e for a finite b >= 0 (clamped to [-400, 400])
__device__ __forceinline__ int bound_exp(double b) {
  const int ex = int((__double_as_longlong(b) >> 52) & 0x7ff);
  const int e = ex == 0 ? -400 : ex - 1022;
  return e < -400 ? -400 : (e > 400 ? 400 : e);
}

__device__ __forceinline__ uint32_t pattern_of(uint32_t src, uint32_t upos, int ubits) {
  uint32_t u = 0;
#pragma unroll
  for (int j = 0; j < kMaxPatternBits; ++j)
    if (j < ubits) u |= ((src >> ((upos >> (8 * j)) & 31u)) & 1u) << j;
  return u;
}

__device__ __forceinline__ GateRec load_gate(const GateRec* p) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(p));
  GateRec r;
  r.flip = uint32_t(a.x);
  r.par = uint32_t(a.y);
  r.sign0 = a.z;
  r.pad = 0;
  return r;
}

// ---------------------------------------------------------------- amplitude algebra
template <bool REAL> struct Amp;

template <> struct Amp<true> {
  typedef double T;
  typedef double C;  // coefficient type
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T unit() { return 1.0; }
  static __device__ __forceinline__ C coef(const InstDesc& d, int64_t slot) { return __ldg(d.vals + slot); }
  // acc += f * p
  static __device__ __forceinline__ void mac(T& acc, C f, T p) { acc = fma(f, p, acc); }
  // Re(conj(a) * b)
  static __device__ __forceinline__ double redot(T a, T b) { return a * b; }
  // (c a - ss b, ss a + c b); nss = -ss comes in precomputed (sign bit flipped
  // in the integer pipe) so that no FP64 negation is issued
  static __device__ __forceinline__ void rot(T& a, T& b, double c, double ss, double nss) {
    const T a0 = a;
    a = fma(nss, b, c * a0);
    b = fma(ss, a0, c * b);
  }
  // lb pa - la pb
  static __device__ __forceinline__ double cross(T lb, T pa, T la, T pb) {
    return fma(lb, pa, -(la * pb));
  }
  static __device__ __forceinline__ double2 to_c(T a) { return make_double2(a, 0.0); }
  static __device__ __forceinline__ T from_c(double2 a) { return a.x; }
};

template <> struct Amp<false> {
  typedef double2 T;
  typedef double2 C;
  static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ T unit() { return make_double2(1.0, 0.0); }
  static __device__ __forceinline__ C coef(const InstDesc& d, int64_t slot) { return __ldg(d.cvals + slot); }
  static __device__ __forceinline__ void mac(T& acc, C f, T p) {
    acc.x = fma(f.x, p.x, fma(-f.y, p.y, acc.x));
    acc.y = fma(f.x, p.y, fma(f.y, p.x, acc.y));
  }
  static __device__ __forceinline__ double redot(T a, T b) { return fma(a.x, b.x, a.y * b.y); }
  static __device__ __forceinline__ void rot(T& a, T& b, double c, double ss, double nss) {
    const T a0 = a;
    a.x = fma(nss, b.x, c * a0.x);
    a.y = fma(nss, b.y, c * a0.y);
    b.x = fma(ss, a0.x, c * b.x);
    b.y = fma(ss, a0.y, c * b.y);
  }
  static __device__ __forceinline__ double cross(T lb, T pa, T la, T pb) {
    return fma(lb.x, pa.x, fma(lb.y, pa.y, -fma(la.x, pb.x, la.y * pb.y)));
  }
  static __device__ __forceinline__ double2 to_c(T a) { return a; }
  static __device__ __forceinline__ T from_c(double2 a) { return a; }
};

__device__ __forceinline__ GroupRec load_group(const GroupRec* p) {
  const int4* q = reinterpret_cast<const int4*>(p);
  const int4 a = q[0];
  const int4 b = q[1];
  GroupRec g;
  g.x = uint32_t(a.x);
  g.upos = uint32_t(a.y);
  g.ebeg = a.z;
  g.eend = a.w;
  g.vbeg = b.x;
  g.ubits = b.y;
  g.kind = b.z;
  g.nq = b.w;
  return g;
}

template <typename C>
__device__ __forceinline__ void cadd(C& f, const C& v) {
  if constexpr (sizeof(C) == sizeof(double)) {
    f += v;
  } else {
    f.x += v.x;
    f.y += v.y;
  }
}

// Folded coefficient f_g(src) of a group (all three forms of GroupRec), from
// tables in shared or global memory. Signs are applied in the integer pipe.
// u is the pattern of src on the group's pattern qubits (pattern_of).
template <bool REAL>
__device__ __forceinline__ typename Amp<REAL>::C group_coef_u(const GroupRec& g, const uint32_t* emask,
                                                              const typename Amp<REAL>::C* vals, uint32_t src,
                                                              uint32_t u) {
  typedef typename Amp<REAL>::C C;
  if (g.kind == 0) {
    const C* vp = vals + g.vbeg + u;
    C f = sflip(vp[0], parity32(src & emask[g.ebeg]));
    for (int e = g.ebeg + 1, j = 1; e < g.eend; ++e, ++j)
      cadd(f, sflip(vp[j << g.ubits], parity32(src & emask[e])));
    return f;
  }
  const uint32_t z0 = emask[g.ebeg];
  uint32_t m = src & emask[g.ebeg + 1];
  C f;
  if (g.kind == 1) {
    const C* vp = vals + g.vbeg + u;
    f = vp[0];
    while (m) {
      const int r = __ffs(m) - 1;
      m &= m - 1;
      cadd(f, vp[(1 + r) << g.ubits]);
    }
  } else {
    const C* q = vals + g.vbeg;
    const int nq = g.nq;
    f = q[0];
    while (m) {
      const int pb = __ffs(m) - 1;
      m &= m - 1;
      cadd(f, q[1 + pb]);
      const C* row = q + 1 + nq + pb * nq;
      uint32_t m2 = m;
      while (m2) {
        const int qb = __ffs(m2) - 1;
        m2 &= m2 - 1;
        cadd(f, row[qb]);
      }
    }
  }
  return sflip(f, parity32(src & z0));
}

template <bool REAL>
__device__ __forceinline__ typename Amp<REAL>::C group_coef(const GroupRec& g, const uint32_t* emask,
                                                            const typename Amp<REAL>::C* vals, uint32_t src) {
  return group_coef_u<REAL>(g, emask, vals, src, pattern_of(src, g.upos, g.ubits));
}

// group_coef split at its first table term: v0 = vals[vbeg + u] and z = emask[ebeg]
// (the first entry's value and mask in the entry form, B[u] or Q[0] and z0 in the
// occupation forms) are loaded by the caller ahead of time; this adds the rest in
// the same order as group_coef, so the result is bitwise the same.
template <bool REAL>
__device__ __forceinline__ typename Amp<REAL>::C group_coef_rest(const GroupRec& g, const uint32_t* emask,
                                                                 const typename Amp<REAL>::C* vals, uint32_t src,
                                                                 typename Amp<REAL>::C v0, uint32_t z) {
  typedef typename Amp<REAL>::C C;
  if (g.kind == 0) {
    const uint32_t u = pattern_of(src, g.upos, g.ubits);
    const C* vp = vals + g.vbeg + u;
    C f = sflip(v0, parity32(src & z));
    for (int e = g.ebeg + 1, j = 1; e < g.eend; ++e, ++j)
      cadd(f, sflip(vp[j << g.ubits], parity32(src & emask[e])));
    return f;
  }
  uint32_t m = src & emask[g.ebeg + 1];
  C f = v0;
  if (g.kind == 1) {
    const uint32_t u = pattern_of(src, g.upos, g.ubits);
    const C* vp = vals + g.vbeg + u;
    while (m) {
      const int r = __ffs(m) - 1;
      m &= m - 1;
      cadd(f, vp[(1 + r) << g.ubits]);
    }
  } else {
    const C* q = vals + g.vbeg;
    const int nq = g.nq;
    while (m) {
      const int pb = __ffs(m) - 1;
      m &= m - 1;
      cadd(f, q[1 + pb]);
      const C* row = q + 1 + nq + pb * nq;
      uint32_t m2 = m;
      while (m2) {
        const int qb = __ffs(m2) - 1;
        m2 &= m2 - 1;
        cadd(f, row[qb]);
      }
    }
  }
  return sflip(f, parity32(src & z));
}


__device__ __forceinline__ bool in_sector(uint32_t k, int n_elec, int n_alpha) {
  if (__popc(k) != n_elec) return false;
  return n_alpha < 0 || __popc(k & 0x55555555u) == n_alpha;
}

// Position of basis state k in the sector's sorted list (k must be in the
// sector): the count of sector states with a smaller high part, plus the rank
// of the low part among low parts with the same electron counts.
__device__ __forceinline__ uint32_t sector_rank(const InstDesc& d, uint32_t k) {
  return __ldg(d.rank_hi + (k >> d.lo_bits)) + __ldg(d.rank_lo + (k & ((1u << d.lo_bits) - 1u)));
}

// Entry j of output r's connectivity row (kEllPad past the row's end).
__device__ __forceinline__ uint32_t ell_at(const uint32_t* ell, const uint16_t* ell16, int64_t idx) {
  if (ell16) {
    const uint32_t v = __ldg(ell16 + idx);
    return v == 0xFFFFu ? kEllPad : v;
  }
  return __ldg(ell + idx);
}

// Calls f(gi) for the group indices of output r's connectivity row at slots
// j = first, first + step, ... in order, up to the first pad. The indices are
// read in chunks of kEllChunk and the next chunk is requested before the
// current one is used, so a thread has a chunk of loads in flight instead of
// one L2 round trip per entry.
constexpr int kEllChunk = 8;
template <class F>
__device__ __forceinline__ void ell_row(const uint32_t* ell, const uint16_t* ell16, int W, int64_t D, int64_t r,
                                       int first, int step, F&& f) {
  constexpr int U = kEllChunk;
  uint32_t cur[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int j = first + u * step;
    cur[u] = j < W ? ell_at(ell, ell16, int64_t(j) * D + r) : kEllPad;
  }
  for (int j0 = first; j0 < W; j0 += U * step) {
    const bool more = cur[U - 1] != kEllPad && j0 + U * step < W;
    uint32_t nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + (U + u) * step;
      nxt[u] = (more && j < W) ? ell_at(ell, ell16, int64_t(j) * D + r) : kEllPad;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cur[u] != kEllPad) f(cur[u]);
    if (!more) break;
#pragma unroll
    for (int u = 0; u < U; ++u) cur[u] = nxt[u];
  }
}

// group_coef on fixed-point tables (int64, one common scale): the same terms,
// summed exactly in the integer pipe.
__device__ __forceinline__ long long group_coef_int(const GroupRec& g, const uint32_t* emask, const long long* vals,
                                                    uint32_t src, uint32_t u) {
  if (g.kind == 0) {
    const long long* vp = vals + g.vbeg + u;
    long long f = neg_if(vp[0], parity32(src & emask[g.ebeg]));
    for (int e = g.ebeg + 1, j = 1; e < g.eend; ++e, ++j) f += neg_if(vp[j << g.ubits], parity32(src & emask[e]));
    return f;
  }
  const uint32_t z0 = emask[g.ebeg];
  uint32_t m = src & emask[g.ebeg + 1];
  long long f;
  if (g.kind == 1) {
    const long long* vp = vals + g.vbeg + u;
    f = vp[0];
    while (m) {
      const int r = __ffs(m) - 1;
      m &= m - 1;
      f += vp[(1 + r) << g.ubits];
    }
  } else {
    const long long* q = vals + g.vbeg;
    const int nq = g.nq;
    f = q[0];
    while (m) {
      const int pb = __ffs(m) - 1;
      m &= m - 1;
      f += q[1 + pb];
      const long long* row = q + 1 + nq + pb * nq;
      uint32_t m2 = m;
      while (m2) {
        const int qb = __ffs(m2) - 1;
        m2 &= m2 - 1;
        f += row[qb];
      }
    }
  }
  return neg_if(f, parity32(src & z0));
}

// One output row of H psi over the compressed state (entry r of psi is sector
// state r): sum over the row's connectivity entries j of f_{g_j}(src) psi[rank(src)],
// src = k ^ x_{g_j}, in row order. Entries are taken in chunks of U: first every
// entry's group record, source rank, psi value and first table term are loaded
// (independent loads, all in flight together), then the chunk is combined in
// order; only groups with more than one table term go back to memory there.
template <bool REAL, int U>
__device__ __forceinline__ typename Amp<REAL>::T hpsi_row(const uint32_t* ell, const uint16_t* ell16, int W, int64_t D,
                                                          int64_t r, uint32_t k, const GroupRec* groups,
                                                          const uint32_t* emask, const typename Amp<REAL>::C* vals,
                                                          const typename Amp<REAL>::T* psi, const uint32_t* rank_hi,
                                                          const uint32_t* rank_lo, int lo_bits) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  typedef typename A::C C;
  const uint32_t lo_mask = (1u << lo_bits) - 1u;
  T acc = A::zero();
  uint32_t cur[U];
#pragma unroll
  for (int u = 0; u < U; ++u) cur[u] = u < W ? ell_at(ell, ell16, int64_t(u) * D + r) : kEllPad;
  for (int j0 = 0; j0 < W; j0 += U) {
    const bool more = cur[U - 1] != kEllPad && j0 + U < W;
    uint32_t nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      nxt[u] = (more && j0 + U + u < W) ? ell_at(ell, ell16, int64_t(j0 + U + u) * D + r) : kEllPad;
    uint32_t src[U], z[U], extra = 0;
    T pv[U];
    C v0[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool live = cur[u] != kEllPad;
      const GroupRec g = load_group(groups + (live ? cur[u] : 0u));
      src[u] = k ^ g.x;
      // a pad slot reads row r itself (a valid index) and is dropped below
      const uint32_t rs = live ? __ldg(rank_hi + (src[u] >> lo_bits)) + __ldg(rank_lo + (src[u] & lo_mask))
                               : uint32_t(r);
      pv[u] = psi[rs];
      v0[u] = vals[g.vbeg + int(pattern_of(src[u], g.upos, g.ubits))];
      z[u] = emask[g.ebeg];
      if (g.kind != 0 || g.eend > g.ebeg + 1) extra |= 1u << u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cur[u] == kEllPad) continue;
      C f;
      if ((extra >> u) & 1u)
        f = group_coef_rest<REAL>(load_group(groups + cur[u]), emask, vals, src[u], v0[u], z[u]);
      else
        f = sflip(v0[u], parity32(src[u] & z[u]));
      A::mac(acc, f, pv[u]);
    }
    if (!more) break;
#pragma unroll
    for (int u = 0; u < U; ++u) cur[u] = nxt[u];
  }
  return acc;
}

// Deterministic block sum; the result is valid in thread 0.
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < int(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------- resident kernel
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void sweep_barrier(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
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
  double2* pl = reinterpret_cast<double2*>(smem + L.psi);  // real: pl[r] = {psi_r, lambda_r}
  double2* cs = reinterpret_cast<double2*>(smem + L.cs);
  GateRec* gates = reinterpret_cast<GateRec*>(smem + L.gates);
  int32_t* poff = reinterpret_cast<int32_t*>(smem + L.poff);
  uint32_t* rp = reinterpret_cast<uint32_t*>(smem + L.pairs);
  double* gbuf = reinterpret_cast<double*>(smem + L.gbuf);
  double* red = reinterpret_cast<double*>(smem + L.red);
  const int64_t row = d.inst;
  const double* th = theta + row * ld_theta;

  // stage ansatz tables, clear the state
  for (int m = tid; m < M; m += bs) {
    double s, c;
    sincos(th[m], &s, &c);
    GateRec gr = load_gate(d.gates + m);
    if constexpr (FIX) {
      // magnitudes in Q0.64 (bit patterns kept in the double2 slot), signs in pad
      cs[m] = make_double2(llbits(static_cast<long long>(fix_mag(c))), llbits(static_cast<long long>(fix_mag(s))));
      gr.pad = (c < 0.0 ? 1 : 0) | (s < 0.0 ? 2 : 0);
    } else {
      cs[m] = make_double2(c, s);
    }
    gates[m] = gr;
  }
  for (int m = tid; m <= M; m += bs) poff[m] = int32_t(__ldg(d.pair_off + m));
  for (int p = tid; p < P; p += bs) {
    const uint2 e = __ldg(d.rpairs + p);
    rp[p] = (e.x & 0x7fffu) | ((e.x >> 31) << 15) | (e.y << 16);
  }
  if constexpr (REAL) {
    for (int r = tid; r < D; r += bs) pl[r] = make_double2(0.0, 0.0);
  } else {
    for (int r = tid; r < D; r += bs) {
      psi[r] = A::zero();
      lam[r] = A::zero();
    }
  }
  // pull the tables H psi reads later into L2 while the forward sweep runs
  {
    const char* ell_b = reinterpret_cast<const char*>(d.ellp);
    const int64_t ell_bytes = int64_t(W) * D * 4;
    for (int64_t o = int64_t(tid) * 128; o < ell_bytes; o += int64_t(bs) * 128) prefetch_l2(ell_b + o);
    const char* val_b = REAL ? reinterpret_cast<const char*>(d.vals) : reinterpret_cast<const char*>(d.cvals);
    const int64_t val_bytes = int64_t(d.S) * (REAL ? 8 : 16);
    for (int64_t o = int64_t(tid) * 128; o < val_bytes; o += int64_t(bs) * 128) prefetch_l2(val_b + o);
    const char* sec_b = reinterpret_cast<const char*>(d.sector);
    for (int64_t o = int64_t(tid) * 128; o < int64_t(D) * 4; o += int64_t(bs) * 128) prefetch_l2(sec_b + o);
  }
  __syncthreads();
  if (tid == 0) {
    if constexpr (FIX)
      pl[d.hf_rank].x = llbits(1ll << 62);
    else if constexpr (REAL)
      pl[d.hf_rank].x = 1.0;
    else
      psi[d.hf_rank] = A::unit();
  }
  __syncthreads();

  // lane-interleaved position of this thread in the sweep: consecutive pairs go
  // to consecutive warps so every sub-partition gets work on small gates
  const int swarps = sw >> 5;
  // complex: one lane per pair, consecutive pairs on consecutive warps;
  // real: two adjacent lanes per pair (role 0 and 1), pairs dealt the same way
  const int role = REAL ? (tid & 1) : 0;
  const int pstride = REAL ? (sw >> 1) : sw;
  const int spos = REAL ? (((tid & 31) >> 1) * swarps + (tid >> 5)) : ((tid & 31) * swarps + (tid >> 5));

  // a2: forward sweep. The next gate's record, cos/sin and first pair are
  // loaded before the current gate runs, off the barrier-to-barrier path.
  if (tid < sw && M > 0) {
    GateRec gr = gates[0];
    int p0 = poff[0], cnt = poff[1] - p0;
    double2 c_s = cs[0];
    uint32_t ef = (spos < cnt) ? rp[p0 + spos] : 0u;
    for (int m = 0; m < M; ++m) {
      GateRec grn = gr;
      int p0n = 0, cntn = 0;
      double2 c_sn = c_s;
      uint32_t efn = 0u;
      if (m + 1 < M) {
        grn = gates[m + 1];
        p0n = poff[m + 1];
        cntn = poff[m + 2] - p0n;
        c_sn = cs[m + 1];
        if (spos < cntn) efn = rp[p0n + spos];
      }
      if constexpr (REAL) {
        // two lanes per pair: role 0 writes c a - s b at ra, role 1 writes c b + s a
        // at rb; both lanes read before either writes (warp-uniform trip count,
        // lanes past the gate's end read entry 0 and store nothing)
        for (int q0 = 0; q0 < cnt; q0 += pstride) {
          const int q = q0 + spos;
          const bool act = q < cnt;
          const uint32_t e = (q0 == 0) ? ef : rp[p0 + min(q, cnt - 1)];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sgn = int((e >> 15) & 1u);
          const uint32_t kd = role ? rb : ra, ko = role ? ra : rb;
          const int slot = 2 * (p0 + q) + role;
          if constexpr (FIX) {
            const long long self = dbits(pl[kd].x), other = dbits(pl[ko].x);
            const int sneg = sgn ^ role ^ 1 ^ ((gr.pad >> 1) & 1);
            __syncwarp();
            const long long out = neg_if(mulhi_su(self, static_cast<unsigned long long>(dbits(c_s.x))), gr.pad & 1) +
                                  neg_if(mulhi_su(other, static_cast<unsigned long long>(dbits(c_s.y))), sneg);
            if (act) {
              pl[kd].x = llbits(out);
              gbuf[slot] = llbits(out);
            }
          } else {
            const double self = pl[kd].x, other = pl[ko].x;
            const double coef = sflip(c_s.y, sgn ^ role ^ 1);
            __syncwarp();
            const double out = fma(coef, other, c_s.x * self);
            if (act) {
              pl[kd].x = out;
              gbuf[slot] = out;
            }
          }
        }
      } else {
        for (int q = spos; q < cnt; q += sw) {
          const uint32_t e = (q == spos) ? ef : rp[p0 + q];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sb = int((e >> 15) & 1u);
          const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
          T a = psi[ra], b = psi[rb];
          A::rot(a, b, c_s.x, ss, nss);
          psi[ra] = a;
          psi[rb] = b;
        }
      }
      sweep_barrier(sw);
      gr = grn;
      p0 = p0n;
      cnt = cntn;
      c_s = c_sn;
      ef = efn;
    }
  }
  // stage the H psi tables
  const GroupRec* tg = d.groups;
  const uint32_t* te = d.emask;
  const C* tv;
  if constexpr (REAL) tv = d.vals; else tv = d.cvals;
  if (stage) {
    GroupRec* sg = reinterpret_cast<GroupRec*>(smem + L.tab);
    uint32_t* se = reinterpret_cast<uint32_t*>(smem + L.tab + uint32_t(G) * 32u);
    C* sv = reinterpret_cast<C*>(smem + L.tab + uint32_t(G) * 32u + align_up(uint32_t(d.E) * 4u, 16u));
    const int4* gsrc = reinterpret_cast<const int4*>(d.groups);
    int4* gdst = reinterpret_cast<int4*>(sg);
    for (int i = tid; i < 2 * G; i += bs) gdst[i] = __ldg(gsrc + i);
    for (int i = tid; i < d.E; i += bs) se[i] = __ldg(d.emask + i);
    if constexpr (FIX) {
      // fixed-point tables: v * 2^(62 - eh), where 2^eh bounds the sum of |v|
      // over every slot and so every row sum of |H|
      const int eh = bound_exp(*d.hbound);
      const double sc = pow2(62 - eh);
      for (int i = tid; i < d.S; i += bs) sv[i] = llbits(__double2ll_rn(__ldg(d.vals + i) * sc));
    } else {
      for (int i = tid; i < d.S; i += bs) sv[i] = A::coef(d, i);
    }
    tg = sg;
    te = se;
    tv = sv;
  }
  __syncthreads();
  // fixed-point H psi: staged integer tables times psi in Q1.62 (needs the
  // staged tables; otherwise psi goes to FP64 for the FP64 H psi)
  const bool int_h = FIX && stage;
  const int eh = int_h ? bound_exp(*d.hbound) : 0;
  if (FIX && !int_h) {
    for (int r = tid; r < D; r += bs) pl[r].x = __ll2double_rn(dbits(pl[r].x)) * 0x1p-62;
    __syncthreads();
  }

  // a3: lambda = H psi on the sector, E = <psi|lambda>
  double e_part = 0.0;
  const int r_half = (D + CL - 1) / CL;
  const int r_lo = crank * r_half, r_hi = min(D, r_lo + r_half);
  double2* pl_peer = pl;
  if constexpr (CL == 2) pl_peer = cooperative_groups::this_cluster().map_shared_rank(pl, crank ^ 1);
  // Real amplitudes: two threads per output row, one on the row's even slots and
  // one on its odd slots, added (even + odd) by a fixed shuffle; the split
  // depends on nothing but the row, so every launch form gives the same bits.
  constexpr int TPR = REAL ? 2 : 1;
  const int rows = r_hi - r_lo, per_pass = bs / TPR, half = tid % TPR;
  for (int base = 0; base < rows; base += per_pass) {  // same trip count in every thread
    const int lr = base + tid / TPR;
    const bool live = lr < rows;
    const int r = r_lo + (live ? lr : 0);
    const uint32_t k = __ldg(d.sector + r);
    if constexpr (FIX) {
      if (int_h) {
        // lambda in units of 2^(eh - 60): the high word of (table value) x (psi)
        long long acc = 0;
        if (live) {
          const long long* tvi = reinterpret_cast<const long long*>(tv);
          ell_row(d.ellp, nullptr, W, D, r, half, TPR, [&](uint32_t e) {
            const GroupRec g = load_group(tg + (e >> 19));
            acc += __mul64hi(group_coef_int(g, te, tvi, k ^ g.x, (e >> 15) & 15u), dbits(pl[e & 0x7fffu].x));
          });
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);  // even + odd slots (exact)
        if (live && half == 0) {
          pl[r].y = llbits(acc);
          if constexpr (CL == 2) pl_peer[r].y = llbits(acc);
          e_part += (__ll2double_rn(dbits(pl[r].x)) * 0x1p-62) * (__ll2double_rn(acc) * pow2(eh - 60));
        }
        continue;
      }
    }
    T acc = A::zero();
    if (live) {
      ell_row(d.ellp, nullptr, W, D, r, half, TPR, [&](uint32_t e) {
        const GroupRec g = load_group(tg + (e >> 19));
        const C f = group_coef_u<REAL>(g, te, tv, k ^ g.x, (e >> 15) & 15u);
        if constexpr (REAL)
          A::mac(acc, f, pl[e & 0x7fffu].x);
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
        pl[r].y = acc;
        if constexpr (CL == 2) pl_peer[r].y = acc;
        e_part += pl[r].x * acc;
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
      const double v = pl[r].y;
      l2 = fma(v, v, l2);
    }
    const double tot = block_sum(l2, red);
    if (tid == 0) red[56] = tot;
    __syncthreads();
    const int ex = int((dbits(red[56]) >> 52) & 0x7ff);
    // ||lambda||^2 < 2^(ex - 1022) <= 2^(2 lam_e)
    lam_e = ex == 0 ? -500 : (ex - 1022 + 1) >> 1;
    const double sc = pow2(61 - lam_e);
    for (int r = tid; r < D; r += bs) pl[r].y = llbits(__double2ll_rn(pl[r].y * sc));
    __syncthreads();
  }

  // a4: reverse sweep (same prefetch of the next gate as the forward sweep)
  if (tid < sw && M > 0) {
    int m = M - 1;
    GateRec gr = gates[m];
    int p0 = poff[m], cnt = poff[m + 1] - p0;
    double2 c_s = cs[m];
    uint32_t ef = (spos < cnt) ? rp[p0 + spos] : 0u;
    for (; m >= 0; --m) {
      GateRec grn = gr;
      int p0n = 0, cntn = 0;
      double2 c_sn = c_s;
      uint32_t efn = 0u;
      if (m > 0) {
        grn = gates[m - 1];
        p0n = poff[m - 1];
        cntn = poff[m] - p0n;
        c_sn = cs[m - 1];
        if (spos < cntn) efn = rp[p0n + spos];
      }
      if constexpr (REAL) {
        // two lanes per pair: the lane's slot holds phi at its own index (role 0
        // at ra, role 1 at rb); role 0 keeps s lambda_b phi_a, role 1 keeps
        // -s lambda_a phi_b, and each un-applies the gate to lambda at its index
        for (int q0 = 0; q0 < cnt; q0 += pstride) {
          const int q = q0 + spos;
          const bool act = q < cnt;
          const int qc = min(q, cnt - 1);
          const uint32_t e = (q0 == 0) ? ef : rp[p0 + qc];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sr_bit = int((e >> 15) & 1u) ^ role;
          const uint32_t ks = role ? rb : ra, ko = role ? ra : rb;
          const int slot = 2 * (p0 + qc) + role;
          if constexpr (FIX) {
            const long long ph = dbits(gbuf[slot]), ls = dbits(pl[ks].y), lo = dbits(pl[ko].y);
            __syncwarp();
            const unsigned long long cm = static_cast<unsigned long long>(dbits(c_s.x));
            const unsigned long long sm = static_cast<unsigned long long>(dbits(c_s.y));
            const int cneg = gr.pad & 1, sneg = ((gr.pad >> 1) & 1) ^ sr_bit;
            const long long g_term = neg_if(__mul64hi(ph, lo), sr_bit);
            const long long nl = neg_if(mulhi_su(ls, cm), cneg) + neg_if(mulhi_su(lo, sm), sneg);
            if (act) {
              gbuf[slot] = llbits(g_term);
              pl[ks].y = llbits(nl);
            }
          } else {
            const double ph = gbuf[slot], ls = pl[ks].y, lo = pl[ko].y;
            __syncwarp();
            const double sr = sflip(c_s.y, sr_bit);
            const double g_term = sflip(lo * ph, sr_bit);
            const double nl = fma(sr, lo, c_s.x * ls);
            if (act) {
              gbuf[slot] = g_term;
              pl[ks].y = nl;
            }
          }
        }
      } else {
        for (int q = spos; q < cnt; q += sw) {
          const uint32_t e = (q == spos) ? ef : rp[p0 + q];
          const uint32_t ra = e & 0x7fffu, rb = e >> 16;
          const int sb = int((e >> 15) & 1u);
          const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
          T pa = psi[ra], pb = psi[rb], la = lam[ra], lb = lam[rb];
          gbuf[p0 + q] = sflip(A::cross(lb, pa, la, pb), sb);
          A::rot(pa, pb, c_s.x, nss, ss);
          A::rot(la, lb, c_s.x, nss, ss);
          psi[ra] = pa;
          psi[rb] = pb;
          lam[ra] = la;
          lam[rb] = lb;
        }
      }
      sweep_barrier(sw);
      gr = grn;
      p0 = p0n;
      cnt = cntn;
      c_s = c_sn;
      ef = efn;
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

template <bool REAL>
__global__ void __launch_bounds__(kStreamThreads, 1)
k_gate_adj(const uint2* __restrict__ rp, int64_t P, const double2* __restrict__ cs,
           typename Amp<REAL>::T* __restrict__ phi, typename Amp<REAL>::T* __restrict__ lam,
           double* __restrict__ gpart) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  __shared__ double red[32];
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

// Groups gi in [g0, g1) of one bucket against a staged source row: for each
// group in order, lanes walk list entries [e0, e1) (this warp's share, or the
// whole list) and add f_g(src) psi_s[Jb] into lam_s[Ib]. The next group's
// record and range are loaded while the current group runs; U list entries per
// lane are in flight (8 with real amplitudes in the wide block form and in the
// warp form, else 4: the best measured for each). Entries of one list have
// distinct Ib, and __syncwarp separates the groups, so each output is updated
// by one lane at a time, in group order (U does not change the order).
template <bool REAL, int U>
__device__ __forceinline__ void str_groups(const StrPlan& sp, int g0, int g1, int w_lo, int w_hi, uint32_t ka,
                                           const GroupRec* __restrict__ groups, const uint32_t* __restrict__ emask,
                                           const typename Amp<REAL>::C* __restrict__ vals, const uint32_t* kb_s,
                                           const typename Amp<REAL>::T* psi_s, typename Amp<REAL>::T* lam_s,
                                           int lane) {
  typedef Amp<REAL> A;
  if (g0 >= g1) return;
  GroupRec g = load_group(groups + __ldg(sp.bgrp + g0));
  int e0 = __ldg(sp.bsplit + int64_t(g0) * (kStrWarps + 1) + w_lo);
  int e1 = __ldg(sp.bsplit + int64_t(g0) * (kStrWarps + 1) + w_hi);
  for (int gi = g0; gi < g1; ++gi) {
    GroupRec gn = g;
    int e0n = 0, e1n = 0;
    if (gi + 1 < g1) {
      gn = load_group(groups + __ldg(sp.bgrp + gi + 1));
      e0n = __ldg(sp.bsplit + int64_t(gi + 1) * (kStrWarps + 1) + w_lo);
      e1n = __ldg(sp.bsplit + int64_t(gi + 1) * (kStrWarps + 1) + w_hi);
    }
    for (int e = e0 + lane; e < e1; e += U * 32) {
      uint32_t ent[U];
#pragma unroll
      for (int u = 0; u < U; ++u) ent[u] = (e + 32 * u < e1) ? __ldg(sp.lists + e + 32 * u) : 0xFFFFFFFFu;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (ent[u] == 0xFFFFFFFFu) break;
        const uint32_t ib = ent[u] & 0xFFFFu, jb = ent[u] >> 16;
        A::mac(lam_s[ib], group_coef<REAL>(g, emask, vals, ka | kb_s[jb]), psi_s[jb]);
      }
    }
    __syncwarp();
    g = gn;
    e0 = e0n;
    e1 = e1n;
  }
}

// String-driven H psi (spin sectors; see StrPlan), block form for large beta
// string sets: lambda[Ia, :] for one output alpha string per block. For each
// bucket with a source alpha string Ja, the source row psi[Ja, :] is staged in
// shared memory; then every warp walks its share (a fixed Ib range) of each
// group's beta pair list. Needs blockDim.x == 32 * kStrWarps and 2 * Db
// amplitudes (+ Db words of beta strings when Db < kStrWideDb; above, they are
// read from global memory through L1) of shared memory.
template <bool REAL, bool WIDE>
__device__ __forceinline__ void hpsi_str_row(const StrPlan& sp, int ia, const GroupRec* __restrict__ groups,
                                             const uint32_t* __restrict__ emask,
                                             const typename Amp<REAL>::C* __restrict__ vals,
                                             const typename Amp<REAL>::T* __restrict__ psi_am,
                                             typename Amp<REAL>::T* __restrict__ lam_am, unsigned char* smem) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  const int tid = threadIdx.x, bs = blockDim.x, w = tid >> 5, lane = tid & 31;
  const int Db = sp.Db, NB = sp.NB;
  T* psi_s = reinterpret_cast<T*>(smem);
  T* lam_s = psi_s + Db;
  uint32_t* kb_stage = reinterpret_cast<uint32_t*>(lam_s + Db);
  const uint32_t* kb_s = WIDE ? sp.kb : kb_stage;
  for (int j = tid; j < Db; j += bs) {
    lam_s[j] = A::zero();
    if (!WIDE) kb_stage[j] = __ldg(sp.kb + j);
  }
  for (int b = 0; b < NB; ++b) {
    const int ja = __ldg(sp.ja + int64_t(ia) * NB + b);
    if (ja < 0) continue;  // same for the whole block
    const T* row = psi_am + int64_t(ja) * Db;
    {
      // A bucket holding a single group that leaves the beta string unchanged
      // (an alpha-alpha double, most buckets at 24-30 qubits): every output
      // beta string takes one term from the same position of the source row, so
      // it is read straight from global memory, without staging or a pair list.
      // Each output still gets its terms in bucket order: the same bits.
      const int g0 = __ldg(sp.boff + b);
      if (__ldg(sp.boff + b + 1) - g0 == 1) {
        const GroupRec g = load_group(groups + __ldg(sp.bgrp + g0));
        if ((g.x & 0xAAAAAAAAu) == 0) {
          __syncthreads();  // outputs were last updated under the list path's thread mapping
          const uint32_t ka = __ldg(sp.ka + ja);
          for (int j = tid; j < Db; j += bs) A::mac(lam_s[j], group_coef<REAL>(g, emask, vals, ka | kb_s[j]), row[j]);
          continue;
        }
      }
    }
    __syncthreads();       // the previous source row is no longer read
    for (int j = tid; j < Db; j += bs) psi_s[j] = row[j];
    __syncthreads();
    str_groups<REAL, (WIDE && REAL) ? 8 : 4>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), w, w + 1, __ldg(sp.ka + ja), groups, emask,
                     vals, kb_s, psi_s, lam_s, lane);
  }
  __syncthreads();
  T* out = lam_am + int64_t(ia) * Db;
  for (int j = tid; j < Db; j += bs) out[j] = lam_s[j];
}

// Warp form for small beta string sets: each warp owns one output alpha string
// (ia0 + warp), stages its own source rows and walks whole lists; the same
// per-output order as the block form, so the same bits. Shared memory: Db
// words of beta strings, then 2 * Db amplitudes per warp.
template <bool REAL>
__device__ __forceinline__ void hpsi_str_warps(const StrPlan& sp, int ia0, const GroupRec* __restrict__ groups,
                                               const uint32_t* __restrict__ emask,
                                               const typename Amp<REAL>::C* __restrict__ vals,
                                               const typename Amp<REAL>::T* __restrict__ psi_am,
                                               typename Amp<REAL>::T* __restrict__ lam_am, unsigned char* smem) {
  typedef Amp<REAL> A;
  typedef typename A::T T;
  const int tid = threadIdx.x, bs = blockDim.x, w = tid >> 5, lane = tid & 31;
  const int Db = sp.Db, NB = sp.NB;
  uint32_t* kb_s = reinterpret_cast<uint32_t*>(smem);
  T* psi_s = reinterpret_cast<T*>(smem + align_up(uint32_t(Db) * 4u, 16u)) + int64_t(w) * 2 * Db;
  T* lam_s = psi_s + Db;
  for (int j = tid; j < Db; j += bs) kb_s[j] = __ldg(sp.kb + j);
  __syncthreads();
  const int ia = ia0 + w;
  if (ia >= sp.Da) return;  // no block-wide barrier follows
  for (int j = lane; j < Db; j += 32) lam_s[j] = A::zero();
  for (int b = 0; b < NB; ++b) {
    const int ja = __ldg(sp.ja + int64_t(ia) * NB + b);
    if (ja < 0) continue;  // same for the whole warp
    const T* row = psi_am + int64_t(ja) * Db;
    {
      // single beta-diagonal group: read the source row directly (as in the block form)
      const int g0 = __ldg(sp.boff + b);
      if (__ldg(sp.boff + b + 1) - g0 == 1) {
        const GroupRec g = load_group(groups + __ldg(sp.bgrp + g0));
        if ((g.x & 0xAAAAAAAAu) == 0) {
          __syncwarp();
          const uint32_t ka = __ldg(sp.ka + ja);
          for (int j = lane; j < Db; j += 32) A::mac(lam_s[j], group_coef<REAL>(g, emask, vals, ka | kb_s[j]), row[j]);
          continue;
        }
      }
    }
    __syncwarp();
    for (int j = lane; j < Db; j += 32) psi_s[j] = row[j];
    __syncwarp();
    str_groups<REAL, REAL ? 8 : 4>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), 0, kStrWarps, __ldg(sp.ka + ja), groups, emask,
                     vals, kb_s, psi_s, lam_s, lane);
  }
  __syncwarp();
  T* out = lam_am + int64_t(ia) * Db;
  for (int j = lane; j < Db; j += 32) out[j] = lam_s[j];
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

// ---------------------------------------------------------------- batched streaming (gate-major)
__device__ __forceinline__ int find_seg(const int64_t* __restrict__ pref, int nseg, int64_t item) {
  int lo = 0, hi = nseg;  // pref[lo] <= item < pref[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(pref + mid) <= item)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// cos/sin of every (instance, gate)
__global__ void kb_trig(BatchDev b, const double* __restrict__ theta, int64_t ld) {
  const int64_t n_items = int64_t(b.n) * b.Mmax;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n_items; t += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(t / b.Mmax), m = int(t % b.Mmax);
    const InstDesc* d = b.desc + i;
    if (m < d->M) {
      double sn, c;
      sincos(theta[d->inst * ld + m], &sn, &c);
      b.cs[t] = make_double2(c, sn);
    }
  }
}

__global__ void kb_init(BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t r = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    double* psi = reinterpret_cast<double*>(b.ws + b.psi_off[i]);
    const uint32_t k = __ldg(d->sector + r);
    psi[r] = (k == d->hf) ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(512) kb_gate_fwd(int m, BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t q = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    double* psi = reinterpret_cast<double*>(b.ws + b.psi_off[i]);
    const double2 c_s = b.cs[int64_t(i) * b.Mmax + m];
    const uint2 pr = __ldg(d->rpairs + __ldg(d->pair_off + m) + q);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
    double a = psi[ra], bb = psi[rb];
    Amp<true>::rot(a, bb, c_s.x, ss, nss);
    psi[ra] = a;
    psi[rb] = bb;
  }
}

__global__ void __launch_bounds__(512, 1) kb_hpsi(BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t r = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    const double* psi = reinterpret_cast<const double*>(b.ws + b.psi_off[i]);
    double* lam = reinterpret_cast<double*>(b.ws + b.lam_off[i]);
    const uint32_t k = __ldg(d->sector + r);
    const GroupRec* groups = d->groups;
    const uint32_t* emask = d->emask;
    const double* vals = d->vals;
    const int W = d->W, G = d->G;
    const int64_t D = d->D;
    double acc = 0.0;
    if (W > 0) {
      const uint32_t* ell = d->ell;
      const uint16_t* ell16 = d->ell16;
      acc = hpsi_row<true, 4>(ell, ell16, W, D, r, k, groups, emask, vals, psi, d->rank_hi, d->rank_lo,
                              d->lo_bits);
    } else {
      const int ne = d->n_elec, na = d->n_alpha;
      for (int gi = 0; gi < G; ++gi) {
        const GroupRec g = load_group(groups + gi);
        const uint32_t src = k ^ g.x;
        if (!in_sector(src, ne, na)) continue;
        acc = fma(group_coef<true>(g, emask, vals, src), psi[sector_rank(*d, src)], acc);
      }
    }
    lam[r] = acc;
    b.ebuf[b.ebase[i] + r] = psi[r] * acc;
  }
}

// String-driven H psi over the batch: block -> (instance slot, output alpha string)
__global__ void __launch_bounds__(kStrWarps * 32, 2) kb_hpsi_str(BatchDev b, BatchSegs sg) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int s = find_seg(sg.pref, sg.nseg, int64_t(blockIdx.x));
  const int i = __ldg(sg.inst + s);
  const int blk = int(int64_t(blockIdx.x) - __ldg(sg.pref + s));
  const InstDesc* d = b.desc + i;
  const StrPlan sp = *d->str;
  const double* psi_am = reinterpret_cast<const double*>(b.ws + b.am_off[i]);
  double* lam_am = reinterpret_cast<double*>(b.ws + b.am_off[i]) + d->D;
  if (sp.Db >= kStrMinDb)
    if (sp.Db >= kStrWideDb)
      hpsi_str_row<true, true>(sp, blk, d->groups, d->emask, d->vals, psi_am, lam_am, smem);
    else
      hpsi_str_row<true, false>(sp, blk, d->groups, d->emask, d->vals, psi_am, lam_am, smem);
  else
    hpsi_str_warps<true>(sp, blk * kStrWarps, d->groups, d->emask, d->vals, psi_am, lam_am, smem);
}

// alpha-major copy of every instance's psi
__global__ void kb_perm_gather(BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t r = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    const double* psi = reinterpret_cast<const double*>(b.ws + b.psi_off[i]);
    double* psi_am = reinterpret_cast<double*>(b.ws + b.am_off[i]);
    psi_am[r] = psi[__ldg(d->str->perm + r)];
  }
}

// lambda back to sector order, and the per-output energy terms psi_r lambda_r
__global__ void kb_perm_scatter(BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t r = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    const double* psi = reinterpret_cast<const double*>(b.ws + b.psi_off[i]);
    double* lam = reinterpret_cast<double*>(b.ws + b.lam_off[i]);
    const double* lam_am = reinterpret_cast<const double*>(b.ws + b.am_off[i]) + d->D;
    const uint32_t k = __ldg(d->str->perm + r);
    const double v = lam_am[r];
    lam[k] = v;
    b.ebuf[b.ebase[i] + k] = psi[k] * v;
  }
}

// E of instance slot blockIdx.x: fixed-order sum of its per-output terms
__global__ void kb_energy(BatchDev b, double* __restrict__ energy) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const InstDesc* d = b.desc + i;
  const double* e = b.ebuf + b.ebase[i];
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < d->D; r += blockDim.x) acc += e[r];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) energy[d->inst] = tot;
}

__global__ void __launch_bounds__(512) kb_gate_adj(int m, BatchDev b, BatchSegs sg) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < sg.total; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(sg.pref, sg.nseg, t);
    const int i = __ldg(sg.inst + s);
    const int64_t q = t - __ldg(sg.pref + s);
    const InstDesc* d = b.desc + i;
    double* phi = reinterpret_cast<double*>(b.ws + b.psi_off[i]);
    double* lam = reinterpret_cast<double*>(b.ws + b.lam_off[i]);
    const double2 c_s = b.cs[int64_t(i) * b.Mmax + m];
    const int64_t p = __ldg(d->pair_off + m) + q;
    const uint2 pr = __ldg(d->rpairs + p);
    const uint32_t ra = pr.x & 0x7fffffffu, rb = pr.y;
    const int sb = int(pr.x >> 31);
    const double ss = sflip(c_s.y, sb), nss = sflip(c_s.y, sb ^ 1);
    double pa = phi[ra], pb = phi[rb], la = lam[ra], lb = lam[rb];
    b.gbuf[b.gbase[i] + p] = sflip(Amp<true>::cross(lb, pa, la, pb), sb);
    Amp<true>::rot(pa, pb, c_s.x, nss, ss);
    Amp<true>::rot(la, lb, c_s.x, nss, ss);
    phi[ra] = pa;
    phi[rb] = pb;
    lam[ra] = la;
    lam[rb] = lb;
  }
}

// g of (instance, gate) pair blockIdx.x: fixed-order sum of its pair contributions
__global__ void kb_grad(BatchDev b, const int32_t* __restrict__ gm_inst, const int32_t* __restrict__ gm_gate,
                        double* __restrict__ grad, int64_t ld_grad) {
  __shared__ double red[32];
  const int i = gm_inst[blockIdx.x], m = gm_gate[blockIdx.x];
  const InstDesc* d = b.desc + i;
  const int64_t p0 = d->pair_off[m], p1 = d->pair_off[m + 1];
  const double* gb = b.gbuf + b.gbase[i];
  double acc = 0.0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) acc += gb[p];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) grad[d->inst * ld_grad + m] = 2.0 * tot;
}

inline int batch_grid(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return int(g);
}

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

// ---------------------------------------------------------------- launchers
cudaError_t set_str_smem_limit(size_t smem) {
  const int b = int(smem);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_hpsi_str<true, false>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<false, false>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<true, true>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hpsi_str<false, true>, a, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_hpsi_str, a, b);
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
template <bool REAL>
cudaError_t stream_forward(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                           const double* theta, cudaStream_t stream) {
  typedef typename Amp<REAL>::T T;
  T* psi = static_cast<T*>(b.psi);
  const int nt = kStreamThreads;
  if (d.M > 0) k_trig<<<(d.M + 255) / 256, 256, 0, stream>>>(theta, d.M, b.cs);
  k_init_sector<REAL><<<stream_grid(d.D), nt, 0, stream>>>(d.sector, d.D, d.hf, psi);
  for (int m = 0; m < d.M; ++m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    if (p1 > p0)
      k_gate_fwd<REAL><<<stream_grid(p1 - p0), nt, 0, stream>>>(d.rpairs + p0, p1 - p0, b.cs + m, psi);
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
  for (int m = d.M - 1; m >= 0; --m) {
    const int64_t p0 = sp.pair_off_host[m], p1 = sp.pair_off_host[m + 1];
    double* gp = b.gpart + int64_t(m) * kMaxPartials;
    k_gate_adj<REAL><<<stream_grid(p1 - p0), kStreamThreads, 0, stream>>>(d.rpairs + p0, p1 - p0, b.cs + m,
                                                                          phi, lam, gp);
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

cudaError_t batch_stream_run(const BatchDev& b, const BatchSegs* gate_segs, const BatchSegs& out_segs,
                             const BatchSegs& str_segs, size_t str_smem,
                             const int32_t* d_gm_inst, const int32_t* d_gm_gate, int64_t n_gm,
                             const double* theta, int64_t ld_theta, double* energy, double* grad,
                             int64_t ld_grad, int threads, cudaStream_t stream) {
  if (b.n == 0) return cudaSuccess;
  const int nt = threads;
  if (b.Mmax > 0) kb_trig<<<batch_grid(int64_t(b.n) * b.Mmax, nt), nt, 0, stream>>>(b, theta, ld_theta);
  kb_init<<<batch_grid(out_segs.total, nt), nt, 0, stream>>>(b, out_segs);
  for (int m = 0; m < b.Mmax; ++m)
    if (gate_segs[m].total > 0)
      kb_gate_fwd<<<batch_grid(gate_segs[m].total, nt), nt, 0, stream>>>(m, b, gate_segs[m]);
  if (str_segs.total > 0) {
    kb_perm_gather<<<batch_grid(out_segs.total, nt), nt, 0, stream>>>(b, out_segs);
    kb_hpsi_str<<<unsigned(str_segs.total), kStrWarps * 32, str_smem, stream>>>(b, str_segs);
    kb_perm_scatter<<<batch_grid(out_segs.total, nt), nt, 0, stream>>>(b, out_segs);
  } else {
    kb_hpsi<<<batch_grid(out_segs.total, nt), nt, 0, stream>>>(b, out_segs);
  }
  kb_energy<<<b.n, 256, 0, stream>>>(b, energy);
  if (grad) {
    for (int m = b.Mmax - 1; m >= 0; --m)
      if (gate_segs[m].total > 0)
        kb_gate_adj<<<batch_grid(gate_segs[m].total, nt), nt, 0, stream>>>(m, b, gate_segs[m]);
    if (n_gm > 0) kb_grad<<<int(n_gm), 128, 0, stream>>>(b, d_gm_inst, d_gm_gate, grad, ld_grad);
  }
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
