// Device helpers shared by the CUDA translation units of libvqe (vqe_kernels.cu,
// vqe_batch.cu): amplitude algebra, the folded group coefficient f_g(src) of
// Eq. 2's Pauli groups, sector ranks, connectivity-row walkers, deterministic
// block sums and the string-driven H psi of a spin sector. Everything lives in
// an unnamed namespace, so each translation unit keeps its own copy.
#pragma once

#include <cuda_runtime.h>

#include "vqe_internal.h"

namespace vqe {
namespace {

// A state-vector load: through L2 only (ld.global.cg) when CG, for state that
// other CTAs of the same launch write while this one runs; a plain load otherwise.
template <bool CG, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

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

// ell_row over packed entries together with their precomputed coefficients
// (InstDesc::hmat, the same [W][D] layout): calls f(entry, coefficient) for the
// thread's slots first, first + step, ... in order. The walk advances two
// pointers by a fixed stride and counts the thread's slots once, so a slot
// costs its two loads and no index arithmetic; the next U slots are loaded
// while the current U are combined.
template <int U, class F>
__device__ __forceinline__ void ell_row_mat(const uint32_t* ell, const long long* mat, int W, int64_t D, int64_t r,
                                            int first, int step, F&& f) {
  const int n = (W - first + step - 1) / step;  // this thread's slots
  const int64_t stride = int64_t(step) * D;
  const uint32_t* pe = ell + int64_t(first) * D + r;
  const long long* pm = mat + int64_t(first) * D + r;
  uint32_t cur[U];
  long long cv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    cur[u] = u < n ? __ldg(pe + u * stride) : kEllPad;
    cv[u] = u < n ? __ldg(pm + u * stride) : 0ll;
  }
  for (int i0 = 0; i0 < n; i0 += U) {
    const bool more = cur[U - 1] != kEllPad && i0 + U < n;
    pe += U * stride;
    pm += U * stride;
    uint32_t nxt[U];
    long long nv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = more && i0 + U + u < n;
      nxt[u] = ok ? __ldg(pe + u * stride) : kEllPad;
      nv[u] = ok ? __ldg(pm + u * stride) : 0ll;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cur[u] != kEllPad) f(cur[u], cv[u]);
    if (!more) break;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cur[u] = nxt[u];
      cv[u] = nv[u];
    }
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
template <bool REAL, int U, bool CG = false>
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
      pv[u] = ld_state<CG>(psi + rs);
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

// The folded coefficient of a single-term group (kind 0 with one entry: every
// double excitation of Jordan-Wigner chemistry) for sources ka | kb that share
// the alpha string ka: the alpha string's pattern bits and sign are taken once
// per group, and only the beta string's bits per source. simple_value gives
// bit for bit what group_coef gives for the same source.
struct SimpleCoef {
  uint32_t base;  // vbeg plus the alpha pattern bits (bits 0-30), sign bit from the alpha string (bit 31)
  uint32_t qu;    // per beta pattern bit t, byte t = qubit position (odd, so never 0) | bit of u << 5
  uint32_t eb;    // beta part of the sign mask
};

__device__ __forceinline__ bool simple_coef(const GroupRec& g, const uint32_t* __restrict__ emask, uint32_t ka,
                                            SimpleCoef& c) {
  if (g.kind != 0 || g.eend != g.ebeg + 1) return false;
  const uint32_t em = __ldg(emask + g.ebeg);
  c.eb = em & 0xAAAAAAAAu;
  uint32_t base = uint32_t(g.vbeg), qu = 0u;
  int nb = 0;
#pragma unroll
  for (int j = 0; j < kMaxPatternBits; ++j) {
    if (j < g.ubits) {
      const uint32_t pos = (g.upos >> (8 * j)) & 31u;
      if (pos & 1u) {
        qu |= (pos | (uint32_t(j) << 5)) << (8 * nb);
        ++nb;
      } else {
        base += ((ka >> pos) & 1u) << j;
      }
    }
  }
  c.base = base | (uint32_t(parity32(ka & em)) << 31);
  c.qu = qu;
  return true;
}

template <typename C>
__device__ __forceinline__ C simple_value(const SimpleCoef& c, const C* __restrict__ vals, uint32_t kb) {
  uint32_t u = 0u;
#pragma unroll
  for (int t = 0; t < kMaxPatternBits; ++t) {
    const uint32_t q = (c.qu >> (8 * t)) & 255u;
    if (q == 0u) break;
    u |= ((kb >> (q & 31u)) & 1u) << (q >> 5);
  }
  return sflip(vals[(c.base & 0x7fffffffu) + u], int(c.base >> 31) ^ parity32(kb & c.eb));
}

// Groups gi in [g0, g1) of one bucket against a staged source row: for each
// group in order, lanes walk list entries [e0, e1) (this warp's share, or the
// whole list) and add f_g(src) psi_s[Jb] into lam_s[Ib]. The next group's
// record and range are loaded while the current group runs; U list entries per
// lane are in flight (4 here; the real wide block form and the real warp form run
// the pipelined str_groups_hot below with 16 and 8). Entries of one list have
// distinct Ib, and __syncwarp separates the groups, so each output is updated
// by one lane at a time, in group order (U does not change the order). HOIST:
// single-term groups take the source alpha string's part once per group
// (SimpleCoef); measured faster in the wide block form and the warp form, and
// slower in the staged block form, which therefore keeps group_coef.
template <bool REAL, int U, bool HOIST = true>
__device__ __forceinline__ void str_groups(const StrPlan& sp, int g0, int g1, int w_lo, int w_hi, uint32_t ka,
                                           const GroupRec* __restrict__ groups, const uint32_t* __restrict__ emask,
                                           const typename Amp<REAL>::C* __restrict__ vals, const uint32_t* kb_s,
                                           const typename Amp<REAL>::T* psi_s, typename Amp<REAL>::T* lam_s,
                                           int lane, uint32_t ob) {
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
    // walks this warp's list entries with coefficient function cf(beta string)
    auto walk = [&](auto&& cf) {
      for (int e = e0 + lane; e < e1; e += U * 32) {
        uint32_t ent[U];
#pragma unroll
        for (int u = 0; u < U; ++u) ent[u] = (e + 32 * u < e1) ? __ldg(sp.lists + e + 32 * u) : 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (ent[u] == 0xFFFFFFFFu) break;
          const uint32_t ib = ent[u] & 0x1FFFu, jb = (ent[u] >> 16) & 0x1FFFu;
          const uint32_t kbv = kb_s[jb];
          // the staged row carries (-1)^{|Jb & ob|}; undo it on the coefficient
          A::mac(lam_s[ib], sflip(cf(kbv), parity32(kbv & ob)), psi_s[jb]);
        }
      }
    };
    SimpleCoef sc;
    if (HOIST && simple_coef(g, emask, ka, sc))  // the same for the whole warp
      walk([&](uint32_t kbv) { return simple_value(sc, vals, kbv); });
    else
      walk([&](uint32_t kbv) { return group_coef<REAL>(g, emask, vals, ka | kbv); });
    __syncwarp();
    g = gn;
    e0 = e0n;
    e1 = e1n;
  }
}

// Real amplitudes, software-pipelined form of str_groups: while group gi's list
// is walked, group gi+1's coefficient state and table values are computed and
// loaded, and group gi+2's record is loaded (StrPlan::bgx, no group record or
// mask needed for single-term groups). A single-term group with at most two
// beta pattern bits has at most four distinct table values; they are loaded
// once per group and each list entry selects one by its beta bits, so the entry
// needs no table load. Every entry gets the same coefficient as from
// group_coef, and outputs are summed in the same order: the same bits. Used by
// the wide block form and the warp form (the staged block form measured
// faster with str_groups).
struct HotCoef {
  SimpleCoef sc;
  double v0, v1, v2, v3;  // vals[base + b0 * o0 + b1 * o1] for beta bits (b0, b1)
  int32_t mode;           // 0: general group (group_coef), 1: preloaded values, 2: one table load per entry,
                          // 3: alpha-hop x beta-hop group (v0, v1 signed; the list entry selects and signs)
};

__device__ __forceinline__ HotCoef hot_prep(uint4 r, uint32_t ka, const double* __restrict__ vals) {
  HotCoef h;
  h.v0 = h.v1 = h.v2 = h.v3 = 0.0;
  h.sc.qu = r.y;
  h.sc.eb = r.w & 0xAAAAAAAAu;
  if (!(r.z >> 31)) {
    h.mode = 0;
    h.sc.base = 0u;
    return h;
  }
  uint32_t base = r.z & 0x7fffffffu;
#pragma unroll
  for (int t = 0; t < kMaxPatternBits; ++t) {
    const uint32_t b = (r.x >> (8 * t)) & 255u;
    if (b == 255u) break;
    base += ((ka >> (b & 31u)) & 1u) << (b >> 5);
  }
  h.sc.base = base | (uint32_t(parity32(ka & r.w)) << 31);
  if (r.y >> 31) {
    // alpha-hop x beta-hop group: the two coefficients, for a source holding the
    // lower or the higher beta hop qubit, with every sign not carried by the
    // staged row or the list entry folded in
    h.mode = 3;
    const uint32_t o0 = 1u << ((r.y >> 5) & 7u), o1 = 1u << ((r.y >> 13) & 7u);
    const int sa = int(h.sc.base >> 31);
    h.v0 = sflip(__ldg(vals + base + o0), sa ^ int((r.y >> 29) & 1u));
    h.v1 = sflip(__ldg(vals + base + o1), sa ^ int((r.y >> 30) & 1u));
    return h;
  }
  if (((r.y >> 16) & 255u) != 0u) {
    h.mode = 2;
    return h;
  }
  h.mode = 1;
  const uint32_t q0 = r.y & 255u, q1 = (r.y >> 8) & 255u;
  const uint32_t o0 = q0 ? (1u << (q0 >> 5)) : 0u, o1 = q1 ? (1u << (q1 >> 5)) : 0u;
  h.v0 = __ldg(vals + base);
  if (o0) h.v1 = __ldg(vals + base + o0);
  if (o1) h.v2 = __ldg(vals + base + o1);
  if (o0 && o1) h.v3 = __ldg(vals + base + o0 + o1);
  return h;
}

template <int U>
__device__ __forceinline__ void str_groups_hot(const StrPlan& sp, int g0, int g1, int w_lo, int w_hi, uint32_t ka,
                                               const GroupRec* __restrict__ groups,
                                               const uint32_t* __restrict__ emask, const double* __restrict__ vals,
                                               const uint32_t* kb_s, const double* psi_s, double* lam_s, int lane,
                                               uint32_t ob) {
  typedef Amp<true> A;
  if (g0 >= g1) return;
  constexpr int S = kStrWarps + 1;
  HotCoef h = hot_prep(__ldg(sp.bgx + g0), ka, vals);
  int e0 = __ldg(sp.bsplit + int64_t(g0) * S + w_lo);
  int e1 = __ldg(sp.bsplit + int64_t(g0) * S + w_hi);
  uint4 rn = g0 + 1 < g1 ? __ldg(sp.bgx + g0 + 1) : make_uint4(0u, 0u, 0u, 0u);
  for (int gi = g0; gi < g1; ++gi) {
    const uint4 rnn = gi + 2 < g1 ? __ldg(sp.bgx + gi + 2) : rn;
    int e0n = 0, e1n = 0;
    HotCoef hn = h;
    if (gi + 1 < g1) {
      e0n = __ldg(sp.bsplit + int64_t(gi + 1) * S + w_lo);
      e1n = __ldg(sp.bsplit + int64_t(gi + 1) * S + w_hi);
      hn = hot_prep(rn, ka, vals);
    }
    // walks this warp's list entries; cf(entry, beta string) gives the coefficient
    // for the staged row (which carries (-1)^{|Jb & ob|})
    auto walk = [&](auto&& cf) {
      for (int e = e0 + lane; e < e1; e += U * 32) {
        uint32_t ent[U];
#pragma unroll
        for (int u = 0; u < U; ++u) ent[u] = (e + 32 * u < e1) ? __ldg(sp.lists + e + 32 * u) : 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (ent[u] == 0xFFFFFFFFu) break;
          const uint32_t ib = ent[u] & 0x1FFFu, jb = (ent[u] >> 16) & 0x1FFFu;
          A::mac(lam_s[ib], cf(ent[u], jb), psi_s[jb]);
        }
      }
    };
    if (h.mode == 3) {
      // no beta string needed: the entry's bit 13 picks the coefficient, bit 14 its sign
      walk([&](uint32_t en, uint32_t) { return sflip((en >> 13) & 1u ? h.v1 : h.v0, int((en >> 14) & 1u)); });
    } else if (h.mode == 1) {
      const uint32_t s0 = h.sc.qu & 31u, s1 = (h.sc.qu >> 8) & 31u;
      walk([&](uint32_t, uint32_t jb) {
        const uint32_t kbv = kb_s[jb];
        const uint32_t b0 = (kbv >> s0) & 1u, b1 = (kbv >> s1) & 1u;  // qubit 0 is alpha: a missing bit reads 0
        const double v = b1 ? (b0 ? h.v3 : h.v2) : (b0 ? h.v1 : h.v0);
        return sflip(v, int(h.sc.base >> 31) ^ parity32(kbv & h.sc.eb) ^ parity32(kbv & ob));
      });
    } else if (h.mode == 2) {
      walk([&](uint32_t, uint32_t jb) {
        const uint32_t kbv = kb_s[jb];
        return sflip(simple_value(h.sc, vals, kbv), parity32(kbv & ob));
      });
    } else {
      const GroupRec g = load_group(groups + __ldg(sp.bgrp + gi));
      walk([&](uint32_t, uint32_t jb) {
        const uint32_t kbv = kb_s[jb];
        return sflip(group_coef<true>(g, emask, vals, ka | kbv), parity32(kbv & ob));
      });
    }
    __syncwarp();
    h = hn;
    e0 = e0n;
    e1 = e1n;
    rn = rnn;
  }
}

// String-driven H psi (spin sectors; see StrPlan), block form for large beta
// string sets: lambda[Ia, :] for one output alpha string per block. For each
// bucket with a source alpha string Ja, the source row psi[Ja, :] is staged in
// shared memory; then every warp walks its share (a fixed Ib range) of each
// group's beta pair list. Needs blockDim.x == 32 * kStrWarps and 2 * Db
// amplitudes (+ Db words of beta strings when Db < kStrWideDb; above, they are
// read from global memory through L1) of shared memory. UW: list entries per lane
// in flight in the real wide form's pipelined group loop (16 for the standalone
// kernel; the persistent batch kernel, which has fewer registers to spare, uses 4).
template <bool REAL, bool WIDE, bool CG = false, int UW = 16>
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
          SimpleCoef sc;
          if (WIDE && simple_coef(g, emask, ka, sc)) {
            for (int j = tid; j < Db; j += bs) A::mac(lam_s[j], simple_value(sc, vals, kb_s[j]), ld_state<CG>(row + j));
          } else {
            for (int j = tid; j < Db; j += bs)
              A::mac(lam_s[j], group_coef<REAL>(g, emask, vals, ka | kb_s[j]), ld_state<CG>(row + j));
          }
          continue;
        }
      }
    }
    __syncthreads();       // the previous source row is no longer read
    // only the pipelined loop of the wide form uses a signed row (measured slower in the staged form)
    const uint32_t ob = (REAL && WIDE) ? __ldg(sp.bob + b) : 0u;  // the same for the whole block
    for (int j = tid; j < Db; j += bs) psi_s[j] = sflip(ld_state<CG>(row + j), parity32(kb_s[j] & ob));
    __syncthreads();
    // UW list entries per lane in flight in the pipelined loop: 16 measured best at
    // 30 qubits (H psi 4: 88.5 ms, 8: 86.3, 12: 87.5, 16: 85.3; the same bits)
    if constexpr (REAL && WIDE)
      str_groups_hot<UW>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), w, w + 1, __ldg(sp.ka + ja), groups, emask,
                        vals, kb_s, psi_s, lam_s, lane, ob);
    else
      str_groups<REAL, (WIDE && REAL) ? 8 : 4, WIDE>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), w, w + 1,
                                                     __ldg(sp.ka + ja), groups, emask, vals, kb_s, psi_s, lam_s, lane,
                                                     ob);
  }
  __syncthreads();
  T* out = lam_am + int64_t(ia) * Db;
  for (int j = tid; j < Db; j += bs) out[j] = lam_s[j];
}

// Warp form for small beta string sets: each warp owns one output alpha string
// (ia0 + warp), stages its own source rows and walks whole lists; the same
// per-output order as the block form, so the same bits. Shared memory: Db
// words of beta strings, then 2 * Db amplitudes per warp.
template <bool REAL, bool CG = false>
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
          SimpleCoef sc;
          if (simple_coef(g, emask, ka, sc)) {
            for (int j = lane; j < Db; j += 32) A::mac(lam_s[j], simple_value(sc, vals, kb_s[j]), ld_state<CG>(row + j));
          } else {
            for (int j = lane; j < Db; j += 32)
              A::mac(lam_s[j], group_coef<REAL>(g, emask, vals, ka | kb_s[j]), ld_state<CG>(row + j));
          }
          continue;
        }
      }
    }
    __syncwarp();
    const uint32_t ob = __ldg(sp.bob + b);  // the same for the whole warp
    for (int j = lane; j < Db; j += 32) psi_s[j] = sflip(ld_state<CG>(row + j), parity32(kb_s[j] & ob));
    __syncwarp();
    if constexpr (REAL)
      str_groups_hot<8>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), 0, kStrWarps, __ldg(sp.ka + ja), groups,
                        emask, vals, kb_s, psi_s, lam_s, lane, ob);
    else
      str_groups<REAL, 4>(sp, __ldg(sp.boff + b), __ldg(sp.boff + b + 1), 0, kStrWarps, __ldg(sp.ka + ja), groups,
                          emask, vals, kb_s, psi_s, lam_s, lane, ob);
  }
  __syncwarp();
  T* out = lam_am + int64_t(ia) * Db;
  for (int j = lane; j < Db; j += 32) out[j] = lam_s[j];
}

}  // namespace
}  // namespace vqe
