// Internal tables shared by the host side (vqe_host.cpp) and the CUDA kernels
// (vqe_kernels.cu) of libvqe. Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

struct vqe_hamiltonian_s;
struct vqe_ansatz_s;

namespace vqe {

constexpr int kMaxQubits = 32;
constexpr int kMaxPatternBits = 4;          // X bits folded into per-pattern tables
constexpr uint32_t kEllPad = 0xFFFFFFFFu;   // empty connectivity slot
constexpr int kResidentThreads = 512;
constexpr int kStreamThreads = 256;
constexpr int kMaxPartials = 1024;          // per-gate reduction partials (streaming)
constexpr int kPoolChunk = 4096;            // pairs per partial sum of the pool screening

// One X-mask group of the Hamiltonian. The group adds f(src) * psi[src] to
// lambda[src ^ x]; u is the pattern of src on the group's pattern qubits
// (bit j of u = bit upos_j of src). Three forms of f:
//  kind 0 (entry form):
//    f(src) = sum_{e=ebeg}^{eend-1} (-1)^{|src & emask[e]|} vals[vbeg + (e-ebeg)*2^ubits + u]
//  kind 1 (linear occupation form), emask[ebeg] = z0, emask[ebeg+1] = R:
//    f(src) = (-1)^{|src & z0|} (B[u] + sum_{r in src & R} B[(1+r)*2^ubits + u]),  B = vals + vbeg
//  kind 2 (quadratic occupation form, ubits = 0), same z0 and R, Q = vals + vbeg:
//    f(src) = (-1)^{|src & z0|} (Q[0] + sum_{p in src&R} Q[1+p] + sum_{p<q in src&R} Q[1+nq+p*nq+q])
struct GroupRec {
  uint32_t x;       // X mask of every term in the group
  uint32_t upos;    // up to 4 pattern-bit positions, 8 bits each
  int32_t ebeg;     // entry range in emask[]
  int32_t eend;
  int32_t vbeg;     // first value slot (in values, real or complex)
  int32_t ubits;    // number of pattern bits (0..4)
  int32_t kind;     // 0, 1 or 2 (above)
  int32_t nq;       // qubit count (row stride of the quadratic table)
};

// One excitation rotation. Its amplitude pairs are (k, k ^ flip) for k in the
// gate's pair list; T|k> = s|k ^ flip> with s = sign0 * (-1)^{|k & par|}.
struct GateRec {
  uint32_t flip;
  uint32_t par;
  int32_t sign0;    // +1 or -1
  int32_t pad;
};

// String-driven H psi of a spin sector: the sector is the product of alpha
// strings (even qubits) and beta strings (odd qubits), and psi is read as a
// Da x Db matrix in alpha-major order. Groups are bucketed by their alpha mask;
// a bucket maps output alpha string Ia to source alpha string ja[Ia * NB + b]
// (-1: none). Each group's beta mask selects a list of (output, source) beta
// string pairs (Ib | Jb << 16, 13 bits each, increasing Ib; for a beta mask of
// one hop {q_lo < q_hi}, bit 13 = the source holds q_hi, bit 14 = parity of the
// source's beta qubits strictly between q_lo and q_hi); bsplit gives, per bucket entry,
// the entry range of its list for each of the kStrWarps warps (a fixed share of
// the Ib range each).
constexpr int kStrWarps = 8;
constexpr int kStrMinDb = 512;    // smaller beta string sets: a warp per output alpha string
constexpr int kStrWideDb = 2048;  // larger ones: beta strings read through L1, four blocks per SM
struct StrPlan {
  int32_t Da, Db, NB, pad;
  const uint32_t* ka;      // [Da] alpha strings as qubit masks, increasing
  const uint32_t* kb;      // [Db] beta strings as qubit masks, increasing
  const int32_t* ja;       // [Da * NB]
  const int32_t* boff;     // [NB + 1] entry range of each bucket in bgrp
  const int32_t* bgrp;     // group index, bucket by bucket, by beta mask
  const int32_t* bsplit;   // [entries * (kStrWarps + 1)] absolute list offsets
  const uint32_t* lists;   // concatenated beta lists
  const uint32_t* perm;    // [Da * Db] alpha-major index -> position in the sorted sector
  // per bucket entry (bgrp order), the parts of a single-term group's coefficient
  // that need no source string: {qa, qb, vbeg | single << 31, em}; qa / qb: per
  // alpha / beta pattern bit t, byte t = qubit | (bit of u) << 5 (qa: 0xFF ends
  // the list; qb: 0 ends it, beta qubits are odd); em: the term's Z mask. For an
  // alpha-hop x beta-hop group whose sign splits as described at bob, qb bit 31
  // is set and bits 29 / 30 hold the remaining sign bit when the source holds
  // the lower / higher beta hop qubit.
  const uint4* bgx;
  // per bucket: for a single alpha hop {p < q}, the beta qubits strictly between
  // p and q (else 0); the staged source row is multiplied by (-1)^{|Jb & bob|}
  const uint32_t* bob;
};

struct InstDesc {
  // ansatz
  int32_t n, M;
  uint32_t hf;
  int32_t ellp_fast;         // 1: ellp entries with bit 31 set are single-slot entries (see below)
  int64_t D;                 // sector dimension
  const uint32_t* sector;    // [D] sorted basis indices of the sector
  const GateRec* gates;      // [M]
  const int64_t* pair_off;   // [M+1]
  const uint32_t* pairs;     // [pair_off[M]] lower index k of each pair
  const uint2* rpairs;       // [pair_off[M]] (rank(k) | sign << 31, rank(k ^ flip)); sign: (-1)-bit of T|k>
  // rank(k) = rank_hi[k >> lo_bits] + rank_lo[k & (2^lo_bits - 1)] is the position
  // of sector state k in sector[]; the streaming kernels store amplitudes there
  const uint32_t* rank_hi;
  const uint32_t* rank_lo;
  int32_t lo_bits, hf_rank;  // hf_rank = rank(hf)
  const StrPlan* str;        // device copy of the string plan, or null
  // resident kernel: [W][D] packed entries rank(src) | pattern(src) << 15 | group << 19
  // (D <= 32767, G <= 8191), pad 0xFFFFFFFF. With ellp_fast (G <= 4095), an entry
  // whose group has a single folded term (f = (-1)^s vals[slot], the double
  // excitations of Jordan-Wigner chemistry) is instead
  // rank(src) | s << 15 | slot << 16 | 1 << 31 (slot < 32768).
  const uint32_t* ellp;
  // resident kernel, same shape as ellp: each entry's coefficient f_g(src) in the
  // fixed-point scale of the staged tables (v * 2^(62 - eh), 2^eh bounding hbound),
  // summed exactly as group_coef_int does; null when not built
  const long long* hmat;
  const double* hbound;      // device: sum of |vals| (bounds every row sum of |H|)
  // Hamiltonian
  int32_t G, W;              // groups, connectivity slots per output
  const GroupRec* groups;    // [G]
  const uint32_t* emask;     // [entries]
  const double* vals;        // real tables (one double per slot)
  const double2* cvals;      // complex tables (one double2 per slot)
  const uint32_t* ell;       // [W][D] column-major: groups connected to each output (host-built)
  const uint16_t* ell16;     // same, 16-bit entries built on the device (pad 0xFFFF); used when set
  // row of this instance in the caller's theta / energy / gradient arrays
  int64_t inst;
  int32_t E, S;              // folded entries and value slots of the Hamiltonian
  int32_t stage_tables;      // resident kernel: copy the group tables to shared memory
  int32_t sweep_threads;     // resident kernel: threads that run the gate sweeps
  int32_t n_elec, n_alpha;   // sector (n_alpha < 0: electron number only)
};

// Persistent batched evaluation (vqe_batch.cu): a device work queue of tasks,
// each instance a chain of levels (see PTaskKind), run by one launch.
constexpr int kPersistThreads = 256;  // == kStrWarps * 32, the string-driven H psi's block
enum PTaskKind : int32_t {
  PT_INIT = 0, PT_FWD = 1, PT_GATHER = 2, PT_HPSI = 3, PT_SCATTER = 4, PT_DOT = 5, PT_ADJ = 6,
  PT_ADJS = 7  // adjoint step of a large gate: partials [lo, hi) of k_gate_adj's grid-strided layout
};
struct PTask {
  int32_t slot;   // persistent slot (instance) of the task
  int32_t kind;   // PTaskKind
  int32_t m;      // gate (FWD, ADJ)
  int32_t need;   // the slot's progress counter must reach this before the task runs
  int64_t lo, hi; // pairs of gate m (FWD, ADJ), alpha-major entries (GATHER, SCATTER), output alpha
                  // strings (HPSI, string form) or rows (HPSI, other sectors), 256-entry blocks (DOT)
  int64_t aux;    // ADJ: index of gate m's first partial among the slot's gradient partials
};
struct PSlot {    // byte offsets in the workspace
  int64_t psi, lam, psi_am, lam_am, cs, ep, gp;
};
struct PFinal {   // one output of the finalising launch
  int64_t off;    // byte offset of its partials in the workspace
  int32_t nb;     // partial count
  int32_t m;      // gate, or -1 for the energy
  int64_t inst;   // row in the caller's arrays
  double scale;   // 2 for gradients, 1 for energies
};
struct PersistDev {
  const InstDesc* desc;  // [n]
  const PSlot* slots;    // [n]
  const PTask* tasks;    // [n_tasks], the queue order
  int32_t n_tasks, n;
  char* ws;
  int* counters;         // [n] progress, then the next-task counter, then the status word
  long long budget_ns;   // bound of every wait
  int32_t probe_task;    // >= 0: that task waits for a count nothing reaches (timeout check)
  int32_t pad;
};

// memset of the counters, the persistent launch (grid CTAs), and the finalising
// launch over rows[0, n_rows) (gradient rows first: n_grad_rows of them, skipped
// when grad is null).
cudaError_t batch_persistent_run(const PersistDev& p, int grid, size_t smem, const PFinal* rows, int n_rows,
                                 int n_grad_rows, const double* theta, int64_t ld_theta, double* energy, double* grad,
                                 int64_t ld_grad, cudaStream_t stream);
cudaError_t set_persist_smem_limit(size_t smem);
cudaError_t persist_occupancy(size_t smem, int* blocks_per_sm);
// memset of the counters and the persistent launch alone (the gate sweeps of a
// large single instance; no dynamic shared memory, no finalising launch)
cudaError_t persistent_sweep_run(const PersistDev& p, int grid, const double* theta, cudaStream_t stream);

// Persistent gate sweeps of one large instance (stream_energy_grad with real
// amplitudes): queues of INIT + FWD tasks and of ADJS tasks for an ansatz, with
// device copies of its descriptor (ansatz fields only) and workspace offsets.
struct SweepPlan {
  InstDesc* d_desc = nullptr;
  PSlot* d_slot = nullptr;
  PTask* d_fwd = nullptr;
  PTask* d_adj = nullptr;
  int32_t n_fwd = 0, n_adj = 0, grid = 0;
};
cudaError_t set_str_smem_limit(size_t smem);

// Shared-memory layout of the resident kernel (byte offsets), computed the same
// way on the host (to size the launch) and on the device (to carve it). The
// state is compressed to the sector (D entries): real amplitudes as D double2
// {psi, lambda}, complex ones as psi[D] and lambda[D].
struct ResidentLayout {
  uint32_t psi, lam, cs, gates, poff, pairs, rank, gbuf, tab, red, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// String-driven H psi: shared memory and blocks of its two forms (a block per
// output alpha string when Db >= kStrMinDb, else a warp per output alpha string).
// The block form stages the beta strings next to the two rows unless
// Db >= kStrWideDb, where leaving them in L1 lets four blocks share an SM.
__host__ __device__ inline size_t str_smem_bytes(int Db, size_t amp) {
  if (Db >= kStrWideDb) return size_t(Db) * 2 * amp;
  return Db >= kStrMinDb ? size_t(Db) * (2 * amp + 4)
                         : align_up(uint32_t(Db) * 4u, 16u) + size_t(kStrWarps) * 2 * size_t(Db) * amp;
}
__host__ __device__ inline int str_blocks(int Da, int Db) {
  return Db >= kStrMinDb ? Da : (Da + kStrWarps - 1) / kStrWarps;
}

// Staged H psi tables: groups, then entry masks, then values.
__host__ __device__ inline uint32_t staged_table_bytes(int G, int E, int S, bool real) {
  return uint32_t(G) * 32u + align_up(uint32_t(E) * 4u, 16u) + uint32_t(S) * (real ? 8u : 16u);
}

__host__ __device__ inline ResidentLayout resident_layout(int n, int M, int P, int G, int E, int S, int D, int lo_bits,
                                                          bool real, bool stage) {
  ResidentLayout L;
  L.psi = 0;
  L.lam = real ? 0u : uint32_t(D) * 16u;
  // real amplitudes: {psi, lambda} rows plus one scratch row (index D) that the
  // sweep lanes past a gate's end read and write
  uint32_t o = real ? (uint32_t(D) + 1u) * 16u : 2u * uint32_t(D) * 16u;
  L.cs = align_up(o, 16u);
  o = L.cs + uint32_t(M) * 16u;
  L.gates = align_up(o, 16u);
  o = L.gates + uint32_t(M) * 16u;
  L.poff = o;
  o += uint32_t(M + 1) * 4u;
  L.pairs = align_up(o, 16u);  // ra | sign << 15 | rb << 16 per pair
  o = L.pairs + uint32_t(P) * 4u;
  L.rank = align_up(o, 16u);   // (no rank tables: the packed entries carry source ranks)
  o = L.rank;
  // per-pair slots: with real amplitudes two per pair (one per lane of the pair),
  // holding the forward sweep's output and later the gradient contribution; with
  // complex amplitudes one gradient contribution per pair
  L.gbuf = align_up(o, 16u);
  o = L.gbuf + (real ? (uint32_t(P) + 1u) * 16u : uint32_t(P) * 8u);  // real: two scratch slots at 2P
  L.tab = align_up(o, 16u);
  o = L.tab + (stage ? staged_table_bytes(G, E, S, real) : 0u);
  L.red = align_up(o, 16u);
  L.total = L.red + 64u * 8u;
  return L;
}

// Kernel launchers (vqe_kernels.cu). All are asynchronous on `stream`.
// ctas_per_instance: 1, or 2 (a cluster per instance; real amplitudes only).
// fixed_point: real sweeps in 64-bit fixed point on the integer pipe (real only).
cudaError_t launch_resident(const InstDesc* d_descs, const InstDesc* one, int n_inst,
                            size_t smem, bool real, bool with_grad, const double* theta,
                            int64_t ld_theta, double* energy, double* grad, int64_t ld_grad,
                            cudaStream_t stream, int ctas_per_instance, bool fixed_point);
cudaError_t set_resident_smem_limit(size_t smem, bool real);

struct StreamBuffers {
  void* psi = nullptr;     // D amplitudes (double or double2), sector order
  void* lam = nullptr;     // D amplitudes
  void* psi_am = nullptr;  // D amplitudes, alpha-major (string-driven H psi)
  void* lam_am = nullptr;  // D amplitudes, alpha-major
  // large real instances: the forward sweep's outputs {phi(k), phi(k ^ flip)} of
  // every pair, in pair order (null: the reverse sweep un-applies the gates to psi)
  double2* phi = nullptr;
  double2* cs;    // [M] (cos, sin)
  double* epart;  // [kMaxPartials]
  double* gpart;  // [M * kMaxPartials]
};

// Host-side facts the streaming launchers need besides the device descriptor.
struct StreamPlan {
  const SweepPlan* sweep = nullptr;  // persistent gate sweeps (null: one launch per gate)
  int64_t counters_off = 0;          // byte offset of the sweep queue's counters in the workspace
  const int64_t* pair_off_host;  // [M+1]
  const int32_t* d_nb_rows;      // device [M+1]: blocks of each gate's adjoint launch, then of H psi
  int n_elec, n_alpha;           // sector test (n_alpha < 0: number sector only)
  bool use_ell;
  bool use_str;                  // string-driven H psi with `str`
  StrPlan str;
};

// Blocks of a streaming launch over `work` items (also the partial count).
inline int stream_grid(int64_t work) {
  int64_t b = (work + kStreamThreads - 1) / kStreamThreads;
  if (b < 1) b = 1;
  if (b > kMaxPartials) b = kMaxPartials;
  return int(b);
}

cudaError_t stream_energy_grad(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                               bool real, bool with_grad, const double* theta, double* energy,
                               double* grad, cudaStream_t stream);
cudaError_t stream_state(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                         const double* theta, double* psi_out, cudaStream_t stream);
cudaError_t stream_apply_h(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                           const double* psi_in, double* lam_out, double* energy,
                           cudaStream_t stream);
// lambda = H psi with real amplitudes compressed to the sector (b.psi in, b.lam out).
// Real amplitudes, b.phi set: energy and gradient with the forward outputs kept
// (vqe_phi.cu); psi, lambda and the energy are those of stream_energy_grad.
cudaError_t stream_energy_grad_kept(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b,
                                    const double* theta, double* energy, double* grad, cudaStream_t stream);
cudaError_t stream_apply_h_real(const InstDesc& d, const StreamPlan& sp, const StreamBuffers& b, double* energy,
                                cudaStream_t stream);

// The fixed-point coefficient of every packed connectivity entry (InstDesc::hmat):
// ivals (S int64) receives the scaled table values first. Asynchronous on stream,
// after the values and hbound are final.
cudaError_t build_hmat(const uint32_t* ellp, int W, int64_t D, const uint32_t* sector, const GroupRec* groups,
                       const uint32_t* emask, const double* vals, int64_t S, const double* hbound, int fast,
                       long long* ivals, long long* hmat, cudaStream_t stream);

// Device-built connectivity table (16-bit group indices) for large sectors:
// len[r] = groups connected to output r; then rows filled in `order`.
cudaError_t ell_device_count(const uint32_t* sector, int64_t D, const GroupRec* groups, int G,
                             const int32_t* order, int n_elec, int n_alpha, int32_t* len, int32_t* wmax,
                             cudaStream_t stream);
cudaError_t ell_device_fill(const uint32_t* sector, int64_t D, const GroupRec* groups, int G,
                            const int32_t* order, int n_elec, int n_alpha, int W, uint16_t* ell,
                            cudaStream_t stream);

// ADAPT pool screening (vqe_pool.cu): grad[m] = 2 Re <lam| T_m - T_m^dagger |psi>
// over the M operators of a pool handle; chunk_off[m] = sum over operators
// before m of ceil(pairs / kPoolChunk); part holds n_chunks = chunk_off[M] doubles;
// pl (16-byte aligned) receives psi and lam side by side, D * 2 amplitudes.
cudaError_t pool_gradients(const uint2* rpairs, const int64_t* pair_off, const int64_t* chunk_off, int M,
                           int64_t n_chunks, bool real, const void* psi, const void* lam, int64_t D, void* pl,
                           double* part, double* grad, cudaStream_t stream);

// Host helpers for the allocation-free entry point (vqe_static.cu).
// off: psi, lambda, alpha-major psi, alpha-major lambda (0 when unused), cos/sin,
// energy partials, gradient partials; *need: total bytes.
// The string-driven H psi is used only if its scratch fits in `limit` bytes.
int prepare_noalloc(vqe_hamiltonian_s* h, vqe_ansatz_s* a, bool with_grad, size_t limit, InstDesc* d,
                    StreamPlan* sp, bool* real, size_t off[7], size_t* need);
int set_error(int code, const char* msg);

// Table refold from new coefficients (vqe_aux.cu): slot s of the value tables is
// sum_{j in [off[s], off[s+1])} w[j] * coefs[term[j] & 0x7fffffff], added to the
// imaginary part when term[j] < 0.
cudaError_t fold_coefs(int64_t n_slots, const int64_t* off, const int32_t* term, const float* w,
                       const double* coefs, double* vals, double2* cvals, cudaStream_t stream);
// *out = sum |v[i]| (deterministic)
cudaError_t abs_sum(const double* v, int64_t n, double* out, cudaStream_t stream);

// Up to kRowPtrs device rows per launch, passed by value: row r (global index
// base + r) has len[r] doubles at p[r].
constexpr int kRowPtrs = 64;
struct RowPtrs {
  const double* p[kRowPtrs];
  int32_t len[kRowPtrs];
  int32_t base, count;
};
// dst[(base + r) * ld + k] = p[r][k]  /  p[r][k] = src[(base + r) * ld + k], k < len[r].
cudaError_t pack_rows(const RowPtrs& rp, double* dst, int64_t ld, int max_len, cudaStream_t stream);
cudaError_t unpack_rows(const RowPtrs& rp, const double* src, int64_t ld, int max_len, cudaStream_t stream);

}  // namespace vqe
