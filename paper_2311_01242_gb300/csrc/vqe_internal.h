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

// One X-mask group of the Hamiltonian. For a source index `src` whose bits on
// the group's pattern qubits form the pattern u (bit j of u = bit upos_j of
// src), the group's coefficient is
//   f(src) = sum_{e=ebeg}^{eend-1} (-1)^{|src & emask[e]|} vals[vbeg + (e-ebeg)*2^ubits + u]
// and the group adds f(src) * psi[src] to lambda[src ^ x].
struct GroupRec {
  uint32_t x;       // X mask of every term in the group
  uint32_t upos;    // up to 4 pattern-bit positions, 8 bits each
  int32_t ebeg;     // entry range in emask[]
  int32_t eend;
  int32_t vbeg;     // first value slot (in values, real or complex)
  int32_t ubits;    // number of pattern bits (0..4)
  int32_t pad0, pad1;
};

// One excitation rotation. Its amplitude pairs are (k, k ^ flip) for k in the
// gate's pair list; T|k> = s|k ^ flip> with s = sign0 * (-1)^{|k & par|}.
struct GateRec {
  uint32_t flip;
  uint32_t par;
  int32_t sign0;    // +1 or -1
  int32_t pad;
};

struct InstDesc {
  // ansatz
  int32_t n, M;
  uint32_t hf;
  int32_t pad0;
  int64_t D;                 // sector dimension
  const uint32_t* sector;    // [D] sorted basis indices of the sector
  const GateRec* gates;      // [M]
  const int64_t* pair_off;   // [M+1]
  const uint32_t* pairs;     // [pair_off[M]] lower index k of each pair
  // Hamiltonian
  int32_t G, W;              // groups, connectivity slots per output
  const GroupRec* groups;    // [G]
  const uint32_t* emask;     // [entries]
  const double* vals;        // real tables (one double per slot)
  const double2* cvals;      // complex tables (one double2 per slot)
  const uint32_t* ell;       // [W][D] column-major: groups connected to each output
  // row of this instance in the caller's theta / energy / gradient arrays
  int64_t inst;
};

// Shared-memory bytes the resident kernel needs for an instance.
inline size_t resident_smem_bytes(int n, int M, int64_t total_pairs, bool real) {
  size_t amp = real ? 8 : 16;
  return 2 * (size_t(1) << n) * amp + size_t(total_pairs) * 8 + size_t(M) * 16 + 64 * 8;
}

// Kernel launchers (vqe_kernels.cu). All are asynchronous on `stream`.
cudaError_t launch_resident(const InstDesc* d_descs, const InstDesc* one, int n_inst,
                            size_t smem, bool real, bool with_grad, const double* theta,
                            int64_t ld_theta, double* energy, double* grad, int64_t ld_grad,
                            cudaStream_t stream);
cudaError_t set_resident_smem_limit(size_t smem, bool real);

struct StreamBuffers {
  void* psi;      // 2^n amplitudes (double or double2)
  void* lam;      // 2^n amplitudes
  double2* cs;    // [M] (cos, sin)
  double* epart;  // [kMaxPartials]
  double* gpart;  // [M * kMaxPartials]
};

// Host-side facts the streaming launchers need besides the device descriptor.
struct StreamPlan {
  const int64_t* pair_off_host;  // [M+1]
  const int32_t* d_nb_rows;      // device [M+1]: blocks of each gate's adjoint launch, then of H psi
  int n_elec, n_alpha;           // sector test (n_alpha < 0: number sector only)
  bool use_ell;
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

// Host helpers for the allocation-free entry point (vqe_static.cu).
int prepare_noalloc(vqe_hamiltonian_s* h, vqe_ansatz_s* a, bool with_grad, InstDesc* d, StreamPlan* sp,
                    bool* real, size_t off[5], size_t* need);
int set_error(int code, const char* msg);

}  // namespace vqe
