// Host side of libvqe: argument validation, the Jordan-Wigner mapping of Eq. 2,
// X-mask grouping and folding of the Pauli sum, excitation records, sector and
// pair lists, the connectivity table, workspace layout and kernel dispatch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/vqe.h"
#include "vqe_internal.h"

using vqe::GateRec;
using vqe::GroupRec;
using vqe::InstDesc;
using cplx = std::complex<double>;

namespace {

thread_local std::string g_err;
int g_flags = 0;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(VQE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline int pc32(uint32_t v) { return __builtin_popcount(v); }
inline int pc64(uint64_t v) { return __builtin_popcountll(v); }

template <typename T>
int upload(const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return VQE_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(out), v.size() * sizeof(T));
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(VQE_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return VQE_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Run f(lo, hi) over [0, n) on up to hardware_concurrency threads.
template <typename F>
void parallel_for(int64_t n, F f) {
  int nt = int(std::thread::hardware_concurrency());
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  if (n < 4096 || nt == 1) {
    f(int64_t(0), n);
    return;
  }
  std::vector<std::thread> ts;
  const int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    ts.emplace_back([=]() { f(lo, hi); });
  }
  for (auto& t : ts) t.join();
}

// Run f(i) for every i in [0, n) on up to hardware_concurrency threads, each
// thread taking the next unclaimed index (for items of uneven, large cost).
template <typename F>
void parallel_items(int64_t n, F f) {
  int nt = int(std::thread::hardware_concurrency());
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  if (n <= 1 || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> ts;
  for (int t = 0; t < nt && t < n; ++t)
    ts.emplace_back([&]() {
      for (int64_t i = next++; i < n; i = next++) f(i);
    });
  for (auto& t : ts) t.join();
}

// ------------------------------------------------------------------ Pauli algebra
// A Pauli string P(x, z) = i^{|x&z|} X^x Z^z. Product rule:
// P(x1,z1) P(x2,z2) = i^{|x1&z1| + |x2&z2| + 2|z1&x2| - |x&z|} P(x, z), x = x1^x2, z = z1^z2.
struct PTerm {
  uint64_t x, z;
  cplx c;
};

inline PTerm pmul(const PTerm& a, const PTerm& b) {
  const uint64_t x = a.x ^ b.x, z = a.z ^ b.z;
  int ph = pc64(a.x & a.z) + pc64(b.x & b.z) + 2 * pc64(a.z & b.x) - pc64(x & z);
  ph = ((ph % 4) + 4) % 4;
  static const cplx ipow[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
  return PTerm{x, z, a.c * b.c * ipow[ph]};
}

// Jordan-Wigner ladder operator of spin orbital p as two Pauli strings:
// a_p = (P(p, <p) + i P(p, <p|p)) / 2, a+_p = (P(p, <p) - i P(p, <p|p)) / 2.
inline void ladder(int p, bool dagger, PTerm out[2]) {
  const uint64_t bit = uint64_t(1) << p, below = bit - 1;
  out[0] = PTerm{bit, below, cplx(0.5, 0.0)};
  out[1] = PTerm{bit, below | bit, cplx(0.0, dagger ? -0.5 : 0.5)};
}

// Adds coef * (product of ladder ops, leftmost first) into acc.
void add_ladder_product(std::unordered_map<uint64_t, cplx>& acc, double coef, const int* orb,
                        const bool* dag, int nops) {
  PTerm f[4][2];
  for (int i = 0; i < nops; ++i) ladder(orb[i], dag[i], f[i]);
  for (int choice = 0; choice < (1 << nops); ++choice) {
    PTerm t{0, 0, cplx(coef, 0.0)};
    for (int i = 0; i < nops; ++i) t = pmul(t, f[i][(choice >> i) & 1]);
    if (t.c == cplx(0, 0)) continue;
    acc[(t.x << 32) | t.z] += t.c;
  }
}

}  // namespace

// ------------------------------------------------------------------ shared connectivity tables
// Hamiltonians with the same X-mask structure (a bond-stretch scan) have the
// same connectivity table for a sector; one device copy serves them all.
namespace {
struct SharedEll {
  uint32_t* d = nullptr;
  std::vector<uint32_t> host;
  int refs = 0;
};
std::mutex g_ell_mu;
std::multimap<uint64_t, SharedEll*> g_ell_reg;

// Handle serial numbers, never reused (keys of the cached batch plans).
std::atomic<uint64_t> g_serial{1};
uint64_t next_serial() { return g_serial.fetch_add(1); }

uint64_t fnv1a(const std::vector<uint32_t>& v) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  for (size_t i = 0; i < v.size() * 4; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h ^ v.size();
}

// Tables above this size are not shared (no host copy is kept for them).
constexpr size_t kShareEllBytes = size_t(16) << 20;
uint64_t g_ell_unique = 0;

int ell_acquire(const std::vector<uint32_t>& v, uint32_t** out) {
  std::lock_guard<std::mutex> lock(g_ell_mu);
  if (v.size() * 4 > kShareEllBytes) {
    SharedEll* e = new SharedEll;
    const int rc = upload(v, &e->d);
    if (rc) {
      delete e;
      return rc;
    }
    e->refs = 1;
    g_ell_reg.emplace(~uint64_t(0) - (g_ell_unique++), e);  // never matched by a hash lookup
    *out = e->d;
    return VQE_OK;
  }
  const uint64_t h = fnv1a(v);
  auto range = g_ell_reg.equal_range(h);
  for (auto it = range.first; it != range.second; ++it) {
    if (it->second->host == v) {
      ++it->second->refs;
      *out = it->second->d;
      return VQE_OK;
    }
  }
  SharedEll* e = new SharedEll;
  const int rc = upload(v, &e->d);
  if (rc) {
    delete e;
    return rc;
  }
  e->host = v;
  e->refs = 1;
  g_ell_reg.emplace(h, e);
  *out = e->d;
  return VQE_OK;
}

void ell_release(uint32_t* d) {
  if (!d) return;
  std::lock_guard<std::mutex> lock(g_ell_mu);
  for (auto it = g_ell_reg.begin(); it != g_ell_reg.end(); ++it) {
    if (it->second->d == d) {
      if (--it->second->refs == 0) {
        dfree(it->second->d);
        delete it->second;
        g_ell_reg.erase(it);
      }
      return;
    }
  }
}
// Device-built 16-bit tables, shared by Hamiltonians with the same group
// X masks (in connectivity order) and the same sector.
struct SharedEll16 {
  uint16_t* d = nullptr;
  int W = 0;
  std::vector<uint32_t> key;
  int refs = 0;
};
std::mutex g_ell16_mu;
std::vector<SharedEll16*> g_ell16_reg;

void ell16_release(uint16_t* d) {
  if (!d) return;
  std::lock_guard<std::mutex> lock(g_ell16_mu);
  for (size_t i = 0; i < g_ell16_reg.size(); ++i) {
    if (g_ell16_reg[i]->d == d) {
      if (--g_ell16_reg[i]->refs == 0) {
        dfree(g_ell16_reg[i]->d);
        delete g_ell16_reg[i];
        g_ell16_reg.erase(g_ell16_reg.begin() + long(i));
      }
      return;
    }
  }
}
}  // namespace

// ------------------------------------------------------------------ handles
struct vqe_hamiltonian_s {
  int n = 0;
  std::vector<uint64_t> x, z;
  std::vector<double> c;
  std::vector<GroupRec> groups;
  std::vector<uint32_t> emask;
  std::vector<cplx> cvals;
  int is_real = 1;
  uint64_t serial = 0;  // never reused: keys cached batch plans
  // value tables as a linear map of the kept terms' coefficients (vqe_set_coefs)
  std::vector<int64_t> lin_off;
  std::vector<int32_t> lin_term;
  std::vector<float> lin_w;
  int64_t* d_lin_off = nullptr;
  int32_t* d_lin_term = nullptr;
  float* d_lin_w = nullptr;
  double* d_bound = nullptr;  // sum of |vals| over all slots (device)
  GroupRec* d_groups = nullptr;
  uint32_t* d_emask = nullptr;
  double* d_vals = nullptr;
  double2* d_cvals = nullptr;
  struct Ell {
    int W = 0;
    bool use_ell = false;
    uint32_t* d_ell = nullptr;
    uint16_t* d_ell16 = nullptr;      // device-built 16-bit table (large sectors)
    uint32_t* d_ellp = nullptr;       // packed entries for the resident kernel (small sectors)
    bool ellp_fast = false;           // d_ellp holds single-slot entries (flag bit 31)
    long long* d_hmat = nullptr;      // fixed-point coefficient of each packed entry (this H's values)
    long long* d_ivals = nullptr;     // scratch of its builds: the value tables in fixed point (one
                                      // per sector, so builds on different streams never share it)
    uint32_t* d_hsec = nullptr;       // the sector's basis states, for rebuilding d_hmat
    int64_t hD = 0;
    int64_t nnz = 0;                  // connected (output, group) pairs
    double extra_adds = 0;            // sum over nnz of (entries - 1)
    // spin sectors: alpha/beta string tables of the string-driven H psi
    bool use_str = false;
    vqe::StrPlan str{};
    vqe::StrPlan* d_str = nullptr;     // device copy of str (batched kernels)
    std::vector<void*> str_alloc;      // device arrays behind str
  };
  std::mutex mu;
  std::map<std::tuple<int, int, int>, Ell> ells;
  ~vqe_hamiltonian_s() {
    dfree(d_groups);
    dfree(d_emask);
    dfree(d_vals);
    dfree(d_cvals);
    dfree(d_lin_off);
    dfree(d_lin_term);
    dfree(d_lin_w);
    dfree(d_bound);
    for (auto& kv : ells) {
      dfree(kv.second.d_hmat);
      dfree(kv.second.d_ivals);
      dfree(kv.second.d_hsec);
      ell_release(kv.second.d_ell);
      ell_release(kv.second.d_ellp);
      ell16_release(kv.second.d_ell16);
      for (void* p : kv.second.str_alloc) dfree(p);
    }
  }
};

struct vqe_ansatz_s {
  int n = 0, M = 0;
  uint64_t hf = 0;
  int n_elec = 0, n_alpha = -1;
  std::vector<int32_t> exc;
  std::vector<GateRec> gates;
  std::vector<int64_t> pair_off;
  std::vector<uint32_t> pairs;
  std::vector<uint32_t> sector;
  int lo_bits = 0;                    // rank(k) = rank_hi[k >> lo_bits] + rank_lo[k & (2^lo_bits - 1)]
  std::vector<uint32_t> rank_hi, rank_lo;
  std::vector<uint2> rpairs;          // (rank(k) | sign << 31, rank(k ^ flip)) per pair
  std::vector<int64_t> chunk_off;     // [M+1] pool screening: chunks of kPoolChunk pairs before gate m
  int64_t* d_chunk_off = nullptr;
  uint32_t* d_rank_hi = nullptr;
  uint32_t* d_rank_lo = nullptr;
  uint2* d_rpairs = nullptr;
  std::vector<int32_t> nb_rows;
  GateRec* d_gates = nullptr;
  int64_t* d_pair_off = nullptr;
  uint32_t* d_pairs = nullptr;
  uint32_t* d_sector = nullptr;
  int32_t* d_nb_rows = nullptr;
  uint64_t serial = 0;  // never reused: keys cached batch plans
  std::mutex sweep_mu;
  std::unique_ptr<vqe::SweepPlan> sweep;  // persistent gate sweeps, built on first streaming use
  std::tuple<int, int, int> key() const { return std::make_tuple(n, n_elec, n_alpha); }
  ~vqe_ansatz_s() {
    if (sweep) {
      dfree(sweep->d_desc);
      dfree(sweep->d_slot);
      dfree(sweep->d_fwd);
      dfree(sweep->d_adj);
    }
    dfree(d_gates);
    dfree(d_pair_off);
    dfree(d_chunk_off);
    dfree(d_pairs);
    dfree(d_sector);
    dfree(d_rank_hi);
    dfree(d_rank_lo);
    dfree(d_rpairs);
    dfree(d_nb_rows);
  }
};

// Persistent evaluation of the batch's instances that do not fit shared memory
// (real-amplitude path): per-slot workspace offsets and two task queues (with
// and without the gradient), built at batch creation and again when the
// tuning changes.
struct PersistQueue {
  std::vector<vqe::PTask> tasks;  // queue order
  std::vector<vqe::PFinal> finals;
  int n_grad_rows = 0;
  vqe::PTask* d_tasks = nullptr;
  vqe::PFinal* d_finals = nullptr;
  ~PersistQueue() {
    dfree(d_tasks);
    dfree(d_finals);
  }
};

struct StreamBatch {
  std::vector<int> slots;                 // batch index of each persistent slot
  std::vector<int> big;                   // batch indices evaluated one by one (too large for a slot)
  std::vector<InstDesc> descs;            // per slot
  std::vector<vqe::PSlot> pslots;
  InstDesc* d_desc = nullptr;
  vqe::PSlot* d_slots = nullptr;
  std::unique_ptr<PersistQueue> q[2];     // 0: energy only, 1: with gradient
  size_t counters_off = 0, persist_bytes = 0, big_bytes = 0;
  size_t smem = 0;
  int grid = 0;
  int ctas_per_sm = 0;                    // 0: as many as fit
  int gate_chunk = 1024;                  // pairs per FWD/ADJ task (multiple of 256)
  long long budget_ns = 2000000000ll;
  int probe_task = -1;
  int last_queue = 1;                     // queue of the last launch (for status messages)
  ~StreamBatch() {
    dfree(d_desc);
    dfree(d_slots);
  }
};

// vqe_batch_energy_grad_host replays its copies and launches from a CUDA graph
// once a call has been seen with the same host buffers, workspace, flags and
// tuning; one graph per batch (a new key replaces it).
struct HostGraph {
  const double* theta = nullptr;
  int64_t ld_theta = 0;
  double* energies = nullptr;
  double* grads = nullptr;
  int64_t ld_grad = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int flags = 0, device = -1;
  uint64_t tuning = 0;
  cudaGraphExec_t exec = nullptr;
  bool same(const HostGraph& o) const {
    return theta == o.theta && ld_theta == o.ld_theta && energies == o.energies && grads == o.grads &&
           ld_grad == o.ld_grad && ws == o.ws && ws_bytes == o.ws_bytes && flags == o.flags &&
           device == o.device && tuning == o.tuning;
  }
};

struct vqe_batch_s {
  int n_inst = 0;
  int32_t max_params = 0;
  StreamBatch sb;
  HostGraph hg;
  uint64_t tuning_version = 0;
  cudaStream_t capture_stream = nullptr;  // private stream the host-call graph is captured on
  std::mutex hg_mu;
  std::vector<vqe_hamiltonian_t> hams;
  std::vector<vqe_ansatz_t> ans;
  std::vector<InstDesc> descs;          // host copies, device pointers inside
  std::vector<InstDesc> res_descs[2];   // resident descriptors per mode, staging fields set
  std::vector<int> resident[2];         // instance indices per mode (0 real, 1 complex)
  std::vector<int> streaming[2];
  InstDesc* d_res[2] = {nullptr, nullptr};
  size_t res_smem[2] = {0, 0};
  ~vqe_batch_s() {
    if (hg.exec) cudaGraphExecDestroy(hg.exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    dfree(d_res[0]);
    dfree(d_res[1]);
  }
};

namespace {

// Builds (or shares) a 16-bit connectivity table on the device when it fits in
// 40% of the free device memory (at most 96 GB); leaves e unchanged otherwise.
int build_ell_device(vqe_hamiltonian_t h, vqe_ansatz_t a, const std::vector<int>& order,
                     vqe_hamiltonian_s::Ell* e) {
  const int G = int(h->groups.size());
  const int64_t D = int64_t(a->sector.size());
  std::vector<uint32_t> key;
  key.reserve(size_t(G) + 4);
  key.push_back(uint32_t(a->n));
  key.push_back(uint32_t(a->n_elec));
  key.push_back(uint32_t(a->n_alpha));
  key.push_back(uint32_t(D));
  for (int g : order) key.push_back(h->groups[g].x);
  {
    std::lock_guard<std::mutex> lock(g_ell16_mu);
    for (auto* s : g_ell16_reg)
      if (s->key == key) {
        ++s->refs;
        e->W = s->W;
        e->d_ell16 = s->d;
        e->use_ell = true;
        return VQE_OK;
      }
  }
  std::vector<int32_t> ord(order.begin(), order.end());
  int32_t *d_order = nullptr, *d_len = nullptr, *d_wmax = nullptr;
  int rc = upload(ord, &d_order);
  if (rc) return rc;
  cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(&d_len), size_t(D) * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(reinterpret_cast<void**>(&d_wmax), 4);
  if (ce == cudaSuccess)
    ce = vqe::ell_device_count(a->d_sector, D, h->d_groups, G, d_order, a->n_elec, a->n_alpha, d_len, d_wmax, 0);
  int32_t W = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(&W, d_wmax, 4, cudaMemcpyDeviceToHost);
  size_t free_b = 0, total_b = 0;
  if (ce == cudaSuccess) ce = cudaMemGetInfo(&free_b, &total_b);
  uint16_t* d_ell = nullptr;
  const double bytes = double(W) * double(D) * 2.0;
  if (ce == cudaSuccess && W > 0 && bytes <= std::min(0.4 * double(free_b), 96.0e9)) {
    ce = cudaMalloc(reinterpret_cast<void**>(&d_ell), size_t(W) * size_t(D) * 2);
    if (ce == cudaSuccess)
      ce = vqe::ell_device_fill(a->d_sector, D, h->d_groups, G, d_order, a->n_elec, a->n_alpha, W, d_ell, 0);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  }
  dfree(d_order);
  dfree(d_len);
  dfree(d_wmax);
  if (ce != cudaSuccess) {
    dfree(d_ell);
    return cuda_fail(ce, "device connectivity table");
  }
  if (d_ell) {
    SharedEll16* s = new SharedEll16;
    s->d = d_ell;
    s->W = W;
    s->key = std::move(key);
    s->refs = 1;
    {
      std::lock_guard<std::mutex> lock(g_ell16_mu);
      g_ell16_reg.push_back(s);
    }
    e->W = W;
    e->d_ell16 = d_ell;
    e->use_ell = true;
  }
  return VQE_OK;
}

// FP64 additions the kernels spend on one group's coefficient for a source index.
double fp64_adds(vqe_hamiltonian_t h, int g, uint32_t src) {
  const GroupRec& r = h->groups[g];
  if (r.kind == 0) return double(r.eend - r.ebeg - 1);
  const int k = pc32(src & h->emask[r.ebeg + 1]);
  return r.kind == 1 ? double(k) : double(k + k * (k - 1) / 2);
}

// String tables of a spin sector (the product of alpha strings on the even
// qubits and beta strings on the odd qubits) for the string-driven H psi:
//  - alpha and beta strings in increasing order, and the alpha-major order's
//    map to the sector's sorted order (perm);
//  - groups that can connect anything (even numbers of flipped alpha and beta
//    bits) in buckets of equal alpha mask, each bucket sorted by beta mask;
//  - for each output alpha string and bucket, the source alpha string (or -1);
//  - for each beta mask, the (output, source) beta string pairs in output
//    order, with the entry range of each warp's fixed share of outputs.
int build_strings(vqe_hamiltonian_t h, vqe_ansatz_t a, vqe_hamiltonian_s::Ell* e) {
  const int n = a->n, Na = a->n_alpha, Nb = a->n_elec - a->n_alpha;
  const uint32_t all = uint32_t((uint64_t(1) << n) - 1);
  const uint32_t even = all & 0x55555555u, odd = all & 0xAAAAAAAAu;
  auto subsets = [](uint32_t pool, int c) {
    std::vector<uint32_t> bits, out;
    for (int q = 0; q < 32; ++q)
      if ((pool >> q) & 1u) bits.push_back(q);
    const int m = int(bits.size());
    if (c < 0 || c > m) return out;
    // every c-subset of the pool, as masks, in increasing order
    std::vector<uint32_t> all_masks;
    for (uint64_t v = 0; v < (uint64_t(1) << m); ++v) {
      if (__builtin_popcountll(v) != c) continue;
      uint32_t w = 0;
      for (int j = 0; j < m; ++j)
        if ((v >> j) & 1) w |= 1u << bits[j];
      all_masks.push_back(w);
    }
    std::sort(all_masks.begin(), all_masks.end());
    return all_masks;
  };
  const std::vector<uint32_t> ka = subsets(even, Na), kb = subsets(odd, Nb);
  const int64_t Da = int64_t(ka.size()), Db = int64_t(kb.size());
  // shared memory of a block (complex amplitudes: the larger of the two)
  const size_t smem = vqe::str_smem_bytes(int(std::min<int64_t>(Db, 65535)), 16);
  if (Da * Db != int64_t(a->sector.size()) || Db > 8191 || smem > size_t(200) * 1024) return VQE_OK;  // not used
  {
    static std::mutex mu;
    static size_t set_to = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (smem > set_to) {
      const cudaError_t ce = vqe::set_str_smem_limit(smem);
      if (ce != cudaSuccess) return cuda_fail(ce, "string-driven H psi shared memory");
      set_to = smem;
    }
  }
  auto index_of = [](const std::vector<uint32_t>& v, uint32_t m) -> int32_t {
    auto it = std::lower_bound(v.begin(), v.end(), m);
    return (it != v.end() && *it == m) ? int32_t(it - v.begin()) : -1;
  };
  const uint32_t lo_mask = (1u << a->lo_bits) - 1u;
  auto rank = [&](uint32_t k) { return a->rank_hi[k >> a->lo_bits] + a->rank_lo[k & lo_mask]; };
  std::vector<uint32_t> perm(size_t(Da * Db));
  parallel_for(Da, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      for (int64_t j = 0; j < Db; ++j) perm[size_t(i * Db + j)] = rank(ka[size_t(i)] | kb[size_t(j)]);
  });
  // buckets of groups by alpha mask, each sorted by beta mask then index
  const int G = int(h->groups.size());
  std::vector<int> keep;
  for (int g = 0; g < G; ++g) {
    const uint32_t x = h->groups[g].x;
    if ((pc32(x & even) & 1) == 0 && (pc32(x & odd) & 1) == 0) keep.push_back(g);
  }
  std::stable_sort(keep.begin(), keep.end(), [&](int p, int q) {
    const uint32_t xp = h->groups[p].x, xq = h->groups[q].x;
    if ((xp & even) != (xq & even)) return (xp & even) < (xq & even);
    return (xp & odd) < (xq & odd);
  });
  std::vector<uint32_t> bxa;
  std::vector<int32_t> boff, bgrp, blist;
  std::vector<uint32_t> lxb;  // beta mask of each list
  for (size_t i = 0; i < keep.size(); ++i) {
    const uint32_t x = h->groups[keep[i]].x;
    if (bxa.empty() || bxa.back() != (x & even)) {
      bxa.push_back(x & even);
      boff.push_back(int32_t(i));
    }
    const uint32_t xb = x & odd;
    auto it = std::lower_bound(lxb.begin(), lxb.end(), xb);
    if (it == lxb.end() || *it != xb) lxb.insert(it, xb);
    bgrp.push_back(keep[i]);
  }
  boff.push_back(int32_t(keep.size()));
  for (size_t i = 0; i < keep.size(); ++i)
    blist.push_back(int32_t(std::lower_bound(lxb.begin(), lxb.end(), h->groups[keep[i]].x & odd) - lxb.begin()));
  const int NB = int(bxa.size()), NL = int(lxb.size());
  // source alpha string per (output alpha string, bucket)
  std::vector<int32_t> ja(size_t(Da) * size_t(std::max(NB, 1)), -1);
  parallel_for(Da, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      for (int b = 0; b < NB; ++b) {
        const uint32_t src = ka[size_t(i)] ^ bxa[size_t(b)];
        if (pc32(src) == Na) ja[size_t(i) * NB + b] = index_of(ka, src);
      }
  });
  // beta pair lists in output order, with each warp's share of outputs
  const int SW = vqe::kStrWarps;
  const int64_t share = (Db + SW - 1) / SW;
  // an entry is Ib | Jb << 16 (13 bits each); for a list whose beta mask is a
  // single hop {q_lo < q_hi}, bit 13 says the source string holds q_hi (else q_lo)
  // and bit 14 is the parity of the source's beta qubits strictly between them
  std::vector<std::vector<uint32_t>> lists(static_cast<size_t>(NL));
  parallel_for(NL, [&](int64_t lo, int64_t hi) {
    for (int64_t l = lo; l < hi; ++l) {
      const uint32_t xb = lxb[size_t(l)];
      const bool hop = pc32(xb) == 2;
      const int q_lo = hop ? __builtin_ctz(xb) : 0, q_hi = hop ? 31 - __builtin_clz(xb) : 0;
      const uint32_t between = hop ? (((1u << q_hi) - 1u) & ~((2u << q_lo) - 1u) & odd) : 0u;
      for (int64_t j = 0; j < Db; ++j) {
        const uint32_t src = kb[size_t(j)] ^ xb;
        if (pc32(src) != Nb) continue;
        uint32_t ent = uint32_t(j) | (uint32_t(index_of(kb, src)) << 16);
        if (hop) ent |= ((src >> q_hi) & 1u) << 13 | uint32_t(pc32(src & between) & 1) << 14;
        lists[size_t(l)].push_back(ent);
      }
    }
  });
  std::vector<uint32_t> flat;
  std::vector<int32_t> split(static_cast<size_t>(NL) * (SW + 1));
  for (int l = 0; l < NL; ++l) {
    const int64_t base = int64_t(flat.size());
    const auto& L = lists[size_t(l)];
    for (int w = 0; w <= SW; ++w) {
      const uint32_t first = uint32_t(std::min<int64_t>(Db, int64_t(w) * share));
      const int64_t pos = std::lower_bound(L.begin(), L.end(), first,
                                           [](uint32_t ent, uint32_t v) { return (ent & 0x1FFFu) < v; }) -
                          L.begin();
      split[size_t(l) * (SW + 1) + w] = int32_t(base + pos);
    }
    flat.insert(flat.end(), L.begin(), L.end());
  }
  if (flat.size() >= (size_t(1) << 31)) return VQE_OK;
  if (flat.empty()) flat.push_back(0);
  // each bucket entry's list range per warp
  std::vector<int32_t> bsplit(blist.size() * (SW + 1));
  for (size_t i = 0; i < blist.size(); ++i)
    for (int w = 0; w <= SW; ++w) bsplit[i * (SW + 1) + w] = split[size_t(blist[i]) * (SW + 1) + w];
  if (bgrp.empty()) {
    bgrp.push_back(0);
    bsplit.assign(SW + 1, 0);
  }
  // per bucket: for a single alpha hop {p < q}, the beta qubits strictly between
  // p and q; the bucket's staged source row is multiplied by (-1)^{|Jb & bob|}
  auto between_odd = [&](uint32_t x2) -> uint32_t {
    if (pc32(x2) != 2) return 0u;
    const int lo_q = __builtin_ctz(x2), hi_q = 31 - __builtin_clz(x2);
    return ((1u << hi_q) - 1u) & ~((2u << lo_q) - 1u) & odd;
  };
  std::vector<uint32_t> bob(size_t(std::max(NB, 1)), 0u);
  for (int b = 0; b < NB; ++b) bob[size_t(b)] = between_odd(bxa[size_t(b)]);
  std::vector<int32_t> bucket_of(bgrp.size(), 0);
  for (int b = 0; b < NB; ++b)
    for (int32_t i = boff[size_t(b)]; i < boff[size_t(b) + 1]; ++i) bucket_of[size_t(i)] = b;
  // compact per-entry records of single-term groups (no source string needed)
  std::vector<uint4> bgx(bgrp.size());
  for (size_t i = 0; i < bgrp.size(); ++i) {
    const GroupRec& g = h->groups[size_t(bgrp[i])];
    const bool single = g.kind == 0 && g.eend == g.ebeg + 1;
    uint32_t qa = 0xFFFFFFFFu, qb = 0u;
    int na = 0, nb = 0;
    for (int j = 0; j < g.ubits; ++j) {
      const uint32_t pos = (g.upos >> (8 * j)) & 31u;
      const uint32_t byte = pos | (uint32_t(j) << 5);
      if (pos & 1u) {
        qb |= byte << (8 * nb);
        ++nb;
      } else {
        qa = (qa & ~(0xFFu << (8 * na))) | (byte << (8 * na));
        ++na;
      }
    }
    // an alpha-hop x beta-hop single-term group whose beta sign is the bucket's
    // row sign times its list entries' sign, up to a term fixed by which hop
    // qubit the source holds: flag (bit 31 of qb) and those two terms (bits 29, 30)
    const uint32_t xb = g.x & odd;
    if (single && na == 2 && nb == 2 && pc32(g.x & even) == 2 && pc32(xb) == 2) {
      const uint32_t em = h->emask[size_t(g.ebeg)];
      const uint32_t rest = (em & odd) ^ bob[size_t(bucket_of[i])] ^ between_odd(xb);
      if ((rest & ~xb) == 0u) {
        const int q_lo = __builtin_ctz(xb), q_hi = 31 - __builtin_clz(xb);
        qb |= 0x80000000u | ((rest >> q_lo) & 1u) << 29 | ((rest >> q_hi) & 1u) << 30;
      }
    }
    bgx[i] = make_uint4(qa, qb, uint32_t(g.vbeg) | (single ? 0x80000000u : 0u), single ? h->emask[size_t(g.ebeg)] : 0u);
  }
  if (bgx.empty()) bgx.push_back(make_uint4(0xFFFFFFFFu, 0u, 0u, 0u));
  vqe::StrPlan& P = e->str;
  P.Da = int32_t(Da);
  P.Db = int32_t(Db);
  P.NB = NB;
  int rc;
  auto up = [&](auto& vec, auto** dst) -> int {
    int r = upload(vec, dst);
    if (r == VQE_OK) e->str_alloc.push_back(static_cast<void*>(*dst));
    return r;
  };
  uint32_t *d_ka, *d_kb, *d_lists, *d_perm;
  int32_t *d_ja, *d_boff, *d_bgrp, *d_bsplit;
  uint4* d_bgx;
  uint32_t* d_bob;
  std::vector<uint32_t> ka_v(ka), kb_v(kb);
  if ((rc = up(ka_v, &d_ka)) || (rc = up(kb_v, &d_kb)) || (rc = up(ja, &d_ja)) || (rc = up(boff, &d_boff)) ||
      (rc = up(bgrp, &d_bgrp)) || (rc = up(bsplit, &d_bsplit)) || (rc = up(flat, &d_lists)) ||
      (rc = up(perm, &d_perm)) || (rc = up(bgx, &d_bgx)) || (rc = up(bob, &d_bob)))
    return rc;
  P.bgx = d_bgx;
  P.bob = d_bob;
  P.ka = d_ka;
  P.kb = d_kb;
  P.ja = d_ja;
  P.boff = d_boff;
  P.bgrp = d_bgrp;
  P.bsplit = d_bsplit;
  P.lists = d_lists;
  P.perm = d_perm;
  std::vector<vqe::StrPlan> one(1, P);
  vqe::StrPlan* d_plan = nullptr;
  if ((rc = up(one, &d_plan))) return rc;
  e->d_str = d_plan;
  e->use_str = true;
  return VQE_OK;
}

const vqe_hamiltonian_s::Ell* get_ell(vqe_hamiltonian_t h, vqe_ansatz_t a, int* err) {
  *err = VQE_OK;
  std::lock_guard<std::mutex> lock(h->mu);
  auto it = h->ells.find(a->key());
  if (it != h->ells.end()) return &it->second;
  vqe_hamiltonian_s::Ell e;
  const int64_t D = int64_t(a->sector.size());
  const int G = int(h->groups.size());
  const int ne = a->n_elec, na = a->n_alpha;
  auto inside = [ne, na](uint32_t k) {
    return pc32(k) == ne && (na < 0 || pc32(k & 0x55555555u) == na);
  };
  // group order inside a row: by entry count, then pattern bits, then index, so
  // that lanes of a warp meet groups of the same shape at the same slot.
  std::vector<int> order(G);
  for (int g = 0; g < G; ++g) order[g] = g;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
    const int ep = h->groups[p].eend - h->groups[p].ebeg, eq = h->groups[q].eend - h->groups[q].ebeg;
    if (ep != eq) return ep < eq;
    return h->groups[p].ubits < h->groups[q].ubits;
  });
  // row lengths
  std::vector<int32_t> len(D, 0);
  const double cost = double(D) * double(G);
  if (na >= 0 && G > 0) {
    const int rc = build_strings(h, a, &e);
    if (rc != VQE_OK) {
      *err = rc;
      return nullptr;
    }
  }
  if (cost > 2.0e7 && G > 0 && G < 65535 && e.use_str) {
    // large spin sector: H psi runs string-driven; no connectivity table
  } else if (cost > 2.0e7 && G > 0 && G < 65535) {
    const int rc = build_ell_device(h, a, order, &e);
    if (rc != VQE_OK) {
      *err = rc;
      return nullptr;
    }
  } else if (cost <= 4.0e9 && G > 0) {
    parallel_for(D, [&](int64_t lo, int64_t hi) {
      for (int64_t r = lo; r < hi; ++r) {
        const uint32_t k = a->sector[r];
        int c = 0;
        for (int g = 0; g < G; ++g) c += inside(k ^ h->groups[g].x);
        len[r] = c;
      }
    });
    int W = 0;
    int64_t nnz = 0;
    for (int64_t r = 0; r < D; ++r) {
      W = std::max(W, int(len[r]));
      nnz += len[r];
    }
    e.nnz = nnz;
    const double bytes = double(W) * double(D) * 4.0;
    if (bytes <= 512.0e6) {
      std::vector<uint32_t> ell(size_t(W) * size_t(D), vqe::kEllPad);
      std::vector<double> extra(D, 0.0);
      parallel_for(D, [&](int64_t lo, int64_t hi) {
        for (int64_t r = lo; r < hi; ++r) {
          const uint32_t k = a->sector[r];
          int j = 0;
          double ex = 0;
          for (int oi = 0; oi < G; ++oi) {
            const int g = order[oi];
            if (inside(k ^ h->groups[g].x)) {
              ell[size_t(j) * size_t(D) + size_t(r)] = uint32_t(g);
              ex += fp64_adds(h, g, k ^ h->groups[g].x);
              ++j;
            }
          }
          extra[r] = ex;
        }
      });
      for (int64_t r = 0; r < D; ++r) e.extra_adds += extra[r];
      e.W = W;
      e.use_ell = true;
      int rc = W > 0 ? ell_acquire(ell, &e.d_ell) : VQE_OK;
      if (rc != VQE_OK) {
        *err = rc;
        return nullptr;
      }
      if (W > 0 && D <= 32767 && G <= 8191) {
        // packed entries for the resident kernel: source rank, source pattern,
        // group; with G <= 4095, single-term groups carry their signed table slot
        // instead (no group record or mask to read in the kernel)
        const uint32_t lo_mask = (1u << a->lo_bits) - 1u;
        const bool fast = G <= 4095;
        e.ellp_fast = fast;
        std::vector<uint32_t> packed(ell.size(), vqe::kEllPad);
        parallel_for(D, [&](int64_t lo, int64_t hi) {
          for (int64_t r = lo; r < hi; ++r) {
            const uint32_t k = a->sector[size_t(r)];
            for (int j = 0; j < W; ++j) {
              const uint32_t g = ell[size_t(j) * size_t(D) + size_t(r)];
              if (g == vqe::kEllPad) break;
              const GroupRec& gr = h->groups[g];
              const uint32_t src = k ^ gr.x;
              uint32_t u = 0;
              for (int b = 0; b < gr.ubits; ++b) u |= ((src >> ((gr.upos >> (8 * b)) & 31u)) & 1u) << b;
              const uint32_t rs = a->rank_hi[src >> a->lo_bits] + a->rank_lo[src & lo_mask];
              const uint32_t slot = uint32_t(gr.vbeg) + u;
              uint32_t v = rs | (u << 15) | (g << 19);
              if (fast && gr.kind == 0 && gr.eend == gr.ebeg + 1 && slot < 32768u)
                v = rs | (uint32_t(pc32(src & h->emask[gr.ebeg]) & 1) << 15) | (slot << 16) | 0x80000000u;
              packed[size_t(j) * size_t(D) + size_t(r)] = v;
            }
          }
        });
        if ((rc = ell_acquire(packed, &e.d_ellp)) != VQE_OK) {
          *err = rc;
          return nullptr;
        }
        // small sectors: each entry's fixed-point coefficient for the resident
        // kernel's H psi (rebuilt by vqe_set_coefs); without it the kernel
        // computes them from the staged tables, with the same bits
        const size_t mat_bytes = size_t(W) * size_t(D) * 8;
        const size_t S = h->cvals.size();
        if (D <= 8192 && mat_bytes <= (size_t(64) << 20) && S > 0) {
          cudaError_t ce = cudaSuccess;
          ce = cudaMalloc(&e.d_ivals, S * sizeof(long long));
          if (ce == cudaSuccess) ce = cudaMalloc(&e.d_hmat, mat_bytes);
          if (ce == cudaSuccess && upload(a->sector, &e.d_hsec) != VQE_OK) ce = cudaErrorMemoryAllocation;
          e.hD = D;
          if (ce == cudaSuccess)
            ce = vqe::build_hmat(e.d_ellp, W, D, e.d_hsec, h->d_groups, h->d_emask, h->d_vals, int64_t(S),
                                 h->d_bound, e.ellp_fast ? 1 : 0, e.d_ivals, e.d_hmat, 0);
          if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
          if (ce != cudaSuccess) {
            cudaGetLastError();
            dfree(e.d_hmat);
            dfree(e.d_hsec);
            dfree(e.d_ivals);
            e.d_hmat = nullptr;  // the table path serves instead
            e.d_hsec = nullptr;
            e.d_ivals = nullptr;
          }
        }
      }
    }
  }
  if (!e.use_ell || e.d_ell16) {
    // device-built table or scan mode: estimate the work from a sample of outputs
    e.nnz = 0;
    e.extra_adds = 0;
    const int64_t step = std::max<int64_t>(1, D / 4096);
    int64_t sampled = 0;
    double nnz = 0, ex = 0;
    for (int64_t r = 0; r < D; r += step) {
      const uint32_t k = a->sector[r];
      for (int g = 0; g < G; ++g)
        if (inside(k ^ h->groups[g].x)) {
          nnz += 1;
          ex += fp64_adds(h, g, k ^ h->groups[g].x);
        }
      ++sampled;
    }
    if (sampled > 0) {
      e.nnz = int64_t(nnz * double(D) / double(sampled));
      e.extra_adds = ex * double(D) / double(sampled);
    }
  }
  auto res = h->ells.emplace(a->key(), e);
  return &res.first->second;
}

InstDesc make_desc(vqe_hamiltonian_t h, vqe_ansatz_t a, const vqe_hamiltonian_s::Ell* e, int64_t inst) {
  InstDesc d;
  std::memset(&d, 0, sizeof(d));
  d.n = a->n;
  d.M = a->M;
  d.hf = uint32_t(a->hf);
  d.D = int64_t(a->sector.size());
  d.sector = a->d_sector;
  d.rpairs = a->d_rpairs;
  d.rank_hi = a->d_rank_hi;
  d.rank_lo = a->d_rank_lo;
  d.lo_bits = a->lo_bits;
  d.hf_rank = int32_t(a->rank_hi[a->hf >> a->lo_bits] + a->rank_lo[a->hf & ((1u << a->lo_bits) - 1u)]);
  d.str = e->use_str ? e->d_str : nullptr;
  d.ellp = e->d_ellp;
  d.ellp_fast = e->ellp_fast ? 1 : 0;
  d.hmat = e->d_hmat;
  d.hbound = h->d_bound;
  d.gates = a->d_gates;
  d.pair_off = a->d_pair_off;
  d.pairs = a->d_pairs;
  d.G = int(h->groups.size());
  d.W = e->use_ell ? e->W : 0;
  d.groups = h->d_groups;
  d.emask = h->d_emask;
  d.vals = h->d_vals;
  d.cvals = h->d_cvals;
  d.ell = e->d_ell;
  d.ell16 = e->d_ell16;
  d.inst = inst;
  d.E = int32_t(h->emask.size());
  d.S = int32_t(h->cvals.size());
  d.stage_tables = 0;
  d.sweep_threads = 128;
  d.n_elec = a->n_elec;
  d.n_alpha = a->n_alpha;
  return d;
}

bool use_real() { return (g_flags & VQE_FLAG_FORCE_COMPLEX) == 0; }
bool use_fixed(bool real) { return real && (g_flags & VQE_FLAG_FP64_SWEEPS) == 0; }

// Whether an instance fits the shared-memory-resident kernel in this mode; if
// so, sets the shared-memory bytes and the descriptor's staging/sweep fields.
bool resident_fit(vqe_ansatz_t a, const vqe_hamiltonian_s::Ell* e, bool real, InstDesc* d, size_t* smem) {
  if (g_flags & VQE_FLAG_FORCE_STREAMING) return false;
  if (!e->use_ell || !e->d_ell || !e->d_ellp || a->n > 16) return false;
  if (a->sector.size() > 32767) return false;  // 15-bit ranks in the staged pair list
  if (a->pairs.size() > (size_t(1) << 24) || d->S > (1 << 24) || d->G > (1 << 20)) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int P = int(a->pairs.size());
  for (int stage = 1; stage >= 0; --stage) {
    const vqe::ResidentLayout L = vqe::resident_layout(a->n, a->M, P, d->G, d->E, d->S, int(a->sector.size()),
                                                       a->lo_bits, real, stage != 0);
    if (L.total <= uint32_t(optin)) {
      d->stage_tables = stage;
      d->sweep_threads = 128;
      *smem = L.total;
      return true;
    }
  }
  return false;
}

struct WsLayout {
  size_t psi, lam, psi_am, lam_am, cs, epart, ctr, gpart, phi, total;
};

// Real sectors from this size keep the forward sweep's pair outputs for the
// reverse sweep: psi and lambda (16 bytes per state together) no longer share
// the L2, and the reverse step's gathers of both would miss it.
constexpr size_t kKeepPhiMinStates = 6000000;

WsLayout ws_layout(vqe_ansatz_t a, bool complex_amp, bool with_grad) {
  WsLayout L;
  const size_t amp = complex_amp ? 16 : 8;
  const size_t vec = align256(std::max<size_t>(a->sector.size(), 1) * amp);  // compressed to the sector
  L.psi = 0;
  L.lam = vec;
  L.psi_am = 2 * vec;  // alpha-major copies for the string-driven H psi
  L.lam_am = 3 * vec;
  L.cs = 4 * vec;
  L.epart = L.cs + align256(size_t(std::max(a->M, 1)) * 16);
  L.ctr = L.epart + align256(size_t(vqe::kMaxPartials) * 8);  // task counters of the persistent sweeps
  L.gpart = L.ctr + 256;
  L.phi = L.gpart + (with_grad ? align256(size_t(std::max(a->M, 1)) * vqe::kMaxPartials * 8) : 0);
  const bool keep = !complex_amp && with_grad && a->sector.size() >= kKeepPhiMinStates;
  L.total = L.phi + (keep ? align256(size_t(a->pair_off.empty() ? 0 : a->pair_off.back()) * 16) : 0);
  if (!keep) L.phi = 0;
  return L;
}

vqe::StreamBuffers buffers(void* ws, const WsLayout& L) {
  char* b = static_cast<char*>(ws);
  vqe::StreamBuffers s;
  s.psi = b + L.psi;
  s.lam = b + L.lam;
  s.psi_am = b + L.psi_am;
  s.lam_am = b + L.lam_am;
  s.cs = reinterpret_cast<double2*>(b + L.cs);
  s.epart = reinterpret_cast<double*>(b + L.epart);
  s.gpart = reinterpret_cast<double*>(b + L.gpart);
  s.phi = L.phi ? reinterpret_cast<double2*>(b + L.phi) : nullptr;
  return s;
}

// Task queues of the persistent gate sweeps of ansatz a (real amplitudes; used
// under VQE_FLAG_PERSISTENT_SWEEPS): the forward queue holds the HF init and
// each gate's rotation in 2,048-pair tasks, the adjoint queue each gate's
// adjoint step in tasks of four partial sums laid out as k_gate_adj's blocks
// (so the gradient has the same bits as with one launch per gate). Built once
// per ansatz, on its first use; null if the device refuses (the caller then
// launches per gate).
const vqe::SweepPlan* get_sweep(vqe_ansatz_t a) {
  std::lock_guard<std::mutex> lk(a->sweep_mu);
  if (a->sweep) return a->sweep->grid > 0 ? a->sweep.get() : nullptr;
  std::unique_ptr<vqe::SweepPlan> sp(new vqe::SweepPlan);
  InstDesc d;
  std::memset(&d, 0, sizeof(d));
  d.n = a->n;
  d.M = a->M;
  d.hf = uint32_t(a->hf);
  d.D = int64_t(a->sector.size());
  d.sector = a->d_sector;
  d.gates = a->d_gates;
  d.pair_off = a->d_pair_off;
  d.pairs = a->d_pairs;
  d.rpairs = a->d_rpairs;
  d.rank_hi = a->d_rank_hi;
  d.rank_lo = a->d_rank_lo;
  d.lo_bits = a->lo_bits;
  d.n_elec = a->n_elec;
  d.n_alpha = a->n_alpha;
  const WsLayout L = ws_layout(a, false, true);
  const vqe::PSlot ps{int64_t(L.psi), int64_t(L.lam), -1, -1, int64_t(L.cs), int64_t(L.epart), int64_t(L.gpart)};
  std::vector<vqe::PTask> fwd, adj;
  auto task = [](std::vector<vqe::PTask>& q, int kind, int m, int need, int64_t lo, int64_t hi, int64_t aux) {
    vqe::PTask t;
    t.slot = 0;
    t.kind = kind;
    t.m = m;
    t.need = need;
    t.lo = lo;
    t.hi = hi;
    t.aux = aux;
    q.push_back(t);
  };
  task(fwd, vqe::PT_INIT, 0, 0, 0, d.D, 0);
  const int64_t gc = 2048;
  for (int m = 0; m < a->M; ++m) {
    const int need = int(fwd.size());
    const int64_t P = a->pair_off[m + 1] - a->pair_off[m];
    for (int64_t lo = 0; lo < P; lo += gc) task(fwd, vqe::PT_FWD, m, need, lo, std::min(P, lo + gc), 0);
  }
  for (int m = a->M - 1; m >= 0; --m) {
    const int need = int(adj.size());
    const int nb = vqe::stream_grid(a->pair_off[m + 1] - a->pair_off[m]);
    for (int b0 = 0; b0 < nb; b0 += 4)
      task(adj, vqe::PT_ADJS, m, need, b0, std::min(nb, b0 + 4), int64_t(m) * vqe::kMaxPartials);
  }
  int dev = 0, sms = 0, per_sm = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            vqe::persist_occupancy(0, &per_sm) == cudaSuccess && per_sm > 0 &&
            fwd.size() < size_t(INT32_MAX / 2) && adj.size() < size_t(INT32_MAX / 2);
  std::vector<InstDesc> dv(1, d);
  std::vector<vqe::PSlot> sv(1, ps);
  ok = ok && upload(dv, &sp->d_desc) == VQE_OK && upload(sv, &sp->d_slot) == VQE_OK &&
       upload(fwd, &sp->d_fwd) == VQE_OK && (adj.empty() || upload(adj, &sp->d_adj) == VQE_OK);
  cudaGetLastError();
  sp->n_fwd = int32_t(fwd.size());
  sp->n_adj = int32_t(adj.size());
  sp->grid = ok ? sms * per_sm : 0;
  a->sweep = std::move(sp);
  return ok ? a->sweep.get() : nullptr;
}

vqe::StreamPlan plan(vqe_ansatz_t a, const vqe_hamiltonian_s::Ell* e) {
  vqe::StreamPlan p;
  if (use_real() && (g_flags & VQE_FLAG_PERSISTENT_SWEEPS)) {
    p.sweep = get_sweep(a);
    p.counters_off = int64_t(ws_layout(a, false, false).ctr);
  }
  p.pair_off_host = a->pair_off.data();
  p.d_nb_rows = a->d_nb_rows;
  p.n_elec = a->n_elec;
  p.n_alpha = a->n_alpha;
  p.use_ell = e->use_ell;
  p.use_str = e->use_str && !(g_flags & VQE_FLAG_NO_STRINGS);
  p.str = e->str;
  return p;
}

int check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return VQE_OK;
  if (ws == nullptr) return fail(VQE_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(VQE_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (have < need)
    return fail(VQE_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes, got " +
                                       std::to_string(have));
  return VQE_OK;
}

int check_pair(vqe_hamiltonian_t h, vqe_ansatz_t a) {
  if (!h || !a) return fail(VQE_ERR_INVALID_ARG, "NULL handle");
  if (h->n != a->n) return fail(VQE_ERR_INVALID_ARG, "Hamiltonian and ansatz qubit counts differ");
  return VQE_OK;
}

// dynamic shared memory opt-in, cached per device and mode
int ensure_smem(size_t smem, bool real) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, real ? 1 : 0);
  auto it = done.find(key);
  if (it != done.end() && it->second >= smem) return VQE_OK;
  e = vqe::set_resident_smem_limit(smem, real);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  done[key] = smem;
  return VQE_OK;
}

// Two CTAs (a cluster) per resident instance when amplitudes are real and every
// instance's pair of CTAs fits on the device at once; one otherwise.
int ctas_per_instance(bool real, int n_inst) {
  if (!real || (g_flags & VQE_FLAG_NO_CLUSTER)) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return 2 * n_inst <= sms ? 2 : 1;
}

// One streamed instance: with its forward outputs kept when the workspace layout
// has room for them (large real sectors) and no flag asks for the un-applying
// reverse sweep, else the plain streaming path.
cudaError_t stream_eval(const InstDesc& d, const vqe::StreamPlan& sp, const vqe::StreamBuffers& b, bool real,
                        bool with_grad, const double* theta, double* energy, double* grad, cudaStream_t stream) {
  if (real && with_grad && b.phi && !sp.sweep && !(g_flags & VQE_FLAG_NO_PHI_STORE))
    return vqe::stream_energy_grad_kept(d, sp, b, theta, energy, grad, stream);
  return vqe::stream_energy_grad(d, sp, b, real, with_grad, theta, energy, grad, stream);
}

int run_single(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta, double* energy, double* grad,
               void* ws, size_t ws_bytes, cudaStream_t stream, bool with_grad) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  if ((!theta && a->M > 0) || !energy || (with_grad && !grad && a->M > 0))
    return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const bool real = use_real();
  InstDesc d = make_desc(h, a, e, 0);
  size_t smem = 0;
  if (resident_fit(a, e, real, &d, &smem)) {
    if ((rc = ensure_smem(smem, real))) return rc;
    cudaError_t ce = vqe::launch_resident(nullptr, &d, 1, smem, real, with_grad, theta, 0, energy, grad, 0,
                                          stream, ctas_per_instance(real, 1), use_fixed(real));
    if (ce != cudaSuccess) return cuda_fail(ce, "resident kernel launch");
    return VQE_OK;
  }
  const WsLayout L = ws_layout(a, !real, with_grad);
  if ((rc = check_ws(ws, ws_bytes, L.total))) return rc;
  cudaError_t ce = stream_eval(d, plan(a, e), buffers(ws, L), real, with_grad, theta, energy, grad, stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "streaming launch");
  return VQE_OK;
}

}  // namespace

namespace vqe {

// Descriptor, streaming plan and scratch layout for vqe_energy_grad_noalloc.
// H psi uses the (Hamiltonian, sector) pair's string or connectivity tables
// when an earlier call already built them, else a scan of all groups with an
// integer sector test; nothing is built or allocated here. Only the buffers the
// chosen path touches get scratch: the alpha-major copies only for the
// string-driven H psi. Real amplitudes unless complex arithmetic is forced.
int prepare_noalloc(vqe_hamiltonian_s* h, vqe_ansatz_s* a, bool with_grad, size_t limit, InstDesc* d,
                    StreamPlan* sp, bool* real, size_t off[7], size_t* need) {
  const int rc = check_pair(h, a);
  if (rc) return rc;
  *real = use_real();
  static const vqe_hamiltonian_s::Ell none;
  const vqe_hamiltonian_s::Ell* e = &none;
  {
    std::lock_guard<std::mutex> lock(h->mu);
    auto it = h->ells.find(a->key());
    if (it != h->ells.end()) e = &it->second;  // entries are never erased while h lives
  }
  *d = make_desc(h, a, e, 0);
  *sp = plan(a, e);
  sp->sweep = nullptr;  // one launch per gate: the sweep queues address the regular workspace layout
  // the string-driven H psi needs two more sector-sized vectors; when they do
  // not fit, the connectivity rows (if built) or the group scan serve instead
  const size_t amp = *real ? 8 : 16;
  const size_t vec0 = align256(std::max<size_t>(a->sector.size(), 1) * amp);
  const size_t fixed = align256(size_t(std::max(a->M, 1)) * 16) + align256(size_t(vqe::kMaxPartials) * 8) +
                       (with_grad ? align256(size_t(std::max(a->M, 1)) * vqe::kMaxPartials * 8) : 0);
  if (sp->use_str && 4 * vec0 + fixed > limit) sp->use_str = false;
  const size_t vec = align256(std::max<size_t>(a->sector.size(), 1) * amp);
  size_t o = 0;
  off[0] = o;  // psi
  o += vec;
  off[1] = o;  // lambda
  o += vec;
  if (sp->use_str) {
    off[2] = o;  // alpha-major psi
    o += vec;
    off[3] = o;  // alpha-major lambda
    o += vec;
  } else {
    off[2] = off[3] = 0;
  }
  off[4] = o;  // cos/sin
  o += align256(size_t(std::max(a->M, 1)) * 16);
  off[5] = o;  // energy partials
  o += align256(size_t(vqe::kMaxPartials) * 8);
  off[6] = o;  // gradient partials
  if (with_grad) o += align256(size_t(std::max(a->M, 1)) * vqe::kMaxPartials * 8);
  *need = o;
  return VQE_OK;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

}  // namespace vqe

// ------------------------------------------------------------------ C ABI
extern "C" {

int vqe_version(void) { return 100; }

int vqe_set_flags(int flags) {
  const int old = g_flags;
  g_flags = flags;
  return old;
}

const char* vqe_last_error(void) { return g_err.c_str(); }

int vqe_jordan_wigner(int n_spatial, const double* h, const double* eri, double c0, double drop_tol,
                      int64_t capacity, uint64_t* x_out, uint64_t* z_out, double* c_out, int64_t* n_out) {
  if (n_spatial < 1 || n_spatial > 16) return fail(VQE_ERR_INVALID_ARG, "n_spatial must be 1..16");
  if (!h || !eri || !n_out) return fail(VQE_ERR_INVALID_ARG, "NULL input");
  if (!(drop_tol >= 0.0) || !std::isfinite(c0)) return fail(VQE_ERR_INVALID_ARG, "bad drop_tol or c0");
  const int ns = n_spatial;
  std::unordered_map<uint64_t, cplx> acc;
  acc.reserve(size_t(1) << 20);
  if (c0 != 0.0) acc[0] += cplx(c0, 0.0);
  for (int p = 0; p < ns; ++p)
    for (int q = 0; q < ns; ++q) {
      const double v = h[p * ns + q];
      if (!std::isfinite(v)) return fail(VQE_ERR_INVALID_ARG, "non-finite h");
      if (v == 0.0) continue;
      for (int s = 0; s < 2; ++s) {
        const int orb[2] = {2 * p + s, 2 * q + s};
        const bool dag[2] = {true, false};
        add_ladder_product(acc, v, orb, dag, 2);
      }
    }
  for (int p = 0; p < ns; ++p)
    for (int q = 0; q < ns; ++q)
      for (int r = 0; r < ns; ++r)
        for (int s = 0; s < ns; ++s) {
          const double v = eri[((p * ns + q) * ns + r) * ns + s];
          if (!std::isfinite(v)) return fail(VQE_ERR_INVALID_ARG, "non-finite eri");
          if (v == 0.0) continue;
          for (int sg = 0; sg < 2; ++sg)
            for (int tau = 0; tau < 2; ++tau) {
              const int P = 2 * p + sg, Q = 2 * q + sg, R = 2 * r + tau, S = 2 * s + tau;
              if (P == R || Q == S) continue;  // a+_P a+_P = 0 and a_Q a_Q = 0
              const int orb[4] = {P, R, S, Q};
              const bool dag[4] = {true, true, false, false};
              add_ladder_product(acc, 0.5 * v, orb, dag, 4);
            }
        }
  std::vector<std::pair<uint64_t, double>> terms;
  terms.reserve(acc.size());
  for (const auto& kv : acc) {
    const cplx c = kv.second;
    if (std::fabs(c.imag()) > 1e-10 * std::max(1.0, std::fabs(c.real())))
      return fail(VQE_ERR_NOT_REAL, "mapped coefficient has an imaginary part; integrals not symmetric?");
    if (std::fabs(c.real()) < drop_tol || c.real() == 0.0) continue;
    terms.emplace_back(kv.first, c.real());
  }
  std::sort(terms.begin(), terms.end(),
            [](const std::pair<uint64_t, double>& a, const std::pair<uint64_t, double>& b) { return a.first < b.first; });
  *n_out = int64_t(terms.size());
  if (capacity < int64_t(terms.size()) || !x_out || !z_out || !c_out)
    return fail(VQE_ERR_INVALID_ARG, "capacity too small: need " + std::to_string(terms.size()));
  for (size_t i = 0; i < terms.size(); ++i) {
    x_out[i] = terms[i].first >> 32;
    z_out[i] = terms[i].first & 0xFFFFFFFFull;
    c_out[i] = terms[i].second;
  }
  return VQE_OK;
}

int vqe_fold_frozen(int n_spatial, const double* h, const double* eri, double c0, int n_frozen,
                    const int32_t* frozen, int n_active, const int32_t* active, double* h_out, double* eri_out,
                    double* c0_out) {
  if (n_spatial < 1 || n_frozen < 0 || n_active < 0 || n_frozen + n_active > n_spatial)
    return fail(VQE_ERR_INVALID_ARG, "bad orbital counts");
  if (!h || !eri || !c0_out || (n_frozen > 0 && !frozen) || (n_active > 0 && (!active || !h_out || !eri_out)))
    return fail(VQE_ERR_INVALID_ARG, "NULL input");
  std::vector<char> seen(size_t(n_spatial), 0);
  for (int i = 0; i < n_frozen + n_active; ++i) {
    const int o = i < n_frozen ? frozen[i] : active[i - n_frozen];
    if (o < 0 || o >= n_spatial || seen[size_t(o)]) return fail(VQE_ERR_INVALID_ARG, "orbital out of range or listed twice");
    seen[size_t(o)] = 1;
  }
  const size_t ns = size_t(n_spatial);
  auto H = [&](int p, int q) { return h[size_t(p) * ns + size_t(q)]; };
  auto V = [&](int p, int q, int r, int t) { return eri[((size_t(p) * ns + size_t(q)) * ns + size_t(r)) * ns + size_t(t)]; };
  // core energy: one-body and the frozen pairs' mutual Coulomb minus exchange
  double e = c0;
  for (int i = 0; i < n_frozen; ++i) {
    const int c = frozen[i];
    e += 2.0 * H(c, c);
    for (int j = 0; j < n_frozen; ++j) {
      const int d = frozen[j];
      e += 2.0 * V(c, c, d, d) - V(c, d, d, c);
    }
  }
  // effective one-body term on the active orbitals (Eq. 3's fold over the core)
  const size_t na = size_t(n_active);
  for (size_t x = 0; x < na; ++x)
    for (size_t y = 0; y < na; ++y) {
      const int p = active[x], q = active[y];
      double v = H(p, q);
      for (int i = 0; i < n_frozen; ++i) v += 2.0 * V(p, q, frozen[i], frozen[i]) - V(p, frozen[i], frozen[i], q);
      h_out[x * na + y] = v;
    }
  for (size_t a = 0; a < na; ++a)
    for (size_t b = 0; b < na; ++b)
      for (size_t c = 0; c < na; ++c)
        for (size_t d = 0; d < na; ++d)
          eri_out[((a * na + b) * na + c) * na + d] = V(active[a], active[b], active[c], active[d]);
  *c0_out = e;
  return VQE_OK;
}

int vqe_hcb_hamiltonian(int n_spatial, const double* h, const double* eri, double c0, double drop_tol,
                        int64_t capacity, uint64_t* x_out, uint64_t* z_out, double* c_out, int64_t* n_out) {
  if (n_spatial < 1 || n_spatial > vqe::kMaxQubits) return fail(VQE_ERR_INVALID_ARG, "n_spatial must be 1..32");
  if (!h || !eri || !n_out) return fail(VQE_ERR_INVALID_ARG, "NULL input");
  if (!(drop_tol >= 0.0) || !std::isfinite(c0)) return fail(VQE_ERR_INVALID_ARG, "bad drop_tol or c0");
  const int ns = n_spatial;
  auto H = [&](int p, int q) { return h[p * ns + q]; };
  auto V = [&](int p, int q, int r, int s) { return eri[((size_t(p) * ns + q) * ns + r) * ns + s]; };
  for (size_t i = 0; i < size_t(ns) * ns; ++i)
    if (!std::isfinite(h[i])) return fail(VQE_ERR_INVALID_ARG, "non-finite h");
  for (size_t i = 0; i < size_t(ns) * ns * ns * ns; ++i)
    if (!std::isfinite(eri[i])) return fail(VQE_ERR_INVALID_ARG, "non-finite eri");
  // Seniority-zero block of Eq. 2 with pair occupations n_p = (1 - Z_p) / 2:
  //   sum_p eps_p n_p + sum_{p<q} W_pq n_p n_q + sum_{p<q} K_pq (b+_p b_q + b+_q b_p),
  //   eps_p = 2 h_pp + (pp|pp), W_pq = 2 [2 (pp|qq) - (pq|qp)], K_pq = (pq|pq),
  //   b+_p b_q + b+_q b_p = (X_p X_q + Y_p Y_q) / 2.
  std::map<std::pair<uint64_t, uint64_t>, double> acc;  // (x, z) -> coefficient
  double id = c0;
  for (int p = 0; p < ns; ++p) {
    const double eps = 2.0 * H(p, p) + V(p, p, p, p);
    id += 0.5 * eps;
    acc[{0, uint64_t(1) << p}] -= 0.5 * eps;
  }
  for (int p = 0; p < ns; ++p)
    for (int q = p + 1; q < ns; ++q) {
      const uint64_t pq = (uint64_t(1) << p) | (uint64_t(1) << q);
      const double W = 2.0 * (2.0 * V(p, p, q, q) - V(p, q, q, p));
      id += 0.25 * W;
      acc[{0, uint64_t(1) << p}] -= 0.25 * W;
      acc[{0, uint64_t(1) << q}] -= 0.25 * W;
      acc[{0, pq}] += 0.25 * W;
      const double K = V(p, q, p, q);
      acc[{pq, 0}] += 0.5 * K;
      acc[{pq, pq}] += 0.5 * K;
    }
  acc[{0, 0}] += id;
  std::vector<std::pair<std::pair<uint64_t, uint64_t>, double>> terms;
  for (const auto& kv : acc)
    if (kv.second != 0.0 && std::fabs(kv.second) >= drop_tol) terms.push_back(kv);
  *n_out = int64_t(terms.size());
  if (capacity < int64_t(terms.size()) || !x_out || !z_out || !c_out)
    return fail(VQE_ERR_INVALID_ARG, "capacity too small: need " + std::to_string(terms.size()));
  for (size_t i = 0; i < terms.size(); ++i) {
    x_out[i] = terms[i].first.first;
    z_out[i] = terms[i].first.second;
    c_out[i] = terms[i].second;
  }
  return VQE_OK;
}

int vqe_create_hamiltonian(int n_qubits, int64_t n_terms, const uint64_t* xs, const uint64_t* zs,
                           const double* cs, double drop_tol, vqe_hamiltonian_t* out) {
  if (!out) return fail(VQE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > vqe::kMaxQubits) return fail(VQE_ERR_INVALID_ARG, "n_qubits must be 1..32");
  if (n_terms < 1) return fail(VQE_ERR_INVALID_ARG, "n_terms must be >= 1");
  if (!xs || !zs || !cs) return fail(VQE_ERR_INVALID_ARG, "NULL term array");
  if (!(drop_tol >= 0.0) || !std::isfinite(drop_tol)) return fail(VQE_ERR_INVALID_ARG, "bad drop_tol");
  const uint64_t full = (n_qubits == 64) ? ~0ull : ((uint64_t(1) << n_qubits) - 1);
  std::map<std::pair<uint64_t, uint64_t>, double> merged;
  for (int64_t t = 0; t < n_terms; ++t) {
    if ((xs[t] & ~full) || (zs[t] & ~full))
      return fail(VQE_ERR_INVALID_ARG, "term " + std::to_string(t) + " has a mask bit >= n_qubits");
    if (!std::isfinite(cs[t])) return fail(VQE_ERR_INVALID_ARG, "non-finite coefficient");
    merged[std::make_pair(xs[t], zs[t])] += cs[t];
  }
  std::unique_ptr<vqe_hamiltonian_s> H(new vqe_hamiltonian_s);
  H->n = n_qubits;
  for (const auto& kv : merged) {
    if (std::fabs(kv.second) < drop_tol || kv.second == 0.0) continue;
    H->x.push_back(kv.first.first);
    H->z.push_back(kv.first.second);
    H->c.push_back(kv.second);
  }
  // Group by x (merged is sorted by x then z). Every table slot is built as a
  // linear combination of the kept terms (term index, weight f * i^p, f a
  // small power of two) so that vqe_set_coefs can refold the tables on the
  // device in the same order; the values come from that same combination.
  using Lin = std::vector<std::pair<int32_t, cplx>>;
  static const cplx ipow[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
  std::vector<Lin> slots;
  auto scaled = [](const Lin& a, double f, Lin& out) {
    for (const auto& tw : a) out.emplace_back(tw.first, tw.second * f);
  };
  size_t t = 0;
  while (t < H->x.size()) {
    size_t t1 = t;
    while (t1 < H->x.size() && H->x[t1] == H->x[t]) ++t1;
    const uint32_t x = uint32_t(H->x[t]);
    GroupRec g;
    std::memset(&g, 0, sizeof(g));
    g.x = x;
    const uint32_t xsel = (pc32(x) <= vqe::kMaxPatternBits) ? x : 0u;
    int pos[4] = {0, 0, 0, 0}, ub = 0;
    for (int q = 0; q < 32; ++q)
      if ((xsel >> q) & 1u) pos[ub++] = q;
    g.ubits = ub;
    g.upos = 0;
    for (int j = 0; j < ub; ++j) g.upos |= uint32_t(pos[j]) << (8 * j);
    const int nu = 1 << ub;
    std::map<uint32_t, std::vector<Lin>> entries;  // z outside the pattern bits -> table
    for (size_t i = t; i < t1; ++i) {
      const uint32_t z = uint32_t(H->z[i]);
      const cplx ph = ipow[pc32(x & z) & 3];
      auto& tab = entries[z & ~xsel];
      if (tab.empty()) tab.assign(nu, Lin());
      for (int u = 0; u < nu; ++u) {
        uint32_t bits = 0;
        for (int j = 0; j < ub; ++j)
          if ((u >> j) & 1) bits |= 1u << pos[j];
        tab[u].emplace_back(int32_t(i), (pc32(bits & z) & 1) ? -ph : ph);
      }
    }
    // Evaluation form (see GroupRec::kind): the entry form, or the occupation
    // form when every entry's Z mask differs from a base mask z0 by at most one
    // bit (linear in the occupations) or, for a single pattern, by at most two
    // bits (quadratic), using (-1)^{n_r} = 1 - 2 n_r.
    int best_w = 99;
    uint32_t z0 = 0;
    for (const auto& cand : entries) {
      int w = 0;
      for (const auto& other : entries) w = std::max(w, pc32(other.first ^ cand.first));
      if (w < best_w) {
        best_w = w;
        z0 = cand.first;
      }
    }
    int kind = 0;
    if (entries.size() > 2 && best_w <= 1)
      kind = 1;
    else if (entries.size() > 3 && ub == 0 && best_w <= 2)
      kind = 2;
    g.kind = kind;
    g.nq = n_qubits;
    g.ebeg = int32_t(H->emask.size());
    g.vbeg = int32_t(slots.size());
    if (kind == 0) {
      for (auto& kv : entries) {
        H->emask.push_back(kv.first);
        for (int u = 0; u < nu; ++u) slots.push_back(std::move(kv.second[u]));
      }
    } else {
      uint32_t R = 0;
      for (const auto& kv : entries) R |= kv.first ^ z0;
      H->emask.push_back(z0);
      H->emask.push_back(R);
      const int nq = n_qubits;
      if (kind == 1) {
        std::vector<Lin> B(size_t(1 + nq) * nu);
        for (const auto& kv : entries) {
          const uint32_t dm = kv.first ^ z0;
          for (int u = 0; u < nu; ++u) {
            scaled(kv.second[u], 1.0, B[u]);
            if (dm) scaled(kv.second[u], -2.0, B[size_t(1 + __builtin_ctz(dm)) * nu + u]);
          }
        }
        for (auto& l : B) slots.push_back(std::move(l));
      } else {
        std::vector<Lin> Q(size_t(1 + nq + nq * nq));
        for (const auto& kv : entries) {
          const uint32_t dm = kv.first ^ z0;
          const Lin& a = kv.second[0];
          scaled(a, 1.0, Q[0]);
          if (pc32(dm) >= 1) {
            const int pb = __builtin_ctz(dm);
            scaled(a, -2.0, Q[1 + pb]);
            if (pc32(dm) == 2) {
              const int qb = 31 - __builtin_clz(dm);
              scaled(a, -2.0, Q[1 + qb]);
              scaled(a, 4.0, Q[size_t(1 + nq) + size_t(pb) * nq + qb]);
            }
          }
        }
        for (auto& l : Q) slots.push_back(std::move(l));
      }
    }
    g.eend = int32_t(H->emask.size());
    H->groups.push_back(g);
    t = t1;
  }
  // Flatten the linear map: weight f * i^p stored as the float f and the sign
  // bit of the term index set when p = 1. The values are summed in the same
  // order as the device refold (each product is exact).
  H->lin_off.assign(slots.size() + 1, 0);
  for (size_t s2 = 0; s2 < slots.size(); ++s2) {
    H->lin_off[s2 + 1] = H->lin_off[s2] + int64_t(slots[s2].size());
    for (const auto& tw : slots[s2]) {
      const bool imag = tw.second.imag() != 0.0;
      const double f = imag ? tw.second.imag() : tw.second.real();
      H->lin_term.push_back(imag ? int32_t(uint32_t(tw.first) | 0x80000000u) : tw.first);
      H->lin_w.push_back(float(f));
    }
  }
  H->cvals.resize(slots.size());
  for (size_t s2 = 0; s2 < slots.size(); ++s2) {
    double re = 0.0, im = 0.0;
    for (int64_t j = H->lin_off[s2]; j < H->lin_off[s2 + 1]; ++j) {
      const int32_t tt = H->lin_term[size_t(j)];
      const double v = double(H->lin_w[size_t(j)]) * H->c[size_t(tt & 0x7fffffff)];
      if (tt < 0)
        im += v;
      else
        re += v;
    }
    H->cvals[s2] = cplx(re, im);
  }
  std::vector<double> vals(H->cvals.size());
  std::vector<double2> cv(H->cvals.size());
  H->is_real = 1;
  for (size_t i = 0; i < H->cvals.size(); ++i) {
    vals[i] = H->cvals[i].real();
    cv[i] = make_double2(H->cvals[i].real(), H->cvals[i].imag());
    if (H->cvals[i].imag() != 0.0) H->is_real = 0;
  }
  if (H->groups.empty()) {
    // H = 0 after dropping: keep one empty identity group so tables are non-empty
    GroupRec g;
    std::memset(&g, 0, sizeof(g));
    g.ebeg = 0;
    g.eend = 1;
    g.vbeg = 0;
    H->emask.push_back(0);
    H->cvals.push_back(cplx(0, 0));
    vals.push_back(0.0);
    cv.push_back(make_double2(0.0, 0.0));
    H->groups.push_back(g);
  }
  int rc;
  if ((rc = upload(H->groups, &H->d_groups))) return rc;
  if ((rc = upload(H->emask, &H->d_emask))) return rc;
  if ((rc = upload(vals, &H->d_vals))) return rc;
  if ((rc = upload(cv, &H->d_cvals))) return rc;
  if (!H->lin_term.empty()) {
    if ((rc = upload(H->lin_off, &H->d_lin_off))) return rc;
    if ((rc = upload(H->lin_term, &H->d_lin_term))) return rc;
    if ((rc = upload(H->lin_w, &H->d_lin_w))) return rc;
  }
  {
    std::vector<double> zero(1, 0.0);
    if ((rc = upload(zero, &H->d_bound))) return rc;
    cudaError_t ce = vqe::abs_sum(H->d_vals, int64_t(vals.size()), H->d_bound, 0);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(0);
    if (ce != cudaSuccess) return cuda_fail(ce, "table bound");
  }
  H->serial = next_serial();
  *out = H.release();
  return VQE_OK;
}

int vqe_hamiltonian_info(vqe_hamiltonian_t h, int* n_qubits, int64_t* n_terms, int64_t* n_groups,
                         int* is_real) {
  if (!h) return fail(VQE_ERR_INVALID_ARG, "NULL handle");
  if (n_qubits) *n_qubits = h->n;
  if (n_terms) *n_terms = int64_t(h->x.size());
  if (n_groups) *n_groups = h->x.empty() ? 0 : int64_t(h->groups.size());
  if (is_real) *is_real = h->is_real;
  return VQE_OK;
}

static void purge_plans(uint64_t serial);

int vqe_hamiltonian_terms(vqe_hamiltonian_t h, uint64_t* x_masks, uint64_t* z_masks, double* coefs) {
  if (!h) return fail(VQE_ERR_INVALID_ARG, "NULL handle");
  for (size_t t = 0; t < h->x.size(); ++t) {
    if (x_masks) x_masks[t] = h->x[t];
    if (z_masks) z_masks[t] = h->z[t];
    if (coefs) coefs[t] = h->c[t];
  }
  return VQE_OK;
}

int vqe_set_coefs(vqe_hamiltonian_t h, const double* coefs_dev, vqe_stream_t stream) {
  if (!h) return fail(VQE_ERR_INVALID_ARG, "NULL handle");
  if (!coefs_dev) return fail(VQE_ERR_INVALID_ARG, "NULL coefficient pointer");
  const int64_t n_slots = int64_t(h->lin_off.size()) - 1;
  if (n_slots <= 0 || h->lin_term.empty()) return VQE_OK;  // every term was dropped: H = 0
  cudaError_t ce = vqe::fold_coefs(n_slots, h->d_lin_off, h->d_lin_term, h->d_lin_w, coefs_dev, h->d_vals,
                                   h->d_cvals, static_cast<cudaStream_t>(stream));
  if (ce == cudaSuccess) ce = vqe::abs_sum(h->d_vals, n_slots, h->d_bound, static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "coefficient refold");
  // the resident kernel's precomputed entry coefficients follow the new values
  std::lock_guard<std::mutex> lock(h->mu);
  for (auto& kv : h->ells) {
    vqe_hamiltonian_s::Ell& e = kv.second;
    if (!e.d_hmat) continue;
    ce = vqe::build_hmat(e.d_ellp, e.W, e.hD, e.d_hsec, h->d_groups, h->d_emask, h->d_vals, n_slots,
                         h->d_bound, e.ellp_fast ? 1 : 0, e.d_ivals, e.d_hmat, static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) return cuda_fail(ce, "entry coefficient rebuild");
  }
  return VQE_OK;
}

void vqe_destroy_hamiltonian(vqe_hamiltonian_t h) {
  if (!h) return;
  purge_plans(h->serial);
  delete h;
}

static int finish_ansatz(std::unique_ptr<vqe_ansatz_s> A, const std::vector<uint32_t>& occv, vqe_ansatz_t* out);

int vqe_create_ansatz(int n_qubits, uint64_t hf_bits, int32_t n_exc, const int32_t* exc,
                      vqe_ansatz_t* out) {
  if (!out) return fail(VQE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > vqe::kMaxQubits) return fail(VQE_ERR_INVALID_ARG, "n_qubits must be 1..32");
  const uint64_t full = (uint64_t(1) << n_qubits) - 1;
  if (hf_bits & ~full) return fail(VQE_ERR_INVALID_ARG, "hf_bits has a bit >= n_qubits");
  if (n_exc < 0 || (n_exc > 0 && !exc)) return fail(VQE_ERR_INVALID_ARG, "bad excitation list");
  std::unique_ptr<vqe_ansatz_s> A(new vqe_ansatz_s);
  A->n = n_qubits;
  A->M = n_exc;
  A->hf = hf_bits;
  A->exc.assign(exc, exc + 4 * size_t(n_exc));
  A->n_elec = pc64(hf_bits);
  bool spin_ok = true;
  std::vector<uint32_t> occv;
  for (int m = 0; m < n_exc; ++m) {
    const int32_t* e = exc + 4 * m;
    const bool single = e[2] < 0;
    int orb[4];
    int nops;
    if (single) {
      if (e[3] >= 0) return fail(VQE_ERR_INVALID_ARG, "single excitation needs {i, a, -1, -1}");
      orb[0] = e[1];  // a+_a
      orb[1] = e[0];  // a_i
      nops = 2;
    } else {
      orb[0] = e[2];  // a+_a
      orb[1] = e[3];  // a+_b
      orb[2] = e[1];  // a_j
      orb[3] = e[0];  // a_i
      nops = 4;
    }
    uint32_t flip = 0;
    for (int i = 0; i < nops; ++i) {
      if (orb[i] < 0 || orb[i] >= n_qubits)
        return fail(VQE_ERR_INVALID_ARG, "excitation " + std::to_string(m) + " index out of range");
      if (flip & (1u << orb[i]))
        return fail(VQE_ERR_INVALID_ARG, "excitation " + std::to_string(m) + " repeats an index");
      flip |= 1u << orb[i];
    }
    const uint32_t occ = single ? (1u << e[0]) : ((1u << e[0]) | (1u << e[1]));
    occv.push_back(occ);
    const uint32_t vir = flip & ~occ;
    if (pc32(occ & 0x55555555u) != pc32(vir & 0x55555555u)) spin_ok = false;
    // sign of T on k0 = occ, applying the rightmost factor first
    uint32_t k = occ;
    int par = 0;
    uint32_t pmask = 0;
    for (int i = nops - 1; i >= 0; --i) {
      const uint32_t bit = 1u << orb[i], below = bit - 1;
      par ^= pc32(k & below) & 1;
      pmask ^= below;
      k ^= bit;
    }
    GateRec g;
    g.flip = flip;
    g.par = pmask & ~flip;
    g.sign0 = par ? -1 : 1;
    g.pad = 0;
    A->gates.push_back(g);
  }
  A->n_alpha = spin_ok ? pc32(uint32_t(hf_bits) & 0x55555555u) : -1;
  return finish_ansatz(std::move(A), occv, out);
}

// Sector, pair lists, rank tables and device copies of an ansatz whose gates
// (A->gates) and annihilated-orbital masks (occv) are set; A->n_alpha < 0
// selects the electron-number sector, else the (N, N_alpha) spin sector.
static int finish_ansatz(std::unique_ptr<vqe_ansatz_s> A, const std::vector<uint32_t>& occv, vqe_ansatz_t* out) {
  const int n_qubits = A->n, n_exc = A->M;
  const uint64_t full = (uint64_t(1) << n_qubits) - 1;
  // sector enumeration
  const int n = n_qubits;
  auto subsets = [](uint32_t pool, int c, std::vector<uint32_t>& outv) {
    std::vector<int> bits;
    for (int q = 0; q < 32; ++q)
      if ((pool >> q) & 1u) bits.push_back(q);
    const int m = int(bits.size());
    outv.clear();
    if (c < 0 || c > m) return;
    if (c == 0) {
      outv.push_back(0);
      return;
    }
    uint64_t v = (uint64_t(1) << c) - 1;
    const uint64_t lim = uint64_t(1) << m;
    while (v < lim) {
      uint32_t w = 0;
      for (int j = 0; j < m; ++j)
        if ((v >> j) & 1) w |= 1u << bits[j];
      outv.push_back(w);
      const uint64_t t = v | (v - 1);
      v = (t + 1) | (((~t & (t + 1)) - 1) >> (__builtin_ctzll(v) + 1));
    }
  };
  const uint32_t all = uint32_t(full);
  const uint32_t even = all & 0x55555555u, odd = all & 0xAAAAAAAAu;
  auto enumerate = [&](uint32_t fixed_occ, uint32_t fixed_all, std::vector<uint32_t>& outv) {
    // states k with k & fixed_all == fixed_occ and the sector's counts
    outv.clear();
    const uint32_t free_bits = all & ~fixed_all;
    if (A->n_alpha >= 0) {
      const int ca = A->n_alpha - pc32(fixed_occ & even);
      const int cb = (A->n_elec - A->n_alpha) - pc32(fixed_occ & odd);
      std::vector<uint32_t> pa, pb;
      subsets(free_bits & even, ca, pa);
      subsets(free_bits & odd, cb, pb);
      outv.reserve(pa.size() * pb.size());
      for (uint32_t u : pa)
        for (uint32_t w : pb) outv.push_back(fixed_occ | u | w);
    } else {
      std::vector<uint32_t> pf;
      subsets(free_bits, A->n_elec - pc32(fixed_occ), pf);
      for (uint32_t u : pf) outv.push_back(fixed_occ | u);
    }
    std::sort(outv.begin(), outv.end());
  };
  enumerate(0, 0, A->sector);
  (void)n;
  // pair lists: lower states (occupied i,j; empty a,b) of each gate
  A->pair_off.assign(size_t(n_exc) + 1, 0);
  std::vector<std::vector<uint32_t>> per(n_exc);
  parallel_items(n_exc, [&](int64_t m) { enumerate(occv[size_t(m)], A->gates[m].flip, per[m]); });
  for (int m = 0; m < n_exc; ++m) A->pair_off[m + 1] = A->pair_off[m] + int64_t(per[m].size());
  A->pairs.resize(size_t(A->pair_off[n_exc]));
  parallel_items(n_exc, [&](int64_t m) {
    std::copy(per[m].begin(), per[m].end(), A->pairs.begin() + A->pair_off[m]);
    std::vector<uint32_t>().swap(per[m]);
  });
  // Rank tables of the sorted sector. A state k splits into a high part h =
  // k >> L and a low part v = k & (2^L - 1); sorted order compares h first, so
  // rank(k) = #{sector states with a smaller high part} + #{low parts below v
  // with the same electron counts as v}. The counts are (alpha, beta) for a
  // spin sector (even / odd qubits) and N otherwise.
  {
    const int L = (n + 1) / 2, Hb = n - L;
    A->lo_bits = L;
    const bool spin = A->n_alpha >= 0;
    const uint32_t lo_mask = uint32_t((uint64_t(1) << L) - 1);
    auto binom = [](int a, int b) -> uint64_t {
      if (b < 0 || b > a) return 0;
      uint64_t r = 1;
      for (int i = 1; i <= b; ++i) r = r * uint64_t(a - b + i) / uint64_t(i);
      return r;
    };
    const int lo_even = (L + 1) / 2, lo_odd = L / 2;
    A->rank_lo.assign(size_t(1) << L, 0u);
    std::vector<uint32_t> counter(33 * 33, 0u);
    for (uint32_t v = 0; v <= lo_mask; ++v) {
      const int key = spin ? pc32(v & even) * 33 + pc32(v & odd) : pc32(v);
      A->rank_lo[v] = counter[size_t(key)]++;
      if (v == lo_mask) break;
    }
    A->rank_hi.assign(size_t(1) << Hb, 0u);
    uint64_t acc = 0;
    const int n_beta = A->n_elec - A->n_alpha;
    for (uint64_t h = 0; h < (uint64_t(1) << Hb); ++h) {
      A->rank_hi[size_t(h)] = uint32_t(acc);
      const uint32_t hk = uint32_t(h << L);
      if (spin)
        acc += binom(lo_even, A->n_alpha - pc32(hk & even)) * binom(lo_odd, n_beta - pc32(hk & odd));
      else
        acc += binom(L, A->n_elec - pc32(hk));
    }
    if (acc != uint64_t(A->sector.size()) || A->sector.size() >= (size_t(1) << 31))
      return fail(VQE_ERR_UNSUPPORTED, "sector rank tables do not cover the sector");
    auto rank = [&](uint32_t k) { return A->rank_hi[k >> L] + A->rank_lo[k & lo_mask]; };
    for (size_t r = 0; r < A->sector.size(); ++r)
      if (rank(A->sector[r]) != uint32_t(r)) return fail(VQE_ERR_UNSUPPORTED, "sector rank mismatch");
    A->rpairs.resize(A->pairs.size());
    parallel_items(n_exc, [&](int64_t m) {
      const GateRec& g = A->gates[size_t(m)];
      for (int64_t p = A->pair_off[m]; p < A->pair_off[m + 1]; ++p) {
        const uint32_t k = A->pairs[size_t(p)];
        const uint32_t sb = uint32_t((pc32(k & g.par) & 1) ^ (g.sign0 < 0 ? 1 : 0));
        A->rpairs[size_t(p)] = make_uint2(rank(k) | (sb << 31), rank(k ^ g.flip));
      }
    });
  }
  A->nb_rows.resize(size_t(n_exc) + 1);
  for (int m = 0; m < n_exc; ++m) A->nb_rows[m] = vqe::stream_grid(A->pair_off[m + 1] - A->pair_off[m]);
  A->nb_rows[n_exc] = vqe::stream_grid(int64_t(A->sector.size()));
  A->chunk_off.assign(size_t(n_exc) + 1, 0);
  for (int m = 0; m < n_exc; ++m)
    A->chunk_off[m + 1] =
        A->chunk_off[m] + (A->pair_off[m + 1] - A->pair_off[m] + vqe::kPoolChunk - 1) / vqe::kPoolChunk;
  int rc;
  if ((rc = upload(A->gates, &A->d_gates))) return rc;
  if ((rc = upload(A->pair_off, &A->d_pair_off))) return rc;
  if ((rc = upload(A->chunk_off, &A->d_chunk_off))) return rc;
  if ((rc = upload(A->pairs, &A->d_pairs))) return rc;
  if ((rc = upload(A->sector, &A->d_sector))) return rc;
  if ((rc = upload(A->rank_hi, &A->d_rank_hi))) return rc;
  if ((rc = upload(A->rank_lo, &A->d_rank_lo))) return rc;
  if (!A->rpairs.empty() && (rc = upload(A->rpairs, &A->d_rpairs))) return rc;
  if ((rc = upload(A->nb_rows, &A->d_nb_rows))) return rc;
  if (A->pairs.empty()) {
    // keep valid (never read) pair pointers for kernels
    std::vector<uint32_t> one(1, 0);
    if ((rc = upload(one, &A->d_pairs))) return rc;
    std::vector<uint2> one2(1, make_uint2(0, 0));
    if ((rc = upload(one2, &A->d_rpairs))) return rc;
  }
  A->serial = next_serial();
  *out = A.release();
  return VQE_OK;
}

int vqe_create_ansatz_hcb(int n_qubits, uint64_t hf_bits, int32_t n_exc, const int32_t* pairs, vqe_ansatz_t* out) {
  if (!out) return fail(VQE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > vqe::kMaxQubits) return fail(VQE_ERR_INVALID_ARG, "n_qubits must be 1..32");
  const uint64_t full = (uint64_t(1) << n_qubits) - 1;
  if (hf_bits & ~full) return fail(VQE_ERR_INVALID_ARG, "hf_bits has a bit >= n_qubits");
  if (n_exc < 0 || (n_exc > 0 && !pairs)) return fail(VQE_ERR_INVALID_ARG, "bad pair-excitation list");
  std::unique_ptr<vqe_ansatz_s> A(new vqe_ansatz_s);
  A->n = n_qubits;
  A->M = n_exc;
  A->hf = hf_bits;
  A->n_elec = pc64(hf_bits);  // boson (electron-pair) count
  A->n_alpha = -1;            // sector: the number of occupied qubits only
  std::vector<uint32_t> occv;
  for (int m = 0; m < n_exc; ++m) {
    const int i = pairs[2 * m], a = pairs[2 * m + 1];
    if (i < 0 || i >= n_qubits || a < 0 || a >= n_qubits || i == a)
      return fail(VQE_ERR_INVALID_ARG, "pair excitation " + std::to_string(m) + " needs two distinct qubits");
    A->exc.insert(A->exc.end(), {i, a, -1, -1});
    // b+_a b_i: hard-core bosons on different qubits commute, so no parity string
    GateRec g;
    g.flip = (1u << i) | (1u << a);
    g.par = 0;
    g.sign0 = 1;
    g.pad = 0;
    A->gates.push_back(g);
    occv.push_back(1u << i);
  }
  return finish_ansatz(std::move(A), occv, out);
}

int vqe_ansatz_info(vqe_ansatz_t a, int* n_qubits, int32_t* n_params, int64_t* sector_dim, int64_t* n_pairs) {
  if (!a) return fail(VQE_ERR_INVALID_ARG, "NULL handle");
  if (n_qubits) *n_qubits = a->n;
  if (n_params) *n_params = a->M;
  if (sector_dim) *sector_dim = int64_t(a->sector.size());
  if (n_pairs) *n_pairs = int64_t(a->pairs.size());
  return VQE_OK;
}

void vqe_destroy_ansatz(vqe_ansatz_t a) {
  if (!a) return;
  purge_plans(a->serial);
  delete a;
}

size_t vqe_workspace_bytes(vqe_hamiltonian_t h, vqe_ansatz_t a, int mode) {
  if (check_pair(h, a)) return 0;
  int rc = VQE_OK;
  if (!get_ell(h, a, &rc)) return 0;
  const bool cplx_amp = (mode & VQE_WS_COMPLEX) || !use_real();
  if (!cplx_amp && (g_flags & VQE_FLAG_PERSISTENT_SWEEPS)) get_sweep(a);  // before any stream capture
  return ws_layout(a, cplx_amp, (mode & VQE_WS_GRAD) != 0).total;
}

int vqe_energy(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta, double* energy, void* ws,
               size_t ws_bytes, vqe_stream_t stream) {
  return run_single(h, a, theta, energy, nullptr, ws, ws_bytes, static_cast<cudaStream_t>(stream), false);
}

int vqe_energy_grad(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta, double* energy, double* grad,
                    void* ws, size_t ws_bytes, vqe_stream_t stream) {
  return run_single(h, a, theta, energy, grad, ws, ws_bytes, static_cast<cudaStream_t>(stream), true);
}

int vqe_state(vqe_ansatz_t a, vqe_hamiltonian_t h, const double* theta, double* psi_out, void* ws,
              size_t ws_bytes, vqe_stream_t stream) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  if ((!theta && a->M > 0) || !psi_out) return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const WsLayout L = ws_layout(a, false, false);
  if ((rc = check_ws(ws, ws_bytes, L.total))) return rc;
  InstDesc d = make_desc(h, a, e, 0);
  cudaError_t ce = vqe::stream_state(d, plan(a, e), buffers(ws, L), theta, psi_out,
                                     static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "state launch");
  return VQE_OK;
}

int vqe_apply_hamiltonian(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* psi, double* lam_out,
                          double* energy, void* ws, size_t ws_bytes, vqe_stream_t stream) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  if (!psi || !lam_out || !energy) return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const WsLayout L = ws_layout(a, true, false);
  if ((rc = check_ws(ws, ws_bytes, L.total))) return rc;
  InstDesc d = make_desc(h, a, e, 0);
  cudaError_t ce = vqe::stream_apply_h(d, plan(a, e), buffers(ws, L), psi, lam_out, energy,
                                       static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "apply_hamiltonian launch");
  return VQE_OK;
}

int vqe_apply_hamiltonian_sector(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* psi, double* lam_out,
                                 double* energy, void* ws, size_t ws_bytes, vqe_stream_t stream) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  if (!psi || !lam_out || !energy) return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  if (psi == lam_out) return fail(VQE_ERR_INVALID_ARG, "psi and lambda must not overlap");
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const WsLayout L = ws_layout(a, false, false);
  if ((rc = check_ws(ws, ws_bytes, L.total))) return rc;
  InstDesc d = make_desc(h, a, e, 0);
  vqe::StreamBuffers b = buffers(ws, L);
  b.psi = const_cast<double*>(psi);  // read only: H psi writes lambda and the alpha-major copies
  b.lam = lam_out;
  cudaError_t ce = vqe::stream_apply_h_real(d, plan(a, e), b, energy, static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "apply_hamiltonian_sector launch");
  return VQE_OK;
}

size_t vqe_pool_workspace_bytes(vqe_hamiltonian_t h, vqe_ansatz_t a, vqe_ansatz_t pool) {
  if (check_pair(h, a)) return 0;
  if (!pool) {
    fail(VQE_ERR_INVALID_ARG, "NULL pool handle");
    return 0;
  }
  int rc = VQE_OK;
  if (!get_ell(h, a, &rc)) return 0;
  const bool real = use_real();
  return ws_layout(a, !real, false).total + align256(size_t(std::max<int64_t>(pool->chunk_off.back(), 1)) * 8) +
         align256(std::max<size_t>(a->sector.size(), 1) * (real ? 16 : 32));
}

int vqe_pool_gradients(vqe_hamiltonian_t h, vqe_ansatz_t a, vqe_ansatz_t pool, const double* theta, double* energy,
                       double* pool_grad, void* ws, size_t ws_bytes, vqe_stream_t stream) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  if (!pool) return fail(VQE_ERR_INVALID_ARG, "NULL pool handle");
  if (pool->n != a->n || pool->key() != a->key())
    return fail(VQE_ERR_INVALID_ARG,
                "pool sector differs from the ansatz's (same qubits, electrons and spin counts needed)");
  if ((!theta && a->M > 0) || !energy || (!pool_grad && pool->M > 0))
    return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const bool real = use_real();
  const WsLayout L = ws_layout(a, !real, false);
  const int64_t n_chunks = pool->chunk_off.back();
  const size_t part_bytes = align256(size_t(std::max<int64_t>(n_chunks, 1)) * 8);
  const size_t need = L.total + part_bytes + align256(std::max<size_t>(a->sector.size(), 1) * (real ? 16 : 32));
  if ((rc = check_ws(ws, ws_bytes, need))) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  InstDesc d = make_desc(h, a, e, 0);
  const vqe::StreamBuffers b = buffers(ws, L);
  cudaError_t ce = vqe::stream_energy_grad(d, plan(a, e), b, real, false, theta, energy, nullptr, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "pool screening forward / H psi launch");
  double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + L.total);
  void* pl = static_cast<char*>(ws) + L.total + part_bytes;
  ce = vqe::pool_gradients(pool->d_rpairs, pool->d_pair_off, pool->d_chunk_off, pool->M, n_chunks, real, b.psi,
                           b.lam, int64_t(a->sector.size()), pl, part, pool_grad, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "pool screening launch");
  return VQE_OK;
}

// Largest instance a persistent slot takes: every per-gate pair list and the
// sector fit one pass of 1024 blocks of 256 threads, so the slot's reductions
// follow the single-instance kernels' partial sums exactly.
constexpr int64_t kSlotMaxItems = int64_t(vqe::kMaxPartials) * vqe::kStreamThreads;

static bool slot_fits(vqe_ansatz_t a) {
  if (int64_t(a->sector.size()) > kSlotMaxItems) return false;
  for (int m = 0; m < a->M; ++m)
    if (a->pair_off[m + 1] - a->pair_off[m] > kSlotMaxItems) return false;
  return true;
}

// Builds both task queues of the persistent launch for the current grid and
// gate chunk. Each slot is a chain of levels (INIT, FWD 0..M-1, [GATHER], HPSI,
// [SCATTER], DOT, then ADJ M-1..0 with the gradient); a task waits for every
// task of the earlier levels of its slot. The queue order comes from a list
// schedule of rough task costs over the grid's CTAs: whenever a CTA frees up,
// it takes the ready task whose level has the longest remaining chain after it
// (critical path first), so long instances start early and short ones fill in.
static int build_queues(vqe_batch_s* B) {
  StreamBatch& sb = B->sb;
  const int n = int(sb.slots.size());
  const int64_t gc = sb.gate_chunk;
  for (int mode = 0; mode < 2; ++mode) {
    const bool grad = mode == 1;
    struct Lvl {
      int slot;
      int64_t t0, nt;  // first task (in `tasks`) and count
      double cost, bottom;
    };
    std::vector<vqe::PTask> tasks;
    std::vector<double> cost;
    std::vector<Lvl> lv;
    std::vector<int64_t> slot_lv0(n + 1, 0);
    std::unique_ptr<PersistQueue> Q(new PersistQueue);
    for (int s = 0; s < n; ++s) {
      const int bi = sb.slots[s];
      vqe_ansatz_t a = B->ans[bi];
      const auto& d = sb.descs[s];
      const int64_t D = int64_t(a->sector.size());
      int rc2 = VQE_OK;
      const auto* e = get_ell(B->hams[bi], a, &rc2);
      if (!e) return rc2;
      const bool str = d.str != nullptr;
      int32_t done = 0;  // tasks of the slot in earlier levels
      slot_lv0[s] = int64_t(lv.size());
      auto level = [&](auto&& add) {
        Lvl L{s, int64_t(tasks.size()), 0, 0.0, 0.0};
        add();
        L.nt = int64_t(tasks.size()) - L.t0;
        if (L.nt == 0) return;
        for (int64_t t = L.t0; t < L.t0 + L.nt; ++t) {
          tasks[t].need = done;
          L.cost = std::max(L.cost, cost[t]);
        }
        done += int32_t(L.nt);
        lv.push_back(L);
      };
      auto task = [&](int kind, int m, int64_t lo, int64_t hi, int64_t aux, double c) {
        vqe::PTask t;
        t.slot = s;
        t.kind = kind;
        t.m = m;
        t.need = 0;
        t.lo = lo;
        t.hi = hi;
        t.aux = aux;
        tasks.push_back(t);
        cost.push_back(c);
      };
      // cost estimates in ns per CTA (only their proportions matter)
      level([&] { task(vqe::PT_INIT, 0, 0, D, 0, 1000.0 + 0.5 * double(D)); });
      for (int m = 0; m < a->M; ++m)
        level([&] {
          const int64_t P = a->pair_off[m + 1] - a->pair_off[m];
          for (int64_t lo = 0; lo < P; lo += gc) {
            const int64_t hi = std::min(P, lo + gc);
            task(vqe::PT_FWD, m, lo, hi, 0, 1500.0 + 0.6 * double(hi - lo));
          }
        });
      const int64_t ch = 16384;  // entries per GATHER / SCATTER task
      if (str)
        level([&] {
          for (int64_t lo = 0; lo < D; lo += ch) task(vqe::PT_GATHER, 0, lo, std::min(D, lo + ch), 0, 1500.0 + 0.3 * double(std::min(ch, D - lo)));
        });
      level([&] {
        const double per_entry = 1.6;  // measured order of magnitude of the string-driven H psi per CTA
        if (str) {
          const int Da = e->str.Da, Db = e->str.Db;
          const int per = Db < vqe::kStrMinDb ? vqe::kStrWarps : 1;
          for (int lo = 0; lo < Da; lo += per) {
            const int hi = std::min(Da, lo + per);
            task(vqe::PT_HPSI, 0, lo, hi, 0, 2000.0 + per_entry * double(e->nnz) * double(hi - lo) / double(Da));
          }
        } else {
          for (int64_t lo = 0; lo < D; lo += vqe::kPersistThreads) {
            const int64_t hi = std::min(D, lo + vqe::kPersistThreads);
            task(vqe::PT_HPSI, 0, lo, hi, 0, 2000.0 + 3.0 * per_entry * double(e->nnz) * double(hi - lo) / double(D));
          }
        }
      });
      if (str)
        level([&] {
          for (int64_t lo = 0; lo < D; lo += ch) task(vqe::PT_SCATTER, 0, lo, std::min(D, lo + ch), 0, 1500.0 + 0.3 * double(std::min(ch, D - lo)));
        });
      const int64_t nbD = (std::max<int64_t>(D, 1) + vqe::kPersistThreads - 1) / vqe::kPersistThreads;
      level([&] {
        for (int64_t lo = 0; lo < nbD; lo += 16) task(vqe::PT_DOT, 0, lo, std::min(nbD, lo + 16), 0, 1500.0 + 150.0 * double(std::min<int64_t>(16, nbD - lo)));
      });
      if (grad) {
        // gate m's partials start after those of gates 0..m-1
        std::vector<int64_t> gbase(a->M + 1, 0);
        for (int m = 0; m < a->M; ++m) {
          const int64_t P = a->pair_off[m + 1] - a->pair_off[m];
          gbase[m + 1] = gbase[m] + std::max<int64_t>(1, (P + vqe::kStreamThreads - 1) / vqe::kStreamThreads);
        }
        for (int m = a->M - 1; m >= 0; --m)
          level([&] {
            const int64_t P = a->pair_off[m + 1] - a->pair_off[m];
            for (int64_t lo = 0; lo < P; lo += gc) {
              const int64_t hi = std::min(P, lo + gc);
              task(vqe::PT_ADJ, m, lo, hi, gbase[m], 2000.0 + 1.0 * double(hi - lo));
            }
          });
      }
    }
    slot_lv0[n] = int64_t(lv.size());
    // remaining chain after each level (inclusive)
    for (int s = 0; s < n; ++s) {
      double acc = 0.0;
      for (int64_t l = slot_lv0[s + 1] - 1; l >= slot_lv0[s]; --l) {
        acc += lv[l].cost;
        lv[l].bottom = acc;
      }
    }
    // list schedule over the grid's CTAs
    std::vector<int64_t> level_of(tasks.size());
    for (int64_t l = 0; l < int64_t(lv.size()); ++l)
      for (int64_t t = lv[l].t0; t < lv[l].t0 + lv[l].nt; ++t) level_of[t] = l;
    typedef std::pair<double, int64_t> PQ;  // (priority, -task) max-heap; (time, level) min-heap
    std::priority_queue<std::pair<double, int64_t>> ready;
    std::priority_queue<PQ, std::vector<PQ>, std::greater<PQ>> running;
    std::vector<int64_t> left(lv.size());
    for (int64_t l = 0; l < int64_t(lv.size()); ++l) left[l] = lv[l].nt;
    auto push_level = [&](int64_t l) {
      for (int64_t t = lv[l].t0; t < lv[l].t0 + lv[l].nt; ++t) ready.push(std::make_pair(lv[l].bottom, -t));
    };
    for (int s = 0; s < n; ++s)
      if (slot_lv0[s] < slot_lv0[s + 1]) push_level(slot_lv0[s]);
    int free_ctas = std::max(1, sb.grid);
    double now = 0.0;
    Q->tasks.reserve(tasks.size());
    while (Q->tasks.size() < tasks.size()) {
      while (free_ctas > 0 && !ready.empty()) {
        const int64_t t = -ready.top().second;
        ready.pop();
        Q->tasks.push_back(tasks[t]);
        running.push(std::make_pair(now + cost[t], level_of[t]));
        --free_ctas;
      }
      if (running.empty()) break;  // cannot happen: every level follows a finished one
      const PQ done = running.top();
      running.pop();
      now = done.first;
      ++free_ctas;
      const int64_t l = done.second;
      if (--left[l] == 0 && l + 1 < int64_t(lv.size()) && lv[l + 1].slot == lv[l].slot) push_level(l + 1);
    }
    if (Q->tasks.size() != tasks.size()) return fail(VQE_ERR_INVALID_ARG, "persistent queue construction failed");
    if (tasks.size() > size_t(INT32_MAX / 2)) return fail(VQE_ERR_UNSUPPORTED, "batch has too many tasks");
    // finalising rows: gradients first, then energies
    if (grad) {
      for (int s = 0; s < n; ++s) {
        vqe_ansatz_t a = B->ans[sb.slots[s]];
        int64_t base = 0;
        for (int m = 0; m < a->M; ++m) {
          const int64_t P = a->pair_off[m + 1] - a->pair_off[m];
          const int64_t nb = std::max<int64_t>(1, (P + vqe::kStreamThreads - 1) / vqe::kStreamThreads);
          Q->finals.push_back(vqe::PFinal{sb.pslots[s].gp + base * 8, int32_t(nb), m, sb.descs[s].inst, 2.0});
          base += nb;
        }
      }
      Q->n_grad_rows = int(Q->finals.size());
    }
    for (int s = 0; s < n; ++s) {
      const int64_t D = int64_t(B->ans[sb.slots[s]]->sector.size());
      const int64_t nbD = (std::max<int64_t>(D, 1) + vqe::kPersistThreads - 1) / vqe::kPersistThreads;
      Q->finals.push_back(vqe::PFinal{sb.pslots[s].ep, int32_t(nbD), -1, sb.descs[s].inst, 1.0});
    }
    int rc;
    if ((rc = upload(Q->tasks, &Q->d_tasks))) return rc;
    if ((rc = upload(Q->finals, &Q->d_finals))) return rc;
    sb.q[mode] = std::move(Q);
  }
  return VQE_OK;
}

// The persistent kernel's dynamic shared-memory limit only ever grows (per
// device), so that every batch created so far can still launch.
static int ensure_persist_smem(size_t smem) {
  static std::mutex mu;
  static std::map<int, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(dev);
  if (it != done.end() && it->second >= smem) return VQE_OK;
  e = vqe::set_persist_smem_limit(smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute (persistent kernel)");
  done[dev] = smem;
  return VQE_OK;
}

// Grid of the persistent launch: the SM count times the CTAs that fit per SM
// (or the tuned count, if smaller).
static int persist_grid(const StreamBatch& sb, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  int rc = ensure_persist_smem(sb.smem);
  if (rc) return rc;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess) ce = vqe::persist_occupancy(sb.smem, &per_sm);
  if (ce != cudaSuccess) return cuda_fail(ce, "persistent launch set-up");
  if (per_sm < 1) return fail(VQE_ERR_UNSUPPORTED, "persistent kernel does not fit an SM");
  if (sb.ctas_per_sm > 0) per_sm = std::min(per_sm, sb.ctas_per_sm);
  *grid = sms * per_sm;
  return VQE_OK;
}

static int build_stream_batch(vqe_batch_s* B) {
  StreamBatch& sb = B->sb;
  for (int i : B->streaming[0]) {
    if (slot_fits(B->ans[i]))
      sb.slots.push_back(i);
    else
      sb.big.push_back(i);
  }
  for (int i : sb.big) sb.big_bytes = std::max(sb.big_bytes, ws_layout(B->ans[i], false, true).total);
  const int n = int(sb.slots.size());
  if (n == 0) return VQE_OK;
  size_t off = 0;
  for (int s = 0; s < n; ++s) {
    const int i = sb.slots[s];
    vqe_ansatz_t a = B->ans[i];
    sb.descs.push_back(B->descs[i]);
    const size_t D = std::max<size_t>(a->sector.size(), 1);
    const size_t vec = align256(D * 8);
    vqe::PSlot ps;
    ps.psi = int64_t(off);
    ps.lam = int64_t(off + vec);
    off += 2 * vec;
    if (B->descs[i].str) {
      ps.psi_am = int64_t(off);
      ps.lam_am = int64_t(off + vec);
      off += 2 * vec;
      int rc2 = VQE_OK;
      const auto* e = get_ell(B->hams[i], a, &rc2);
      if (!e) return rc2;
      sb.smem = std::max(sb.smem, vqe::str_smem_bytes(e->str.Db, 8));
    } else {
      ps.psi_am = ps.lam_am = -1;
    }
    ps.cs = int64_t(off);
    off += align256(size_t(std::max(a->M, 1)) * 16);
    ps.ep = int64_t(off);
    off += align256(((D + vqe::kPersistThreads - 1) / vqe::kPersistThreads) * 8);
    ps.gp = int64_t(off);
    int64_t nbg = 0;
    for (int m = 0; m < a->M; ++m)
      nbg += std::max<int64_t>(1, (a->pair_off[m + 1] - a->pair_off[m] + vqe::kStreamThreads - 1) / vqe::kStreamThreads);
    off += align256(size_t(std::max<int64_t>(nbg, 1)) * 8);
    sb.pslots.push_back(ps);
  }
  sb.counters_off = off;
  sb.persist_bytes = off + align256(size_t(n + 2) * sizeof(int));
  int rc;
  if ((rc = upload(sb.descs, &sb.d_desc))) return rc;
  if ((rc = upload(sb.pslots, &sb.d_slots))) return rc;
  if ((rc = persist_grid(sb, &sb.grid))) return rc;
  return build_queues(B);
}

int vqe_create_batch(int n_inst, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans, vqe_batch_t* out) {
  if (!out) return fail(VQE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  if (n_inst < 1 || !hams || !ans) return fail(VQE_ERR_INVALID_ARG, "bad batch arrays");
  std::unique_ptr<vqe_batch_s> B(new vqe_batch_s);
  B->n_inst = n_inst;
  for (int i = 0; i < n_inst; ++i) {
    int rc = check_pair(hams[i], ans[i]);
    if (rc) return fail(rc, "instance " + std::to_string(i) + ": " + g_err);
    const auto* e = get_ell(hams[i], ans[i], &rc);
    if (!e) return rc;
    B->hams.push_back(hams[i]);
    B->ans.push_back(ans[i]);
    B->descs.push_back(make_desc(hams[i], ans[i], e, i));
    B->max_params = std::max(B->max_params, ans[i]->M);
    for (int mode = 0; mode < 2; ++mode) {
      const bool real = mode == 0;
      InstDesc d = B->descs.back();
      size_t smem = 0;
      if (resident_fit(ans[i], e, real, &d, &smem)) {
        B->resident[mode].push_back(i);
        B->res_descs[mode].push_back(d);
        B->res_smem[mode] = std::max(B->res_smem[mode], smem);
      } else {
        B->streaming[mode].push_back(i);
      }
    }
  }
  for (int mode = 0; mode < 2; ++mode) {
    int rc = upload(B->res_descs[mode], &B->d_res[mode]);
    if (rc) return rc;
  }
  int rc = build_stream_batch(B.get());
  if (rc) return rc;
  *out = B.release();
  return VQE_OK;
}

int32_t vqe_batch_max_params(vqe_batch_t b) { return b ? b->max_params : 0; }

// Streamed instances run one by one (stream_energy_grad) in complex mode, under
// VQE_FLAG_NO_STRINGS, and for instances too large for a persistent slot.
static bool persistent_mode(vqe_batch_t b, bool real) {
  return real && !(g_flags & VQE_FLAG_NO_STRINGS) && !b->sb.slots.empty();
}

size_t vqe_batch_workspace_bytes(vqe_batch_t b, int with_grad) {
  if (!b) return 0;
  const int mode = use_real() ? 0 : 1;
  size_t one = 0;  // largest one-by-one instance
  if (mode == 0 && persistent_mode(b, true)) {
    for (int i : b->sb.big) one = std::max(one, ws_layout(b->ans[i], false, with_grad != 0).total);
    return b->sb.persist_bytes + one;
  }
  for (int i : b->streaming[mode]) one = std::max(one, ws_layout(b->ans[i], mode == 1, with_grad != 0).total);
  return one;
}

static int run_one_by_one(vqe_batch_t b, const std::vector<int>& which, bool real, const double* theta,
                          int64_t ld_theta, double* energies, double* grads, int64_t ld_grad, char* ws,
                          size_t ws_bytes, cudaStream_t stream) {
  const bool with_grad = grads != nullptr;
  for (int i : which) {
    vqe_ansatz_t a = b->ans[i];
    int rc2 = VQE_OK;
    const auto* e = get_ell(b->hams[i], a, &rc2);
    if (!e) return rc2;
    const WsLayout L = ws_layout(a, !real, with_grad);
    if ((rc2 = check_ws(ws, ws_bytes, L.total))) return rc2;
    cudaError_t ce = stream_eval(b->descs[i], plan(a, e), buffers(ws, L), real, with_grad,
                                 theta + int64_t(i) * ld_theta, energies + i,
                                 with_grad ? grads + int64_t(i) * ld_grad : nullptr, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "batched streaming launch");
  }
  return VQE_OK;
}

static int batch_run(vqe_batch_t b, const double* theta, int64_t ld_theta, double* energies, double* grads,
                     int64_t ld_grad, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  const bool with_grad = grads != nullptr;
  if (!theta || !energies) return fail(VQE_ERR_INVALID_ARG, "NULL device pointer");
  if (ld_theta < b->max_params || (with_grad && ld_grad < b->max_params))
    return fail(VQE_ERR_INVALID_ARG, "leading dimension smaller than max params");
  const bool real = use_real();
  const int mode = real ? 0 : 1;
  int rc;
  if (!b->resident[mode].empty()) {
    if ((rc = ensure_smem(b->res_smem[mode], real))) return rc;
    cudaError_t ce = vqe::launch_resident(b->d_res[mode], nullptr, int(b->resident[mode].size()),
                                          b->res_smem[mode], real, with_grad, theta, ld_theta, energies,
                                          grads, ld_grad, stream,
                                          ctas_per_instance(real, int(b->resident[mode].size())),
                                          use_fixed(real));
    if (ce != cudaSuccess) return cuda_fail(ce, "batched resident launch");
  }
  if (persistent_mode(b, real)) {
    const StreamBatch& sb = b->sb;
    const size_t need = vqe_batch_workspace_bytes(b, with_grad);
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    const PersistQueue& Q = *sb.q[with_grad ? 1 : 0];
    b->sb.last_queue = with_grad ? 1 : 0;
    vqe::PersistDev pd;
    pd.desc = sb.d_desc;
    pd.slots = sb.d_slots;
    pd.tasks = Q.d_tasks;
    pd.n_tasks = int32_t(Q.tasks.size());
    pd.n = int32_t(sb.slots.size());
    pd.ws = static_cast<char*>(ws);
    pd.counters = reinterpret_cast<int*>(static_cast<char*>(ws) + sb.counters_off);
    pd.budget_ns = sb.budget_ns;
    pd.probe_task = sb.probe_task;
    pd.pad = 0;
    if ((rc = ensure_persist_smem(sb.smem))) return rc;
    cudaError_t ce = vqe::batch_persistent_run(pd, sb.grid, sb.smem, Q.d_finals, int(Q.finals.size()),
                                               Q.n_grad_rows, theta, ld_theta, energies,
                                               with_grad ? grads : nullptr, ld_grad, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "persistent batch launch");
    if (!sb.big.empty())
      return run_one_by_one(b, sb.big, true, theta, ld_theta, energies, grads, ld_grad,
                            static_cast<char*>(ws) + sb.persist_bytes, ws_bytes - sb.persist_bytes, stream);
  } else if (!b->streaming[mode].empty()) {
    const size_t need = vqe_batch_workspace_bytes(b, with_grad);
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    return run_one_by_one(b, b->streaming[mode], real, theta, ld_theta, energies, grads, ld_grad,
                          static_cast<char*>(ws), ws_bytes, stream);
  }
  return VQE_OK;
}

int vqe_batch_energy_grad(vqe_batch_t b, const double* theta, int64_t ld_theta, double* energies,
                          double* grads, int64_t ld_grad, void* ws, size_t ws_bytes, vqe_stream_t stream) {
  return batch_run(b, theta, ld_theta, energies, grads, ld_grad, ws, ws_bytes,
                   static_cast<cudaStream_t>(stream));
}

size_t vqe_batch_host_workspace_bytes(vqe_batch_t b, int with_grad) {
  if (!b) return 0;
  const size_t io = align256(size_t(b->n_inst) * size_t(std::max(b->max_params, 1)) * 8) +
                    align256(size_t(b->n_inst) * 8) +
                    (with_grad ? align256(size_t(b->n_inst) * size_t(std::max(b->max_params, 1)) * 8) : 0);
  return io + vqe_batch_workspace_bytes(b, with_grad);
}

int vqe_batch_energy_grad_host(vqe_batch_t b, const double* theta_host, int64_t ld_theta, double* energies_host,
                               double* grads_host, int64_t ld_grad, void* ws, size_t ws_bytes,
                               vqe_stream_t stream_) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const bool with_grad = grads_host != nullptr;
  if (!theta_host || !energies_host) return fail(VQE_ERR_INVALID_ARG, "NULL host pointer");
  const int64_t Mx = std::max(b->max_params, 1);
  if (ld_theta < b->max_params || (with_grad && ld_grad < b->max_params))
    return fail(VQE_ERR_INVALID_ARG, "leading dimension smaller than max params");
  const size_t need = vqe_batch_host_workspace_bytes(b, with_grad);
  int rc = check_ws(ws, ws_bytes, need);
  if (rc) return rc;
  char* base = static_cast<char*>(ws);
  double* d_theta = reinterpret_cast<double*>(base);
  size_t off = align256(size_t(b->n_inst) * size_t(Mx) * 8);
  double* d_e = reinterpret_cast<double*>(base + off);
  off += align256(size_t(b->n_inst) * 8);
  double* d_g = nullptr;
  if (with_grad) {
    d_g = reinterpret_cast<double*>(base + off);
    off += align256(size_t(b->n_inst) * size_t(Mx) * 8);
  }
  // upload, evaluate, download, all asynchronous on s
  // (rows packed back to back on both sides: one plain copy instead of a
  // strided one, which the copy engine would run row by row)
  const size_t rows_bytes = size_t(b->n_inst) * size_t(Mx) * 8;
  const bool packed_theta = b->max_params == Mx && ld_theta == Mx;
  const bool packed_grad = b->max_params == Mx && ld_grad == Mx;
  auto issue = [&](cudaStream_t s) -> int {
    cudaError_t ce =
        packed_theta ? cudaMemcpyAsync(d_theta, theta_host, rows_bytes, cudaMemcpyHostToDevice, s)
                       : cudaMemcpy2DAsync(d_theta, size_t(Mx) * 8, theta_host, size_t(ld_theta) * 8,
                                           size_t(b->max_params) * 8, size_t(b->n_inst), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "theta upload");
    const int r = batch_run(b, d_theta, Mx, d_e, d_g, Mx, base + off, ws_bytes - off, s);
    if (r) return r;
    ce = cudaMemcpyAsync(energies_host, d_e, size_t(b->n_inst) * 8, cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) return cuda_fail(ce, "energy download");
    if (with_grad) {
      ce = packed_grad ? cudaMemcpyAsync(grads_host, d_g, rows_bytes, cudaMemcpyDeviceToHost, s)
                         : cudaMemcpy2DAsync(grads_host, size_t(ld_grad) * 8, d_g, size_t(Mx) * 8,
                                             size_t(b->max_params) * 8, size_t(b->n_inst), cudaMemcpyDeviceToHost, s);
      if (ce != cudaSuccess) return cuda_fail(ce, "gradient download");
    }
    return VQE_OK;
  };
  // after the synchronisation: a wait of the persistent launch that ran out
  // (status word in the batch's part of the workspace) returns VQE_ERR_TIMEOUT
  auto persist_check = [&]() -> int {
    if (!persistent_mode(b, use_real())) return VQE_OK;
    return vqe_batch_status(b, base + off, ws_bytes - off, stream);
  };
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();  // status unknown: plain copies and launches, then synchronise
    if ((rc = issue(stream))) return rc;
    const cudaError_t se = cudaStreamSynchronize(stream);
    return se == cudaSuccess ? persist_check() : cuda_fail(se, "stream synchronize");
  }
  if (cap != cudaStreamCaptureStatusNone) return issue(stream);  // inside the caller's capture: no sync
  HostGraph key;
  key.theta = theta_host;
  key.ld_theta = ld_theta;
  key.energies = energies_host;
  key.grads = grads_host;
  key.ld_grad = ld_grad;
  key.ws = ws;
  key.ws_bytes = ws_bytes;
  key.flags = g_flags;
  key.tuning = b->tuning_version;
  cudaGetDevice(&key.device);
  std::lock_guard<std::mutex> lk(b->hg_mu);
  cudaError_t ce;
  if (b->hg.exec && b->hg.same(key)) {
    ce = cudaGraphLaunch(b->hg.exec, stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph launch");
  } else {
    // first call with these buffers: run directly, then capture the same
    // sequence (nothing executes during capture) for the next calls
    if ((rc = issue(stream))) return rc;
    if (b->hg.exec) {
      cudaGraphExecDestroy(b->hg.exec);
      b->hg.exec = nullptr;
    }
    if (!b->capture_stream) cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (b->capture_stream &&
        cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const std::string saved = g_err;
      const int rc2 = issue(b->capture_stream);
      const cudaError_t ce2 = cudaStreamEndCapture(b->capture_stream, &graph);
      cudaGraphExec_t exec = nullptr;
      if (rc2 == VQE_OK && ce2 == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        key.exec = exec;
        b->hg = key;
      }
      if (graph) cudaGraphDestroy(graph);
      g_err = saved;  // a failed capture only means no graph: the call itself succeeded
    }
    cudaGetLastError();
  }
  ce = cudaStreamSynchronize(stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "stream synchronize");
  return persist_check();
}

int vqe_batch_set_tuning(vqe_batch_t b, int ctas_per_sm, int gate_chunk, int sweep_threads) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  if (ctas_per_sm < 0 || ctas_per_sm > 16) return fail(VQE_ERR_INVALID_ARG, "ctas_per_sm: 1..16, or 0 for all that fit");
  if (gate_chunk < 0 || gate_chunk % vqe::kStreamThreads || gate_chunk > (1 << 20))
    return fail(VQE_ERR_INVALID_ARG, "gate_chunk: a multiple of 256 up to 2^20, or 0 to keep");
  if (sweep_threads != 0 && (sweep_threads < 32 || sweep_threads > vqe::kResidentThreads || sweep_threads % 32))
    return fail(VQE_ERR_INVALID_ARG, "sweep_threads: a multiple of 32 in [32, 512], or 0 to keep");
  ++b->tuning_version;  // launch shapes are captured in the host-call graph
  StreamBatch& sb = b->sb;
  if (!sb.slots.empty() && (ctas_per_sm != sb.ctas_per_sm || (gate_chunk && gate_chunk != sb.gate_chunk))) {
    sb.ctas_per_sm = ctas_per_sm;
    if (gate_chunk) sb.gate_chunk = gate_chunk;
    int rc = persist_grid(sb, &sb.grid);
    if (rc == VQE_OK) rc = build_queues(b);
    if (rc) return rc;
  }
  if (sweep_threads) {
    for (int mode = 0; mode < 2; ++mode) {
      for (auto& d : b->res_descs[mode]) d.sweep_threads = sweep_threads;
      if (!b->res_descs[mode].empty()) {
        cudaError_t e = cudaMemcpy(b->d_res[mode], b->res_descs[mode].data(),
                                   b->res_descs[mode].size() * sizeof(InstDesc), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
      }
    }
  }
  return VQE_OK;
}

int vqe_batch_get_tuning(vqe_batch_t b, int* ctas_per_sm, int* gate_chunk, int* grid, int64_t* n_tasks) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  if (ctas_per_sm) *ctas_per_sm = b->sb.ctas_per_sm;
  if (gate_chunk) *gate_chunk = b->sb.gate_chunk;
  if (grid) *grid = b->sb.slots.empty() ? 0 : b->sb.grid;
  if (n_tasks) *n_tasks = b->sb.q[1] ? int64_t(b->sb.q[1]->tasks.size()) : 0;
  return VQE_OK;
}

int vqe_batch_set_wait(vqe_batch_t b, int64_t budget_ns, int32_t probe_task) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  if (budget_ns < 1000 || budget_ns > int64_t(600) * 1000000000ll)
    return fail(VQE_ERR_INVALID_ARG, "budget_ns: 1e3 .. 6e11");
  if (probe_task < -1) return fail(VQE_ERR_INVALID_ARG, "probe_task: a task index, or -1");
  ++b->tuning_version;
  b->sb.budget_ns = budget_ns;
  b->sb.probe_task = probe_task;
  return VQE_OK;
}

int vqe_batch_status(vqe_batch_t b, const void* ws, size_t ws_bytes, vqe_stream_t stream) {
  if (!b) return fail(VQE_ERR_INVALID_ARG, "NULL batch");
  const StreamBatch& sb = b->sb;
  if (sb.slots.empty()) return VQE_OK;
  if (!ws || ws_bytes < sb.persist_bytes) return fail(VQE_ERR_WORKSPACE, "workspace smaller than the batch's");
  int status = 0;
  cudaError_t ce = cudaMemcpyAsync(&status, static_cast<const char*>(ws) + sb.counters_off + (sb.slots.size() + 1) * sizeof(int),
                                   sizeof(int), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "status read");
  if (status == 0) return VQE_OK;
  const int t = status - 1;
  const PersistQueue* Q = sb.q[sb.last_queue].get();
  std::string what = "task " + std::to_string(t);
  if (Q && t >= 0 && size_t(t) < Q->tasks.size())
    what += " (instance " + std::to_string(sb.descs[Q->tasks[t].slot].inst) + ")";
  return fail(VQE_ERR_TIMEOUT, "persistent batch: a wait of " + what + " ran out of its " +
                                   std::to_string(sb.budget_ns) + " ns budget; outputs are NaN");
}

void vqe_destroy_batch(vqe_batch_t b) { delete b; }

// Batch plans behind the pointer-array calls, keyed by the instances' handle
// serial numbers; the least recently used plan is dropped beyond kMaxPlans.
namespace {
constexpr size_t kMaxPlans = 16;
struct CachedPlan {
  vqe_batch_t b = nullptr;
  uint64_t last_use = 0;
};
std::mutex g_plan_mu;
std::map<std::vector<uint64_t>, CachedPlan> g_plans;
uint64_t g_plan_clock = 0;

int plan_for(int n, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans, vqe_batch_t* out) {
  *out = nullptr;
  if (n < 1 || !hams || !ans) return fail(VQE_ERR_INVALID_ARG, "bad instance arrays");
  std::vector<uint64_t> key;
  key.reserve(2 * size_t(n));
  for (int i = 0; i < n; ++i) {
    if (!hams[i] || !ans[i]) return fail(VQE_ERR_INVALID_ARG, "NULL handle in instance " + std::to_string(i));
    key.push_back(hams[i]->serial);
    key.push_back(ans[i]->serial);
  }
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    vqe_batch_t b = nullptr;
    int rc = vqe_create_batch(n, hams, ans, &b);
    if (rc) return rc;
    if (g_plans.size() >= kMaxPlans) {
      auto old = g_plans.begin();
      for (auto j = g_plans.begin(); j != g_plans.end(); ++j)
        if (j->second.last_use < old->second.last_use) old = j;
      vqe_destroy_batch(old->second.b);
      g_plans.erase(old);
    }
    it = g_plans.emplace(std::move(key), CachedPlan{b, 0}).first;
  }
  it->second.last_use = ++g_plan_clock;
  *out = it->second.b;
  return VQE_OK;
}

struct PackedLayout {
  int64_t ld = 1;
  size_t theta_off = 0, grad_off = 0, batch_off = 0, total = 0;
};

PackedLayout packed_layout(vqe_batch_t b, bool with_grad) {
  PackedLayout L;
  L.ld = std::max<int64_t>(b->max_params, 1);
  const size_t mat = align256(size_t(b->n_inst) * size_t(L.ld) * 8);
  L.theta_off = 0;
  L.grad_off = mat;
  L.batch_off = mat + (with_grad ? mat : 0);
  L.total = L.batch_off + vqe_batch_workspace_bytes(b, with_grad);
  return L;
}

int batched_run(int n, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans, const double* const* theta,
                double* energies, double* const* grads, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (!theta || !energies) return fail(VQE_ERR_INVALID_ARG, "NULL theta array or energies pointer");
  vqe_batch_t b = nullptr;
  int rc = plan_for(n, hams, ans, &b);
  if (rc) return rc;
  const bool with_grad = grads != nullptr;
  for (int i = 0; i < n; ++i) {
    if (ans[i]->M > 0 && !theta[i]) return fail(VQE_ERR_INVALID_ARG, "NULL theta pointer, instance " + std::to_string(i));
    if (with_grad && ans[i]->M > 0 && !grads[i])
      return fail(VQE_ERR_INVALID_ARG, "NULL gradient pointer, instance " + std::to_string(i));
  }
  const PackedLayout L = packed_layout(b, with_grad);
  if ((rc = check_ws(ws, ws_bytes, L.total))) return rc;
  char* base = static_cast<char*>(ws);
  double* d_theta = reinterpret_cast<double*>(base + L.theta_off);
  double* d_grad = with_grad ? reinterpret_cast<double*>(base + L.grad_off) : nullptr;
  auto rows = [&](bool pack) -> int {
    for (int r0 = 0; r0 < n; r0 += vqe::kRowPtrs) {
      vqe::RowPtrs rp;
      std::memset(&rp, 0, sizeof(rp));
      rp.base = r0;
      rp.count = std::min(vqe::kRowPtrs, n - r0);
      int max_len = 0;
      for (int r = 0; r < rp.count; ++r) {
        rp.p[r] = pack ? theta[r0 + r] : grads[r0 + r];
        rp.len[r] = ans[r0 + r]->M;
        max_len = std::max(max_len, rp.len[r]);
      }
      cudaError_t ce = pack ? vqe::pack_rows(rp, d_theta, L.ld, max_len, stream)
                            : vqe::unpack_rows(rp, d_grad, L.ld, max_len, stream);
      if (ce != cudaSuccess) return cuda_fail(ce, pack ? "theta gather" : "gradient scatter");
    }
    return VQE_OK;
  };
  if ((rc = rows(true))) return rc;
  rc = batch_run(b, d_theta, L.ld, energies, d_grad, L.ld, base + L.batch_off, ws_bytes - L.batch_off, stream);
  if (rc) return rc;
  return with_grad ? rows(false) : VQE_OK;
}
}  // namespace

static void purge_plans(uint64_t serial) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (std::find(it->first.begin(), it->first.end(), serial) != it->first.end()) {
      vqe_destroy_batch(it->second.b);
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

size_t vqe_batched_workspace_bytes(int n_inst, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans,
                                   int with_grad) {
  vqe_batch_t b = nullptr;
  if (plan_for(n_inst, hams, ans, &b)) return 0;
  return packed_layout(b, with_grad != 0).total;
}

int vqe_energy_batched(int n_inst, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans,
                       const double* const* theta_dev, double* energies_dev, void* ws, size_t ws_bytes,
                       vqe_stream_t stream) {
  return batched_run(n_inst, hams, ans, theta_dev, energies_dev, nullptr, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

int vqe_energy_grad_batched(int n_inst, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ans,
                            const double* const* theta_dev, double* energies_dev, double* const* grads_dev,
                            void* ws, size_t ws_bytes, vqe_stream_t stream) {
  if (!grads_dev) return fail(VQE_ERR_INVALID_ARG, "NULL gradient array");
  return batched_run(n_inst, hams, ans, theta_dev, energies_dev, grads_dev, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

int vqe_work_counts(vqe_hamiltonian_t h, vqe_ansatz_t a, int64_t* n_pairs, int64_t* n_entries,
                    double* extra_adds) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  if (n_pairs) *n_pairs = int64_t(a->pairs.size());
  if (n_entries) *n_entries = e->nnz;
  if (extra_adds) *extra_adds = e->extra_adds;
  return VQE_OK;
}

int vqe_work_estimate(vqe_hamiltonian_t h, vqe_ansatz_t a, int with_grad, double* flops, double* bytes) {
  int rc = check_pair(h, a);
  if (rc) return rc;
  const auto* e = get_ell(h, a, &rc);
  if (!e) return rc;
  const double P = double(a->pairs.size());
  const double D = double(a->sector.size());
  // forward rotation 6 flops/pair; H psi: 2 per connected (output, group) plus
  // the table adds, 2 per output for <psi|lambda>; adjoint 16 flops/pair.
  double f = 6.0 * P + 2.0 * double(e->nnz) + e->extra_adds + 2.0 * D;
  // compulsory state traffic (real amplitudes): 4 amplitude moves per pair
  // forward, psi read + lambda written once on the sector, 8 moves per pair adjoint.
  double by = 32.0 * P + 16.0 * D;
  if (with_grad) {
    f += 16.0 * P;
    by += 64.0 * P;
  }
  if (flops) *flops = f;
  if (bytes) *bytes = by;
  return VQE_OK;
}

}  // extern "C"
