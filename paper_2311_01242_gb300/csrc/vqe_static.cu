// Energy + gradient without any device allocation: the streaming kernels run
// on a fixed scratch array that lives in the library's own device memory.
//
// Who needs this: a caller that is not allowed to call cudaMalloc, for
// example code running inside another framework whose allocator owns the
// device memory (raw allocations would bypass its pool and its accounting),
// or a service with a fixed device-memory budget that is set when the process
// starts. Such a caller still passes theta, the energy and the gradient
// buffers; the library provides the scratch.
//
// The scratch is one file-scope __device__ array of VQE_NOALLOC_SCRATCH_BYTES
// (16 MiB). Every GPU that loads the library holds it until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and keeps it; that first call should come before any
// stream capture. All calls share the array and it keeps the previous call's
// contents: every scratch entry a call reads is written earlier in the same
// call (the state's sector entries, H psi, the cos/sin table and every
// reduction partial), so nothing needs clearing. Calls whose work overlaps on
// the GPU (two streams, or two threads) race on the array.
//
// H psi takes the fastest path that needs no new tables: when an earlier call
// (vqe_workspace_bytes, vqe_energy_grad, a batch) already built the string or
// connectivity tables of this (Hamiltonian, sector) pair, they are used, with
// the same kernels and results as vqe_energy_grad; otherwise every output
// scans all X-mask groups. The scratch holds only the vectors that path uses.
#include <atomic>
#include <string>

#include <cuda_runtime.h>

#include "../../include/vqe.h"
#include "vqe_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(VQE_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices];

}  // namespace

extern "C" int vqe_energy_grad_noalloc(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta_dev,
                                       double* energy_dev, double* grad_dev, vqe_stream_t stream) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess)
    return vqe::set_error(VQE_ERR_CUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(ce)).c_str());
  if (dev < 0 || dev >= kMaxDevices) return vqe::set_error(VQE_ERR_UNSUPPORTED, "device index above 63");
  void* base = g_scratch_addr[dev].load();
  if (base == nullptr) {
    ce = cudaGetSymbolAddress(&base, g_scratch);
    if (ce != cudaSuccess || base == nullptr)
      return vqe::set_error(VQE_ERR_CUDA,
                            (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce)).c_str());
    g_scratch_addr[dev].store(base);
  }
  const bool with_grad = grad_dev != nullptr;
  vqe::InstDesc d;
  vqe::StreamPlan sp;
  bool real = true;
  size_t off[7], need = 0;
  int rc = vqe::prepare_noalloc(h, a, with_grad, kScratchBytes, &d, &sp, &real, off, &need);
  if (rc != VQE_OK) return rc;
  if ((theta_dev == nullptr && d.M > 0) || energy_dev == nullptr)
    return vqe::set_error(VQE_ERR_INVALID_ARG, "NULL device pointer");
  if (need > kScratchBytes)
    return vqe::set_error(VQE_ERR_INVALID_ARG,
                          ("instance needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                           std::to_string(kScratchBytes) + " (use vqe_energy_grad with a workspace)")
                              .c_str());
  char* b = static_cast<char*>(base);
  vqe::StreamBuffers buf;
  buf.psi = b + off[0];
  buf.lam = b + off[1];
  if (sp.use_str) {
    buf.psi_am = b + off[2];
    buf.lam_am = b + off[3];
  }
  buf.cs = reinterpret_cast<double2*>(b + off[4]);
  buf.epart = reinterpret_cast<double*>(b + off[5]);
  buf.gpart = reinterpret_cast<double*>(b + off[6]);
  ce = vqe::stream_energy_grad(d, sp, buf, real, with_grad, theta_dev, energy_dev, grad_dev,
                               static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess)
    return vqe::set_error(VQE_ERR_CUDA, (std::string("launch: ") + cudaGetErrorString(ce)).c_str());
  return VQE_OK;
}
