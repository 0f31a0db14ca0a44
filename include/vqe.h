/*
 * vqe.h - C ABI of the GB300 state-vector VQE library (libvqe).
 *
 * The library evaluates the variational energy of Eq. 1,
 *     E(theta) = <HF| U(theta)^dagger H U(theta) |HF>,
 * and its gradient dE/dtheta_k, where
 *   - H is the qubit Hamiltonian: a real-weighted sum of Pauli strings, as the
 *     Jordan-Wigner mapping of Eq. 2 produces (Sec. 2.1.1);
 *   - U(theta) = U_M ... U_1, U_k = exp(theta_k (T_k - T_k^dagger)), one
 *     rotation per single or double excitation of the UCCSD ansatz (Sec. 2.1.2);
 *   - |HF> is the Hartree-Fock reference bitstring of Eq. 1.
 * Around that evaluation it also provides ADAPT-VQE's pool screening (Sec.
 * 2.1.1), pUCCD's hard-core boson form and generalised excitation lists
 * (Sec. 2.1.2), and the frozen-core folding of Eq. 3 (Sec. 2.1.3).
 *
 * Conventions shared by every call:
 *   - Bit q of a basis index is qubit q; qubit q is spin orbital q (spatial
 *     orbital q/2, alpha when q is even, beta when odd).
 *   - A Pauli term is (x_mask, z_mask, coef): X where only x has bit q, Z where
 *     only z has it, Y where both do, P|k> = i^{|x&z|} (-1)^{|k&z|} |k ^ x>.
 *   - Excitations are int32 quadruples: {i, a, -1, -1} is the single
 *     T = a+_a a_i; {i, j, a, b} is the double T = a+_a a+_b a_j a_i. Ladder
 *     operators carry the sign (-1)^(occupied orbitals below their index).
 *   - theta_k is the full rotation angle (no factor 1/2).
 *   - n_qubits is 1..32.
 *
 * Memory ownership: create calls copy their host inputs and own device copies
 * of the derived tables until the matching destroy call. theta, energies,
 * gradients and the workspace are caller-owned device memory. One allocation
 * happens outside the create calls: the first use of a (Hamiltonian, sector)
 * pair (vqe_workspace_bytes, vqe_work_counts, vqe_create_batch, or the first
 * compute call with that pair) builds the pair's connectivity or string tables,
 * synchronously, and the pair keeps them until the Hamiltonian is destroyed.
 * Under VQE_FLAG_PERSISTENT_SWEEPS the first streaming evaluation of an ansatz
 * (or vqe_workspace_bytes with it) also builds the task queues of its
 * persistent gate sweeps. After that the compute calls allocate nothing, so
 * make those first calls before any stream capture. Every compute call is asynchronous on the given
 * stream (a cudaStream_t; NULL is the legacy default stream) except where
 * noted.
 *
 * Errors: every int-returning call returns VQE_OK (0) or a VQE_ERR_* code and
 * sets a thread-local message readable with vqe_last_error(). Invalid
 * arguments are rejected before anything is enqueued.
 */
#ifndef VQE_H
#define VQE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  VQE_OK = 0,
  VQE_ERR_INVALID_ARG = 1,  /* bad size, mask bit >= n, index clash, NaN ... */
  VQE_ERR_WORKSPACE = 2,    /* workspace pointer NULL/misaligned or too small */
  VQE_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has details) */
  VQE_ERR_TIMEOUT = 4,      /* a bounded device wait gave up (status word set) */
  VQE_ERR_NOT_REAL = 5,     /* a Pauli coefficient of the mapped H is not real */
  VQE_ERR_UNSUPPORTED = 6,  /* valid request outside what this build implements */
  VQE_ERR_NO_MEMORY = 7     /* create-time allocation failed */
};

typedef struct vqe_hamiltonian_s* vqe_hamiltonian_t;
typedef struct vqe_ansatz_s* vqe_ansatz_t;
typedef struct vqe_batch_s* vqe_batch_t;
typedef void* vqe_stream_t;

/* Library version as 10000*major + 100*minor + patch. */
int vqe_version(void);

/*
 * Process-wide switches, for verification only (0 = normal operation):
 *   VQE_FLAG_FORCE_COMPLEX   evaluate E and g with complex amplitudes and full
 *                            complex coefficients instead of the real path;
 *   VQE_FLAG_FORCE_STREAMING never use the shared-memory-resident kernel;
 *   VQE_FLAG_NO_CLUSTER      run each resident instance on one CTA instead of
 *                            a cluster of two;
 *   VQE_FLAG_FP64_SWEEPS     run the resident kernel's gate sweeps in FP64
 *                            instead of 64-bit fixed point (H psi, the energy
 *                            and every streaming kernel are FP64 either way);
 *   VQE_FLAG_NO_STRINGS      streaming H psi by connectivity rows (or a scan of
 *                            all groups) instead of alpha/beta strings;
 *   VQE_FLAG_PERSISTENT_SWEEPS streaming gate sweeps of a single instance as
 *                            one persistent launch per sweep (a task queue)
 *                            instead of one launch per gate; the same bits as
 *                            one launch per gate without the kept forward
 *                            outputs (below), and slower on the GPUs measured
 *                            (kept for comparison);
 *   VQE_FLAG_NO_PHI_STORE    real instances of 6,000,000 sector states or more
 *                            normally keep the forward sweep's outputs of every
 *                            amplitude pair in the workspace (16 bytes per pair)
 *                            and run the reverse sweep on them and lambda alone;
 *                            with this flag (or VQE_FLAG_PERSISTENT_SWEEPS) the
 *                            reverse sweep un-applies each gate to psi instead.
 *                            The gradients agree to rounding; psi, lambda and the
 *                            energy are the same bits either way.
 * Returns the previous flags. Not thread-safe against concurrent compute calls.
 */
enum {
  VQE_FLAG_FORCE_COMPLEX = 1,
  VQE_FLAG_FORCE_STREAMING = 2,
  VQE_FLAG_NO_CLUSTER = 4,
  VQE_FLAG_FP64_SWEEPS = 8,
  VQE_FLAG_NO_STRINGS = 16,
  VQE_FLAG_PERSISTENT_SWEEPS = 32,
  VQE_FLAG_NO_PHI_STORE = 64
};
int vqe_set_flags(int flags);

/* Message of the last failed call on this thread ("" if none). */
const char* vqe_last_error(void);

/*
 * Jordan-Wigner mapping of Eq. 2 (Sec. 2.1.1), host only, synchronous.
 *   H = c0 + sum_{pq,s} h[p*n_s+q] a+_{ps} a_{qs}
 *          + 1/2 sum_{pqrs,s,t} eri[((p*n_s+q)*n_s+r)*n_s+s] a+_{ps} a+_{rt} a_{st} a_{qs}
 * with eri in chemists' order (pq|rs) and spin orbital (p, s) = qubit 2p+s.
 * Terms with equal masks are merged; |coef| < drop_tol are dropped. Output is
 * sorted by (x_mask, z_mask). If capacity is smaller than the term count,
 * nothing is written to the arrays, *n_out receives the count and the call
 * returns VQE_ERR_INVALID_ARG (query with capacity 0 and NULL arrays).
 * Returns VQE_ERR_NOT_REAL if the mapped coefficients are not real (the
 * integrals were not symmetric).
 */
int vqe_jordan_wigner(int n_spatial, const double* h, const double* eri, double c0,
                      double drop_tol, int64_t capacity, uint64_t* x_out,
                      uint64_t* z_out, double* c_out, int64_t* n_out);

/*
 * Frozen-core folding (Sec. 2.1.3, Eq. 3), host only, synchronous: the
 * integrals of a smaller problem on the active spatial orbitals, with the
 * frozen ones doubly occupied in every determinant. Same h, eri layout as
 * vqe_jordan_wigner; frozen[n_frozen] and active[n_active] list distinct
 * orbitals < n_spatial (active in the order of the new problem).
 *   h_out[x*n_active+y] = h[p][q] + sum_{c frozen} (2 (pq|cc) - (pc|cq)),
 *       p = active[x], q = active[y];
 *   eri_out = eri on the active orbitals;
 *   *c0_out = c0 + sum_{c frozen} 2 h_cc + sum_{c,d frozen} (2 (cc|dd) - (cd|dc)).
 * Eq. 3's constant lists only the one-body core sum; the core-core two-body
 * energy is part of it as well (without it the folded energies shift by a
 * constant). Returns VQE_ERR_INVALID_ARG for bad counts, indices or NULLs.
 */
int vqe_fold_frozen(int n_spatial, const double* h, const double* eri, double c0, int n_frozen,
                    const int32_t* frozen, int n_active, const int32_t* active, double* h_out,
                    double* eri_out, double* c0_out);

/*
 * pUCCD's hard-core boson form (Sec. 2.1.2, pUCCD: half the qubits of the
 * other UCC ansatze): the block of Eq. 2 on seniority-zero determinants (every
 * spatial orbital empty or doubly occupied) as a Pauli sum on n_spatial qubits,
 * qubit p set when orbital p holds a pair. With the same h, eri layout as
 * vqe_jordan_wigner and pair occupations n_p = (1 - Z_p)/2,
 *   H = c0 + sum_p (2 h_pp + (pp|pp)) n_p
 *          + sum_{p<q} 2 [2 (pp|qq) - (pq|qp)] n_p n_q
 *          + sum_{p<q} (pq|pq) (X_p X_q + Y_p Y_q) / 2,
 * exact on that block for real orbitals (pair moves p -> q carry sign +1 in the
 * interleaved Jordan-Wigner order, so no Z strings appear). n_spatial 1..32;
 * output, capacity and errors as vqe_jordan_wigner (terms sorted by (x, z)).
 */
int vqe_hcb_hamiltonian(int n_spatial, const double* h, const double* eri, double c0,
                        double drop_tol, int64_t capacity, uint64_t* x_masks,
                        uint64_t* z_masks, double* coefs, int64_t* n_out);

/*
 * Qubit Hamiltonian from host arrays of n_terms Pauli terms (Eq. 1's H after
 * the mapping of Sec. 2.1.1). Equal (x, z) are merged, |coef| < drop_tol
 * dropped, and terms grouped by x_mask. Each group's terms are folded into
 * per-pattern coefficient tables: for the pattern u of the source index on
 * the group's X bits (up to 4 bits), and the terms' Z bits outside them.
 * The Hamiltonian is flagged real when every folded coefficient
 * c * i^{|x&z|} is real (informational: the energy and gradient kernels use
 * real amplitudes either way, because psi(theta) is real for every theta and
 * only the real parts of the folded coefficients enter E and g).
 * Synchronous; allocates device memory.
 */
int vqe_create_hamiltonian(int n_qubits, int64_t n_terms, const uint64_t* x_masks,
                           const uint64_t* z_masks, const double* coefs,
                           double drop_tol, vqe_hamiltonian_t* out);

/* Counts after merging/dropping; is_real as described above. Any out may be NULL. */
int vqe_hamiltonian_info(vqe_hamiltonian_t h, int* n_qubits, int64_t* n_terms,
                         int64_t* n_groups, int* is_real);

/*
 * The kept terms (after merging and dropping) in the order vqe_set_coefs
 * expects: sorted by (x_mask, z_mask), n_terms of vqe_hamiltonian_info each.
 * coefs are the create-time values (vqe_set_coefs does not update them). Any
 * output may be NULL. Host only.
 */
int vqe_hamiltonian_terms(vqe_hamiltonian_t h, uint64_t* x_masks, uint64_t* z_masks,
                          double* coefs);

/*
 * New coefficients for the same Pauli structure: the Hamiltonian at another
 * point r of a scan (Sec. 2.1.1's mapping applied to the integrals at r gives
 * the same strings with new weights). coefs_dev: n_terms device doubles in the
 * kept-term order above. The group tables are refolded on the device (each
 * table entry is a fixed combination of term coefficients with weights
 * +-1, +-2, +-4 times 1 or i), giving the same bits as vqe_create_hamiltonian
 * with these coefficients when it keeps the same terms. The term set, the
 * grouping and the connectivity tables do not change: a coefficient that is
 * now below the create-time drop tolerance is kept, and a string that was
 * dropped at create time cannot come back. Asynchronous on stream; every
 * later call that uses h (on any stream, including batches and captured
 * graphs holding h) reads the new tables once this work has run, so order
 * the streams accordingly. Allocates nothing; graph-capturable.
 */
int vqe_set_coefs(vqe_hamiltonian_t h, const double* coefs_dev, vqe_stream_t stream);

void vqe_destroy_hamiltonian(vqe_hamiltonian_t h);

/*
 * Ansatz U(theta) (Sec. 2.1.2) on n_qubits from the reference bitstring
 * hf_bits and n_exc excitations (host array of 4*n_exc int32, see above).
 * Indices must lie in [0, n_qubits) and be distinct within an excitation.
 * The reachable sector is fixed here: popcount(hf_bits) electrons, and, when
 * every excitation conserves the alpha/beta counts, the reference's
 * (N_alpha, N_beta). Amplitudes outside it are exactly zero for every theta,
 * and no energy or gradient depends on them, so kernels touch only the
 * sector. Synchronous; allocates device memory.
 */
int vqe_create_ansatz(int n_qubits, uint64_t hf_bits, int32_t n_exc,
                      const int32_t* excitations, vqe_ansatz_t* out);

/*
 * pUCCD ansatz in the hard-core boson form (Sec. 2.1.2, pUCCD) for a
 * Hamiltonian from vqe_hcb_hamiltonian: n_exc pair excitations
 * pairs[2m] = i -> pairs[2m+1] = a, each U_m = exp(theta_m (b+_a b_i - b+_i b_a))
 * with no parity sign (hard-core bosons on different qubits commute);
 * hf_bits: the doubly occupied orbitals of the reference. The state lives in
 * the sector of popcount(hf_bits) occupied qubits. The handle works with every
 * evaluation call (energy, gradient, batches, screening). Errors as
 * vqe_create_ansatz (distinct qubits < n_qubits <= 32).
 */
int vqe_create_ansatz_hcb(int n_qubits, uint64_t hf_bits, int32_t n_exc, const int32_t* pairs,
                          vqe_ansatz_t* out);

/* Sector dimension, parameter count and number of (gate, amplitude-pair) units. */
int vqe_ansatz_info(vqe_ansatz_t a, int* n_qubits, int32_t* n_params,
                    int64_t* sector_dim, int64_t* n_pairs);

void vqe_destroy_ansatz(vqe_ansatz_t a);

/*
 * Bytes of device workspace a call needs for this pair, by mode:
 *   VQE_WS_ENERGY (vqe_energy), VQE_WS_GRAD (vqe_energy_grad, vqe_state),
 *   VQE_WS_COMPLEX (vqe_apply_hamiltonian, or any call while
 *   VQE_FLAG_FORCE_COMPLEX is set); modes may be OR-ed.
 * It holds two state vectors (|psi> or |phi>, and |lambda>) compressed to the
 * ansatz's sector (entry r is the amplitude of the r-th sector state in
 * increasing order), their copies in alpha-major order (string-driven H psi),
 * and reduction partials; with VQE_WS_GRAD and real amplitudes, for sectors of
 * 6,000,000 states or more, also the forward sweep's outputs of every
 * (gate, amplitude pair) unit (16 bytes each: 4.5 GB at 30 qubits with 512
 * angles), which the reverse sweep reads (see VQE_FLAG_NO_PHI_STORE). The
 * workspace must be 256-byte aligned.
 * The first call for a (Hamiltonian, sector) pair builds that pair's
 * connectivity table (synchronous, allocates); call it before any stream
 * capture. Returns 0 and sets the error message on failure.
 */
enum { VQE_WS_ENERGY = 0, VQE_WS_GRAD = 1, VQE_WS_COMPLEX = 2 };
size_t vqe_workspace_bytes(vqe_hamiltonian_t h, vqe_ansatz_t a, int mode);

/*
 * E(theta) of Eq. 1 into energy_dev[0]. theta_dev: n_params device doubles.
 */
int vqe_energy(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta_dev,
               double* energy_dev, void* workspace, size_t workspace_bytes,
               vqe_stream_t stream);

/*
 * E(theta) and grad_dev[k] = dE/dtheta_k by one forward sweep, one H|psi>, and
 * one reverse (adjoint) sweep that un-applies each gate to |lambda> = H|psi>
 * while reducing g_k = 2 Re <lambda| T_k - T_k^dagger |phi_k>, phi_k being the
 * state after gate k: un-applied from the final psi, or, for large real
 * sectors, read from the forward sweep's kept outputs (vqe_workspace_bytes).
 */
int vqe_energy_grad(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta_dev,
                    double* energy_dev, double* grad_dev, void* workspace,
                    size_t workspace_bytes, vqe_stream_t stream);

/*
 * psi(theta) = U(theta)|HF> as a full 2^n complex128 vector (interleaved
 * re, im) in psi_out_dev; every entry, inside the sector or not, is written.
 */
int vqe_state(vqe_ansatz_t a, vqe_hamiltonian_t h, const double* theta_dev,
              double* psi_out_dev, void* workspace, size_t workspace_bytes,
              vqe_stream_t stream);

/*
 * lambda = H psi restricted to the ansatz's sector, for a caller-given full
 * 2^n complex128 vector psi_dev that vanishes outside the sector. lam_out_dev
 * (2^n complex128) receives lambda on the sector and 0 elsewhere;
 * energy_dev[0] receives Re <psi|H|psi>.
 */
int vqe_apply_hamiltonian(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* psi_dev,
                          double* lam_out_dev, double* energy_dev, void* workspace,
                          size_t workspace_bytes, vqe_stream_t stream);

/*
 * lambda = H psi on the ansatz's sector with REAL amplitudes compressed to the
 * sector: psi_dev and lam_dev hold D = sector_dim (vqe_ansatz_info) device
 * doubles, entry r the amplitude of the r-th sector state in increasing order
 * of basis index; energy_dev[0] receives <psi|lambda>. This runs the same
 * real-amplitude H psi kernels as vqe_energy and vqe_energy_grad (string-driven
 * for spin sectors, connectivity rows or a scan of all groups otherwise), which
 * keep the real part of each folded coefficient c * i^{|x&z|}; for the real
 * Hamiltonians of Eq. 2 that is the whole of H. psi_dev and lam_dev must not
 * overlap. workspace: vqe_workspace_bytes(h, a, VQE_WS_ENERGY) bytes,
 * 256-byte aligned. Asynchronous on `stream`.
 */
int vqe_apply_hamiltonian_sector(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* psi_dev,
                                 double* lam_dev, double* energy_dev, void* workspace,
                                 size_t workspace_bytes, vqe_stream_t stream);

/*
 * ADAPT-VQE operator screening (Sec. 2.1.1, ADAPT-VQE: the ansatz grows one pool
 * operator at a time, chosen and stopped by the energy gradients with respect
 * to the pool). For psi = U(theta)|HF> of ansatz a and lambda = H psi, writes
 *   pool_grad_dev[j] = 2 Re <lambda| T_j - T_j^dagger |psi>,   j < n_pool,
 * the derivative of E at angle 0 of pool operator j appended after U(theta),
 * and energy_dev[0] = E(theta).
 *   pool: an ansatz handle whose excitation list is the operator pool (its
 *     angles are not used); it must have a's qubit count and sector (the same
 *     electron count, and the same alpha/beta counts when a is spin-conserving),
 *     else VQE_ERR_INVALID_ARG. Operators may repeat those of a.
 *   theta_dev: a's n_params angles (may be NULL when a has none, the empty
 *     starting ansatz of ADAPT).
 *   pool_grad_dev: device, n_pool doubles, caller-owned (may be NULL when the
 *     pool is empty).
 *   workspace: vqe_pool_workspace_bytes(h, a, pool) bytes, 256-byte aligned
 *     (the sector-compressed psi and lambda, a copy of both side by side, and
 *     one partial sum per started 4096 pairs of each operator); a smaller or
 *     misaligned workspace returns VQE_ERR_WORKSPACE before any launch.
 * Asynchronous on `stream`; allocates nothing, so it can be captured in a CUDA
 * graph. Deterministic: fixed reduction order, independent of the grid size.
 */
size_t vqe_pool_workspace_bytes(vqe_hamiltonian_t h, vqe_ansatz_t a, vqe_ansatz_t pool);
int vqe_pool_gradients(vqe_hamiltonian_t h, vqe_ansatz_t a, vqe_ansatz_t pool,
                       const double* theta_dev, double* energy_dev, double* pool_grad_dev,
                       void* workspace, size_t workspace_bytes, vqe_stream_t stream);

/*
 * A batch of independent instances (the paper runs hundreds of independent
 * simulation jobs over geometries and molecules, abstract and Sec. 4).
 * Instances whose sector and tables fit shared memory run in one resident
 * launch (a CTA pair each). All other instances run in ONE persistent launch:
 * a device work queue of tasks (per instance: HF init, each gate's rotation on
 * a range of pairs, H psi on a range of output strings or rows, the energy's
 * partial sums, each gate's adjoint step and gradient partials), taken in a
 * fixed list-scheduled order by a grid sized to the device, where a task waits
 * (bounded in time, see vqe_batch_set_wait) only for the earlier tasks of its
 * own instance; a small finalising launch then sums the partials. Instances
 * with a gate or sector of more than 262,144 pairs or states are evaluated
 * after it, one by one. Results equal vqe_energy_grad's on each instance bit
 * for bit. hams/ansatze: n_inst handles (they may repeat) that must outlive
 * the batch. Synchronous; allocates the batch's device descriptors and queues.
 */
int vqe_create_batch(int n_inst, const vqe_hamiltonian_t* hams,
                     const vqe_ansatz_t* ansatze, vqe_batch_t* out);

/* Largest n_params over the batch (the minimum leading dimension of theta). */
int32_t vqe_batch_max_params(vqe_batch_t b);

size_t vqe_batch_workspace_bytes(vqe_batch_t b, int with_grad);

/*
 * Energies (and gradients when grads_dev != NULL) of every instance.
 * theta_dev: row i holds instance i's n_params angles at theta_dev + i*ld_theta.
 * grads_dev: row i at grads_dev + i*ld_grad. energies_dev: n_inst doubles.
 */
int vqe_batch_energy_grad(vqe_batch_t b, const double* theta_dev, int64_t ld_theta,
                          double* energies_dev, double* grads_dev, int64_t ld_grad,
                          void* workspace, size_t workspace_bytes, vqe_stream_t stream);

/*
 * Same as vqe_batch_energy_grad with HOST arrays: copies theta host->device,
 * runs, copies energies and gradients device->host, and synchronises the
 * stream before returning. Uses the workspace for the staged copies too
 * (vqe_batch_host_workspace_bytes). The first call with a given set of host
 * buffers, workspace, flags and tuning runs the copies and launches directly
 * and captures them in a CUDA graph (on a private stream; nothing runs twice);
 * later calls with the same set replay that graph, reading the buffers'
 * current contents. Pageable host memory cannot be captured: such calls always
 * run directly. Called while `stream` is being captured, it only enqueues the
 * work (no synchronisation). One graph per batch (a new set of buffers
 * replaces it); calls on one batch handle from several threads are serialised.
 */
size_t vqe_batch_host_workspace_bytes(vqe_batch_t b, int with_grad);
int vqe_batch_energy_grad_host(vqe_batch_t b, const double* theta_host, int64_t ld_theta,
                               double* energies_host, double* grads_host, int64_t ld_grad,
                               void* workspace, size_t workspace_bytes, vqe_stream_t stream);

/*
 * Launch shape of a batch (used by the autotuner): CTAs per SM of the
 * persistent launch (1..16; 0 = as many as fit), amplitude pairs per gate task
 * of the persistent launch (a multiple of 256; 0 keeps the current value,
 * initially 1024), and threads that run the gate sweeps of shared-memory-
 * resident instances (a multiple of 32 in [32, 512]; 0 keeps the current
 * value). Rebuilds the task queues; synchronous. Results do not depend on any
 * of them. vqe_batch_get_tuning reports the current values, the persistent
 * grid and the task count of the gradient queue (any output may be NULL).
 */
int vqe_batch_set_tuning(vqe_batch_t b, int ctas_per_sm, int gate_chunk, int sweep_threads);
int vqe_batch_get_tuning(vqe_batch_t b, int* ctas_per_sm, int* gate_chunk, int* grid, int64_t* n_tasks);

/*
 * Bounded waits of the persistent launch. A CTA whose task depends on
 * unfinished tasks of the same instance polls that instance's progress counter
 * for at most budget_ns nanoseconds (default 2e9; 1e3 .. 6e11 accepted), then
 * writes its task's index + 1 into the status word in the workspace, takes no
 * more tasks and returns; the other CTAs stop at their next task or wait, and
 * every energy and gradient of the persistent instances is written as NaN.
 * vqe_batch_energy_grad_host then returns VQE_ERR_TIMEOUT; after the device
 * call, vqe_batch_status does. probe_task >= 0 makes that task of the queue
 * wait for a count that no task reaches, so its wait runs out (a check of the
 * timeout path that stops no GPU); -1 for normal operation.
 */
int vqe_batch_set_wait(vqe_batch_t b, int64_t budget_ns, int32_t probe_task);

/*
 * Status of the last persistent launch that used `workspace` (the batch's
 * workspace as passed to vqe_batch_energy_grad): synchronises `stream`, reads
 * the status word, and returns VQE_OK or VQE_ERR_TIMEOUT (the message names the
 * task and instance whose wait ran out).
 */
int vqe_batch_status(vqe_batch_t b, const void* workspace, size_t workspace_bytes, vqe_stream_t stream);

void vqe_destroy_batch(vqe_batch_t b);

/*
 * The batched calls by instance list, without a batch handle: instance i is
 * (hams[i], ansatze[i]) with its angles at theta_dev[i] (n_params_i device
 * doubles) and, for the gradient, its output at grads_dev[i]. theta_dev and
 * grads_dev are HOST arrays of n_inst device pointers; energies_dev holds
 * n_inst device doubles. The library keeps a batch plan per instance list
 * (keyed by the handles, at most 16 plans, least recently used dropped; a
 * destroyed handle drops the plans that use it). The plan is built by
 * vqe_batched_workspace_bytes, or by the first compute call for that list
 * (synchronous, allocates); later calls with the same list allocate nothing
 * and can be captured in a CUDA graph. The angles are gathered into the
 * workspace and the gradients scattered back by two small kernels around the
 * batch's own launches. Results equal vqe_batch_energy_grad's bit for bit.
 * vqe_batched_workspace_bytes returns 0 and sets the error message on failure.
 */
size_t vqe_batched_workspace_bytes(int n_inst, const vqe_hamiltonian_t* hams,
                                   const vqe_ansatz_t* ansatze, int with_grad);
int vqe_energy_batched(int n_inst, const vqe_hamiltonian_t* hams, const vqe_ansatz_t* ansatze,
                       const double* const* theta_dev, double* energies_dev,
                       void* workspace, size_t workspace_bytes, vqe_stream_t stream);
int vqe_energy_grad_batched(int n_inst, const vqe_hamiltonian_t* hams,
                            const vqe_ansatz_t* ansatze, const double* const* theta_dev,
                            double* energies_dev, double* const* grads_dev,
                            void* workspace, size_t workspace_bytes, vqe_stream_t stream);

/*
 * Learned warm start: a small network that predicts the UCCSD angles at a new
 * geometry from angles the VQE itself converged to along a bond-stretch scan
 * (the paper scans bond lengths, Sec. 3.1, and starts each VQE from the
 * Hartree-Fock state; the network is not from the paper). Architecture:
 * n_in -> n_hidden -> n_hidden -> n_out, SiLU after the first two layers, BF16
 * weights and BF16 GEMM operands on the tensor cores with FP32 accumulation,
 * FP32 biases, Adam on FP32 master weights.
 * Parameters are one FP32 array (length vqe_mlp_param_count) laid out as
 *   W1 [n_hidden x Ip], b1 [n_hidden], W2 [n_hidden x n_hidden], b2 [n_hidden],
 *   W3 [Op x n_hidden], b3 [Op],
 * Ip = n_in rounded up to 16, Op = n_out rounded up to 16, padding zero; the
 * BF16 copy (uint16 bit patterns) has the same layout. x: [batch x n_in] FP32
 * row-major; target and y: [batch x n_out] FP32 row-major. n_hidden must be a
 * multiple of 16. All device pointers; asynchronous on `stream`.
 * BF16 rounding points: x, both hidden activations, the output gradient and
 * both pre-activation gradients; loss = mean over batch and outputs of
 * (y - target)^2.
 */
int64_t vqe_mlp_param_count(int n_in, int n_hidden, int n_out);
size_t vqe_mlp_workspace_bytes(int batch, int n_in, int n_hidden, int n_out);
/* dst[i] = bf16(src[i]) (round to nearest even) for i < n. */
int vqe_mlp_to_bf16(int64_t n, const float* src, uint16_t* dst, vqe_stream_t stream);
/* y = network(x). */
int vqe_mlp_forward(int batch, int n_in, int n_hidden, int n_out, const float* x, const float* params,
                    const uint16_t* params_bf16, float* y, void* workspace, size_t workspace_bytes,
                    vqe_stream_t stream);
/* loss[0] and the full parameter gradient (same layout as params). */
int vqe_mlp_loss_grad(int batch, int n_in, int n_hidden, int n_out, const float* x, const float* target,
                      const float* params, const uint16_t* params_bf16, float* grads, float* loss,
                      void* workspace, size_t workspace_bytes, vqe_stream_t stream);
/* One bias-corrected Adam step on params, refreshing params_bf16. step_dev is a
 * device int holding this update's 1-based step number; it is incremented on
 * the device afterwards, so a captured training step can be replayed. */
int vqe_mlp_adam(int64_t n, float* params, const float* grads, float* m, float* v, int* step_dev, float lr,
                 float beta1, float beta2, float eps, uint16_t* params_bf16, vqe_stream_t stream);

/*
 * Energy (and gradient when grad_dev != NULL) with no device allocation at all.
 * The paper has no counterpart; this exists for callers that may not call
 * cudaMalloc: code that runs inside another framework whose allocator owns the
 * device memory (a raw allocation would escape its pool and its accounting),
 * or a service whose device-memory budget is fixed when the process starts.
 * The caller passes theta, the energy and the gradient as for vqe_energy_grad;
 * the scratch comes from one static device array of VQE_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library keeps until the process exits.
 * H psi uses the string or connectivity tables of the (h, sector) pair when an
 * earlier call already built them (vqe_workspace_bytes, vqe_energy_grad or a
 * batch; the results then equal vqe_energy_grad's), else a scan of all X-mask
 * groups per output; the call itself builds nothing.
 * Limit: instances whose scratch exceeds that size are rejected with
 * VQE_ERR_INVALID_ARG and a message. The scratch is two sector-sized vectors
 * (8-byte real amplitudes, 16-byte complex ones), two more for the string
 * tables (left out, with those tables, when they would not fit), the cos/sin
 * table and 8 KiB of partials per parameter: for example 20 qubits with 10
 * electrons (63,504 sector states) and 512 parameters fits on every path, 24
 * qubits with 10 electrons (627,264 states) and 512 parameters fits with real
 * amplitudes without the string tables, 26 qubits with 13 electrons (2.9M
 * states) does not fit.
 * The first call on each device looks up the array's device address (with the
 * device current); make that first call before any stream capture. All calls
 * share the array and it keeps the last call's contents; each call writes every
 * scratch entry it reads, so nothing needs clearing, but calls that overlap on
 * the GPU (other streams or threads) race on it. Asynchronous on `stream`.
 */
#define VQE_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int vqe_energy_grad_noalloc(vqe_hamiltonian_t h, vqe_ansatz_t a, const double* theta_dev,
                            double* energy_dev, double* grad_dev, vqe_stream_t stream);

/*
 * Algorithmic work of one energy(+gradient) evaluation, counted exactly on the
 * host from the tables: FP64 flops (an FMA counts 2) and the bytes of state
 * vector a streaming implementation must move. Used for roofline reports.
 */
int vqe_work_estimate(vqe_hamiltonian_t h, vqe_ansatz_t a, int with_grad,
                      double* fp64_flops, double* state_bytes);

/*
 * The exact counts behind vqe_work_estimate: amplitude pairs over all gates of
 * the ansatz (*n_pairs), connected (output, X-mask group) entries of H psi on
 * the ansatz's sector (*n_entries), and the folded-table additions beyond the
 * first term of each entry (*extra_adds). Any output may be NULL. Host only;
 * like vqe_workspace_bytes, the first call for a (Hamiltonian, sector) pair
 * builds that pair's connectivity or string tables (synchronous, allocates).
 */
int vqe_work_counts(vqe_hamiltonian_t h, vqe_ansatz_t a, int64_t* n_pairs, int64_t* n_entries,
                    double* extra_adds);

/*
 * Device probe (synchronous, allocates and frees a small buffer): the rate of
 * independent FP64 FMAs over the whole device (per second and per clock per SM
 * at the nominal SM clock), the clocks of one dependent FMA in a warp, the SM
 * count and clock, the opt-in shared memory per block and the L2 size. The
 * FP64 rate bounds the state-vector kernels (the paper has no counterpart).
 * Any output pointer may be NULL.
 */
int vqe_probe_fp64(double* dfma_per_sec, double* dfma_per_clock_per_sm, double* dependent_dfma_clocks,
                   int* sm_count, int* sm_clock_khz, size_t* smem_optin, int* l2_bytes);

#ifdef __cplusplus
}
#endif

#endif /* VQE_H */
