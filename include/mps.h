/*
 * libmps: GB300-native (sm_103a) differentiable matrix-product-state simulator
 * for variational quantum chemistry circuits (arXiv:2211.07983).
 *
 * C ABI: plain pointers and sizes, no C++ types, no exceptions.  Every entry
 * point returns an mps_status; on error the outputs are left untouched and
 * mps_last_error() returns a thread-local message.  Nothing aborts, traps or
 * asserts on the device: device-side failures are reported through a status
 * word that the host reads after the call's stream work completes.
 *
 * Memory: the library allocates and owns the device memory of every handle it
 * returns (mps_state, mps_circuit, mps_hamiltonian_dev) until the matching
 * *_free call.  Inputs are copied; the caller keeps ownership of its arrays.
 * Arrays marked "host or device" may point to host memory or to device memory
 * of the current CUDA device (the library asks the driver which it is).
 *
 * Streams: all device work of a call is ordered on mps_config.cuda_stream
 * (NULL = the legacy default stream).  Every call that launches device work
 * synchronises that stream before returning, because it reads the device status
 * word; outputs may still be device pointers (no host round trip of the data).
 *
 * Instances: a state may hold n_inst >= 1 independent instances of the same qubit count
 * and configuration (mps_init_product_batch), e.g. the points of a batched VQE step.  Every
 * kernel of a call then runs over all instances at once.  For such a state, every per-call
 * array below holds one row per instance, instance-major: theta is n_inst x n_theta, E_out
 * n_inst values, grad_out n_inst x n_theta, gate_grad_out n_inst x n_gates, expect_out
 * n_inst x (strings).  With n_inst = 1 (mps_init_product) these are the plain shapes.  A
 * device-side error reports the first failing instance in mps_last_error().
 *
 * Notation (Sec. 3): n qubits = n sites; site tensor B_s[Dl][2][Dr], row-major,
 * Dr fastest; bond b joins sites b and b+1 and carries the Schmidt vector
 * lambda_b; bond dimensions never exceed min(2^(b+1), 2^(n-b-1), max_bond).
 */
#ifndef MPS_H
#define MPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPS_OK = 0,
  MPS_EINVAL = 1,    /* invalid argument (sizes, indices, non-finite angle) */
  MPS_ENOMEM = 2,    /* device or host allocation failed */
  MPS_ECUDA = 3,     /* a CUDA runtime call failed */
  MPS_ENOCONV = 4,   /* one-sided Jacobi SVD did not converge within its sweep cap */
  MPS_ENUMERIC = 5,  /* NaN/Inf met in a singular value, a norm or the energy */
  MPS_ETIMEOUT = 6   /* a bounded device wait gave up */
} mps_status;

enum { MPS_PRECISION_FP64 = 0, MPS_PRECISION_MIXED = 1 };

/* Simulation settings (Sec. 3 truncation rule; Sec. 4 checkpointed reverse pass). */
typedef struct {
  int32_t max_bond;          /* D: bond-dimension cap, >= 1 */
  double cutoff;             /* eps: keep singular values with s_i/||s||_2 > eps (values
                                at or below 1e-13 s_1 are numerical zeros, never kept) */
  int32_t precision;         /* MPS_PRECISION_FP64: every contraction in FP64.
                                MPS_PRECISION_MIXED: the Pauli transfer sweeps of the energy
                                and the reverse pass's recomputed two-site tensors run on the
                                tensor cores in split-TF32 (3xTF32, FP32 accumulation).  All
                                that reaches the reverse pass's cotangents stays FP64 (gate
                                contractions, the energy cotangent): the SVD adjoint amplifies
                                rounding at nearly degenerate Schmidt values, and in 3xTF32 those
                                exceeded 1e-5 in |dE/dtheta|.  The SVD, truncation, SVD adjoint
                                and term sums are FP64.  Tensors are stored in FP64 either way. */
  int32_t checkpoint_every;  /* reverse pass: MPS snapshot every k gates, the segment
                                re-run with a tape; 0 = automatic: one tape for the whole
                                circuit when it fits in 60% of free device memory, else 512 */
  void* cuda_stream;         /* cudaStream_t, NULL = default stream */
} mps_config;

/*
 * One fused nearest-neighbour gate on sites (bond, bond+1) (Sec. 3, two-qubit
 * gate; gate fusion).  Matrices are 4x4 complex, row-major, interleaved
 * (re, im), basis index 2*i_bond + i_{bond+1}.
 *   theta_idx < 0 : G = mat (pre/post ignored)
 *   theta_idx >= 0: G(phi) = post * Rz_site(phi) * pre, phi = theta_scale *
 *                   theta[theta_idx], Rz(phi) = diag(e^{-i phi/2}, e^{i phi/2})
 *                   on the lower (rz_site = 0) or upper (rz_site = 1) site.
 */
typedef struct {
  int32_t bond;
  int32_t theta_idx;
  int32_t rz_site;
  int32_t pad_;
  double theta_scale;
  double mat[32];
  double pre[32];
  double post[32];
} mps_gate;

/*
 * Weighted Pauli strings H = sum_k coeff[k] P_k (Sec. 2, Eq. expect-val).
 * Bit s of x_mask/z_mask is qubit s: (x,z) = (1,0) X, (0,1) Z, (1,1) Y.
 * Host arrays; any order (the library sorts them canonically).
 */
typedef struct {
  int32_t n_terms;
  const uint64_t* x_mask;
  const uint64_t* z_mask;
  const double* coeff;
} mps_hamiltonian;

typedef struct mps_state mps_state;              /* MPS on the device */
typedef struct mps_circuit mps_circuit;          /* gate list resident on the device */
typedef struct mps_hamiltonian_dev mps_hamiltonian_dev; /* strings + sweep trie on the device */

/* ---- host-side problem builders (step S0: once per problem) ----------------------- */

/*
 * Jordan-Wigner qubit Hamiltonian of H = sum h_pq a+_p a_q
 * + 1/2 sum (pq|rs) a+_p a+_r a_s a_q (Sec. 2, Eq. ham-pbc, chemist notation),
 * with a_p = Z_0..Z_{p-1} (X_p + iY_p)/2.  Contributions to one string are merged
 * by their correctly rounded exact sum; strings with |c| <= 1e-14 max|c| are
 * dropped; output in canonical order (first non-identity site, then the
 * per-site symbols I<X<Y<Z; the identity first).
 *   n      : spin orbitals, 1..64
 *   h      : host, n*n doubles, h[p*n+q]
 *   eri    : host, n^4 doubles, eri[((p*n+q)*n+r)*n+s] = (pq|rs)
 *   capacity, x_mask, z_mask, coeff: host output arrays of `capacity` entries
 *   n_terms_out: number of strings.  If it exceeds capacity, nothing is written
 *           to the arrays and MPS_EINVAL is returned (call again with room).
 */
mps_status mps_build_hamiltonian(int32_t n, const double* h, const double* eri, int64_t capacity,
                                 uint64_t* x_mask, uint64_t* z_mask, double* coeff,
                                 int64_t* n_terms_out);

/*
 * UCC excitations -> fused nearest-neighbour gates (Sec. 2, UCC ansatz with a
 * first-order Trotter step of "V-shaped" blocks; Sec. 3, gate fusion).
 *   exc: host, 4*n_exc ints (i, j, a, b); a single i->a has j = b = -1 and
 *        generator a+_a a_i - h.c.; a double has a+_a a+_b a_j a_i - h.c.
 *        Excitation t uses angle theta[t]; excitations are applied in order.
 *   gates_out: host array of `capacity` gates; n_gates_out: count.  Too small a
 *        capacity writes nothing and returns MPS_EINVAL with the count set.
 */
mps_status mps_compile_excitations(int32_t n, const int32_t* exc, int32_t n_exc, int64_t capacity,
                                   mps_gate* gates_out, int64_t* n_gates_out);

/* ---- simulator (steps S1-S9) --------------------------------------------------------- */

/* Product state |b_0 ... b_{n-1}> as a D = 1 MPS with all lambda = [1] (Sec. 3, Eq. hf).
 * bits: host, n bytes of 0/1.  n in 2..64. */
mps_status mps_init_product(int32_t n_qubits, const uint8_t* bits, const mps_config* cfg,
                            mps_state** out);

/*
 * n_inst product states in one state object (1 <= n_inst <= 4096).  bits: host, n_inst x
 * n_qubits bytes of 0/1 (row r is instance r).  The instances are replicas of one device
 * address layout (driver virtual-memory mappings, grown on demand), so one kernel launch
 * serves all of them; each instance's memory is committed only as it is used.
 */
mps_status mps_init_product_batch(int32_t n_inst, int32_t n_qubits, const uint8_t* bits,
                                  const mps_config* cfg, mps_state** out);

/* Number of instances of a state. */
mps_status mps_state_instances(const mps_state* s, int32_t* n_inst);

/* Deep copy of a state (same config, stream and instance count). */
mps_status mps_clone(const mps_state* s, mps_state** out);

/* Copy a state back to the host.  dims: n+1 ints (bond dims, dims[0] = dims[n] = 1);
 * lam: sum of dims[1..n-1] doubles (lambda_0, lambda_1, ...), or NULL;
 * tensors: sum_s dims[s]*2*dims[s+1] complex values as interleaved doubles,
 * sites in order, each [Dl][2][Dr] row-major, or NULL. */
mps_status mps_read_state(const mps_state* s, int32_t* dims, double* lam, double* tensors);
/* The same for instance `inst` (0 <= inst < n_inst); mps_read_state reads instance 0. */
mps_status mps_read_state_instance(const mps_state* s, int32_t inst, int32_t* dims, double* lam,
                                   double* tensors);

/* Upload a gate list once (validated: bonds in range, finite matrices). */
mps_status mps_circuit_create(int32_t n_qubits, const mps_gate* gates, int32_t n_gates,
                              mps_circuit** out);
void mps_circuit_free(mps_circuit* c);

/* Upload a Hamiltonian once; builds the sweep trie (strings sharing a first site
 * form a batch; strings sharing a prefix share its environments). */
mps_status mps_hamiltonian_create(int32_t n_qubits, const mps_hamiltonian* h,
                                  mps_hamiltonian_dev** out);
void mps_hamiltonian_free(mps_hamiltonian_dev* h);

/*
 * In place |s> <- U(theta)|s> (Sec. 3: each gate = two-site contraction, lambda
 * scaling, SVD, truncation, update; Sec. 4, Eq. pqc).  theta: host or device,
 * n_theta doubles, finite; every theta_idx must be < n_theta.
 */
mps_status mps_apply_circuit(mps_state* s, const mps_gate* gates, int32_t n_gates,
                             const double* theta, int32_t n_theta);
mps_status mps_apply_circuit_dev(mps_state* s, const mps_circuit* c, const double* theta,
                                 int32_t n_theta);

/*
 * E = sum_k c_k Re<psi|P_k|psi> / <psi|psi> (Sec. 2, Eq. expect-val; Sec. 3, Eq.
 * paulistringexp) by batched transfer-matrix sweeps.  E_out: host or device double.
 * expect_out: NULL, or host/device array with one double per non-identity string,
 * receiving Re<psi|P_k|psi>/<psi|psi> in canonical order (first non-identity site,
 * then the per-site symbols I<X<Y<Z).
 */
mps_status mps_energy(const mps_state* s, const mps_hamiltonian* h, double* E_out);
mps_status mps_energy_dev(const mps_state* s, const mps_hamiltonian_dev* h, double* E_out,
                          double* expect_out);

/*
 * Energy cotangent (step S7): E and Bbar_s = dE/dB_s* of the state itself, i.e.
 * [sum_k c_k env_k(s) - E env_I(s)] / <psi|psi> with env_P(s) the network of
 * <psi|P|psi> with conj(B_s) removed (Sec. 4, Eq. expecgrad: dE/d<psi| = H|psi>
 * normalised).  Bbar_out: host or device, complex values as interleaved doubles in the
 * layout of mps_read_state's `tensors` (current bond dims), of instance 0; E_out: one value
 * per instance.
 */
mps_status mps_energy_cotangent_dev(const mps_state* s, const mps_hamiltonian_dev* h, double* E_out,
                                    double* Bbar_out);

/*
 * E(theta) and dE/dtheta for |psi> = U(theta)|s0> (s0 is not modified): forward
 * pass with snapshots, energy, energy cotangent dE/dB* (Sec. 4, Eq. expecgrad),
 * then the exact reverse pass through every truncated gate (Eq. circuitevolvegrad,
 * App. A rules), k held fixed.  grad_out: n_theta doubles; gate_grad_out: NULL or
 * n_gates doubles receiving dE/dphi of each gate's Rz angle (0 for fixed gates).
 * All three outputs: host or device.
 */
/* The host-argument calls mps_apply_circuit, mps_energy and mps_energy_grad upload their gate
 * list and Hamiltonian into the state's workspace.  The last upload of each is kept with a copy of
 * its contents and reused while later calls on the same state pass equal contents, so a repeated
 * call reuses the sweep trie, the energy plan and the captured evaluation graph. */
mps_status mps_energy_grad(const mps_state* s0, const mps_gate* gates, int32_t n_gates,
                           const double* theta, int32_t n_theta, const mps_hamiltonian* h,
                           double* E_out, double* grad_out, double* gate_grad_out);
mps_status mps_energy_grad_dev(const mps_state* s0, const mps_circuit* c, const double* theta,
                               int32_t n_theta, const mps_hamiltonian_dev* h, double* E_out,
                               double* grad_out, double* gate_grad_out);

/*
 * Which SVD a single-instance state's gates use.  MPS_SVD_AUTO (the default): a gate whose
 * two-site matrix can exceed 128 rows or columns (bond caps above 64) runs the cooperative SVD,
 * which spreads one matrix over every SM; smaller ones, and every gate of a batched state, run one
 * CTA per matrix.  MPS_SVD_ONE_CTA: always one CTA per matrix (its work arrays in global memory
 * when they exceed shared memory), for callers that run many problems at once
 * (mps_energy_grad_multi), where one SM per problem keeps the GPU full and a whole-GPU SVD would
 * have to run alone.  Results agree with the other policy to rounding.  MPS_EINVAL for a NULL
 * state or an unknown policy.
 */
enum { MPS_SVD_AUTO = 0, MPS_SVD_ONE_CTA = 1 };
mps_status mps_set_svd_policy(mps_state* s, int32_t policy);

/*
 * E and dE/dtheta of n_prob independent problems of uneven size (their own qubit counts, bond
 * dimensions, circuits and Hamiltonians), evaluated together: problem i is exactly
 * mps_energy_grad_dev(states[i], circuits[i], theta[i], n_theta[i], hams[i], E_out[i],
 * grad_out[i], NULL), with the same results bit for bit.  The problems whose SVDs fit one CTA
 * (every two-site matrix at most 128 on a side, or batched states) are enqueued on one
 * library-owned stream each, so the GPU runs them concurrently, and each replays its own captured
 * graph from its third evaluation on; the problems that need the cooperative whole-GPU SVD run
 * afterwards, one at a time.  Each problem's work starts after the work already enqueued on its
 * state's stream, and the call returns when every problem has finished.  E_out[i], grad_out[i]:
 * host or device, n_inst and n_inst * n_theta[i] doubles.  Errors: MPS_EINVAL for NULL arguments,
 * n_prob < 1 or a state passed twice; otherwise the first failing problem's status and message
 * (the others are still waited for).  No counterpart in the paper; this is the batching of
 * independent instances of uneven size.
 */
mps_status mps_energy_grad_multi(int32_t n_prob, mps_state* const* states, const mps_circuit* const* circuits,
                                 const double* const* theta, const int32_t* n_theta,
                                 const mps_hamiltonian_dev* const* hams, double* const* E_out,
                                 double* const* grad_out);

/*
 * E and dE/dtheta with the Pauli strings split over processes (one process per GPU).  E and the
 * energy cotangent dE/dB* are linear in the strings once divided by the common <psi|psi>
 * (Sec. 2, Eq. expect-val; Sec. 4, Eq. expecgrad): with H = sum_r H_r, E = sum_r E_r and
 * dE/dB* = sum_r [env_{H_r} - E_r env_I] / <psi|psi>.  So every rank runs the (replicated) forward
 * pass, the energy and cotangent of its own strings, one sum-allreduce of (E_r, Bbar_r) by the
 * caller, then the (replicated) reverse pass from the summed cotangent.  The identity string
 * belongs to exactly one rank's H_r.
 *   begin: forward + energy + cotangent of h_shard (its strings only); E_out: one value per
 *          instance, host or device; Bbar_out: device memory of mps_cotangent_size() doubles
 *          (instance-major, the state's site slots at the bond caps, interleaved complex).
 *   end:   reverse pass from Bbar_in (device, the summed cotangent, same layout); grad_out and
 *          gate_grad_out as in mps_energy_grad_dev.  Requires a begin with the same circuit on
 *          this state just before it (no other call on the state in between); n_theta as in begin.
 */
mps_status mps_energy_grad_shard_begin(const mps_state* s0, const mps_circuit* c, const double* theta,
                                       int32_t n_theta, const mps_hamiltonian_dev* h_shard, double* E_out,
                                       double* Bbar_out);
mps_status mps_energy_grad_shard_end(const mps_state* s0, const mps_circuit* c, int32_t n_theta,
                                     const double* Bbar_in, double* grad_out, double* gate_grad_out);
/* Number of doubles of a state's cotangent buffer (all instances). */
mps_status mps_cotangent_size(const mps_state* s, int64_t* n_doubles);

/*
 * The gate SVD on its own (steps S3-S4, Sec. 3): one-sided Jacobi SVD of a complex m x ncol
 * matrix A (m, ncol even, <= 512) on its shorter side, FP32 preconditioning sweeps followed by
 * FP64 re-orthonormalisation and FP64 sweeps (FP64-accurate result), sorted descending, then
 * the truncation rule k = max(1, min(D, #{s_i/||s||_2 > eps, s_i > 1e-13 s_1})).  With K = min(m, ncol):
 *   A: host or device, row-major, interleaved (re, im)
 *   s_out: K doubles; V_out: ncol x K complex (row-major, V[r][j] = component r of right
 *   singular vector j; zero for numerically-zero s_j when m < ncol); W_out: m x K complex,
 *   W = A V (row-major; zero columns for numerically-zero s_j); k_out: one int.
 *   Outputs: host or device.  Uses the default stream and synchronises.
 */
mps_status mps_svd_dev(int32_t m, int32_t ncol, const double* A, int32_t D, double eps, double* s_out,
                       double* V_out, double* W_out, int32_t* k_out);

/*
 * Autotuning of the one-CTA gate SVD's work split (no counterpart in the paper).  A column pair of
 * a Jacobi round is handled by 8, 16 or 32 lanes, chosen separately for the FP32 and the FP64
 * sweeps; without a tuned table a rule picks them from the number of pairs.
 *   mps_svd_tune: mean device time in ms (*ms_out, from CUDA events on the default stream) of
 *     `reps` (1..1000) SVDs of the row-major m x ncol complex matrix A (host or device; m, ncol
 *     even, 2..128) by one CTA with jg32 / jg64 lanes per pair (8, 16, 32, or 0 for the rule),
 *     after one warm-up.  Synchronises; MPS_ENOCONV etc. if the SVD fails.
 *   mps_set_svd_tiles: installs the process-wide table used by every later one-CTA gate SVD whose
 *     bond caps give an m_cap x n_cap matrix: n_entries rows of 4 ints {m_cap, n_cap, jg32, jg64}
 *     (host; caps 2..512; lanes 0, 8, 16 or 32, 0 = the rule for that phase).  n_entries = 0
 *     clears the table.  A captured evaluation graph keeps the choice it was captured with.
 *     MPS_EINVAL for malformed entries (the table is then unchanged).
 */
mps_status mps_svd_tune(int32_t m, int32_t ncol, const double* A, int32_t jg32, int32_t jg64, int32_t reps,
                        double* ms_out);
mps_status mps_set_svd_tiles(int32_t n_entries, const int32_t* entries);

/*
 * The gate SVD of mps_svd_dev without any memory allocation.  Some callers cannot call
 * cudaMalloc: embedders whose device memory is owned by another allocator (a framework's caching
 * allocator, a memory pool sized once at start-up) or that run under a fixed device-memory budget,
 * and latency-critical loops that cannot pay for the device-wide synchronisation that
 * cudaMalloc/cudaFree can imply.  This entry point serves them from a fixed scratch array inside
 * the library.  The paper has no counterpart; this is a service of the library.
 *   m, ncol: even, 2..128 (larger sizes are rejected with MPS_EINVAL: the scratch is fixed).
 *   A, s_out, V_out, W_out, k_out: device memory of the current device, owned by the caller, same
 *   layouts and meaning as in mps_svd_dev (K = min(m, ncol)); memory of another device is
 *   rejected with MPS_EINVAL.  cuda_stream: cudaStream_t or NULL.
 * Scratch: one file-scope device array of about 1.25 MiB inside the library, held by every GPU
 * that loads the library until the process exits.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current.  All calls on a device
 * share the array, which keeps the last call's contents (the call clears what must start at
 * zero): calls that overlap on the GPU (different streams or threads) race and must be
 * serialised by the caller.  The call synchronises `cuda_stream` to read the status word.
 */
mps_status mps_svd_noalloc(int32_t m, int32_t ncol, const double* A, int32_t D, double eps, double* s_out,
                           double* V_out, double* W_out, int32_t* k_out, void* cuda_stream);

/*
 * One complex GEMM C = op(A) op(B) (M x N, inner size K) through the kernels of the contractions,
 * for testing them on their own; the paper has no counterpart.  op codes: 0 N, 1 T (transpose),
 * 2 H (conjugate transpose), 3 C (conjugate).  A, B, C: device memory of the current device,
 * row-major, interleaved (re, im), leading dimensions lda, ldb, ldc in complex elements; C is
 * overwritten.  engine: 0 = split-TF32 on mma.sync tensor-core instructions, 1 = split-TF32 on
 * tcgen05.mma with tensor-memory accumulators (the mixed path's large sweep contractions), 2 =
 * FP64 (the FP64 path's kernel).  Uses the default stream and synchronises.
 */
mps_status mps_zgemm_mixed_dev(int32_t M, int32_t N, int32_t K, const double* A, int32_t lda, int32_t opA,
                               const double* B, int32_t ldb, int32_t opB, double* C, int32_t ldc, int32_t engine);

/*
 * Profiling of the gate SVD, the dominant kernel.  While enabled, every SVD launch of calls on
 * this state is bracketed by CUDA events on the state's stream and the SVD kernel adds the
 * floating-point operations its sweeps actually performed to a device counter.
 * mps_profile_read fills out6 = {SVD time in ms from the CUDA events, SVD launches timed by
 * events, FP64 flops, FP32 flops, SVD time in ms from the kernel's own %globaltimer reads, SVD
 * launches counted on the device} since the last read and resets them; counters are summed over
 * the instances (one launch serves every instance, and its %globaltimer time is summed over its
 * CTAs).  The flop and device-time counters run whether or not profiling is enabled; the events
 * only while it is enabled.  Both work inside captured graphs (the events are recorded as
 * external event nodes).  No counterpart in the paper.
 */
mps_status mps_profile(mps_state* s, int32_t enable);
mps_status mps_profile_read(mps_state* s, double* out6);

/*
 * Where the gate SVD's device time went, gathered by the mps_profile_read calls since the last
 * call of this one (then reset): out6 = {ms in FP32 sweeps, ms re-orthonormalising Q and
 * re-forming X = X0 Q in FP64, ms in FP64 sweeps, ms writing the outputs, FP32 sweeps run, FP64
 * sweeps run}, each summed over launches and CTAs.  No counterpart in the paper.
 */
mps_status mps_profile_svd_phases(mps_state* s, double* out6);

/* Release a state (NULL-safe). */
void mps_free(mps_state* s);

/* Thread-local text of the last error of this thread ("" if none). */
const char* mps_last_error(void);

/* Kernel launches issued by this process so far (instrumentation for benchmarks). */
int64_t mps_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* MPS_H */
