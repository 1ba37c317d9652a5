// Kernel launchers of libmps (internal).  All sizes that depend on truncation are read from
// device memory (`dims`), so every launcher can be enqueued without a host synchronisation.
//
// dims layout of a state with n sites: dims[i], i = 0..n, is the dimension of the bond left
// of site i (dims[0] = dims[n] = 1), so site s is B_s[dims[s]][2][dims[s+1]].  Schmidt vectors
// use the same slot numbering: slot i holds lambda of the bond between sites i-1 and i, slot 0
// is the trivial left boundary [1].
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mpsk {

void note_launch();
void add_launches(long long k);
long long launches();
long long thread_launches();

// Every launcher takes the batch of instances it runs over (see Batch in common.cuh).
void launch_zgemm_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n,
                          cudaStream_t st);
// up to 4 descriptors passed by value (no device-side descriptor storage needed)
struct GemmBatch {
  GemmDesc d[4];
  int count;
};
void launch_zgemm_small(const Batch& bt, const GemmBatch& b, int max_m, int max_n, cudaStream_t st);
// The same two GEMMs on the tensor cores in split-TF32 (3xTF32) arithmetic, FP32 accumulation
// (mixed-precision path; gemm_tf32.cu).
void launch_zgemm_tf32x3_small(const Batch& bt, const GemmBatch& b, int max_m, int max_n, cudaStream_t st);
void launch_zgemm_tf32x3_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n,
                                 cudaStream_t st);

// The same batched GEMM on the 5th-generation tensor cores (tcgen05.mma kind::tf32, accumulators in
// tensor memory), split-TF32, 128 x 128 tiles (gemm_tc.cu); `status` is the per-instance status
// word (a bounded wait that gives up records MPS_ETIMEOUT).  zgemm_tc_available() is false when the
// kernel's shared memory cannot be configured.
bool zgemm_tc_available();
void launch_zgemm_tc_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n, int* status,
                             cudaStream_t st);
// Batched GEMM steps of the mixed path use the tcgen05 kernel when both output sides can reach this
constexpr int TC_MIN_SIDE = 64;

// G (16 complex per gate) and dG/dphi from the gate table and theta (device).
void launch_gate_matrices(const Batch& bt, const void* d_gates, int n_gates, const double* d_theta, int n_theta,
                          double2* G, double2* dG, int* status, cudaStream_t st);

// C[(a,i'),(j',c)] = sum_ij G[(i'j'),(ij)] sum_m B_b[a,i,m] B_{b+1}[m,j,c]  (row-major, optional)
// A = lambda_{slot b} * C, column-major (input of the SVD).  When Bl_tape is non-null the kernel
// also copies B_b (2 Dl Dm values) to Bl_tape and B_{b+1} (2 Dm Dr values) to Br_tape.
void launch_contract(const Batch& bt, const double2* Bl, const double2* Br, const int* dims, int b,
                     const double2* G, const double* lam_left, double2* C, double2* A, double2* Bl_tape,
                     double2* Br_tape, int max_dl, int max_dr, cudaStream_t st);

// Per instance i: (dst + i dst_stride)[0..n) = (src + i src_stride)[0..n), strides in bytes, on
// the SMs.  Device-to-device copies stay off the copy engines, whose queues are shared by all
// streams: a copy that waits for one evaluation would hold back every other one behind it.
void launch_copy_f64(const Batch& bt, double* dst, size_t dst_stride, const double* src, size_t src_stride,
                     size_t n, cudaStream_t st);
// out[0] = the first non-zero status word over the instances, out[1] = its instance (-1 if
// none); every status word is cleared.
void launch_status_fetch(const Batch& bt, int* status, double* out, cudaStream_t st);
// dst[0..n) = 0 in every instance, on the SMs (for the same reason).
void launch_zero_f64(const Batch& bt, double* dst, size_t n, cudaStream_t st);

// Gate SVD (steps S3-S4): A = lambda-scaled C~ (m x n, column-major).  FP32 preconditioning
// sweeps, FP64 re-orthonormalisation, FP64 sweeps; orthogonalises K = min(m, n) columns.
// Writes s (K values, descending), Vs (K right singular vectors of length n, column j at
// Vs + j*n), lam_out (slot b+1), dims[b+1] = k, and when non-null: W (K columns of length m,
// W_j = C~ v_j, zero for numerical zeros), tape_dims {Dl, Dm, Dr, k, K, kz} (kz = k when K < n,
// else 0: the width of the adjoint's complement term, empty when the K vectors span C^n),
// lam_left_copy.
// scratch: global buffer of (K^2 + R K) complex values used when shared memory is too small.
struct SvdArgs {
  const double2* A;
  double2* scratch;
  int* dims;
  int b;
  int D;
  double eps;
  double2* Vs;
  double* s;
  double* lam_out;
  double2* W;
  int* tape_dims;
  const double* lam_left;
  double* lam_left_copy;
  int* status;
  double* stats;   // optional, 10 doubles: [0] += FP64 flops, [1] += FP32 flops, [2] += kernel ns, [3] += 1,
                   // [4..7] += ns in FP32 sweeps / re-orthonormalisation and X0 Q / FP64 sweeps / output,
                   // [8], [9] += FP32 and FP64 sweeps run
  int jg32, jg64;  // lanes per column pair of the FP32 / FP64 sweeps (8, 16 or 32); <= 0: a rule from
                   // the pair count.  launch_svd replaces 0, 0 by the tuned table's entry
                   // (svd_tiles_set) for the launch's caps, if it has one.
};
size_t svd_smem_bytes(int m_cap, int n_cap);
bool svd_fits_smem(int m_cap, int n_cap);
// one CTA per instance
void launch_svd(const Batch& bt, const SvdArgs& a, int m_cap, int n_cap, cudaStream_t st);
// The tuned table of lanes per column pair, keyed by the bond caps' matrix shape (m_cap, n_cap):
// entries of 4 ints {m_cap, n_cap, jg32, jg64}; n = 0 clears it.  Read by launch_svd (a launch
// captured in a graph keeps the choice it was captured with).
void svd_tiles_set(const int* entries, int n);
void svd_tiles_get(int m_cap, int n_cap, int* jg32, int* jg64);
// The same SVD of one large matrix (one instance) over the whole GPU: a cooperative launch of one
// CTA per SM with bounded grid barriers between Jacobi rounds (svd_coop.cu), FP64 sweeps.  scratch:
// svd_coop_scratch_bytes(m_cap, n_cap) bytes of device memory; a.scratch is not used.
size_t svd_coop_scratch_bytes(int m_cap, int n_cap);
cudaError_t launch_svd_coop(const SvdArgs& a, void* scratch, int m_cap, int n_cap, cudaStream_t st);
// Gates whose two-site matrix can exceed this many rows or columns use the cooperative SVD when the
// state holds one instance (batched states keep one CTA per instance).
constexpr int SVD_COOP_MIN_SIDE = 129;

// B_{b+1} <- (Vs[:, :k])^H reshaped [k][2][Dr]
void launch_vh_rows(const Batch& bt, const double2* Vs, const int* dims, int b, double2* Br_out, int max_k,
                    int max_ncol, cudaStream_t st);

// ---- gate adjoint pieces; `td` = tape dims {Dl, Dm, Dr, k, K} ------------------------------------
void launch_conjT(const Batch& bt, const double2* Bbar_r, const int* td, double2* Vbar, int max_k, int max_ncol,
                  cudaStream_t st);
void launch_sbar(const Batch& bt, double* lambar_slot, const double* s, const int* td, double* wbar,
                 cudaStream_t st);
void launch_build_K(const Batch& bt, const double2* Y, const double* s, const double* wbar, const int* td,
                    double2* K, int max_K, cudaStream_t st);
void launch_zscale(const Batch& bt, double2* Z, const double* s, const int* td, int max_n, int max_k,
                   cudaStream_t st);
void launch_lam_scale(const Batch& bt, double2* Cbar, const double2* Ctbar, const double2* C,
                      const double* lam_left, const int* td, double* lambar_left, int max_dl, cudaStream_t st);
void launch_gbar(const Batch& bt, const double2* Cbar, const double2* Theta, const int* td, const double2* dG,
                 double2* Gbar, double* gate_grad, cudaStream_t st);
void launch_thetabar(const Batch& bt, const double2* Cbar, const double2* G, const int* td, double2* Thbar,
                     int max_dl, int max_dr, cudaStream_t st);
// csr tables are shared by all instances
void launch_theta_reduce(const Batch& bt, const double* gate_grad, const int* csr_off, const int* csr_gate,
                         const double* csr_scale, int n_theta, double* grad, cudaStream_t st);

// ---- energy ----------------------------------------------------------------------------------
// OB[ob_off[3s+o]] = O applied to the physical index of B_s, o = 0 X, 1 Y, 2 Z.
void launch_apply_paulis(const Batch& bt, const double2* B, const size_t* site_off, const size_t* ob_off,
                         const int* dims, int n, double2* OB, int max_site, cudaStream_t st);
// e[t] = sum_{x,y} L_t[x][y] R_t[x][y] for pairs given by pointer tables; D from dims[didx[t]]
void launch_env_dots(const Batch& bt, const double2* const* Ls, const double2* const* Rs, const int* didx,
                     const int* dims, int count, double2* e, cudaStream_t st);
// E = (sum_k c_k Re e_k) / Re Z with compensated (Neumaier) summation, deterministic order;
// expect (optional) = Re e_k / Re Z.
// c (the coefficients) is shared by all instances.
void launch_energy_sum(const Batch& bt, const double2* e, const double* c, int n_terms, double c0,
                       const double2* Z, double* E_out, double* expect, int* status, cudaStream_t st);
// Y[t] = sum over a list of sources (alpha_j * X_j), fixed order; used for trie reductions.
struct AxpyList {
  double2* out;
  int src_begin, src_end;   // into the src tables
  int didx;                 // element count = dims[didx]^2 * mult
  int mult;
  int accumulate;           // 1: out += ..., 0: out = ...
};
void launch_axpy_lists(const Batch& bt, const AxpyList* lists, int count, const double2* const* src,
                       const double* src_coef, const int* dims, int max_elems, cudaStream_t st);
// out = AR + (c0 - *E) * RI over dims[slot]^2 elements
void launch_rsum(const Batch& bt, double2* out, const double2* AR, const double2* RI, double c0, const double* E,
                 const int* dims, int slot, int max_elems, cudaStream_t st);
// Bbar_s = (sum_nodes O_node . E_node + Eid) / Z for one site; node_op: 0 I, 1 X, 2 Y, 3 Z
struct SeedSite {
  double2* out;        // Bbar_s [Dl][2][Dr]
  const double2* Eid;  // identity-part environment [Dl][2][Dr]
  int node_begin, node_end;
  int s;               // site
};
void launch_seed_assemble(const Batch& bt, const SeedSite* sites, int n_sites, const double2* const* Enode,
                          const int* node_op, const int* dims, const double2* Z, int max_site, cudaStream_t st);

}  // namespace mpsk
