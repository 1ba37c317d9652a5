// libmps host engine and C ABI (see include/mps.h).
//
// Pipeline of one energy + gradient evaluation (all on the caller's stream, bond dimensions
// kept on the device so nothing waits on the host between gates):
//   1. gate matrices G(phi), dG/dphi from theta                         (gate_kernels.cu)
//   2. forward: per gate contract -> Jacobi SVD + truncation -> update  (Sec. 3), MPS snapshot
//      every `checkpoint_every` gates
//   3. energy by trie-shared transfer sweeps, and its cotangent Bbar = dE/dB*  (Sec. 2-3; Sec. 4
//      Eq. expecgrad)
//   4. reverse: per segment, restore the snapshot, recompute with a tape, then run the exact
//      adjoint of every gate backwards (Sec. 4, Eq. circuitevolvegrad; App. A rules)
//   5. dE/dtheta = sum over the Rz angles that share a theta (fixed order)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <numeric>

#include "engine.h"

using namespace mpsk;

namespace mpsk {
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // launches issued by this thread (graph capture)
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches() { return g_launches.load(); }
long long thread_launches() { return t_launches; }
}  // namespace mpsk

namespace mpsi {

static std::atomic<long long> g_uid{0};
long long next_uid() { return ++g_uid; }

static thread_local std::string g_err;

mps_status fail(mps_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }

// Waits for the legacy default stream, on which allocations are zeroed and host tables are
// uploaded (cudaMemset/cudaMemcpy).  A pageable host-to-device cudaMemcpy may return before its
// DMA has landed, and the library's kernels run on non-blocking streams that do not order
// themselves after the legacy stream, so every such batch ends with this fence.
mps_status legacy_fence() {
  MPS_CU(cudaStreamSynchronize(cudaStreamLegacy));
  return MPS_OK;
}

mps_status DevBuf::alloc(size_t nbytes) {
  reset();
  if (nbytes == 0) nbytes = 16;
  if (arena) {
    MPS_TRY(arena->alloc(nbytes, &p));
    bytes = nbytes;
    return MPS_OK;
  }
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(MPS_ENOMEM, "cudaMalloc(" + std::to_string(nbytes) + " bytes): " + cudaGetErrorString(e));
  }
  bytes = nbytes;
  MPS_CU(cudaMemset(p, 0, nbytes));
  return legacy_fence();
}

mps_status DevBuf::ensure(size_t nbytes) {
  if (p && bytes >= nbytes) return MPS_OK;
  return alloc(nbytes);
}

void Layout::build(int n_, int D_) {
  n = n_;
  D = D_;
  cap.assign(n + 1, 1);
  max_cap = 1;
  for (int i = 1; i < n; ++i) {
    int e = std::min(i, n - i);
    long long c = e >= 30 ? (long long)D : std::min<long long>(1ll << e, D);
    cap[i] = (int)c;
    max_cap = std::max(max_cap, cap[i]);
  }
  site_off.assign(n + 1, 0);
  for (int s = 0; s < n; ++s) site_off[s + 1] = site_off[s] + (size_t)cap[s] * 2 * cap[s + 1];
  lam_off.assign(n + 2, 0);
  for (int i = 0; i <= n; ++i) lam_off[i + 1] = lam_off[i] + (size_t)cap[i];
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

mps_status StateBuf::alloc(const Layout& L) {
  size_t b1 = align256(L.site_elems() * sizeof(double2));
  size_t b2 = align256(L.lam_elems() * sizeof(double));
  size_t b3 = align256((L.n + 1) * sizeof(int));
  MPS_TRY(mem.alloc(b1 + b2 + b3));
  char* base = mem.as<char>();
  B = reinterpret_cast<double2*>(base);
  lam = reinterpret_cast<double*>(base + b1);
  dims = reinterpret_cast<int*>(base + b1 + b2);
  return MPS_OK;
}

mps_status StateBuf::copy_from(const StateBuf& o, const Layout& L, cudaStream_t st) {
  (void)L;
  const Batch bt = mem.arena ? mem.arena->batch() : Batch{1, 0};
  launch_copy_f64(bt, mem.as<double>(), bt.stride, o.mem.as<double>(), bt.stride, mem.bytes / sizeof(double), st);
  return MPS_OK;
}

PtrLocation ptr_location(const void* p) {
  if (!p) return PTR_HOST;
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (a.type != cudaMemoryTypeDevice) return PTR_HOST;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PTR_OTHER_DEVICE;
  }
  return a.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
}

// A caller's array: host (false) or device memory of the current device (true).  Memory of
// another device is rejected with MPS_EINVAL (the kernels run on the current device only).
static mps_status where_is(const void* p, const char* what, bool* dev) {
  const PtrLocation l = ptr_location(p);
  if (l == PTR_OTHER_DEVICE)
    return fail(MPS_EINVAL, std::string(what) + " points to memory of another device");
  *dev = l == PTR_DEVICE;
  return MPS_OK;
}

// ---- workspace ------------------------------------------------------------------------------
struct TapeSlot {
  double2 *Bl, *Br, *C, *W, *Vs;
  double *s, *lamL;
  int* dims;
};

// Every device buffer of a workspace is per instance (a range of the state's arena).
struct Workspace {
  Arena* arena;
  DevBuf A, svd, C, Vs, s;                        // forward scratch at the largest bond
  DevBuf svdc;                                    // scratch of the cooperative (multi-SM) SVD
  DevBuf G, dG, theta, scalars, gate_grad, grad;  // per call
  StateBuf work, rec;                             // energy_grad working states
  std::vector<std::unique_ptr<StateBuf>> snaps;
  DevBuf tape;
  DevBuf Bbar, lambar;
  DevBuf rv;                                      // reverse scratch
  double2 *Vbar = nullptr, *Cbar = nullptr, *Y = nullptr, *Km = nullptr, *T1 = nullptr, *Ctbar = nullptr,
          *Theta = nullptr, *Thbar = nullptr, *Gbar = nullptr;
  double* wbar = nullptr;
  bool work_ok = false;
  // profiling of the gate SVD (mps_profile): events around every launch, flop counters
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  DevBuf stats;            // 10 doubles per instance (see SvdArgs::stats)
  double phases[6] = {0, 0, 0, 0, 0, 0};   // phase ms and sweeps, gathered by mps_profile_read
  double svd_ms = 0.0;
  long long svd_launches = 0;
  // captured energy+gradient call (see mps_energy_grad_dev)
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<const void*> graph_key, graph_seen;
  long long graph_kernels = 0;
  size_t graph_ev_used = 0;       // profiling events recorded by the captured graph
  // Host inputs and outputs of a call pass through pinned host memory that kernels read and
  // write directly (slot 0 receives the status word).  No call queues work on a copy engine:
  // copy-engine queues are shared by all streams, so an output copy that waits for one
  // evaluation would hold back every other evaluation behind it.
  double* stage = nullptr;        // host view
  double* stage_dev = nullptr;    // device view
  size_t stage_n = 0, stage_used = 0;
  struct Pending {
    double* dst;
    size_t off, count;
  };
  std::vector<Pending> pending;   // host outputs to copy out of the staging after the call
  cudaEvent_t done = nullptr;     // blocking-sync event: waiting threads sleep instead of spinning
  long long shard_uid = -1;       // circuit of a pending mps_energy_grad_shard_begin
  long long auto_uid = -1;        // circuit for which the automatic checkpoint interval was chosen
  int auto_K = 0;
  // Host-argument calls (mps_apply_circuit, mps_energy, mps_energy_grad) upload their gate list
  // and Hamiltonian; the last uploads are kept with a copy of their contents and reused while a
  // caller passes the same contents, so that the energy plan and the captured graph of a
  // repeated call are reused too.
  std::unique_ptr<mps_circuit> host_circ;
  std::vector<mps_gate> host_circ_gates;
  std::unique_ptr<mps_hamiltonian_dev> host_ham;
  std::vector<uint64_t> host_ham_x, host_ham_z;
  std::vector<double> host_ham_c;
  explicit Workspace(Arena* a)
      : arena(a), A(a), svd(a), C(a), Vs(a), s(a), G(a), dG(a), theta(a), scalars(a), gate_grad(a), grad(a),
        work(a), rec(a), tape(a), Bbar(a), lambar(a), rv(a), stats(a) {}
  ~Workspace() {
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (stage) cudaFreeHost(stage);
    if (done) cudaEventDestroy(done);
  }
};

struct Ctx {
  const Layout* L;
  const mps_config* cfg;
  cudaStream_t st;
  int* status;
  Workspace* ws;
  Batch bt;
};

// A gate on bond b runs the cooperative multi-SM SVD when the state holds one instance, its
// policy allows it, and the gate's two-site matrix can exceed SVD_COOP_MIN_SIDE - 1 rows or columns.
static bool gate_uses_coop(const Layout& L, int n_inst, int b) {
  return !L.one_cta_svd && n_inst == 1 && std::max(2 * L.cap[b], 2 * L.cap[b + 2]) >= SVD_COOP_MIN_SIDE;
}
static bool state_uses_coop(const Layout& L, int n_inst) {
  return !L.one_cta_svd && n_inst == 1 && 2 * L.max_cap >= SVD_COOP_MIN_SIDE;
}

static mps_status ensure_forward_scratch(const Layout& L, Workspace& w) {
  const size_t mc = 2 * (size_t)L.max_cap, nc = 2 * (size_t)L.max_cap;
  if (state_uses_coop(L, w.arena->n)) MPS_TRY(w.svdc.ensure(svd_coop_scratch_bytes((int)mc, (int)nc)));
  MPS_TRY(w.A.ensure(mc * nc * sizeof(double2)));
  MPS_TRY(w.svd.ensure(2 * nc * nc * sizeof(double2)));   // SVD scratch if shared memory is too small
  MPS_TRY(w.C.ensure(mc * nc * sizeof(double2)));
  MPS_TRY(w.Vs.ensure(nc * nc * sizeof(double2)));
  MPS_TRY(w.s.ensure(nc * sizeof(double)));
  return MPS_OK;
}

static GemmDesc make_desc(const int* dims, const double2* A, int opA, const double2* B, int opB, double2* C,
                          DimExpr M, DimExpr N, DimExpr K, DimExpr lda, DimExpr ldb, DimExpr ldc,
                          bool accumulate = false, double alpha = 1.0) {
  GemmDesc d{};
  d.A = A;
  d.B = B;
  d.C = C;
  d.dims = dims;
  d.M = M;
  d.N = N;
  d.K = K;
  d.lda = lda;
  d.ldb = ldb;
  d.ldc = ldc;
  d.opA = opA;
  d.opB = opB;
  d.alpha = make_double2(alpha, 0.0);
  d.beta = make_double2(accumulate ? 1.0 : 0.0, 0.0);
  return d;
}

// Profiling event on the stream; under stream capture it is recorded as an external event node,
// so that replays of the captured graph re-record it.
static mps_status record_profile_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MPS_CU(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    MPS_CU(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
  else
    MPS_CU(cudaEventRecord(e, st));
  return MPS_OK;
}

// one gate on bond b: contract -> SVD/truncate -> update (Sec. 3); with a tape when `tp`
// A per-gate GEMM; `mixed_ok` GEMMs run on the tensor cores in 3xTF32 on the mixed-precision
// path.  Only the recomputed Theta = B_b B_{b+1} is: it feeds dE/dphi of its own gate and nothing
// upstream.  Every other gate GEMM stays FP64.  The forward site update's FP32-level rounding
// accumulates over the circuit: 1.5e-6 relative in E after 1400 gates, where the tolerance is
// 1e-6.  The cotangents of the reverse pass reach the SVD adjoints of all earlier gates, whose
// 1/(s_i^2 - s_j^2) factors amplify rounding at nearly degenerate Schmidt values: 1.1e-4
// relative in |dE/dtheta| with them in 3xTF32, where the tolerance is 1e-5.
static void gemm_small(const Ctx& cx, const GemmBatch& g, int max_m, int max_n, bool mixed_ok) {
  if (mixed_ok && cx.cfg->precision == MPS_PRECISION_MIXED)
    launch_zgemm_tf32x3_small(cx.bt, g, max_m, max_n, cx.st);
  else
    launch_zgemm_small(cx.bt, g, max_m, max_n, cx.st);
}

static mps_status forward_gate(Ctx& cx, StateBuf& sb, int b, const double2* Gt, const TapeSlot* tp) {
  const Layout& L = *cx.L;
  Workspace& w = *cx.ws;
  double2* Bl = sb.B + L.site_off[b];
  double2* Br = sb.B + L.site_off[b + 1];
  double2* C = tp ? tp->C : w.C.as<double2>();
  double2* Vs = tp ? tp->Vs : w.Vs.as<double2>();
  double* s = tp ? tp->s : w.s.as<double>();
  launch_contract(cx.bt, Bl, Br, sb.dims, b, Gt, sb.lam + L.lam_off[b], C, w.A.as<double2>(), tp ? tp->Bl : nullptr,
                  tp ? tp->Br : nullptr, L.cap[b], L.cap[b + 2], cx.st);
  SvdArgs a{};
  a.A = w.A.as<double2>();
  a.scratch = w.svd.as<double2>();
  a.dims = sb.dims;
  a.b = b;
  a.D = cx.cfg->max_bond;
  a.eps = cx.cfg->cutoff;
  a.Vs = Vs;
  a.s = s;
  a.lam_out = sb.lam + L.lam_off[b + 1];
  a.W = tp ? tp->W : nullptr;
  a.tape_dims = tp ? tp->dims : nullptr;
  a.lam_left = sb.lam + L.lam_off[b];
  a.lam_left_copy = tp ? tp->lamL : nullptr;
  a.status = cx.status;
  a.stats = w.stats.as<double>();
  if (w.profile) {
    if (w.ev_used + 2 > w.ev_pool.size()) {
      for (int q = 0; q < 256; ++q) {
        cudaEvent_t e;
        MPS_CU(cudaEventCreate(&e));
        w.ev_pool.push_back(e);
      }
    }
    MPS_TRY(record_profile_event(w.ev_pool[w.ev_used], cx.st));
  }
  if (gate_uses_coop(L, cx.bt.n, b)) {
    const cudaError_t e = launch_svd_coop(a, w.svdc.p, 2 * L.cap[b], 2 * L.cap[b + 2], cx.st);
    if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("cooperative SVD launch: ") + cudaGetErrorString(e));
  } else {
    launch_svd(cx.bt, a, 2 * L.cap[b], 2 * L.cap[b + 2], cx.st);
  }
  if (w.profile) {
    MPS_TRY(record_profile_event(w.ev_pool[w.ev_used + 1], cx.st));
    w.ev_used += 2;
  }
  GemmBatch g{};
  g.count = 1;
  g.d[0] = make_desc(sb.dims, C, OP_N, Vs, OP_T, Bl, dref(b, 2), dref(b + 1), dref(b + 2, 2), dref(b + 2, 2),
                     dref(b + 2, 2), dref(b + 1));
  gemm_small(cx, g, 2 * L.cap[b], L.cap[b + 1], false);   // FP64: its rounding would accumulate over the circuit
  launch_vh_rows(cx.bt, Vs, sb.dims, b, Br, L.cap[b + 1], 2 * L.cap[b + 2], cx.st);
  return MPS_OK;
}

static mps_status forward_gates(Ctx& cx, StateBuf& sb, const mps_circuit* c, const double2* G, int g0, int g1,
                                const std::vector<TapeSlot>* tapes) {
  for (int t = g0; t < g1; ++t) {
    const TapeSlot* tp = tapes ? &(*tapes)[t - g0] : nullptr;
    MPS_TRY(forward_gate(cx, sb, c->host[t].bond, G + 16 * (size_t)t, tp));
  }
  MPS_CU(cudaGetLastError());
  return MPS_OK;
}

// exact adjoint of one gate (Sec. 4 / App. A): cotangents of the gate's outputs
// (Bbar_b, Bbar_{b+1}, lambar of bond b) -> cotangents of its inputs and dE/dphi.
static mps_status reverse_gate(Ctx& cx, int t, int b, const TapeSlot& tp, double2* Bbar, double* lambar,
                               const double2* G, const double2* dG, double* gate_grad) {
  const Layout& L = *cx.L;
  Workspace& w = *cx.ws;
  const int* td = tp.dims;
  const DimExpr m = dref(0, 2), Dm = dref(1), nc = dref(2, 2), k = dref(3), Ks = dref(4), kz = dref(5);
  double2* Bbl = Bbar + L.site_off[b];
  double2* Bbr = Bbar + L.site_off[b + 1];
  const int mcap = 2 * L.cap[b], ncap = 2 * L.cap[b + 2], kcap = L.cap[b + 1], Kcap = std::min(mcap, ncap);
  launch_conjT(cx.bt, Bbr, td, w.Vbar, kcap, ncap, cx.st);                          // Vbar = Bbar_{b+1}^H
  GemmBatch g{};
  g.count = 2;
  g.d[0] = make_desc(td, tp.C, OP_H, Bbl, OP_N, w.Vbar, nc, k, m, nc, k, k, true);     // Vbar += C^H Bbar_b
  g.d[1] = make_desc(td, Bbl, OP_N, tp.Vs, OP_C, w.Cbar, m, nc, k, k, nc, nc);         // Cbar = Bbar_b V_k^H
  gemm_small(cx, g, std::max(mcap, ncap), std::max(kcap, ncap), false);
  g.count = 1;
  g.d[0] = make_desc(td, tp.Bl, OP_N, tp.Br, OP_N, w.Theta, m, nc, Dm, Dm, nc, nc);    // Theta = B_b B_{b+1}
  gemm_small(cx, g, mcap, ncap, true);
  launch_sbar(cx.bt, lambar + L.lam_off[b + 1], tp.s, td, w.wbar, cx.st);              // sbar -> wbar
  g.count = 1;
  g.d[0] = make_desc(td, tp.Vs, OP_C, w.Vbar, OP_N, w.Y, Ks, k, nc, nc, k, k);         // Y = V_e^H Vbar
  gemm_small(cx, g, Kcap, kcap, false);
  // The complement Z = (I - V_e V_e^H) Vbar has kz = k columns when K < ncol and none when the K
  // vectors span C^ncol (kz = 0: these GEMMs and the complement term below do nothing).
  g.d[0] = make_desc(td, tp.Vs, OP_T, w.Y, OP_N, w.Vbar, nc, kz, Ks, nc, k, k, true, -1.0);   // Z = Vbar - V_e Y
  gemm_small(cx, g, ncap, kcap, false);
  // Z again minus its part in span(V_e): the subtraction above leaves rounding of size eps |Vbar|
  // inside the span, which 1/w_k would amplify for small kept values; the second pass removes it
  // (T1 is free until T1 = W K below).
  g.d[0] = make_desc(td, tp.Vs, OP_C, w.Vbar, OP_N, w.T1, Ks, kz, nc, nc, k, k);       // Y2 = V_e^H Z
  gemm_small(cx, g, Kcap, kcap, false);
  g.d[0] = make_desc(td, tp.Vs, OP_T, w.T1, OP_N, w.Vbar, nc, kz, Ks, nc, k, k, true, -1.0);  // Z -= V_e Y2
  gemm_small(cx, g, ncap, kcap, false);
  launch_build_K(cx.bt, w.Y, tp.s, w.wbar, td, w.Km, Kcap, cx.st);                            // diag(wbar)+J+J^H
  launch_zscale(cx.bt, w.Vbar, tp.s, td, ncap, kcap, cx.st);                                  // Z diag(1/w_k)
  g.d[0] = make_desc(td, tp.W, OP_T, w.Km, OP_N, w.T1, m, Ks, Ks, m, Ks, Ks);          // T1 = W K
  gemm_small(cx, g, mcap, Kcap, false);
  g.d[0] = make_desc(td, w.T1, OP_N, tp.Vs, OP_C, w.Ctbar, m, nc, Ks, Ks, nc, nc);     // C~bar = T1 V_e^H
  gemm_small(cx, g, mcap, ncap, false);
  g.d[0] = make_desc(td, tp.W, OP_T, w.Vbar, OP_H, w.Ctbar, m, nc, kz, m, k, nc, true);  // += W_k (Z/w)^H
  gemm_small(cx, g, mcap, ncap, false);
  launch_lam_scale(cx.bt, w.Cbar, w.Ctbar, tp.C, tp.lamL, td, b > 0 ? lambar + L.lam_off[b] : nullptr, L.cap[b],
                   cx.st);
  launch_gbar(cx.bt, w.Cbar, w.Theta, td, dG + 16 * (size_t)t, w.Gbar, gate_grad + t, cx.st);
  launch_thetabar(cx.bt, w.Cbar, G + 16 * (size_t)t, td, w.Thbar, L.cap[b], L.cap[b + 2], cx.st);
  g.count = 2;
  g.d[0] = make_desc(td, w.Thbar, OP_N, tp.Br, OP_H, Bbl, m, Dm, nc, nc, nc, Dm);      // Bbar_b = Thbar B_{b+1}^H
  g.d[1] = make_desc(td, tp.Bl, OP_H, w.Thbar, OP_N, Bbr, Dm, nc, m, Dm, nc, nc);      // Bbar_{b+1} = B_b^H Thbar
  gemm_small(cx, g, std::max(mcap, kcap), std::max(kcap, ncap), false);
  return MPS_OK;
}

}  // namespace mpsi

// ===================================================================================================
// energy engine
// ===================================================================================================
namespace mpsi {

struct Step {
  enum Kind { GEMM, AXPY, PAULIS, DOTS, SUM, RSUM, SEED } kind;
  int off = 0, count = 0, max_m = 0, max_n = 0;
  int slot = 0;
};

// Energy plan of one Hamiltonian for one state: `bufs` is per instance (a range of the state's
// arena); the descriptor and pointer tables are shared by the instances and hold instance-0
// addresses, which the kernels shift.
struct EnergyCache {
  long long key_arena = 0;
  const void* key_B = nullptr;
  const int* key_dims = nullptr;
  const void* key_Bbar = nullptr;
  DevBuf bufs, tables;
  std::vector<Step> plan_e, plan_seed;
  // device views
  GemmDesc* d_desc = nullptr;
  AxpyList* d_axpy = nullptr;
  const double2** d_src = nullptr;
  double* d_srccoef = nullptr;
  const double2** d_dotL = nullptr;
  const double2** d_dotR = nullptr;
  int* d_dotdidx = nullptr;
  SeedSite* d_seed = nullptr;
  const double2** d_Enode = nullptr;
  int* d_nodeop = nullptr;
  size_t* d_site_off = nullptr;
  size_t* d_ob_off = nullptr;
  double2* OB = nullptr;
  double2* e = nullptr;
  double2* Z = nullptr;
  std::vector<double2*> RI, AR, Rsum;
  int max_site = 1;
  size_t bytes = 0;        // device bytes of `bufs` per instance
};

}  // namespace mpsi

mps_hamiltonian_dev::~mps_hamiltonian_dev() = default;

namespace mpsi {

// Build every buffer, descriptor and step of the energy (+ cotangent) pass for one state layout.
//
// Memory is bounded by the widest trie level, not by the trie: only the left environment L_v of
// every node is kept (the cotangent needs it again); the other per-node intermediates live in
// slabs that hold one trie level (one site) and are reused level after level:
//   T  (site-sized): T_p = L_p B_s of the parents of the level being formed
//   X  (bond^2):     right environment of each node's subtree, X_v = c_v R^I + sum_children Y_c
//   Y  (bond^2, two slabs by site parity): Y_v = T^R_{O_v}(X_v), read by the level above
//   UE (site-sized): U_v = B_t X_v^T, then E_v = T_par(v) X_v^T (U is consumed first)
// The cotangent walks the sites from right to left; at each site it finishes the right identity
// accumulator A^R, the identity-part environment Eid and the seed of that site before the slabs
// move on, so no level's intermediates are needed after its site is done.
static mps_status build_energy_cache(const Layout& L, const StateBuf& sb, mps_hamiltonian_dev* h,
                                     double2* d_Bbar, EnergyCache& ec) {
  const int n = L.n;
  const int nn = (int)h->node_site.size();
  const int nt = (int)h->x.size();
  const std::vector<int>& cap = L.cap;
  auto sq = [&](int i) { return (size_t)cap[i] * cap[i]; };
  auto site_sz = [&](int s) { return (size_t)cap[s] * 2 * cap[s + 1]; };
  auto level_n = [&](int s) { return (size_t)(h->site_begin[s + 1] - h->site_begin[s]); };
  auto local = [&](int v) { return (size_t)(v - h->site_begin[h->node_site[v]]); };
  // ---- buffer plan (complex elements) ----
  size_t total = 0;
  auto take = [&](size_t elems) {
    size_t o = total;
    total += (elems + 15) & ~size_t(15);
    return o;
  };
  size_t o_one = take(1), o_zero = take(1);
  std::vector<size_t> oLI(n), oTL(n), oUR(n), oRI(n + 1), oTA(n), oAL(n), oAR(n + 1), oRsum(n + 1), oEid(n),
      oOB(3 * n), oURa(n);
  for (int s = 0; s < n; ++s) {
    oLI[s] = take(sq(s + 1));
    oTL[s] = take(site_sz(s));
    oUR[s] = take(site_sz(s));
    oRI[s] = take(sq(s));
    oTA[s] = take(site_sz(s));
    oAL[s] = take(sq(s + 1));
    oAR[s] = take(sq(s));
    oRsum[s] = take(sq(s));
    oEid[s] = take(site_sz(s));
    oURa[s] = take(site_sz(s));
    for (int o = 0; o < 3; ++o) oOB[3 * s + o] = take(site_sz(s));
  }
  oRI[n] = o_one;
  oAR[n] = take(1);
  oRsum[n] = take(1);
  std::vector<size_t> oL(nn);
  for (int v = 0; v < nn; ++v) oL[v] = take(sq(h->node_site[v] + 1));
  size_t xs = 1, ys = 1, ues = 1, ts = 1;
  for (int s = 0; s < n; ++s) {
    xs = std::max(xs, level_n(s) * sq(s + 1));
    ys = std::max(ys, level_n(s) * sq(s));
    ues = std::max(ues, level_n(s) * site_sz(s));
    if (s > 0) ts = std::max(ts, level_n(s - 1) * site_sz(s));
  }
  const size_t o_X = take(xs), o_Y0 = take(ys), o_Y1 = take(ys), o_UE = take(ues), o_T = take(ts);
  size_t o_e = take(2 * (size_t)std::max(nt, 1));
  Arena* arena = sb.mem.arena;
  ec.bufs.arena = arena;
  MPS_TRY(ec.bufs.alloc(total * sizeof(double2)));
  double2* base = ec.bufs.as<double2>();
  auto P = [&](size_t o) { return base + o; };
  // slab addresses of node v (at site s = node_site[v])
  auto Xv = [&](int v) { return P(o_X + local(v) * sq(h->node_site[v] + 1)); };
  auto Yv = [&](int v) {
    const int s = h->node_site[v];
    return P(((s & 1) ? o_Y1 : o_Y0) + local(v) * sq(s));
  };
  auto UEv = [&](int v) { return P(o_UE + local(v) * site_sz(h->node_site[v])); };
  auto Tp = [&](int p) { return P(o_T + local(p) * site_sz(h->node_site[p] + 1)); };   // T of parent p
  double2 one_val = make_double2(1.0, 0.0);
  for (int i = 0; i < arena->n; ++i)
    MPS_CU(cudaMemcpy(ish(P(o_one), (size_t)i * arena->stride), &one_val, sizeof(double2), cudaMemcpyHostToDevice));
  ec.e = P(o_e);
  ec.Z = P(oLI[n - 1]);
  ec.OB = base;
  ec.RI.resize(n + 1);
  ec.AR.resize(n + 1);
  ec.Rsum.resize(n + 1);
  for (int s = 0; s <= n; ++s) {
    ec.RI[s] = P(oRI[s]);
    ec.AR[s] = P(oAR[s]);
    ec.Rsum[s] = P(oRsum[s]);
  }
  ec.max_site = 1;
  for (int s = 0; s < n; ++s) ec.max_site = std::max<int>(ec.max_site, cap[s] * cap[s + 1]);
  ec.bytes = total * sizeof(double2);

  // ---- descriptors and steps ----
  std::vector<GemmDesc> D;
  std::vector<AxpyList> AX;
  std::vector<const double2*> SRC;
  std::vector<double> SRCC;
  const int* dims = sb.dims;
  auto Bs = [&](int s) { return (const double2*)(sb.B + L.site_off[s]); };
  auto OBp = [&](int s, int op) -> const double2* { return op == 0 ? Bs(s) : P(oOB[3 * s + op - 1]); };
  auto gemm_step = [&](std::vector<Step>& plan, size_t first, int mm, int mn) {
    for (size_t c0 = first; c0 < D.size(); c0 += 65535) {   // grid z limit per launch
      Step st{Step::GEMM};
      st.off = (int)c0;
      st.count = (int)std::min<size_t>(65535, D.size() - c0);
      st.max_m = mm;
      st.max_n = mn;
      plan.push_back(st);
    }
  };
  auto axpy_step = [&](std::vector<Step>& plan, size_t first, int max_elems) {
    for (size_t c0 = first; c0 < AX.size(); c0 += 65535) {
      Step st{Step::AXPY};
      st.off = (int)c0;
      st.count = (int)std::min<size_t>(65535, AX.size() - c0);
      st.max_m = max_elems;
      plan.push_back(st);
    }
  };
  std::vector<Step>& PE = ec.plan_e;
  std::vector<Step>& PS = ec.plan_seed;
  PE.clear();
  PS.clear();
  PE.push_back(Step{Step::PAULIS});
  // identity environments L^I (left) and R^I (right), interleaved two per launch
  for (int q = 0; q < n; ++q) {
    size_t f = D.size();
    int s = q;   // left chain, first half-step: TL_s = L^I_{s-1} B_s
    const double2* Lp = s == 0 ? P(o_one) : P(oLI[s - 1]);
    D.push_back(make_desc(dims, Lp, OP_N, Bs(s), OP_N, P(oTL[s]), dref(s), dref(s + 1, 2), dref(s), dref(s),
                          dref(s + 1, 2), dref(s + 1, 2)));
    int r = n - 1 - q;   // right chain: UR_r = B_r R^I_{r+1}^T
    D.push_back(make_desc(dims, Bs(r), OP_N, P(oRI[r + 1]), OP_T, P(oUR[r]), dref(r, 2), dref(r + 1),
                          dref(r + 1), dref(r + 1), dref(r + 1), dref(r + 1)));
    gemm_step(PE, f, std::max(cap[s], 2 * cap[r]), std::max(2 * cap[s + 1], cap[r + 1]));
    f = D.size();
    // L^I_s = B_s^H TL_s ; R^I_r = conj(B_r) UR_r^T
    D.push_back(make_desc(dims, Bs(s), OP_H, P(oTL[s]), OP_N, P(oLI[s]), dref(s + 1), dref(s + 1), dref(s, 2),
                          dref(s + 1), dref(s + 1), dref(s + 1)));
    D.push_back(make_desc(dims, Bs(r), OP_C, P(oUR[r]), OP_T, P(oRI[r]), dref(r), dref(r), dref(r + 1, 2),
                          dref(r + 1, 2), dref(r + 1, 2), dref(r)));
    gemm_step(PE, f, std::max(cap[s + 1], cap[r]), std::max(cap[s + 1], cap[r]));
  }
  // T of the parents of the nodes at site s: T_p = L_p B_s (into the T slab)
  auto parents_T = [&](std::vector<Step>& plan, int s) {
    int v0 = h->site_begin[s], v1 = h->site_begin[s + 1];
    size_t f = D.size();
    std::vector<char> done(nn, 0);
    for (int v = v0; v < v1; ++v) {
      int p = h->node_parent[v];
      if (p < 0 || done[p]) continue;
      done[p] = 1;
      D.push_back(make_desc(dims, P(oL[p]), OP_N, Bs(s), OP_N, Tp(p), dref(s), dref(s + 1, 2), dref(s), dref(s),
                            dref(s + 1, 2), dref(s + 1, 2)));
    }
    gemm_step(plan, f, cap[s], 2 * cap[s + 1]);
  };
  auto Tpar = [&](int v) -> double2* {
    int p = h->node_parent[v];
    return p < 0 ? P(oTL[h->node_site[v]]) : Tp(p);
  };
  // trie forward sweep, site by site: L_v = (O_v B_s)^H T_par(v)
  for (int s = 0; s < n; ++s) {
    int v0 = h->site_begin[s], v1 = h->site_begin[s + 1];
    if (v0 == v1) continue;
    parents_T(PE, s);
    size_t f = D.size();
    for (int v = v0; v < v1; ++v)
      D.push_back(make_desc(dims, OBp(s, h->node_op[v]), OP_H, Tpar(v), OP_N, P(oL[v]), dref(s + 1), dref(s + 1),
                            dref(s, 2), dref(s + 1), dref(s + 1), dref(s + 1)));
    gemm_step(PE, f, cap[s + 1], cap[s + 1]);
  }
  // string expectations and the energy
  std::vector<const double2*> dotL(nt), dotR(nt);
  std::vector<int> dotd(nt);
  for (int k = 0; k < nt; ++k) {
    int v = h->term_node[k];
    int b = h->node_site[v];
    dotL[k] = P(oL[v]);
    dotR[k] = P(oRI[b + 1]);
    dotd[k] = b + 1;
  }
  PE.push_back(Step{Step::DOTS});
  PE.push_back(Step{Step::SUM});

  // ---- cotangent ----
  // A^L_s = T_I(A^L_{s-1}) + sum_{strings ending at s} c L_leaf;  TA_s = A^L_{s-1} B_s
  for (int s = 0; s < n; ++s) {
    size_t f = D.size();
    const double2* Ap = s == 0 ? P(o_zero) : P(oAL[s - 1]);
    D.push_back(make_desc(dims, Ap, OP_N, Bs(s), OP_N, P(oTA[s]), dref(s), dref(s + 1, 2), dref(s), dref(s),
                          dref(s + 1, 2), dref(s + 1, 2)));
    gemm_step(PS, f, cap[s], 2 * cap[s + 1]);
    if (s == n - 1) break;
    f = D.size();
    D.push_back(make_desc(dims, Bs(s), OP_H, P(oTA[s]), OP_N, P(oAL[s]), dref(s + 1), dref(s + 1), dref(s, 2),
                          dref(s + 1), dref(s + 1), dref(s + 1)));
    gemm_step(PS, f, cap[s + 1], cap[s + 1]);
    size_t fa = AX.size();
    AxpyList a{};
    a.out = P(oAL[s]);
    a.src_begin = (int)SRC.size();
    for (int v = h->site_begin[s]; v < h->site_begin[s + 1]; ++v)
      if (h->node_is_end[v]) {
        SRC.push_back(P(oL[v]));
        SRCC.push_back(h->node_end_coeff[v]);
      }
    a.src_end = (int)SRC.size();
    a.didx = s + 1;
    a.mult = 1;
    a.accumulate = 1;
    if (a.src_end > a.src_begin) AX.push_back(a);
    axpy_step(PS, fa, cap[s + 1] * cap[s + 1]);
  }
  // right to left, one site per iteration
  for (int t = n - 1; t >= 0; --t) {
    const int v0 = h->site_begin[t], v1 = h->site_begin[t + 1];
    // X_v = c_v R^I_{t+1} + sum_children Y_child
    if (v1 > v0) {
      size_t fa = AX.size();
      for (int v = v0; v < v1; ++v) {
        AxpyList a{};
        a.out = Xv(v);
        a.src_begin = (int)SRC.size();
        if (h->node_is_end[v]) {
          SRC.push_back(P(oRI[t + 1]));
          SRCC.push_back(h->node_end_coeff[v]);
        }
        for (int e = h->child_off[v]; e < h->child_off[v + 1]; ++e) {
          SRC.push_back(Yv(h->child_idx[e]));
          SRCC.push_back(1.0);
        }
        a.src_end = (int)SRC.size();
        a.didx = t + 1;
        a.mult = 1;
        a.accumulate = 0;
        AX.push_back(a);
      }
      axpy_step(PS, fa, cap[t + 1] * cap[t + 1]);
    }
    if (t > 0 && v1 > v0) {
      // Y_v = T^R_{O_v}(X_v): U_v = B_t X_v^T, Y_v = conj(O_v B_t) U_v^T
      size_t f = D.size();
      for (int v = v0; v < v1; ++v)
        D.push_back(make_desc(dims, Bs(t), OP_N, Xv(v), OP_T, UEv(v), dref(t, 2), dref(t + 1), dref(t + 1),
                              dref(t + 1), dref(t + 1), dref(t + 1)));
      gemm_step(PS, f, 2 * cap[t], cap[t + 1]);
      f = D.size();
      for (int v = v0; v < v1; ++v)
        D.push_back(make_desc(dims, OBp(t, h->node_op[v]), OP_C, UEv(v), OP_T, Yv(v), dref(t), dref(t),
                              dref(t + 1, 2), dref(t + 1, 2), dref(t + 1, 2), dref(t)));
      gemm_step(PS, f, cap[t], cap[t]);
    }
    if (t >= 1) {
      // A^R_t = T^R_I(A^R_{t+1}) + sum_{roots at t} Y_root
      size_t f = D.size();
      D.push_back(make_desc(dims, Bs(t), OP_N, P(oAR[t + 1]), OP_T, P(oURa[t]), dref(t, 2), dref(t + 1),
                            dref(t + 1), dref(t + 1), dref(t + 1), dref(t + 1)));
      gemm_step(PS, f, 2 * cap[t], cap[t + 1]);
      f = D.size();
      D.push_back(make_desc(dims, Bs(t), OP_C, P(oURa[t]), OP_T, P(oAR[t]), dref(t), dref(t), dref(t + 1, 2),
                            dref(t + 1, 2), dref(t + 1, 2), dref(t)));
      gemm_step(PS, f, cap[t], cap[t]);
      size_t fa = AX.size();
      AxpyList a{};
      a.out = P(oAR[t]);
      a.src_begin = (int)SRC.size();
      for (int v = v0; v < v1; ++v)
        if (h->node_parent[v] < 0) {
          SRC.push_back(Yv(v));
          SRCC.push_back(1.0);
        }
      a.src_end = (int)SRC.size();
      a.didx = t;
      a.mult = 1;
      a.accumulate = 1;
      if (a.src_end > a.src_begin) AX.push_back(a);
      axpy_step(PS, fa, cap[t] * cap[t]);
    }
    // Rsum_{t+1} = A^R_{t+1} + (c0 - E) R^I_{t+1}
    {
      Step st{Step::RSUM};
      st.slot = t + 1;
      st.max_m = cap[t + 1] * cap[t + 1];
      PS.push_back(st);
    }
    // Eid_t = TA_t R^I_{t+1}^T + TL_t Rsum_{t+1}^T
    {
      size_t f = D.size();
      D.push_back(make_desc(dims, P(oTA[t]), OP_N, P(oRI[t + 1]), OP_T, P(oEid[t]), dref(t, 2), dref(t + 1),
                            dref(t + 1), dref(t + 1), dref(t + 1), dref(t + 1)));
      gemm_step(PS, f, 2 * cap[t], cap[t + 1]);
      f = D.size();
      D.push_back(make_desc(dims, P(oTL[t]), OP_N, P(oRsum[t + 1]), OP_T, P(oEid[t]), dref(t, 2), dref(t + 1),
                            dref(t + 1), dref(t + 1), dref(t + 1), dref(t + 1), true));
      gemm_step(PS, f, 2 * cap[t], cap[t + 1]);
    }
    if (v1 > v0) {
      // E_v = T_par(v) X_v^T (T of the parents recomputed into the T slab)
      parents_T(PS, t);
      size_t f = D.size();
      for (int v = v0; v < v1; ++v)
        D.push_back(make_desc(dims, Tpar(v), OP_N, Xv(v), OP_T, UEv(v), dref(t, 2), dref(t + 1), dref(t + 1),
                              dref(t + 1), dref(t + 1), dref(t + 1)));
      gemm_step(PS, f, 2 * cap[t], cap[t + 1]);
    }
    Step st{Step::SEED};
    st.slot = t;
    PS.push_back(st);
  }
  std::vector<SeedSite> seeds(n);
  std::vector<const double2*> Enode(nn);
  for (int v = 0; v < nn; ++v) Enode[v] = UEv(v);
  for (int s = 0; s < n; ++s) {
    seeds[s].out = d_Bbar ? d_Bbar + L.site_off[s] : nullptr;
    seeds[s].Eid = P(oEid[s]);
    seeds[s].node_begin = h->site_begin[s];
    seeds[s].node_end = h->site_begin[s + 1];
    seeds[s].s = s;
  }
  std::vector<size_t> ob_off(3 * n);
  for (int i = 0; i < 3 * n; ++i) ob_off[i] = oOB[i];
  // ---- upload tables ----
  size_t tb = 0;
  auto tk = [&](size_t bytes) {
    size_t o = tb;
    tb += align256(std::max<size_t>(bytes, 16));
    return o;
  };
  size_t t_desc = tk(D.size() * sizeof(GemmDesc)), t_ax = tk(AX.size() * sizeof(AxpyList)),
         t_src = tk(SRC.size() * sizeof(void*)), t_srcc = tk(SRCC.size() * sizeof(double)),
         t_dl = tk(nt * sizeof(void*)), t_dr = tk(nt * sizeof(void*)), t_dd = tk(nt * sizeof(int)),
         t_seed = tk(n * sizeof(SeedSite)), t_en = tk(nn * sizeof(void*)), t_op = tk(nn * sizeof(int)),
         t_so = tk((n + 1) * sizeof(size_t)), t_ob = tk(3 * n * sizeof(size_t));
  MPS_TRY(ec.tables.alloc(tb));
  char* tbase = ec.tables.as<char>();
  auto up = [&](size_t o, const void* src, size_t bytes) -> mps_status {
    if (bytes) MPS_CU(cudaMemcpy(tbase + o, src, bytes, cudaMemcpyHostToDevice));
    return MPS_OK;
  };
  MPS_TRY(up(t_desc, D.data(), D.size() * sizeof(GemmDesc)));
  MPS_TRY(up(t_ax, AX.data(), AX.size() * sizeof(AxpyList)));
  MPS_TRY(up(t_src, SRC.data(), SRC.size() * sizeof(void*)));
  MPS_TRY(up(t_srcc, SRCC.data(), SRCC.size() * sizeof(double)));
  MPS_TRY(up(t_dl, dotL.data(), nt * sizeof(void*)));
  MPS_TRY(up(t_dr, dotR.data(), nt * sizeof(void*)));
  MPS_TRY(up(t_dd, dotd.data(), nt * sizeof(int)));
  MPS_TRY(up(t_seed, seeds.data(), n * sizeof(SeedSite)));
  MPS_TRY(up(t_en, Enode.data(), nn * sizeof(void*)));
  MPS_TRY(up(t_op, h->node_op.data(), nn * sizeof(int)));
  MPS_TRY(up(t_so, L.site_off.data(), (n + 1) * sizeof(size_t)));
  MPS_TRY(up(t_ob, ob_off.data(), 3 * n * sizeof(size_t)));
  ec.d_desc = reinterpret_cast<GemmDesc*>(tbase + t_desc);
  ec.d_axpy = reinterpret_cast<AxpyList*>(tbase + t_ax);
  ec.d_src = reinterpret_cast<const double2**>(tbase + t_src);
  ec.d_srccoef = reinterpret_cast<double*>(tbase + t_srcc);
  ec.d_dotL = reinterpret_cast<const double2**>(tbase + t_dl);
  ec.d_dotR = reinterpret_cast<const double2**>(tbase + t_dr);
  ec.d_dotdidx = reinterpret_cast<int*>(tbase + t_dd);
  ec.d_seed = reinterpret_cast<SeedSite*>(tbase + t_seed);
  ec.d_Enode = reinterpret_cast<const double2**>(tbase + t_en);
  ec.d_nodeop = reinterpret_cast<int*>(tbase + t_op);
  ec.d_site_off = reinterpret_cast<size_t*>(tbase + t_so);
  ec.d_ob_off = reinterpret_cast<size_t*>(tbase + t_ob);
  ec.key_arena = arena->uid;
  ec.key_B = sb.B;
  ec.key_dims = sb.dims;
  ec.key_Bbar = d_Bbar;
  return legacy_fence();
}

// Energy (and, when d_Bbar != null, the cotangent dE/dB* written in the state's site layout).
// mixed: the transfer-matrix GEMMs of the energy itself run in 3xTF32 on the tensor cores (the
// sums stay FP64).  The cotangent dE/dB* is always FP64: it seeds the reverse pass, whose SVD
// adjoints amplify its rounding at nearly degenerate Schmidt values (3xTF32 seeds moved
// |dE/dtheta| by up to 7.7x its norm on some random-angle config-1 instances).
static mps_status energy_pass_impl(const Layout& L, const StateBuf& sb, cudaStream_t st, int* status,
                                   mps_hamiltonian_dev* h, double* d_E, double* d_expect, double2* d_Bbar,
                                   bool mixed) {
  const Batch bt = sb.mem.arena->batch();
  if (!h->cache || h->cache->key_arena != sb.mem.arena->uid || h->cache->key_B != sb.B ||
      h->cache->key_dims != sb.dims || (d_Bbar && h->cache->key_Bbar != d_Bbar)) {
    MPS_CU(cudaStreamSynchronize(st));
    h->cache.reset(new EnergyCache());
    MPS_TRY(build_energy_cache(L, sb, h, d_Bbar, *h->cache));
  }
  EnergyCache& ec = *h->cache;
  const int nt = (int)h->x.size();
  auto run = [&](const std::vector<Step>& plan, bool tf32) -> mps_status {
    for (const Step& s : plan) {
      switch (s.kind) {
        case Step::GEMM:
          if (tf32 && s.max_m >= TC_MIN_SIDE && s.max_n >= TC_MIN_SIDE && zgemm_tc_available())
            launch_zgemm_tc_batched(bt, ec.d_desc + s.off, s.count, s.max_m, s.max_n, status, st);
          else if (tf32)
            launch_zgemm_tf32x3_batched(bt, ec.d_desc + s.off, s.count, s.max_m, s.max_n, st);
          else
            launch_zgemm_batched(bt, ec.d_desc + s.off, s.count, s.max_m, s.max_n, st);
          break;
        case Step::AXPY:
          launch_axpy_lists(bt, ec.d_axpy + s.off, s.count, ec.d_src, ec.d_srccoef, sb.dims, s.max_m, st);
          break;
        case Step::PAULIS:
          launch_apply_paulis(bt, sb.B, ec.d_site_off, ec.d_ob_off, sb.dims, L.n, ec.OB, ec.max_site, st);
          break;
        case Step::DOTS: launch_env_dots(bt, ec.d_dotL, ec.d_dotR, ec.d_dotdidx, sb.dims, nt, ec.e, st); break;
        case Step::SUM:
          launch_energy_sum(bt, ec.e, h->d_coeff.as<double>(), nt, h->c0, ec.Z, d_E, d_expect, status, st);
          break;
        case Step::RSUM:
          launch_rsum(bt, ec.Rsum[s.slot], ec.AR[s.slot], ec.RI[s.slot], h->c0, d_E, sb.dims, s.slot, s.max_m, st);
          break;
        case Step::SEED:   // the seed of one site (its trie level's E slab is reused next)
          launch_seed_assemble(bt, ec.d_seed + s.slot, 1, ec.d_Enode, ec.d_nodeop, sb.dims, ec.Z, ec.max_site, st);
          break;
      }
    }
    MPS_CU(cudaGetLastError());
    return MPS_OK;
  };
  MPS_TRY(run(ec.plan_e, mixed));
  if (d_Bbar) MPS_TRY(run(ec.plan_seed, false));
  return MPS_OK;
}

// ---- hamiltonian upload: canonical order + trie ------------------------------------------
static int first_site(uint64_t x, uint64_t z) {
  uint64_t s = x | z;
  return s ? __builtin_ctzll(s) : -1;
}
static int last_site(uint64_t x, uint64_t z) {
  uint64_t s = x | z;
  return s ? 63 - __builtin_clzll(s) : -1;
}
static int sym(uint64_t x, uint64_t z, int s) {
  int xb = (x >> s) & 1, zb = (z >> s) & 1;
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

static mps_status build_trie(mps_hamiltonian_dev* h) {
  const int n = h->n;
  const int nt = (int)h->x.size();
  // DFS order over the canonically sorted strings: reuse the longest common prefix
  std::vector<int> site, op, parent, is_end;
  std::vector<double> endc;
  h->term_node.assign(nt, -1);
  std::vector<int> path;  // node ids of the previous string's path
  int prev_a = -2;
  for (int k = 0; k < nt; ++k) {
    uint64_t x = h->x[k], z = h->z[k];
    int a = first_site(x, z), b = last_site(x, z);
    int lcp = 0;
    if (a == prev_a) {
      while (lcp < (int)path.size() && a + lcp <= b && op[path[lcp]] == sym(x, z, a + lcp)) ++lcp;
    }
    path.resize(lcp);
    for (int s = a + lcp; s <= b; ++s) {
      site.push_back(s);
      op.push_back(sym(x, z, s));
      parent.push_back(path.empty() ? -1 : path.back());
      is_end.push_back(0);
      endc.push_back(0.0);
      path.push_back((int)site.size() - 1);
    }
    int leaf = path[b - a];
    if (is_end[leaf]) return fail(MPS_EINVAL, "mps_hamiltonian_create: duplicate Pauli string");
    is_end[leaf] = 1;
    endc[leaf] = h->c[k];
    h->term_node[k] = leaf;
    path.resize(b - a + 1);
    prev_a = a;
  }
  // stable sort nodes by site
  const int nn = (int)site.size();
  std::vector<int> order(nn);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return site[u] < site[v]; });
  std::vector<int> newid(nn);
  for (int i = 0; i < nn; ++i) newid[order[i]] = i;
  h->node_site.resize(nn);
  h->node_op.resize(nn);
  h->node_parent.resize(nn);
  h->node_is_end.resize(nn);
  h->node_end_coeff.resize(nn);
  for (int i = 0; i < nn; ++i) {
    int u = order[i];
    h->node_site[i] = site[u];
    h->node_op[i] = op[u];
    h->node_parent[i] = parent[u] < 0 ? -1 : newid[parent[u]];
    h->node_is_end[i] = is_end[u];
    h->node_end_coeff[i] = endc[u];
  }
  for (int k = 0; k < nt; ++k) h->term_node[k] = newid[h->term_node[k]];
  h->site_begin.assign(n + 1, 0);
  for (int i = 0; i < nn; ++i) h->site_begin[h->node_site[i] + 1]++;
  for (int s = 0; s < n; ++s) h->site_begin[s + 1] += h->site_begin[s];
  h->child_off.assign(nn + 1, 0);
  for (int i = 0; i < nn; ++i)
    if (h->node_parent[i] >= 0) h->child_off[h->node_parent[i] + 1]++;
  for (int i = 0; i < nn; ++i) h->child_off[i + 1] += h->child_off[i];
  h->child_idx.assign(h->child_off[nn], 0);
  std::vector<int> fill(h->child_off.begin(), h->child_off.end() - 1);
  for (int i = 0; i < nn; ++i)
    if (h->node_parent[i] >= 0) h->child_idx[fill[h->node_parent[i]]++] = i;
  return MPS_OK;
}

// Sum the durations of the profiled SVD launches of the finished call (stream already idle).
static mps_status harvest_profile(Workspace& w) {
  for (size_t i = 0; i + 1 < w.ev_used; i += 2) {
    float ms = 0.f;
    MPS_CU(cudaEventElapsedTime(&ms, w.ev_pool[i], w.ev_pool[i + 1]));
    w.svd_ms += ms;
    ++w.svd_launches;
  }
  w.ev_used = 0;
  return MPS_OK;
}

static mps_status validate_config(const mps_config* cfg) {
  if (!cfg) return fail(MPS_EINVAL, "config is NULL");
  if (cfg->max_bond < 1 || cfg->max_bond > 256)
    return fail(MPS_EINVAL, "max_bond must be in 1..256");
  if (!(cfg->cutoff >= 0.0) || !std::isfinite(cfg->cutoff)) return fail(MPS_EINVAL, "cutoff must be finite and >= 0");
  if (cfg->precision != MPS_PRECISION_FP64 && cfg->precision != MPS_PRECISION_MIXED)
    return fail(MPS_EINVAL, "precision must be MPS_PRECISION_FP64 or MPS_PRECISION_MIXED");
  if (cfg->checkpoint_every < 0) return fail(MPS_EINVAL, "checkpoint_every must be >= 0");
  return MPS_OK;
}

// Starts a call: staging room for `count` doubles of host inputs and outputs per instance
// (plus the status).
static mps_status begin_call(mps_state* s, size_t count) {
  Workspace& w = *s->ws;
  count = count * (size_t)s->n_inst() + 2;
  if (!w.stage || w.stage_n < count) {
    if (w.stage) cudaFreeHost(w.stage);
    w.stage = w.stage_dev = nullptr;
    w.stage_n = 0;
    MPS_CU(cudaHostAlloc(reinterpret_cast<void**>(&w.stage), count * sizeof(double), cudaHostAllocMapped));
    MPS_CU(cudaHostGetDevicePointer(reinterpret_cast<void**>(&w.stage_dev), w.stage, 0));
    w.stage_n = count;
  }
  w.stage_used = 2;
  w.pending.clear();
  return MPS_OK;
}

static size_t stage_take(Workspace& w, size_t count) {
  const size_t o = w.stage_used;
  w.stage_used += count;
  return o;
}

// Ends a call: fetch the status word through the staging, wait for the stream, and copy the
// host outputs out only when the call succeeded (outputs are untouched on error).
static mps_status complete_call(mps_state* s, const char* where);
static mps_status finish_call(mps_state* s, const char* where) {
  Workspace& w = *s->ws;
  launch_status_fetch(s->batch(), s->status.as<int>(), w.stage_dev, s->st);
  return complete_call(s, where);
}

// The second half of finish_call, for calls whose status fetch is already enqueued.
static mps_status complete_call(mps_state* s, const char* where) {
  Workspace& w = *s->ws;
  if (!w.done) MPS_CU(cudaEventCreateWithFlags(&w.done, cudaEventBlockingSync | cudaEventDisableTiming));
  MPS_CU(cudaEventRecord(w.done, s->st));
  MPS_CU(cudaEventSynchronize(w.done));
  const int code = (int)w.stage[0];
  if (code != 0) {
    const char* what = code == MPS_ENOCONV   ? "Jacobi SVD did not converge"
                       : code == MPS_ENUMERIC ? "non-finite or zero norm met on the device"
                       : code == MPS_EINVAL   ? "invalid angle index or non-finite angle"
                                              : "device error";
    std::string inst = s->n_inst() > 1 ? " (instance " + std::to_string((int)w.stage[1]) + ")" : "";
    return fail((mps_status)code, std::string(where) + ": " + what + inst);
  }
  for (const auto& p : w.pending) std::memcpy(p.dst, w.stage + p.off, p.count * sizeof(double));
  w.pending.clear();
  return MPS_OK;
}

// theta (host or device; one row of n_theta values per instance) -> the workspace's per-instance
// copy
static mps_status stage_theta(mps_state* s, const double* theta, int n_theta, const double** d_theta) {
  Workspace& w = *s->ws;
  const Batch bt = s->batch();
  if (n_theta < 0) return fail(MPS_EINVAL, "n_theta < 0");
  if (n_theta > 0 && !theta) return fail(MPS_EINVAL, "theta is NULL");
  MPS_TRY(w.theta.ensure(std::max(1, n_theta) * sizeof(double)));
  *d_theta = w.theta.as<double>();
  if (n_theta == 0) return MPS_OK;
  const size_t row = (size_t)n_theta * sizeof(double);
  bool theta_dev = false;
  MPS_TRY(where_is(theta, "theta", &theta_dev));
  if (theta_dev) {   // finiteness is checked by the gate-matrix kernel
    launch_copy_f64(bt, w.theta.as<double>(), bt.stride, theta, row, n_theta, s->st);
    return MPS_OK;
  }
  const size_t total = (size_t)n_theta * bt.n;
  for (size_t i = 0; i < total; ++i)
    if (!std::isfinite(theta[i])) return fail(MPS_EINVAL, "theta contains a non-finite value");
  const size_t o = stage_take(w, total);
  std::memcpy(w.stage + o, theta, total * sizeof(double));
  launch_copy_f64(bt, w.theta.as<double>(), bt.stride, w.stage_dev + o, row, n_theta, s->st);
  return MPS_OK;
}

// per-instance device result (count values) -> caller's array of one row per instance (device:
// copy kernel; host: through the staging)
static mps_status put_out(mps_state* s, double* dst, const double* dsrc, size_t count) {
  if (!dst || count == 0) return MPS_OK;
  Workspace& w = *s->ws;
  const Batch bt = s->batch();
  const size_t row = count * sizeof(double);
  bool dst_dev = false;
  MPS_TRY(where_is(dst, "an output array", &dst_dev));
  if (dst_dev) {
    launch_copy_f64(bt, dst, row, dsrc, bt.stride, count, s->st);
    return MPS_OK;
  }
  const size_t o = stage_take(w, count * bt.n);
  launch_copy_f64(bt, w.stage_dev + o, row, dsrc, bt.stride, count, s->st);
  w.pending.push_back({dst, o, count * bt.n});
  return MPS_OK;
}

static mps_status ensure_gate_matrices(mps_state* s, const mps_circuit* c) {
  Workspace& w = *s->ws;
  MPS_TRY(w.G.ensure(std::max(1, c->n_gates) * 16 * sizeof(double2)));
  MPS_TRY(w.dG.ensure(std::max(1, c->n_gates) * 16 * sizeof(double2)));
  return MPS_OK;
}

static void gate_matrices_launch(mps_state* s, const mps_circuit* c, const double* d_theta, int n_theta) {
  Workspace& w = *s->ws;
  launch_gate_matrices(s->batch(), c->gates.p, c->n_gates, d_theta, n_theta, w.G.as<double2>(),
                       w.dG.as<double2>(), s->status.as<int>(), s->st);
}

static mps_status gate_matrices(mps_state* s, const mps_circuit* c, const double* d_theta, int n_theta) {
  MPS_TRY(ensure_gate_matrices(s, c));
  gate_matrices_launch(s, c, d_theta, n_theta);
  return MPS_OK;
}

// The state's upload of a host gate list: reused when the contents equal the last upload's.
static mps_status host_circuit(mps_state* s, const mps_gate* gates, int32_t n_gates, const mps_circuit** out) {
  Workspace& w = *s->ws;
  if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(MPS_EINVAL, "bad gate array");
  if (w.host_circ && (int)w.host_circ_gates.size() == n_gates &&
      (n_gates == 0 || std::memcmp(w.host_circ_gates.data(), gates, (size_t)n_gates * sizeof(mps_gate)) == 0)) {
    *out = w.host_circ.get();
    return MPS_OK;
  }
  mps_circuit* c = nullptr;
  MPS_TRY(mps_circuit_create(s->L.n, gates, n_gates, &c));
  w.host_circ.reset(c);
  w.host_circ_gates.assign(gates, gates + n_gates);
  *out = c;
  return MPS_OK;
}

// The state's upload of a host Hamiltonian: reused when the strings and coefficients equal the
// last upload's.
static mps_status host_hamiltonian(mps_state* s, const mps_hamiltonian* h, const mps_hamiltonian_dev** out) {
  Workspace& w = *s->ws;
  if (!h || h->n_terms < 0 || (h->n_terms > 0 && (!h->x_mask || !h->z_mask || !h->coeff)))
    return fail(MPS_EINVAL, "bad Hamiltonian arrays");
  const size_t nt = (size_t)h->n_terms;
  if (w.host_ham && w.host_ham_c.size() == nt &&
      (nt == 0 || (std::memcmp(w.host_ham_x.data(), h->x_mask, nt * 8) == 0 &&
                   std::memcmp(w.host_ham_z.data(), h->z_mask, nt * 8) == 0 &&
                   std::memcmp(w.host_ham_c.data(), h->coeff, nt * 8) == 0))) {
    *out = w.host_ham.get();
    return MPS_OK;
  }
  mps_hamiltonian_dev* hd = nullptr;
  MPS_TRY(mps_hamiltonian_create(s->L.n, h, &hd));
  w.host_ham.reset(hd);
  w.host_ham_x.assign(h->x_mask, h->x_mask + nt);
  w.host_ham_z.assign(h->z_mask, h->z_mask + nt);
  w.host_ham_c.assign(h->coeff, h->coeff + nt);
  *out = hd;
  return MPS_OK;
}

static mps_status check_circuit(const mps_state* s, const mps_circuit* c, int n_theta) {
  if (!c) return fail(MPS_EINVAL, "circuit is NULL");
  if (c->n != s->L.n) return fail(MPS_EINVAL, "circuit and state have different qubit counts");
  if (c->max_theta_idx >= n_theta) return fail(MPS_EINVAL, "a gate's theta_idx is >= n_theta");
  return MPS_OK;
}

// One matrix's SVD on the device, as the gate kernels see it: the row-major input A (host or
// device, m x ncol complex) copied column-major, dims {m/2, 1, ncol/2}, lambda_left = 1.
struct SvdJob {
  DevBuf buf, status;
  double2 *Acm = nullptr, *W = nullptr, *Vs = nullptr, *scratch = nullptr;
  double *s = nullptr, *lam = nullptr, *one = nullptr;
  int* dims = nullptr;
  SvdArgs a{};
};

static mps_status svd_job_setup(SvdJob& j, int m, int ncol, const double* A, int D, double eps) {
  const size_t mn = (size_t)m * ncol, Kc = (size_t)std::min(m, ncol);
  const size_t sizes[] = {mn * 16, Kc * m * 16, Kc * ncol * 16, 2 * mn * 16 + Kc * Kc * 16, Kc * 8, Kc * 8, 256,
                          (size_t)m * 8};
  size_t bytes = 0;
  for (size_t z : sizes) bytes += align256(z);
  MPS_TRY(j.buf.alloc(bytes));
  MPS_TRY(j.status.alloc(sizeof(int)));
  MPS_CU(cudaMemset(j.status.p, 0, sizeof(int)));
  char* p = j.buf.as<char>();
  int part = 0;
  auto take = [&]() {
    char* q = p;
    p += align256(sizes[part++]);
    return q;
  };
  j.Acm = reinterpret_cast<double2*>(take());
  j.W = reinterpret_cast<double2*>(take());
  j.Vs = reinterpret_cast<double2*>(take());
  j.scratch = reinterpret_cast<double2*>(take());
  j.s = reinterpret_cast<double*>(take());
  j.lam = reinterpret_cast<double*>(take());
  j.dims = reinterpret_cast<int*>(take());
  j.one = reinterpret_cast<double*>(take());
  bool dev_in = false;
  MPS_TRY(where_is(A, "mps_svd: A", &dev_in));
  // row-major input -> column-major working copy (host transpose)
  std::vector<double2> hin(mn), hcm(mn);
  MPS_CU(cudaMemcpy(hin.data(), A, mn * 16, dev_in ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < ncol; ++c) hcm[(size_t)c * m + r] = hin[(size_t)r * ncol + c];
  MPS_CU(cudaMemcpy(j.Acm, hcm.data(), mn * 16, cudaMemcpyHostToDevice));
  int hd[3] = {m / 2, 1, ncol / 2};
  MPS_CU(cudaMemcpy(j.dims, hd, sizeof(hd), cudaMemcpyHostToDevice));
  std::vector<double> ones(m / 2, 1.0);
  MPS_CU(cudaMemcpy(j.one, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice));
  SvdArgs& a = j.a;
  a.A = j.Acm;
  a.scratch = j.scratch;
  a.dims = j.dims;
  a.b = 0;
  a.D = D;
  a.eps = eps;
  a.Vs = j.Vs;
  a.s = j.s;
  a.lam_out = j.lam;
  a.W = j.W;
  a.tape_dims = nullptr;
  a.lam_left = j.one;
  a.lam_left_copy = nullptr;
  a.status = j.status.as<int>();
  return MPS_OK;
}

}  // namespace mpsi

using namespace mpsi;

// ===================================================================================================
// C ABI
// ===================================================================================================
extern "C" {

const char* mps_last_error(void) { return mpsi::g_err.c_str(); }

int64_t mps_kernel_launches(void) { return (int64_t)mpsk::launches(); }

mps_status mps_init_product_batch(int32_t n_inst, int32_t n_qubits, const uint8_t* bits, const mps_config* cfg,
                                  mps_state** out) {
  clear_error();
  if (!out) return fail(MPS_EINVAL, "mps_init_product: out is NULL");
  if (n_inst < 1 || n_inst > 4096) return fail(MPS_EINVAL, "mps_init_product: n_inst must be in 1..4096");
  if (n_qubits < 2 || n_qubits > 64) return fail(MPS_EINVAL, "mps_init_product: n_qubits must be in 2..64");
  if (!bits) return fail(MPS_EINVAL, "mps_init_product: bits is NULL");
  MPS_TRY(validate_config(cfg));
  for (int i = 0; i < n_qubits * n_inst; ++i)
    if (bits[i] > 1) return fail(MPS_EINVAL, "mps_init_product: bits must be 0 or 1");
  std::unique_ptr<mps_state> s(new mps_state());
  s->uid = next_uid();
  s->cfg = *cfg;   // checkpoint_every == 0: automatic (whole-circuit tape when it fits)
  s->st = (cudaStream_t)cfg->cuda_stream;
  s->L.build(n_qubits, cfg->max_bond);
  s->arena.reset(new Arena());
  MPS_TRY(s->arena->init(n_inst));
  s->buf.mem.arena = s->arena.get();
  s->status.arena = s->arena.get();
  s->ws.reset(new Workspace(s->arena.get()));
  MPS_TRY(s->buf.alloc(s->L));
  MPS_TRY(s->status.alloc(sizeof(int)));
  const Layout& L = s->L;
  std::vector<double2> hB(L.site_elems());
  std::vector<double> hl(L.lam_elems(), 0.0);
  std::vector<int> hd(n_qubits + 1, 1);
  for (int i = 0; i <= n_qubits; ++i) hl[L.lam_off[i]] = 1.0;
  for (int r = 0; r < n_inst; ++r) {
    const size_t io = (size_t)r * s->arena->stride;
    std::fill(hB.begin(), hB.end(), make_double2(0.0, 0.0));
    for (int q = 0; q < n_qubits; ++q)   // [1][2][1]
      hB[L.site_off[q] + bits[(size_t)r * n_qubits + q]] = make_double2(1.0, 0.0);
    MPS_CU(cudaMemcpy(ish(s->buf.B, io), hB.data(), hB.size() * sizeof(double2), cudaMemcpyHostToDevice));
    MPS_CU(cudaMemcpy(ish(s->buf.lam, io), hl.data(), hl.size() * sizeof(double), cudaMemcpyHostToDevice));
    MPS_CU(cudaMemcpy(ish(s->buf.dims, io), hd.data(), hd.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  MPS_TRY(legacy_fence());
  *out = s.release();
  return MPS_OK;
}

mps_status mps_init_product(int32_t n_qubits, const uint8_t* bits, const mps_config* cfg, mps_state** out) {
  return mps_init_product_batch(1, n_qubits, bits, cfg, out);
}

mps_status mps_state_instances(const mps_state* s, int32_t* n_inst) {
  clear_error();
  if (!s || !n_inst) return fail(MPS_EINVAL, "mps_state_instances: NULL argument");
  *n_inst = s->n_inst();
  return MPS_OK;
}

mps_status mps_clone(const mps_state* s, mps_state** out) {
  clear_error();
  if (!s || !out) return fail(MPS_EINVAL, "mps_clone: NULL argument");
  std::unique_ptr<mps_state> c(new mps_state());
  c->uid = next_uid();
  c->cfg = s->cfg;
  c->st = s->st;
  c->L = s->L;
  c->arena.reset(new Arena());
  MPS_TRY(c->arena->init(s->n_inst()));
  c->buf.mem.arena = c->arena.get();
  c->status.arena = c->arena.get();
  c->ws.reset(new Workspace(c->arena.get()));
  MPS_TRY(c->buf.alloc(c->L));
  MPS_TRY(c->status.alloc(sizeof(int)));
  // instance i of the clone <- instance i of s (the two arenas have different strides)
  const Batch bs = s->batch();
  const Batch bc = c->batch();
  launch_copy_f64(Batch{bs.n, 0}, c->buf.mem.as<double>(), bc.stride, s->buf.mem.as<double>(), bs.stride,
                  c->buf.mem.bytes / sizeof(double), s->st);
  MPS_CU(cudaStreamSynchronize(s->st));
  *out = c.release();
  return MPS_OK;
}

mps_status mps_profile(mps_state* s, int32_t enable) {
  clear_error();
  if (!s) return fail(MPS_EINVAL, "mps_profile: state is NULL");
  Workspace& w = *s->ws;
  MPS_TRY(w.stats.ensure(10 * sizeof(double)));
  w.profile = enable != 0;
  return MPS_OK;
}

mps_status mps_profile_read(mps_state* s, double* out6) {
  clear_error();
  if (!s || !out6) return fail(MPS_EINVAL, "mps_profile_read: NULL argument");
  Workspace& w = *s->ws;
  double fl[4] = {0.0, 0.0, 0.0, 0.0};
  if (w.stats.p) {   // summed over the instances
    MPS_CU(cudaStreamSynchronize(s->st));
    for (int i = 0; i < s->n_inst(); ++i) {
      double* di = ish(w.stats.as<double>(), (size_t)i * s->arena->stride);
      double fi[10];
      MPS_CU(cudaMemcpy(fi, di, sizeof(fi), cudaMemcpyDeviceToHost));
      MPS_CU(cudaMemset(di, 0, sizeof(fi)));
      for (int q = 0; q < 4; ++q) fl[q] += fi[q];
      for (int q = 0; q < 6; ++q) w.phases[q] += q < 4 ? fi[4 + q] * 1e-6 : fi[4 + q];
    }
  }
  out6[0] = w.svd_ms;
  out6[1] = (double)w.svd_launches;
  out6[2] = fl[0];
  out6[3] = fl[1];
  out6[4] = fl[2] * 1e-6;
  out6[5] = fl[3];
  w.svd_ms = 0.0;
  w.svd_launches = 0;
  return MPS_OK;
}

mps_status mps_profile_svd_phases(mps_state* s, double* out6) {
  clear_error();
  if (!s || !out6) return fail(MPS_EINVAL, "mps_profile_svd_phases: NULL argument");
  Workspace& w = *s->ws;
  for (int q = 0; q < 6; ++q) {
    out6[q] = w.phases[q];
    w.phases[q] = 0.0;
  }
  return MPS_OK;
}

void mps_free(mps_state* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  delete s;
}

mps_status mps_read_state(const mps_state* s, int32_t* dims, double* lam, double* tensors) {
  return mps_read_state_instance(s, 0, dims, lam, tensors);
}

mps_status mps_read_state_instance(const mps_state* s, int32_t inst, int32_t* dims, double* lam,
                                   double* tensors) {
  clear_error();
  if (!s || !dims) return fail(MPS_EINVAL, "mps_read_state: NULL argument");
  if (inst < 0 || inst >= s->n_inst()) return fail(MPS_EINVAL, "mps_read_state: instance out of range");
  const Layout& L = s->L;
  const size_t io = (size_t)inst * s->arena->stride;
  struct {
    const double2* B;
    const double* lam;
    const int* dims;
  } view{ish(s->buf.B, io), ish(s->buf.lam, io), ish(s->buf.dims, io)};
  const auto* sbp = &view;
  MPS_CU(cudaStreamSynchronize(s->st));
  std::vector<int> d(L.n + 1);
  MPS_CU(cudaMemcpy(d.data(), sbp->dims, (L.n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  std::memcpy(dims, d.data(), (L.n + 1) * sizeof(int));
  if (lam) {
    size_t o = 0;
    for (int i = 1; i < L.n; ++i) {
      MPS_CU(cudaMemcpy(lam + o, sbp->lam + L.lam_off[i], d[i] * sizeof(double), cudaMemcpyDeviceToHost));
      o += d[i];
    }
  }
  if (tensors) {
    size_t o = 0;
    for (int q = 0; q < L.n; ++q) {
      size_t e = (size_t)d[q] * 2 * d[q + 1];
      MPS_CU(cudaMemcpy(tensors + 2 * o, sbp->B + L.site_off[q], e * sizeof(double2), cudaMemcpyDeviceToHost));
      o += e;
    }
  }
  return MPS_OK;
}

mps_status mps_circuit_create(int32_t n_qubits, const mps_gate* gates, int32_t n_gates, mps_circuit** out) {
  clear_error();
  if (!out) return fail(MPS_EINVAL, "mps_circuit_create: out is NULL");
  if (n_qubits < 2 || n_qubits > 64) return fail(MPS_EINVAL, "mps_circuit_create: n_qubits must be in 2..64");
  if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(MPS_EINVAL, "mps_circuit_create: bad gate array");
  std::unique_ptr<mps_circuit> c(new mps_circuit());
  c->uid = next_uid();
  c->n = n_qubits;
  c->n_gates = n_gates;
  c->host.assign(gates, gates + n_gates);
  for (int t = 0; t < n_gates; ++t) {
    const mps_gate& g = gates[t];
    if (g.bond < 0 || g.bond > n_qubits - 2)
      return fail(MPS_EINVAL, "mps_circuit_create: gate " + std::to_string(t) + " bond out of range");
    if (g.theta_idx >= 0 && (g.rz_site < 0 || g.rz_site > 1 || !std::isfinite(g.theta_scale)))
      return fail(MPS_EINVAL, "mps_circuit_create: gate " + std::to_string(t) + " has a bad Rz description");
    const double* arrs[3] = {g.mat, g.pre, g.post};
    for (int q = 0; q < 3; ++q)
      for (int e = 0; e < 32; ++e)
        if (!std::isfinite(arrs[q][e])) return fail(MPS_EINVAL, "mps_circuit_create: non-finite gate matrix");
    c->max_theta_idx = std::max(c->max_theta_idx, g.theta_idx);
  }
  MPS_TRY(c->gates.alloc(std::max(1, n_gates) * sizeof(mps_gate)));
  if (n_gates) MPS_CU(cudaMemcpy(c->gates.p, gates, n_gates * sizeof(mps_gate), cudaMemcpyHostToDevice));
  const int nth = c->max_theta_idx + 1;
  std::vector<int> off(nth + 1, 0), gi;
  std::vector<double> sc;
  for (int t = 0; t < n_gates; ++t)
    if (gates[t].theta_idx >= 0) off[gates[t].theta_idx + 1]++;
  for (int i = 0; i < nth; ++i) off[i + 1] += off[i];
  gi.assign(off[nth], 0);
  sc.assign(off[nth], 0.0);
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int t = 0; t < n_gates; ++t)   // gate order inside each theta: fixed, ascending
    if (gates[t].theta_idx >= 0) {
      int p = fill[gates[t].theta_idx]++;
      gi[p] = t;
      sc[p] = gates[t].theta_scale;
    }
  MPS_TRY(c->csr_off.alloc((nth + 1) * sizeof(int)));
  MPS_TRY(c->csr_gate.alloc(std::max<size_t>(1, gi.size()) * sizeof(int)));
  MPS_TRY(c->csr_scale.alloc(std::max<size_t>(1, sc.size()) * sizeof(double)));
  MPS_CU(cudaMemcpy(c->csr_off.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!gi.empty()) {
    MPS_CU(cudaMemcpy(c->csr_gate.p, gi.data(), gi.size() * sizeof(int), cudaMemcpyHostToDevice));
    MPS_CU(cudaMemcpy(c->csr_scale.p, sc.data(), sc.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  MPS_TRY(legacy_fence());
  *out = c.release();
  return MPS_OK;
}

void mps_circuit_free(mps_circuit* c) { delete c; }

mps_status mps_hamiltonian_create(int32_t n_qubits, const mps_hamiltonian* hin, mps_hamiltonian_dev** out) {
  clear_error();
  if (!out || !hin) return fail(MPS_EINVAL, "mps_hamiltonian_create: NULL argument");
  if (n_qubits < 2 || n_qubits > 64) return fail(MPS_EINVAL, "mps_hamiltonian_create: n_qubits must be in 2..64");
  if (hin->n_terms < 0 || (hin->n_terms > 0 && (!hin->x_mask || !hin->z_mask || !hin->coeff)))
    return fail(MPS_EINVAL, "mps_hamiltonian_create: bad term arrays");
  std::unique_ptr<mps_hamiltonian_dev> h(new mps_hamiltonian_dev());
  h->uid = next_uid();
  h->n = n_qubits;
  const uint64_t valid = n_qubits == 64 ? ~0ull : ((1ull << n_qubits) - 1ull);
  struct T {
    uint64_t x, z;
    double c;
  };
  std::vector<T> terms;
  for (int k = 0; k < hin->n_terms; ++k) {
    uint64_t x = hin->x_mask[k], z = hin->z_mask[k];
    double c = hin->coeff[k];
    if (!std::isfinite(c)) return fail(MPS_EINVAL, "mps_hamiltonian_create: non-finite coefficient");
    if ((x | z) & ~valid) return fail(MPS_EINVAL, "mps_hamiltonian_create: string acts beyond n_qubits");
    if ((x | z) == 0) {
      h->c0 += c;
      continue;
    }
    terms.push_back({x, z, c});
  }
  std::sort(terms.begin(), terms.end(), [&](const T& A, const T& B) {
    int a1 = first_site(A.x, A.z), a2 = first_site(B.x, B.z);
    if (a1 != a2) return a1 < a2;
    for (int s = a1; s < n_qubits; ++s) {
      int u = sym(A.x, A.z, s), v = sym(B.x, B.z, s);
      if (u != v) return u < v;
    }
    return false;
  });
  for (const auto& t : terms) {
    h->x.push_back(t.x);
    h->z.push_back(t.z);
    h->c.push_back(t.c);
  }
  MPS_TRY(build_trie(h.get()));
  MPS_TRY(h->d_coeff.alloc(std::max<size_t>(1, h->c.size()) * sizeof(double)));
  if (!h->c.empty())
    MPS_CU(cudaMemcpy(h->d_coeff.p, h->c.data(), h->c.size() * sizeof(double), cudaMemcpyHostToDevice));
  MPS_TRY(legacy_fence());
  *out = h.release();
  return MPS_OK;
}

void mps_hamiltonian_free(mps_hamiltonian_dev* h) { delete h; }

mps_status mps_apply_circuit_dev(mps_state* s, const mps_circuit* c, const double* theta, int32_t n_theta) {
  clear_error();
  if (!s) return fail(MPS_EINVAL, "mps_apply_circuit: state is NULL");
  MPS_TRY(check_circuit(s, c, n_theta));
  MPS_TRY(begin_call(s, std::max(0, n_theta)));
  const double* d_theta = nullptr;
  MPS_TRY(stage_theta(s, theta, n_theta, &d_theta));
  MPS_TRY(ensure_forward_scratch(s->L, *s->ws));
  MPS_TRY(gate_matrices(s, c, d_theta, n_theta));
  s->ws->ev_used = 0;
  Ctx cx{&s->L, &s->cfg, s->st, s->status.as<int>(), s->ws.get(), s->batch()};
  MPS_TRY(forward_gates(cx, s->buf, c, s->ws->G.as<double2>(), 0, c->n_gates, nullptr));
  MPS_TRY(finish_call(s, "mps_apply_circuit"));
  return harvest_profile(*s->ws);
}

mps_status mps_apply_circuit(mps_state* s, const mps_gate* gates, int32_t n_gates, const double* theta,
                             int32_t n_theta) {
  clear_error();
  if (!s) return fail(MPS_EINVAL, "mps_apply_circuit: state is NULL");
  const mps_circuit* c = nullptr;
  MPS_TRY(host_circuit(s, gates, n_gates, &c));
  return mps_apply_circuit_dev(s, c, theta, n_theta);
}

mps_status mps_energy_dev(const mps_state* s, const mps_hamiltonian_dev* h, double* E_out, double* expect_out) {
  clear_error();
  if (!s || !h || !E_out) return fail(MPS_EINVAL, "mps_energy: NULL argument");
  if (h->n != s->L.n) return fail(MPS_EINVAL, "mps_energy: Hamiltonian and state have different qubit counts");
  mps_state* ms = const_cast<mps_state*>(s);
  Workspace& w = *ms->ws;
  const int nt = (int)h->x.size();
  MPS_TRY(begin_call(ms, 1 + (size_t)nt));
  MPS_TRY(w.scalars.ensure((2 + std::max(1, nt)) * sizeof(double)));
  double* dE = w.scalars.as<double>();
  double* dX = expect_out ? dE + 2 : nullptr;
  MPS_TRY(energy_pass_impl(s->L, s->buf, s->st, ms->status.as<int>(), const_cast<mps_hamiltonian_dev*>(h), dE, dX,
                           nullptr, s->cfg.precision == MPS_PRECISION_MIXED));
  MPS_TRY(put_out(ms, E_out, dE, 1));
  MPS_TRY(put_out(ms, expect_out, dX, nt));
  return finish_call(ms, "mps_energy");
}

mps_status mps_energy_cotangent_dev(const mps_state* s, const mps_hamiltonian_dev* h, double* E_out,
                                    double* Bbar_out) {
  clear_error();
  if (!s || !h || !E_out || !Bbar_out) return fail(MPS_EINVAL, "mps_energy_cotangent: NULL argument");
  if (h->n != s->L.n) return fail(MPS_EINVAL, "mps_energy_cotangent: qubit counts differ");
  mps_state* ms = const_cast<mps_state*>(s);
  Workspace& w = *ms->ws;
  const Layout& L = s->L;
  MPS_TRY(begin_call(ms, 1));
  MPS_TRY(w.scalars.ensure(4 * sizeof(double)));
  MPS_TRY(w.Bbar.ensure(L.site_elems() * sizeof(double2)));
  double* dE = w.scalars.as<double>();
  MPS_TRY(energy_pass_impl(L, s->buf, s->st, ms->status.as<int>(), const_cast<mps_hamiltonian_dev*>(h), dE, nullptr,
                           w.Bbar.as<double2>(), s->cfg.precision == MPS_PRECISION_MIXED));
  MPS_TRY(put_out(ms, E_out, dE, 1));
  MPS_TRY(finish_call(ms, "mps_energy_cotangent"));
  // dE/dB* of instance 0
  std::vector<int> d(L.n + 1);
  MPS_CU(cudaMemcpy(d.data(), s->buf.dims, (L.n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  bool dev = false;
  MPS_TRY(where_is(Bbar_out, "Bbar_out", &dev));
  size_t o = 0;
  for (int q = 0; q < L.n; ++q) {
    size_t e = (size_t)d[q] * 2 * d[q + 1];
    MPS_CU(cudaMemcpy(Bbar_out + 2 * o, w.Bbar.as<double2>() + L.site_off[q], e * sizeof(double2),
                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    o += e;
  }
  return MPS_OK;
}

mps_status mps_svd_dev(int32_t m, int32_t ncol, const double* A, int32_t D, double eps, double* s_out,
                       double* V_out, double* W_out, int32_t* k_out) {
  clear_error();
  if (!A || !s_out || !V_out || !W_out || !k_out) return fail(MPS_EINVAL, "mps_svd: NULL argument");
  if (m < 2 || ncol < 2 || (m & 1) || (ncol & 1) || m > 512 || ncol > 512)
    return fail(MPS_EINVAL, "mps_svd: m and ncol must be even and in 2..512");
  if (D < 1 || !(eps >= 0.0)) return fail(MPS_EINVAL, "mps_svd: bad D or eps");
  for (const void* o : {(const void*)s_out, (const void*)V_out, (const void*)W_out, (const void*)k_out}) {
    bool od = false;
    MPS_TRY(where_is(o, "mps_svd: an output array", &od));
  }
  const size_t Kc = (size_t)std::min(m, ncol);
  SvdJob job;
  MPS_TRY(svd_job_setup(job, m, ncol, A, D, eps));
  SvdArgs& a = job.a;
  DevBuf& status = job.status;
  int* dims = job.dims;
  double2* W = job.W;
  double2* Vs = job.Vs;
  double* s = job.s;
  DevBuf coop;
  if (std::max(m, ncol) >= SVD_COOP_MIN_SIDE) {   // the multi-SM SVD that large gates use
    MPS_TRY(coop.alloc(svd_coop_scratch_bytes(m, ncol)));
    MPS_CU(launch_svd_coop(a, coop.p, m, ncol, 0));
  } else {
    launch_svd(Batch{1, 0}, a, m, ncol, 0);
  }
  MPS_CU(cudaGetLastError());
  MPS_CU(cudaDeviceSynchronize());
  int code = 0, k = 0;
  MPS_CU(cudaMemcpy(&code, status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) return fail((mps_status)code, "mps_svd: device status");
  MPS_CU(cudaMemcpy(&k, dims + 1, sizeof(int), cudaMemcpyDeviceToHost));
  // Vs, W are column-major (column j contiguous); return them row-major
  std::vector<double2> hV(Kc * ncol), hW(Kc * m), tV(Kc * ncol), tW(Kc * m);
  MPS_CU(cudaMemcpy(hV.data(), Vs, Kc * ncol * 16, cudaMemcpyDeviceToHost));
  MPS_CU(cudaMemcpy(hW.data(), W, Kc * m * 16, cudaMemcpyDeviceToHost));
  for (size_t j = 0; j < Kc; ++j) {
    for (int r = 0; r < ncol; ++r) tV[(size_t)r * Kc + j] = hV[j * ncol + r];
    for (int r = 0; r < m; ++r) tW[(size_t)r * Kc + j] = hW[j * m + r];
  }
  auto out = [&](void* dst, const void* src, size_t b) -> mps_status {
    MPS_CU(cudaMemcpy(dst, src, b, ptr_location(dst) == PTR_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    return MPS_OK;
  };
  std::vector<double> hs(Kc);
  MPS_CU(cudaMemcpy(hs.data(), s, Kc * 8, cudaMemcpyDeviceToHost));
  MPS_TRY(out(s_out, hs.data(), Kc * 8));
  MPS_TRY(out(V_out, tV.data(), Kc * ncol * 16));
  MPS_TRY(out(W_out, tW.data(), Kc * m * 16));
  MPS_TRY(out(k_out, &k, sizeof(int)));
  return MPS_OK;
}

mps_status mps_svd_tune(int32_t m, int32_t ncol, const double* A, int32_t jg32, int32_t jg64, int32_t reps,
                        double* ms_out) {
  clear_error();
  if (!A || !ms_out) return fail(MPS_EINVAL, "mps_svd_tune: NULL argument");
  if (m < 2 || ncol < 2 || (m & 1) || (ncol & 1) || std::max(m, ncol) >= SVD_COOP_MIN_SIDE)
    return fail(MPS_EINVAL, "mps_svd_tune: m and ncol must be even and in 2..128");
  auto ok_jg = [](int g) { return g == 0 || g == 8 || g == 16 || g == 32; };
  if (!ok_jg(jg32) || !ok_jg(jg64)) return fail(MPS_EINVAL, "mps_svd_tune: lanes per pair must be 0, 8, 16 or 32");
  if (reps < 1 || reps > 1000) return fail(MPS_EINVAL, "mps_svd_tune: reps must be in 1..1000");
  SvdJob job;
  MPS_TRY(svd_job_setup(job, m, ncol, A, std::min(m, ncol), 0.0));
  // 0 asks for the kernel's rule; it is passed as -1 so that launch_svd does not read the table
  job.a.jg32 = jg32 ? jg32 : -1;
  job.a.jg64 = jg64 ? jg64 : -1;
  const SvdArgs a = job.a;
  auto launch = [&]() { launch_svd(Batch{1, 0}, a, m, ncol, 0); };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MPS_CU(cudaEventCreate(&e0));
  MPS_CU(cudaEventCreate(&e1));
  launch();   // warm-up
  MPS_CU(cudaEventRecord(e0, 0));
  for (int r = 0; r < reps; ++r) launch();
  MPS_CU(cudaEventRecord(e1, 0));
  MPS_CU(cudaEventSynchronize(e1));
  float ms = 0.f;
  const cudaError_t ce = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MPS_CU(ce);
  MPS_CU(cudaGetLastError());
  int code = 0;
  MPS_CU(cudaMemcpy(&code, job.status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) return fail((mps_status)code, "mps_svd_tune: device status");
  *ms_out = (double)ms / reps;
  return MPS_OK;
}

mps_status mps_set_svd_tiles(int32_t n_entries, const int32_t* entries) {
  clear_error();
  if (n_entries < 0 || (n_entries > 0 && !entries)) return fail(MPS_EINVAL, "mps_set_svd_tiles: bad arguments");
  for (int i = 0; i < n_entries; ++i) {
    const int32_t* e = entries + 4 * i;
    auto ok_jg = [](int g) { return g == 0 || g == 8 || g == 16 || g == 32; };
    if (e[0] < 2 || e[1] < 2 || e[0] > 512 || e[1] > 512 || !ok_jg(e[2]) || !ok_jg(e[3]))
      return fail(MPS_EINVAL, "mps_set_svd_tiles: entry " + std::to_string(i) +
                                  " must be {m_cap, n_cap in 2..512, lanes 0/8/16/32, lanes 0/8/16/32}");
  }
  svd_tiles_set(entries, n_entries);
  return MPS_OK;
}

mps_status mps_zgemm_mixed_dev(int32_t M, int32_t N, int32_t K, const double* A, int32_t lda, int32_t opA,
                               const double* B, int32_t ldb, int32_t opB, double* C, int32_t ldc, int32_t engine) {
  clear_error();
  if (!A || !B || !C) return fail(MPS_EINVAL, "mps_zgemm_mixed: NULL argument");
  if (M < 1 || N < 1 || K < 1 || opA < 0 || opA > 3 || opB < 0 || opB > 3 || engine < 0 || engine > 2)
    return fail(MPS_EINVAL, "mps_zgemm_mixed: bad sizes, op codes or engine");
  if (ldc < N) return fail(MPS_EINVAL, "mps_zgemm_mixed: ldc < N");
  if (lda < ((opA == OP_N || opA == OP_C) ? K : M) || ldb < ((opB == OP_N || opB == OP_C) ? N : K))
    return fail(MPS_EINVAL, "mps_zgemm_mixed: leading dimension too small");
  for (const void* q : {(const void*)A, (const void*)B, (const void*)C})
    if (ptr_location(q) != PTR_DEVICE) return fail(MPS_EINVAL, "mps_zgemm_mixed: arrays must be device memory");
  if (engine == 1 && !zgemm_tc_available()) return fail(MPS_ECUDA, "mps_zgemm_mixed: tcgen05 kernel unavailable");
  GemmDesc d = make_desc(nullptr, reinterpret_cast<const double2*>(A), opA, reinterpret_cast<const double2*>(B), opB,
                         reinterpret_cast<double2*>(C), dconst(M), dconst(N), dconst(K), dconst(lda), dconst(ldb),
                         dconst(ldc));
  DevBuf dd, status;
  MPS_TRY(dd.alloc(sizeof(GemmDesc)));
  MPS_TRY(status.alloc(sizeof(int)));
  MPS_CU(cudaMemcpy(dd.p, &d, sizeof(GemmDesc), cudaMemcpyHostToDevice));
  if (engine == 1)
    launch_zgemm_tc_batched(Batch{1, 0}, dd.as<GemmDesc>(), 1, M, N, status.as<int>(), 0);
  else if (engine == 0)
    launch_zgemm_tf32x3_batched(Batch{1, 0}, dd.as<GemmDesc>(), 1, M, N, 0);
  else
    launch_zgemm_batched(Batch{1, 0}, dd.as<GemmDesc>(), 1, M, N, 0);
  MPS_CU(cudaGetLastError());
  MPS_CU(cudaDeviceSynchronize());
  int code = 0;
  MPS_CU(cudaMemcpy(&code, status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) return fail((mps_status)code, "mps_zgemm_mixed: device status");
  return MPS_OK;
}

mps_status mps_energy(const mps_state* s, const mps_hamiltonian* h, double* E_out) {
  clear_error();
  if (!s || !h) return fail(MPS_EINVAL, "mps_energy: NULL argument");
  const mps_hamiltonian_dev* hd = nullptr;
  MPS_TRY(host_hamiltonian(const_cast<mps_state*>(s), h, &hd));
  return mps_energy_dev(s, hd, E_out, nullptr);
}

}  // extern "C"

namespace mpsi {

// The energy + gradient evaluation, whole (RUN_FULL) or in the two halves of a string-sharded
// evaluation: RUN_BEGIN = forward pass, energy and cotangent of this rank's strings (the
// cotangent copied to Bbar_io); RUN_END = the reverse pass from the cotangent in Bbar_io (summed
// over the ranks by the caller).  Between the halves the workspace keeps the forward's snapshots
// or tape and the gate matrices.
enum RunMode { RUN_FULL = 0, RUN_BEGIN = 1, RUN_END = 2 };

// With defer (RUN_FULL only) the call returns once everything, the status fetch included, is
// enqueued on the state's stream; complete_call and harvest_profile finish it.
static mps_status energy_grad_run(int mode, const mps_state* s0, const mps_circuit* c, const double* theta,
                                  int32_t n_theta, const mps_hamiltonian_dev* hc, double* E_out, double* grad_out,
                                  double* gate_grad_out, double* Bbar_io, bool defer = false) {
  const char* where = mode == RUN_FULL ? "mps_energy_grad" : mode == RUN_BEGIN ? "mps_energy_grad_shard_begin"
                                                                               : "mps_energy_grad_shard_end";
  if (!s0) return fail(MPS_EINVAL, std::string(where) + ": state is NULL");
  if (mode != RUN_END && (!hc || !E_out)) return fail(MPS_EINVAL, std::string(where) + ": NULL argument");
  if (mode != RUN_BEGIN && n_theta > 0 && !grad_out) return fail(MPS_EINVAL, std::string(where) + ": grad_out is NULL");
  mps_state* s = const_cast<mps_state*>(s0);
  mps_hamiltonian_dev* h = const_cast<mps_hamiltonian_dev*>(hc);
  if (h && h->n != s->L.n) return fail(MPS_EINVAL, std::string(where) + ": Hamiltonian and state have different qubit counts");
  MPS_TRY(check_circuit(s, c, n_theta));
  const Layout& L = s->L;
  Workspace& w = *s->ws;
  const size_t bbar_doubles = 2 * L.site_elems();
  if (mode != RUN_FULL) {
    if (!Bbar_io) return fail(MPS_EINVAL, std::string(where) + ": Bbar is NULL");
    if (ptr_location(Bbar_io) != PTR_DEVICE)
      return fail(MPS_EINVAL, std::string(where) + ": Bbar must be device memory of the current device");
  }
  if (mode == RUN_END && w.shard_uid != c->uid)
    return fail(MPS_EINVAL, "mps_energy_grad_shard_end: no mps_energy_grad_shard_begin with this circuit on this state");
  MPS_TRY(begin_call(s, 1 + 2 * (size_t)std::max(0, n_theta) + (gate_grad_out ? (size_t)c->n_gates : 0)));
  const double* d_theta = nullptr;
  if (mode != RUN_END) MPS_TRY(stage_theta(s, theta, n_theta, &d_theta));
  MPS_TRY(ensure_forward_scratch(L, w));
  MPS_TRY(ensure_gate_matrices(s, c));
  MPS_TRY(w.stats.ensure(10 * sizeof(double)));
  w.ev_used = 0;
  const int ng = c->n_gates;
  // tape slot of one gate: pre-gate tensors, C, W, V, s, lambda_left, dims
  auto slot_elems = [&](int b, size_t* cplx, size_t* dbl) {
    const size_t Dl = L.cap[b], Dm = L.cap[b + 1], Dr = L.cap[b + 2], m = 2 * Dl, nc = 2 * Dr;
    const size_t Kc = std::min(m, nc);
    *cplx = Dl * 2 * Dm + Dm * 2 * Dr + m * nc + m * Kc + nc * Kc;   // Bl, Br, C, W, Vs
    *dbl = Kc + Dl + 4;   // s, lambda_left, dims (8 ints)
  };
  auto slot_bytes = [&](int b) {
    size_t cp, db;
    slot_elems(b, &cp, &db);
    return align256(cp * sizeof(double2)) + align256(db * sizeof(double));
  };
  int K = s->cfg.checkpoint_every;
  if (K <= 0 && w.auto_uid == c->uid) {
    K = w.auto_K;   // decided on the first call with this circuit
  } else if (K <= 0) {   // automatic: keep the whole circuit's tape when it takes < 60% of free memory
    size_t all = 0;
    for (int t = 0; t < ng; ++t) all += slot_bytes(c->host[t].bond);
    size_t fr = 0, tot = 0;
    MPS_CU(cudaMemGetInfo(&fr, &tot));
    const double ni = (double)s->n_inst();
    K = (ni * (double)(all + w.tape.bytes) <= 0.6 * ((double)fr + ni * (double)w.tape.bytes)) ? std::max(1, ng) : 512;
    w.auto_uid = c->uid;
    w.auto_K = K;
  }
  const int nseg = (ng + K - 1) / K;
  if (!w.work_ok) {
    MPS_TRY(w.work.alloc(L));
    MPS_TRY(w.rec.alloc(L));
    w.work_ok = true;
  }
  if (nseg > 1)
    while ((int)w.snaps.size() < nseg) {
      w.snaps.emplace_back(new StateBuf(w.arena));
      MPS_TRY(w.snaps.back()->alloc(L));
    }
  // tape arena for the largest segment
  size_t arena = 0;
  for (int seg = 0; seg < nseg; ++seg) {
    size_t tot = 0;
    for (int t = seg * K; t < std::min(ng, (seg + 1) * K); ++t) tot += slot_bytes(c->host[t].bond);
    arena = std::max(arena, tot);
  }
  MPS_TRY(w.tape.ensure(std::max<size_t>(arena, 256)));
  const size_t mc = 2 * (size_t)L.max_cap, nc = 2 * (size_t)L.max_cap, kc = L.max_cap;
  const size_t rv_elems[] = {nc * kc, mc * nc, nc * kc, nc * nc, mc * nc, mc * nc, mc * nc, mc * nc, 16};
  size_t rv_total = 0;
  for (size_t e : rv_elems) rv_total += align256(e * sizeof(double2));
  rv_total += align256(nc * sizeof(double));
  MPS_TRY(w.rv.ensure(rv_total));
  {
    char* p = w.rv.as<char>();
    double2** dst[] = {&w.Vbar, &w.Cbar, &w.Y, &w.Km, &w.T1, &w.Ctbar, &w.Theta, &w.Thbar, &w.Gbar};
    for (int i = 0; i < 9; ++i) {
      *dst[i] = reinterpret_cast<double2*>(p);
      p += align256(rv_elems[i] * sizeof(double2));
    }
    w.wbar = reinterpret_cast<double*>(p);
  }
  MPS_TRY(w.Bbar.ensure(L.site_elems() * sizeof(double2)));
  MPS_TRY(w.lambar.ensure(L.lam_elems() * sizeof(double)));
  MPS_TRY(w.gate_grad.ensure(std::max(1, ng) * sizeof(double)));
  MPS_TRY(w.grad.ensure(std::max(1, n_theta) * sizeof(double)));
  MPS_TRY(w.scalars.ensure(4 * sizeof(double)));
  Ctx cx{&L, &s->cfg, s->st, s->status.as<int>(), &w, s->batch()};
  const double2* G = w.G.as<double2>();
  const double2* dG = w.dG.as<double2>();
  double* dE = w.scalars.as<double>();
  std::vector<TapeSlot> tapes;
  auto layout_tapes = [&](int g0, int g1) {
    tapes.assign(g1 - g0, TapeSlot{});
    char* p = w.tape.as<char>();
    for (int t = g0; t < g1; ++t) {
      const int b = c->host[t].bond;
      const size_t Dl = L.cap[b], Dm = L.cap[b + 1], Dr = L.cap[b + 2], m = 2 * Dl, ncol = 2 * Dr;
      const size_t Kc = std::min(m, ncol);
      size_t cp, db;
      slot_elems(b, &cp, &db);
      TapeSlot& tp = tapes[t - g0];
      double2* z = reinterpret_cast<double2*>(p);
      tp.Bl = z;
      tp.Br = tp.Bl + Dl * 2 * Dm;
      tp.C = tp.Br + Dm * 2 * Dr;
      tp.W = tp.C + m * ncol;
      tp.Vs = tp.W + m * Kc;
      p += align256(cp * sizeof(double2));
      double* dd = reinterpret_cast<double*>(p);
      tp.s = dd;
      tp.lamL = dd + Kc;
      tp.dims = reinterpret_cast<int*>(dd + Kc + Dl);
      p += align256(db * sizeof(double));
    }
  };
  // Everything from the gate matrices to dE/dtheta, enqueued on the state's stream with no host
  // round trip, so that it can be captured once as a CUDA graph and replayed.
  auto fwd_part = [&]() -> mps_status {
    gate_matrices_launch(s, c, d_theta, n_theta);
    MPS_TRY(w.work.copy_from(s->buf, L, s->st));
    if (nseg == 1) {
      // whole-circuit tape: one forward pass records everything the reverse pass needs
      layout_tapes(0, ng);
      MPS_TRY(forward_gates(cx, w.work, c, G, 0, ng, &tapes));
    } else {
      // forward with an MPS snapshot at the start of every segment
      for (int seg = 0; seg < nseg; ++seg) {
        MPS_TRY(w.snaps[seg]->copy_from(w.work, L, s->st));
        MPS_TRY(forward_gates(cx, w.work, c, G, seg * K, std::min(ng, (seg + 1) * K), nullptr));
      }
    }
    // energy and its cotangent
    MPS_TRY(energy_pass_impl(L, w.work, s->st, s->status.as<int>(), h, dE, nullptr, w.Bbar.as<double2>(),
                             s->cfg.precision == MPS_PRECISION_MIXED));
    return MPS_OK;
  };
  auto rev_part = [&]() -> mps_status {
    if (nseg == 1) layout_tapes(0, ng);   // the whole-circuit tape the forward pass recorded
    launch_zero_f64(cx.bt, w.lambar.as<double>(), L.lam_elems(), s->st);
    launch_zero_f64(cx.bt, w.gate_grad.as<double>(), std::max(1, ng), s->st);
    // reverse, segment by segment (re-running a segment's forward from its snapshot with a tape)
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int g0 = seg * K, g1 = std::min(ng, (seg + 1) * K);
      if (nseg > 1) {
        layout_tapes(g0, g1);
        MPS_TRY(w.rec.copy_from(*w.snaps[seg], L, s->st));
        MPS_TRY(forward_gates(cx, w.rec, c, G, g0, g1, &tapes));
      }
      for (int t = g1 - 1; t >= g0; --t)
        MPS_TRY(reverse_gate(cx, t, c->host[t].bond, tapes[t - g0], w.Bbar.as<double2>(), w.lambar.as<double>(), G,
                             dG, w.gate_grad.as<double>()));
      MPS_CU(cudaGetLastError());
    }
    if (n_theta > 0) {
      launch_zero_f64(cx.bt, w.grad.as<double>(), n_theta, s->st);
      launch_theta_reduce(cx.bt, w.gate_grad.as<double>(), c->csr_off.as<int>(), c->csr_gate.as<int>(),
                          c->csr_scale.as<double>(), c->max_theta_idx + 1, w.grad.as<double>(), s->st);
    }
    return MPS_OK;
  };
  auto body = [&]() -> mps_status {
    MPS_TRY(fwd_part());
    return rev_part();
  };
  if (mode == RUN_BEGIN) {   // this rank's energy and cotangent; the caller sums them over ranks
    MPS_TRY(fwd_part());
    launch_copy_f64(cx.bt, Bbar_io, bbar_doubles * sizeof(double), w.Bbar.as<double>(), cx.bt.stride, bbar_doubles,
                    s->st);
    MPS_TRY(put_out(s, E_out, dE, 1));
    w.shard_uid = c->uid;
    MPS_TRY(finish_call(s, where));
    return harvest_profile(w);
  }
  if (mode == RUN_END) {     // the reverse pass from the summed cotangent
    launch_copy_f64(cx.bt, w.Bbar.as<double>(), cx.bt.stride, Bbar_io, bbar_doubles * sizeof(double), bbar_doubles,
                    s->st);
    MPS_TRY(rev_part());
    w.shard_uid = -1;
    MPS_TRY(put_out(s, grad_out, w.grad.as<double>(), n_theta));
    MPS_TRY(put_out(s, gate_grad_out, w.gate_grad.as<double>(), ng));
    MPS_TRY(finish_call(s, where));
    return harvest_profile(w);
  }
  // The graph is valid while none of the buffers it touches has moved.
  const EnergyCache* ec = h->cache.get();
  std::vector<const void*> key = {(const void*)s->arena->uid, (const void*)c->uid, (const void*)h->uid,
                                  (const void*)(intptr_t)n_theta,
                                  (const void*)(intptr_t)K, w.tape.p, w.rv.p, w.Bbar.p, w.lambar.p,
                                  w.gate_grad.p, w.grad.p, w.theta.p, w.G.p, w.dG.p, w.A.p, w.svd.p, w.C.p,
                                  w.Vs.p, w.s.p, w.stats.p, w.scalars.p, w.work.mem.p, w.rec.mem.p,
                                  ec, ec ? ec->bufs.p : nullptr, ec ? ec->tables.p : nullptr,
                                  (const void*)(intptr_t)w.profile, (const void*)(intptr_t)L.one_cta_svd};
  for (auto& sp : w.snaps) key.push_back(sp->mem.p);
  if (w.graph_exec && key == w.graph_key) {
    MPS_CU(cudaGraphLaunch(w.graph_exec, s->st));
    add_launches(w.graph_kernels);
    w.ev_used = w.graph_ev_used;   // the graph re-records the profiling events of its capture
  } else if (key == w.graph_seen && s->cfg.cuda_stream != nullptr && !state_uses_coop(L, s->n_inst())) {
    // second call with the same buffers: capture the call as a graph, then replay it
    if (w.graph_exec) {
      cudaGraphExecDestroy(w.graph_exec);
      w.graph_exec = nullptr;
    }
    const long long l0 = mpsk::thread_launches();
    MPS_CU(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    mps_status st = body();
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s->st, &graph);
    if (st != MPS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return fail(MPS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&w.graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      w.graph_exec = nullptr;
      return fail(MPS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    }
    w.graph_kernels = mpsk::thread_launches() - l0;
    mpsk::add_launches(-w.graph_kernels);   // captured, not launched: counted at each replay
    w.graph_key = key;
    w.graph_ev_used = w.ev_used;
    MPS_CU(cudaGraphLaunch(w.graph_exec, s->st));
    add_launches(w.graph_kernels);
  } else {
    MPS_TRY(body());
    w.graph_seen = key;
  }
  MPS_TRY(put_out(s, E_out, dE, 1));
  MPS_TRY(put_out(s, grad_out, w.grad.as<double>(), n_theta));
  MPS_TRY(put_out(s, gate_grad_out, w.gate_grad.as<double>(), ng));
  if (defer) {
    launch_status_fetch(s->batch(), s->status.as<int>(), w.stage_dev, s->st);
    return MPS_OK;
  }
  MPS_TRY(finish_call(s, "mps_energy_grad"));
  return harvest_profile(w);
}

// Streams and events of mps_energy_grad_multi, created once per device and kept.
struct MultiPool {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
};

static mps_status multi_pool(int need, MultiPool** out) {
  static std::mutex mu;
  static std::map<int, MultiPool> pools;
  int dev = 0;
  MPS_CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  MultiPool& p = pools[dev];
  while ((int)p.streams.size() < need) {
    cudaStream_t st = nullptr;
    MPS_CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    p.streams.push_back(st);
  }
  while ((int)p.events.size() < 2 * need) {
    cudaEvent_t ev = nullptr;
    MPS_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    p.events.push_back(ev);
  }
  *out = &p;
  return MPS_OK;
}

}  // namespace mpsi

extern "C" {

mps_status mps_energy_grad_dev(const mps_state* s0, const mps_circuit* c, const double* theta, int32_t n_theta,
                               const mps_hamiltonian_dev* hc, double* E_out, double* grad_out,
                               double* gate_grad_out) {
  clear_error();
  return energy_grad_run(RUN_FULL, s0, c, theta, n_theta, hc, E_out, grad_out, gate_grad_out, nullptr);
}

mps_status mps_set_svd_policy(mps_state* s, int32_t policy) {
  clear_error();
  if (!s) return fail(MPS_EINVAL, "mps_set_svd_policy: state is NULL");
  if (policy != MPS_SVD_AUTO && policy != MPS_SVD_ONE_CTA)
    return fail(MPS_EINVAL, "mps_set_svd_policy: policy must be MPS_SVD_AUTO or MPS_SVD_ONE_CTA");
  s->L.one_cta_svd = policy == MPS_SVD_ONE_CTA;
  return MPS_OK;
}

mps_status mps_energy_grad_multi(int32_t n_prob, mps_state* const* states, const mps_circuit* const* circuits,
                                 const double* const* theta, const int32_t* n_theta,
                                 const mps_hamiltonian_dev* const* hams, double* const* E_out,
                                 double* const* grad_out) {
  clear_error();
  if (n_prob < 1 || !states || !circuits || !theta || !n_theta || !hams || !E_out || !grad_out)
    return fail(MPS_EINVAL, "mps_energy_grad_multi: NULL argument or n_prob < 1");
  for (int i = 0; i < n_prob; ++i) {
    if (!states[i] || !circuits[i] || !hams[i])
      return fail(MPS_EINVAL, "mps_energy_grad_multi: NULL state, circuit or Hamiltonian at " + std::to_string(i));
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i])
        return fail(MPS_EINVAL, "mps_energy_grad_multi: the same state appears twice (" + std::to_string(j) +
                                    ", " + std::to_string(i) + ")");
  }
  MultiPool* pool = nullptr;
  MPS_TRY(multi_pool(n_prob + 1, &pool));
  std::vector<cudaStream_t> saved_st(n_prob);
  std::vector<void*> saved_cfg(n_prob);
  std::vector<char> enqueued(n_prob, 0);
  mps_status first = MPS_OK;
  std::string first_msg;
  auto note = [&](mps_status st) {
    if (st != MPS_OK && first == MPS_OK) {
      first = st;
      first_msg = mps_last_error();
    }
  };
  // every problem's own stream order: its pool stream starts after the work already on it
  for (int i = 0; i < n_prob; ++i) {
    mps_state* s = states[i];
    saved_st[i] = s->st;
    saved_cfg[i] = s->cfg.cuda_stream;
    note(cudaEventRecord(pool->events[i], s->st) == cudaSuccess ? MPS_OK : fail(MPS_ECUDA, "event record"));
  }
  const cudaStream_t join = pool->streams[n_prob];
  // problems on the one-CTA SVD: concurrently, one pool stream each
  for (int i = 0; i < n_prob && first == MPS_OK; ++i) {
    mps_state* s = states[i];
    if (state_uses_coop(s->L, s->n_inst())) continue;
    const cudaStream_t st = pool->streams[i];
    if (cudaStreamWaitEvent(st, pool->events[i], 0) != cudaSuccess) {
      note(fail(MPS_ECUDA, "stream wait"));
      break;
    }
    s->st = st;
    s->cfg.cuda_stream = st;
    const mps_status r = energy_grad_run(RUN_FULL, s, circuits[i], theta[i], n_theta[i], hams[i], E_out[i],
                                         grad_out[i], nullptr, nullptr, true);
    note(r);
    if (r == MPS_OK) {
      enqueued[i] = 1;
      note(cudaEventRecord(pool->events[n_prob + i], st) == cudaSuccess ? MPS_OK : fail(MPS_ECUDA, "event record"));
      note(cudaStreamWaitEvent(join, pool->events[n_prob + i], 0) == cudaSuccess ? MPS_OK
                                                                                  : fail(MPS_ECUDA, "stream wait"));
    }
  }
  // problems on the cooperative (whole-GPU) SVD: one after another on the join stream, after all
  // of the above, so that a cooperative grid never shares the GPU with them
  for (int i = 0; i < n_prob && first == MPS_OK; ++i) {
    mps_state* s = states[i];
    if (!state_uses_coop(s->L, s->n_inst())) continue;
    if (cudaStreamWaitEvent(join, pool->events[i], 0) != cudaSuccess) {
      note(fail(MPS_ECUDA, "stream wait"));
      break;
    }
    s->st = join;
    s->cfg.cuda_stream = join;
    note(energy_grad_run(RUN_FULL, s, circuits[i], theta[i], n_theta[i], hams[i], E_out[i], grad_out[i], nullptr,
                         nullptr, false));
  }
  for (int i = 0; i < n_prob; ++i) {
    if (enqueued[i]) {
      mps_state* s = states[i];
      note(complete_call(s, "mps_energy_grad_multi"));
      note(harvest_profile(*s->ws));
    }
  }
  if (first == MPS_OK && cudaStreamSynchronize(join) != cudaSuccess) note(fail(MPS_ECUDA, "join stream"));
  if (first != MPS_OK)   // a problem that failed part-way may have left work on its pool stream
    for (int i = 0; i <= n_prob; ++i) cudaStreamSynchronize(pool->streams[i]);
  for (int i = 0; i < n_prob; ++i) {
    states[i]->st = saved_st[i];
    states[i]->cfg.cuda_stream = saved_cfg[i];
  }
  if (first != MPS_OK) return fail(first, first_msg);
  return MPS_OK;
}

mps_status mps_energy_grad_shard_begin(const mps_state* s0, const mps_circuit* c, const double* theta,
                                       int32_t n_theta, const mps_hamiltonian_dev* h_shard, double* E_out,
                                       double* Bbar_out) {
  clear_error();
  return energy_grad_run(RUN_BEGIN, s0, c, theta, n_theta, h_shard, E_out, nullptr, nullptr, Bbar_out);
}

mps_status mps_energy_grad_shard_end(const mps_state* s0, const mps_circuit* c, int32_t n_theta,
                                     const double* Bbar_in, double* grad_out, double* gate_grad_out) {
  clear_error();
  return energy_grad_run(RUN_END, s0, c, nullptr, n_theta, nullptr, nullptr, grad_out, gate_grad_out,
                         const_cast<double*>(Bbar_in));
}

mps_status mps_cotangent_size(const mps_state* s, int64_t* n_doubles) {
  clear_error();
  if (!s || !n_doubles) return fail(MPS_EINVAL, "mps_cotangent_size: NULL argument");
  *n_doubles = (int64_t)(2 * s->L.site_elems()) * s->n_inst();
  return MPS_OK;
}

mps_status mps_energy_grad(const mps_state* s0, const mps_gate* gates, int32_t n_gates, const double* theta,
                           int32_t n_theta, const mps_hamiltonian* h, double* E_out, double* grad_out,
                           double* gate_grad_out) {
  clear_error();
  if (!s0 || !h) return fail(MPS_EINVAL, "mps_energy_grad: NULL argument");
  mps_state* s = const_cast<mps_state*>(s0);
  const mps_circuit* c = nullptr;
  MPS_TRY(host_circuit(s, gates, n_gates, &c));
  const mps_hamiltonian_dev* hd = nullptr;
  MPS_TRY(host_hamiltonian(s, h, &hd));
  return mps_energy_grad_dev(s0, c, theta, n_theta, hd, E_out, grad_out, gate_grad_out);
}

}  // extern "C"
