// Gate SVD (steps S3-S4, Sec. 3) of one large two-site matrix spread over the whole GPU.
//
// The one-CTA kernel in gate_kernels.cu keeps a matrix in shared memory and serves one instance
// per CTA; a single instance at D = 256 has one (2D) x (2D) = 512 x 512 complex matrix per gate,
// which does not fit in one SM's shared memory and would run on one SM out of 152.  Here the
// same cyclic one-sided Jacobi method runs on one matrix with every SM of the GPU:
//
//   * X (R x K, the K columns being orthogonalised) and the accumulated rotation Q (K x K) live in
//     global memory (8 MB at 512 x 512, resident in L2);
//   * a round of the round-robin ordering rotates K/2 disjoint column pairs; each pair is handled
//     by a group of PW warps of one CTA (rows split between the warps, a shared-memory reduction
//     of the inner product), and consecutive rounds are separated by a grid-wide barrier;
//   * the kernel is launched cooperatively, so every CTA is resident and the barrier is a plain
//     arrive-and-wait on a generation counter.  Every wait is bounded: after two seconds it
//     records MPS_ETIMEOUT and the whole grid returns.
//
// Arithmetic is FP64 throughout (no FP32 preconditioning): the rotation, screening, early-stop
// and output rules are those of the one-CTA kernel, so the results agree with it to rounding.
#include <cooperative_groups.h>

#include <algorithm>

#include "../../include/mps.h"
#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

constexpr int CO_THREADS = 256;                // 8 warps
constexpr int CO_PW = 4;                       // warps per column pair
constexpr int CO_SLOTS = CO_THREADS / 32 / CO_PW;   // pairs per CTA per round
constexpr int CO_MAX_SWEEPS = 60;
constexpr double CO_NULL_REL = 1e-13;          // numerical zeros (same rule as the one-CTA kernel)
constexpr unsigned long long CO_WAIT_NS = 2000000000ull;   // bound of every barrier wait

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Synchronisation words of one launch (zeroed by svd_coop_reset before it).
struct CoopSync {
  unsigned count;           // arrivals at the current barrier
  unsigned gen;             // barrier generation
  int abort;                // set when a wait gave up: every CTA returns
  int rotated[2];           // per sweep parity: some pair was rotated
  unsigned long long maxrel[2];   // per sweep parity: largest rotated |gamma|^2/(alpha beta)
  double fro2;              // unused slot kept for alignment
};

struct CoopArgs {
  SvdArgs p;
  double2* X;       // R x K, column j at X + j R
  double2* Q;       // K x K
  double* nrm;      // K
  double* sv;       // K
  double* part;     // per CTA partial sums
  CoopSync* sync;
};

__global__ void svd_coop_reset(CoopSync* s) {
  s->count = 0;
  s->abort = 0;
  s->rotated[0] = s->rotated[1] = 0;
  s->maxrel[0] = s->maxrel[1] = 0ull;
}

// Grid-wide barrier of a cooperative launch, bounded: false when the grid must stop.
__device__ bool grid_sync(CoopSync* s, int* status) {
  __syncthreads();
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &s->gen;
    volatile int* ab = &s->abort;
    int ok = 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&s->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&s->count, 0u);
      __threadfence();
      atomicAdd(&s->gen, 1u);
    } else {
      const unsigned long long t0 = now_ns();
      while (*gen == g) {
        if (*ab) {
          ok = 0;
          break;
        }
        if (now_ns() - t0 > CO_WAIT_NS) {
          set_status(status, MPS_ETIMEOUT);
          atomicExch(&s->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*ab) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Named barrier of the PW warps that share one column pair.
__device__ __forceinline__ void slot_sync(int slot) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(CO_PW * 32));
}

__global__ void __launch_bounds__(CO_THREADS) svd_coop_kernel(const CoopArgs ca) {
  const SvdArgs& p = ca.p;
  const unsigned long long t_start = now_ns();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int slot = warp / CO_PW, sw = warp % CO_PW;          // pair slot in the CTA, warp in the slot
  const int gwarp = blockIdx.x * (CO_THREADS / 32) + warp;   // global warp index
  const int nwarps = gridDim.x * (CO_THREADS / 32);
  const int b = p.b;
  const int Dl = p.dims[b], Dr = p.dims[b + 2];
  const int m = 2 * Dl, n = 2 * Dr;
  const bool tall = m >= n;
  const int R = tall ? m : n, K = tall ? n : m;
  const int Kp = K + (K & 1);
  double2* X = ca.X;
  double2* Q = ca.Q;
  double* nrm = ca.nrm;
  const double2* A = p.A;   // C~ column-major (m x n)
  __shared__ double red_sh[CO_SLOTS][CO_PW][2];
  __shared__ double blk_sh[CO_THREADS / 32];

  // ---- X = X0 (C~ for m >= n, C~^H otherwise), Q = I, ||X||_F^2 ----
  const size_t nthreads = (size_t)gridDim.x * CO_THREADS;
  const size_t gtid = (size_t)blockIdx.x * CO_THREADS + tid;
  double f = 0.0;
  for (size_t e = gtid; e < (size_t)R * K; e += nthreads) {
    const int j = (int)(e / R), r = (int)(e % R);
    const double2 v = tall ? A[(size_t)j * m + r] : conjd(A[(size_t)r * m + j]);
    X[e] = v;
    f += v.x * v.x + v.y * v.y;
  }
  for (size_t e = gtid; e < (size_t)K * K; e += nthreads)
    Q[e] = make_double2((e / K) == (e % K) ? 1.0 : 0.0, 0.0);
  f = wsum(f);
  if (lane == 0) blk_sh[warp] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < CO_THREADS / 32; ++w) t += blk_sh[w];
    ca.part[blockIdx.x] = t;
  }
  if (!grid_sync(ca.sync, p.status)) return;
  double fro2 = 0.0;
  for (int c = 0; c < (int)gridDim.x; ++c) fro2 += __ldcg(ca.part + c);   // same order in every CTA
  const double tiny = 1e-30 * fro2;
  const double tol = 4.0 * 2.220446049250313e-16 * sqrt((double)R);
  const double tol2 = tol * tol, early = 100.0 * tol2;

  // ---- cyclic sweeps ----
  long long checks = 0, rots = 0;   // counted by the first thread of each pair slot
  int sweep = 0, converged = 0;
  for (; sweep < CO_MAX_SWEEPS; ++sweep) {
    const int par = sweep & 1;
    for (int j = gwarp; j < K; j += nwarps) {   // column norms, one warp per column
      double v = 0.0;
      for (int i = lane; i < R; i += 32) {
        const double2 x = __ldcg(X + (size_t)j * R + i);
        v += x.x * x.x + x.y * x.y;
      }
      v = wsum(v);
      if (lane == 0) nrm[j] = v;
    }
    if (!grid_sync(ca.sync, p.status)) return;
    // The next sweep's flags share a slot with the previous sweep's, which every CTA read before
    // arriving at the barrier above; the next sweep first touches them after its own norm barrier.
    if (blockIdx.x == 0 && tid == 0) {
      ca.sync->rotated[par ^ 1] = 0;
      ca.sync->maxrel[par ^ 1] = 0ull;
    }
    for (int r = 0; r < Kp - 1; ++r) {
      for (int t = blockIdx.x * CO_SLOTS + slot; t < Kp / 2; t += gridDim.x * CO_SLOTS) {
        int pc, qc;
        if (t == 0) {
          pc = r;
          qc = Kp - 1;
        } else {
          pc = (r + t) % (Kp - 1);
          qc = (r - t + Kp - 1) % (Kp - 1);
        }
        if (pc >= K || qc >= K) continue;           // uniform over the slot's warps
        const double al = __ldcg(nrm + pc), be = __ldcg(nrm + qc);
        if (al < tiny || be < tiny) continue;
        double2* ap = X + (size_t)pc * R;
        double2* aq = X + (size_t)qc * R;
        double gr = 0.0, gi = 0.0;
        for (int i = sw * 32 + lane; i < R; i += CO_PW * 32) {
          const double2 x = __ldcg(ap + i), y = __ldcg(aq + i);
          gr += x.x * y.x + x.y * y.y;   // conj(x) y
          gi += x.x * y.y - x.y * y.x;
        }
        gr = wsum(gr);
        gi = wsum(gi);
        if (lane == 0) {
          red_sh[slot][sw][0] = gr;
          red_sh[slot][sw][1] = gi;
        }
        slot_sync(slot);
        gr = 0.0;
        gi = 0.0;
#pragma unroll
        for (int w = 0; w < CO_PW; ++w) {   // fixed order: every thread gets the same bits
          gr += red_sh[slot][w][0];
          gi += red_sh[slot][w][1];
        }
        slot_sync(slot);                    // red_sh is reused by the slot's next pair
        if (sw == 0 && lane == 0) ++checks;
        const double g2 = gr * gr + gi * gi;
        const double ab = al * be;
        if (!(g2 > tol2 * ab)) continue;
        const double inv_g = rsqrt(g2);
        const double g = g2 * inv_g;
        const double zeta = (be - al) * (0.5 * inv_g);
        const double az = fabs(zeta);
        const double tt = az > 1e150 ? 0.5 / zeta : copysign(1.0 / (az + sqrt(1.0 + zeta * zeta)), zeta);
        const double c = rsqrt(1.0 + tt * tt), s = c * tt;
        const double pr = gr * inv_g, pim = gi * inv_g;   // e^{i phi}
        const double spr = s * pr, spi = s * pim;
        // a_p' = c a_p - s e^{-i phi} a_q ; a_q' = s e^{i phi} a_p + c a_q
        for (int i = sw * 32 + lane; i < R; i += CO_PW * 32) {
          const double2 x = __ldcg(ap + i), y = __ldcg(aq + i);
          ap[i] = make_double2(c * x.x - (spr * y.x + spi * y.y), c * x.y - (spr * y.y - spi * y.x));
          aq[i] = make_double2(spr * x.x - spi * x.y + c * y.x, spr * x.y + spi * x.x + c * y.y);
        }
        double2* vp = Q + (size_t)pc * K;
        double2* vq = Q + (size_t)qc * K;
        for (int i = sw * 32 + lane; i < K; i += CO_PW * 32) {
          const double2 x = __ldcg(vp + i), y = __ldcg(vq + i);
          vp[i] = make_double2(c * x.x - (spr * y.x + spi * y.y), c * x.y - (spr * y.y - spi * y.x));
          vq[i] = make_double2(spr * x.x - spi * x.y + c * y.x, spr * x.y + spi * x.x + c * y.y);
        }
        if (sw == 0 && lane == 0) {
          ++rots;
          nrm[pc] = al - tt * g;
          nrm[qc] = be + tt * g;
          ca.sync->rotated[par] = 1;
          atomicMax(&ca.sync->maxrel[par], (unsigned long long)__double_as_longlong(g2 / ab));
        }
      }
      if (!grid_sync(ca.sync, p.status)) return;
    }
    const volatile CoopSync* vs = ca.sync;
    const int rot = vs->rotated[par];
    const double mr = __longlong_as_double((long long)vs->maxrel[par]);
    if (!rot || mr <= early) {   // same stopping rule as the FP64 phase of the one-CTA kernel
      converged = 1;
      ++sweep;
      break;
    }
  }
  if (p.stats && sw == 0 && lane == 0 && (checks | rots)) {
    const double fl = 8.0 * R * (double)checks + (24.0 * R + 24.0 * K) * (double)rots;
    atomicAdd(p.stats, fl);
  }
  if (p.stats && blockIdx.x == 0 && tid == 0) atomicAdd(p.stats, 4.0 * R * K * (double)sweep);
  if (blockIdx.x == 0 && tid == 0 && !converged) set_status(p.status, MPS_ENOCONV);

  // ---- singular values, order, outputs (same layout and rules as the one-CTA kernel) ----
  for (int j = gwarp; j < K; j += nwarps) {
    double v = 0.0;
    for (int i = lane; i < R; i += 32) {
      const double2 x = __ldcg(X + (size_t)j * R + i);
      v += x.x * x.x + x.y * x.y;
    }
    v = wsum(v);
    if (lane == 0) ca.sv[j] = sqrt(v);
  }
  if (!grid_sync(ca.sync, p.status)) return;
  const double* sv = ca.sv;
  double smax = 0.0;
  for (int j = 0; j < K; ++j) smax = fmax(smax, __ldcg(sv + j));
  for (int j = gwarp; j < K; j += nwarps) {
    const double sj = __ldcg(sv + j);
    int rank = 0;
    for (int i = lane; i < K; i += 32) {
      const double si = __ldcg(sv + i);
      rank += (si > sj) || (si == sj && i < j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const bool null_col = !(sj > CO_NULL_REL * smax);
    if (lane == 0) p.s[rank] = sj;
    double2* vs = p.Vs + (size_t)rank * n;
    double2* w = p.W ? p.W + (size_t)rank * m : nullptr;
    if (tall) {   // V = Q, W = X
      for (int i = lane; i < n; i += 32) vs[i] = __ldcg(Q + (size_t)j * K + i);
      if (w)
        for (int i = lane; i < m; i += 32) w[i] = null_col ? make_double2(0, 0) : __ldcg(X + (size_t)j * R + i);
    } else {      // X = V S, Q = U: v_j = X_j / s_j, W_j = U_j s_j
      const double inv = null_col ? 0.0 : 1.0 / sj;
      for (int i = lane; i < n; i += 32) vs[i] = cscale(__ldcg(X + (size_t)j * R + i), inv);
      if (w)
        for (int i = lane; i < m; i += 32) w[i] = null_col ? make_double2(0, 0) : cscale(__ldcg(Q + (size_t)j * K + i), sj);
    }
  }
  if (!grid_sync(ca.sync, p.status)) return;
  if (blockIdx.x != 0) return;
  __shared__ int k_sh;
  __shared__ double nk_sh;
  if (tid == 0) {
    double n2 = 0.0;
    const double* ps = p.s;
    for (int j = 0; j < K; ++j) n2 += __ldcg(ps + j) * __ldcg(ps + j);
    const double nrm2 = sqrt(n2);
    int cnt = 0;
    if (nrm2 > 0.0 && isfinite(nrm2)) {
      for (int j = 0; j < K; ++j) cnt += (__ldcg(ps + j) / nrm2 > p.eps) && (__ldcg(ps + j) > CO_NULL_REL * smax);
    } else {
      set_status(p.status, MPS_ENUMERIC);
    }
    int k = cnt < p.D ? cnt : p.D;
    if (k < 1) k = 1;
    double nk2 = 0.0;
    for (int j = 0; j < k; ++j) nk2 += __ldcg(ps + j) * __ldcg(ps + j);
    k_sh = k;
    nk_sh = sqrt(nk2);
    if (!(nk_sh > 0.0) || !isfinite(nk_sh)) set_status(p.status, MPS_ENUMERIC);
  }
  __syncthreads();
  const int k = k_sh;
  for (int j = tid; j < k; j += CO_THREADS) p.lam_out[j] = __ldcg(p.s + j) / nk_sh;
  if (p.lam_left_copy)
    for (int a = tid; a < Dl; a += CO_THREADS) p.lam_left_copy[a] = p.lam_left[a];
  __syncthreads();
  if (tid == 0) {
    if (p.tape_dims) {
      p.tape_dims[0] = Dl;
      p.tape_dims[1] = p.dims[b + 1];
      p.tape_dims[2] = Dr;
      p.tape_dims[3] = k;
      p.tape_dims[4] = K;
      p.tape_dims[5] = K < n ? k : 0;   // columns of the SVD adjoint's complement term
    }
    p.dims[b + 1] = k;
    if (p.stats) {
      const unsigned long long t_end = now_ns();
      atomicAdd(p.stats + 2, (double)(t_end - t_start));
      atomicAdd(p.stats + 3, 1.0);
      atomicAdd(p.stats + 6, (double)(t_end - t_start));   // all of it is FP64 sweeps and outputs
      atomicAdd(p.stats + 9, (double)sweep);
    }
  }
}

int coop_grid_size() {
  static const int g = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_coop_kernel, CO_THREADS, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    // one CTA per SM: 2 pair slots each, so 152 SMs cover the 256 pairs of a 512-column round
    return per_sm >= 1 ? std::min(sms, 256) : 0;
  }();
  return g;
}

}  // namespace

size_t svd_coop_scratch_bytes(int m_cap, int n_cap) {
  const size_t R = std::max(m_cap, n_cap), K = std::min(m_cap, n_cap);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(R * K * sizeof(double2)) + al(K * K * sizeof(double2)) + 2 * al(K * sizeof(double)) +
         al(256 * sizeof(double)) + al(sizeof(CoopSync));
}

cudaError_t launch_svd_coop(const SvdArgs& a, void* scratch, int m_cap, int n_cap, cudaStream_t st) {
  const int grid = coop_grid_size();
  if (grid < 1) return cudaErrorNotSupported;
  const size_t R = std::max(m_cap, n_cap), K = std::min(m_cap, n_cap);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* q = static_cast<char*>(scratch);
  CoopArgs ca{};
  ca.p = a;
  ca.p.scratch = nullptr;
  ca.X = reinterpret_cast<double2*>(q);
  q += al(R * K * sizeof(double2));
  ca.Q = reinterpret_cast<double2*>(q);
  q += al(K * K * sizeof(double2));
  ca.nrm = reinterpret_cast<double*>(q);
  q += al(K * sizeof(double));
  ca.sv = reinterpret_cast<double*>(q);
  q += al(K * sizeof(double));
  ca.part = reinterpret_cast<double*>(q);
  q += al(256 * sizeof(double));
  ca.sync = reinterpret_cast<CoopSync*>(q);
  svd_coop_reset<<<1, 1, 0, st>>>(ca.sync);
  note_launch();
  void* args[] = {&ca};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)svd_coop_kernel, dim3(grid), dim3(CO_THREADS), args, 0, st);
  note_launch();
  return e;
}

}  // namespace mpsk
