// Gate application (Sec. 3, two-qubit gate with Hastings' canonical-form update) and the
// custom pieces of its exact adjoint (Sec. 4 / App. A rules), FP64.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/mps.h"
#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

// mps_gate is read field by field (its double arrays sit at an 8-byte offset).
struct GateView {
  const mps_gate* g;
  __device__ double2 m(const double* arr, int e) const { return make_double2(arr[2 * e], arr[2 * e + 1]); }
};

__global__ void gate_matrices_kernel(const mps_gate* __restrict__ gates, int n_gates,
                                     const double* __restrict__ theta, int n_theta, double2* G, double2* dG,
                                     int* status, size_t stride) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_gates) return;
  const size_t io = (size_t)blockIdx.y * stride;
  theta = ish(theta, io);
  G = ish(G, io);
  dG = ish(dG, io);
  status = ish(status, io);
  const mps_gate& g = gates[t];
  GateView v{&g};
  if (g.theta_idx < 0) {
    for (int e = 0; e < 16; ++e) {
      G[16 * t + e] = v.m(g.mat, e);
      dG[16 * t + e] = make_double2(0.0, 0.0);
    }
    return;
  }
  if (g.theta_idx >= n_theta) {
    set_status(status, MPS_EINVAL);
    return;
  }
  double th = theta[g.theta_idx];
  if (!isfinite(th)) {
    set_status(status, MPS_EINVAL);
    return;
  }
  double phi = g.theta_scale * th;
  double sn, cs;
  sincos(0.5 * phi, &sn, &cs);
  // Rz(phi) = diag(e^{-i phi/2}, e^{+i phi/2}); dRz/dphi = diag(-i/2 e^{-i phi/2}, i/2 e^{i phi/2})
  double2 r[2] = {make_double2(cs, -sn), make_double2(cs, sn)};
  double2 dr[2] = {make_double2(-0.5 * sn, -0.5 * cs), make_double2(-0.5 * sn, 0.5 * cs)};
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) {
      double2 a = make_double2(0.0, 0.0), da = make_double2(0.0, 0.0);
      for (int k = 0; k < 4; ++k) {
        int bit = (g.rz_site == 0) ? (k >> 1) : (k & 1);
        double2 pk = cmul(v.m(g.post, i * 4 + k), v.m(g.pre, k * 4 + j));
        a = cadd(a, cmul(pk, r[bit]));
        da = cadd(da, cmul(pk, dr[bit]));
      }
      G[16 * t + i * 4 + j] = a;
      dG[16 * t + i * 4 + j] = da;
    }
  }
}

__global__ void contract_kernel(const double2* __restrict__ Bl, const double2* __restrict__ Br,
                                const int* __restrict__ dims, int b, const double2* __restrict__ Gm,
                                const double* __restrict__ lam_left, double2* C, double2* A,
                                double2* __restrict__ Bl_tape, double2* __restrict__ Br_tape, size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Bl = ish(Bl, io);
  Br = ish(Br, io);
  dims = ish(dims, io);
  Gm = ish(Gm, io);
  lam_left = ish(lam_left, io);
  C = ish(C, io);
  A = ish(A, io);
  Bl_tape = ish(Bl_tape, io);
  Br_tape = ish(Br_tape, io);
  const int Dl = dims[b], Dm = dims[b + 1], Dr = dims[b + 2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (Bl_tape) {   // tape copies of the two input tensors at their current (compact) sizes
    const int nl = 2 * Dl * Dm, nr = 2 * Dm * Dr, stride = gridDim.x * blockDim.x;
    for (int i = t; i < nl; i += stride) Bl_tape[i] = Bl[i];
    for (int i = t; i < nr; i += stride) Br_tape[i] = Br[i];
  }
  if (t >= Dl * Dr) return;
  const int a = t / Dr, c = t % Dr;
  const int m = 2 * Dl, ncol = 2 * Dr;
  double2 th[4] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int mm = 0; mm < Dm; ++mm) {
    double2 l0 = Bl[(size_t)(2 * a) * Dm + mm], l1 = Bl[(size_t)(2 * a + 1) * Dm + mm];
    double2 r0 = Br[(size_t)(2 * mm) * Dr + c], r1 = Br[(size_t)(2 * mm + 1) * Dr + c];
    th[0] = cfma(l0, r0, th[0]);
    th[1] = cfma(l0, r1, th[1]);
    th[2] = cfma(l1, r0, th[2]);
    th[3] = cfma(l1, r1, th[3]);
  }
  const double la = lam_left[a];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    double2 v = make_double2(0, 0);
#pragma unroll
    for (int y = 0; y < 4; ++y) v = cfma(Gm[4 * x + y], th[y], v);
    const int row = 2 * a + (x >> 1), col = (x & 1) * Dr + c;
    if (C) C[(size_t)row * ncol + col] = v;
    A[(size_t)col * m + row] = cscale(v, la);
  }
}

// ---- one-sided Jacobi SVD (FP32 preconditioning sweeps + FP64 sweeps) ----------------------
//
// The two-site matrix C~ (m x n) is orthogonalised on its shorter side: for m >= n the n columns
// of X0 = C~ are rotated (Q accumulates V), for m < n the m columns of X0 = C~^H (Q accumulates
// U).  GB300 runs FP64 at about 1/60 of its FP32 rate, so the sweeps first run in FP32 on a complex64
// copy; the accumulated rotation is then re-orthonormalised in FP64 (modified Gram-Schmidt),
// X = X0 Q is re-formed in FP64 from the untouched input, and FP64 sweeps (scaled rotations,
// numerically-zero columns cleaned first) finish to the FP64 convergence criterion.  The result
// is an FP64-accurate SVD whose FP64 work is a few sweeps.
// X, Q live in shared memory when they fit (the launcher decides), else in global scratch.
constexpr int SVD_THREADS = 512;
constexpr int SVD_MAX_SWEEPS = 60;
constexpr double SVD_NULL_REL = 1e-13;   // numerical-zero singular values (relative to s_max)
constexpr double SVD_DEGEN_REL = 1e-10;  // exactly degenerate pairs of squared singular values
constexpr double SVD_DEGEN_ABS = 1e-13;  // pairs of singular values closer than this times s_1

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
struct Cplx;
template <>
struct Cplx<double> {
  using t = double2;
  __device__ static double2 mk(double x, double y) { return make_double2(x, y); }
  __device__ static double sum(double v) { return warp_sum(v); }
};
template <>
struct Cplx<float> {
  using t = float2;
  __device__ static float2 mk(float x, float y) { return make_float2(x, y); }
  __device__ static float sum(float v) { return warp_sumf(v); }
};

// Cyclic (round-robin) sweeps over the K columns of X (R rows, column j at X + j*R) with the
// rotations accumulated into Q (K x K, column j at Q + j*K).  A column pair is handled by a group
// of JG lanes; with JG = 8 one warp works on 4 pairs of a round at once: each lane strides over
// the rows by 8, the inner product is reduced over the group in three shuffles, and the pairs' memory
// accesses and reductions overlap (instruction-level parallelism across pairs, which hides the
// shared-memory and shuffle latencies that a warp-per-pair ordering exposes).  Column norms are
// recomputed at the start of every sweep and updated by each rotation (alpha' = alpha - t g,
// beta' = beta + t g), so a pair costs one inner product.
//
// A pair (p, q) with inner product gamma is rotated when |gamma|^2 > tol^2 alpha beta.  The
// rotation's tangent t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)), zeta = (beta - alpha)/(2|gamma|),
// is computed in FP32; c = 1/sqrt(1 + t^2), s = c t and the phase gamma/|gamma| are then formed
// in the working precision T, so every rotation is unitary to T's precision whatever the
// accuracy of t (a t off by 1e-7 relative leaves |gamma| 1e-7 of its size, removed by the next
// sweep at no extra sweep count, since the sweeps converge quadratically).  FP64 on GB300 runs at
// about 1/60 of the FP32 rate, and this keeps the divisions and square roots of a rotation in FP32.
//
// Stopping: a sweep that rotates nothing.  This generic version runs the FP32 phase; the FP64
// phase uses the scaled variant below, which also stops early.
// Returns the number of sweeps run; *converged = 1 when a stopping rule was met.
//
// JG (lanes per column pair, 8, 16 or 32) is chosen by the caller from the number of pairs in a
// round, so that a round's pairs spread over every warp scheduler of the SM: with few pairs, more
// lanes per pair shorten each lane's serial loop and bring more warps (FP32 phase, latency bound)
// or more of the four FP64 pipes (FP64 phase) into use.
template <int JG, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = JG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T, int JG>
__device__ int jacobi_sweeps(typename Cplx<T>::t* X, typename Cplx<T>::t* Q, int R, int K, T tol, T tiny,
                             int max_sweeps, int* flag_sh, int* converged, T* nrm, double* flops) {
  using C2 = typename Cplx<T>::t;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int grp = lane / JG, gl = lane % JG, per_warp = 32 / JG;
  const int Kp = K + (K & 1);
  const T tol2 = tol * tol;
  int sweep = 0;
  long long checks = 0, rots = 0;   // per group (its first lane's count is used)
  *converged = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = warp; j < K; j += nwarp) {
      T v = 0;
      for (int i = lane; i < R; i += 32) {
        const C2 x = X[(size_t)j * R + i];
        v += x.x * x.x + x.y * x.y;
      }
      v = Cplx<T>::sum(v);
      if (lane == 0) nrm[j] = v;
    }
    if (tid == 0) {
      *flag_sh = 0;
    }
    __syncthreads();
    for (int r = 0; r < Kp - 1; ++r) {
      for (int t0 = warp * per_warp; t0 < Kp / 2; t0 += nwarp * per_warp) {   // uniform over the warp
        const int t = t0 + grp;
        int pc = 0, qc = 0;
        bool live = t < Kp / 2;
        if (live) {
          if (t == 0) {
            pc = r;
            qc = Kp - 1;
          } else {
            pc = (r + t) % (Kp - 1);
            qc = (r - t + Kp - 1) % (Kp - 1);
          }
          live = pc < K && qc < K;
        }
        T al = 0, be = 0;
        if (live) {
          al = nrm[pc];
          be = nrm[qc];
          live = !(al < tiny || be < tiny);
        }
        C2* ap = X + (size_t)pc * R;
        C2* aq = X + (size_t)qc * R;
        T gr = 0, gi = 0;
        if (live) {
          for (int i = gl; i < R; i += JG) {
            const C2 x = ap[i], y = aq[i];
            gr += x.x * y.x + x.y * y.y;   // conj(x) y
            gi += x.x * y.y - x.y * y.x;
          }
        }
        gr = group_sum<JG>(gr);   // every lane of the warp takes part in the shuffles
        gi = group_sum<JG>(gi);
        if (!live) continue;
        if (gl == 0) ++checks;
        const T g2 = gr * gr + gi * gi;
        const T ab = al * be;
        if (!(g2 > tol2 * ab)) continue;
        const T inv_g = rsqrt(g2);
        const T g = g2 * inv_g;
        const float zf = (float)((be - al) * (T(0.5) * inv_g));
        const float af = fabsf(zf);
        const float tf = af > 1e15f ? 0.5f / zf : copysignf(1.f / (af + sqrtf(1.f + zf * zf)), zf);
        const T tt = (T)tf;
        const T c = rsqrt(T(1) + tt * tt), s = c * tt;
        const T pr = gr * inv_g, pim = gi * inv_g;                 // e^{i phi}
        // a_p' = c a_p - s e^{-i phi} a_q ; a_q' = s e^{i phi} a_p + c a_q
        const T spr = s * pr, spi = s * pim;
        for (int i = gl; i < R; i += JG) {
          const C2 x = ap[i], y = aq[i];
          ap[i] = Cplx<T>::mk(c * x.x - (spr * y.x + spi * y.y), c * x.y - (spr * y.y - spi * y.x));
          aq[i] = Cplx<T>::mk(spr * x.x - spi * x.y + c * y.x, spr * x.y + spi * x.x + c * y.y);
        }
        C2* vp = Q + (size_t)pc * K;
        C2* vq = Q + (size_t)qc * K;
        for (int i = gl; i < K; i += JG) {
          const C2 x = vp[i], y = vq[i];
          vp[i] = Cplx<T>::mk(c * x.x - (spr * y.x + spi * y.y), c * x.y - (spr * y.y - spi * y.x));
          vq[i] = Cplx<T>::mk(spr * x.x - spi * x.y + c * y.x, spr * x.y + spi * x.x + c * y.y);
        }
        if (gl == 0) {
          ++rots;
          nrm[pc] = al - tt * g;
          nrm[qc] = be + tt * g;
          *flag_sh = 1;
        }
      }
      __syncthreads();
    }
    const int rot = *flag_sh;
    __syncthreads();
    if (!rot) {
      *converged = 1;
      ++sweep;
      break;
    }
  }
  // work actually done: per sweep K column norms (4R flops each), per checked pair one complex
  // inner product (8R), per rotation the update of two columns of X (24R) and of Q (24K)
  if (flops && gl == 0 && (checks | rots)) {
    const double f = 8.0 * R * (double)checks + (24.0 * R + 24.0 * K) * (double)rots;
    atomicAdd(flops, f);
  }
  if (flops && tid == 0) atomicAdd(flops, 4.0 * R * K * (double)sweep);
  return sweep;
}

// The FP64 sweeps, with the rotations applied in scaled form.  Each column carries a scale
// d_j (and e_j = 1/d_j, kept as its own product so that no division is needed): the true column
// is x_j = d_j xh_j.  The rotation a_p' = c (a_p - t e^{-i phi} a_q), a_q' = c (a_q + t e^{i phi} a_p)
// then becomes xh_p' = xh_p - mu_p xh_q, xh_q' = xh_q + mu_q xh_p with mu_p = t (d_q e_p) e^{-i phi},
// mu_q = t (d_p e_q) e^{i phi}, d_p' = c d_p, d_q' = c d_q: two FMAs per real output instead of
// three, a third less work on GB300's FP64 pipe, which bounds this phase.  (This is the
// square-root-free "fast Givens" idea applied to one-sided Jacobi.)  The scales start at 1 in every
// sweep and are folded into X and Q at its end, so they never leave [0.7^K, 1].  For the small
// rotations of this phase (t^2 < 1e-6) c = 1/sqrt(1 + t^2) and 1/c come from their Taylor series to
// t^4 (error below t^6/3 < 4e-19); larger ones use the square root.
//
// Cleaning sweep: after the FP32 phase the numerically-zero columns of a rank-deficient C~ still
// hold components of size ~1e-7 s_1 along the large singular vectors.  Rotating them against each
// other while those components are being removed mixes them back in, and the sweeps converge only
// linearly on them.  So when there are columns below clean_rel (1e-5) of the largest, the first
// sweep skips the pairs of two such columns and only rotates them against the larger ones; every
// later sweep rotates every pair.  (Skipping them in later sweeps too was tried: without their
// mutual rotations a small kept column rotated against several of them can cycle without
// converging.)
//
// Stopping: a sweep after the cleaning sweep that rotates nothing, or whose every rotated pair had
// |gamma|^2 <= early alpha beta.  With early = (10 tol)^2 such a sweep leaves inner products of
// order K (10 tol)^2, far below tol, so the confirming sweep would rotate nothing.  (A looser
// bound, early = tol/(2K), was measured to cost 1e-9 in energies.)
template <int JG>
__device__ int jacobi_sweeps_scaled(double2* X, double2* Q, int R, int K, double tol, double tiny, int max_sweeps,
                                    int* flag_sh, int* notdone_sh, int* converged, double* nrm, double* dsc,
                                    double* esc, double* maxn_sh, double* flops, double early, double clean_rel) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int grp = lane / JG, gl = lane % JG, per_warp = 32 / JG;
  const int Kp = K + (K & 1);
  const double tol2 = tol * tol;
  int sweep = 0;
  long long checks = 0, rots = 0;
  *converged = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = warp; j < K; j += nwarp) {
      double v = 0;
      for (int i = lane; i < R; i += 32) {
        const double2 x = X[(size_t)j * R + i];
        v += x.x * x.x + x.y * x.y;
      }
      v = warp_sum(v);
      if (lane == 0) {
        nrm[j] = v;
        dsc[j] = 1.0;
        esc[j] = 1.0;
      }
    }
    if (tid == 0) {
      *flag_sh = 0;
      *notdone_sh = 0;
    }
    __syncthreads();
    if (warp == 0) {
      double mx = 0.0;
      for (int j = lane; j < K; j += 32) mx = fmax(mx, nrm[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) *maxn_sh = mx;
    }
    __syncthreads();
    const double maxn = *maxn_sh;
    // the cleaning rule applies to the first sweep, and only when there is something to clean
    bool cleaning = false;
    if (sweep == 0) {
      int any_small = 0;
      for (int j = tid; j < K; j += blockDim.x) any_small |= nrm[j] >= tiny && nrm[j] < clean_rel * clean_rel * maxn;
      cleaning = __syncthreads_or(any_small) != 0;
    }
    const double thr = cleaning ? clean_rel * clean_rel * maxn : 0.0;
    for (int r = 0; r < Kp - 1; ++r) {
      for (int t0 = warp * per_warp; t0 < Kp / 2; t0 += nwarp * per_warp) {   // uniform over the warp
        const int t = t0 + grp;
        int pc = 0, qc = 0;
        bool live = t < Kp / 2;
        if (live) {
          if (t == 0) {
            pc = r;
            qc = Kp - 1;
          } else {
            pc = (r + t) % (Kp - 1);
            qc = (r - t + Kp - 1) % (Kp - 1);
          }
          live = pc < K && qc < K;
        }
        double al = 0, be = 0;
        if (live) {
          al = nrm[pc];
          be = nrm[qc];
          live = !(al < tiny || be < tiny) && !(al < thr && be < thr);
        }
        double2* ap = X + (size_t)pc * R;
        double2* aq = X + (size_t)qc * R;
        double gr = 0, gi = 0;
        if (live) {
          for (int i = gl; i < R; i += JG) {
            const double2 x = ap[i], y = aq[i];
            gr = fma(x.x, y.x, gr);   // conj(x) y
            gr = fma(x.y, y.y, gr);
            gi = fma(x.x, y.y, gi);
            gi = fma(-x.y, y.x, gi);
          }
        }
        gr = group_sum<JG>(gr);   // every lane of the warp takes part in the shuffles
        gi = group_sum<JG>(gi);
        if (!live) continue;
        if (gl == 0) ++checks;
        const double dp = dsc[pc], dq = dsc[qc], dd = dp * dq;
        gr *= dd;   // inner product of the true columns
        gi *= dd;
        const double g2 = gr * gr + gi * gi;
        const double ab = al * be;
        if (!(g2 > tol2 * ab)) continue;
        const double inv_g = rsqrt(g2);
        const double g = g2 * inv_g;
        const float zf = (float)((be - al) * (0.5 * inv_g));
        const float af = fabsf(zf);
        const float tf = af > 1e15f ? 0.5f / zf : copysignf(1.f / (af + sqrtf(1.f + zf * zf)), zf);
        const double tt = (double)tf;
        const double t2 = tt * tt;
        double c, rc;   // c = 1/sqrt(1 + t^2), rc = 1/c
        if (t2 < 1e-6) {
          c = fma(t2, fma(0.375, t2, -0.5), 1.0);
          rc = fma(t2, fma(-0.125, t2, 0.5), 1.0);
        } else {
          c = rsqrt(1.0 + t2);
          rc = (1.0 + t2) * c;
        }
        const double ep = esc[pc], eq = esc[qc];
        const double kp = tt * (dq * ep) * inv_g, kq = tt * (dp * eq) * inv_g;
        const double mpr = kp * gr, mpi = -kp * gi;   // mu_p = t (d_q/d_p) e^{-i phi}
        const double mqr = kq * gr, mqi = kq * gi;    // mu_q = t (d_p/d_q) e^{i phi}
        for (int i = gl; i < R; i += JG) {
          const double2 x = ap[i], y = aq[i];
          ap[i] = make_double2(fma(-mpr, y.x, fma(mpi, y.y, x.x)), fma(-mpr, y.y, fma(-mpi, y.x, x.y)));
          aq[i] = make_double2(fma(mqr, x.x, fma(-mqi, x.y, y.x)), fma(mqr, x.y, fma(mqi, x.x, y.y)));
        }
        double2* vp = Q + (size_t)pc * K;
        double2* vq = Q + (size_t)qc * K;
        for (int i = gl; i < K; i += JG) {
          const double2 x = vp[i], y = vq[i];
          vp[i] = make_double2(fma(-mpr, y.x, fma(mpi, y.y, x.x)), fma(-mpr, y.y, fma(-mpi, y.x, x.y)));
          vq[i] = make_double2(fma(mqr, x.x, fma(-mqi, x.y, y.x)), fma(mqr, x.y, fma(mqi, x.x, y.y)));
        }
        if (gl == 0) {
          ++rots;
          nrm[pc] = al - tt * g;
          nrm[qc] = be + tt * g;
          dsc[pc] = dp * c;
          dsc[qc] = dq * c;
          esc[pc] = ep * rc;
          esc[qc] = eq * rc;
          *flag_sh = 1;
          if (g2 > early * ab) *notdone_sh = 1;
        }
      }
      __syncthreads();
    }
    // fold the scales into the columns
    for (int e = tid; e < R * K; e += blockDim.x) X[e] = cscale(X[e], dsc[e / R]);
    for (int e = tid; e < K * K; e += blockDim.x) Q[e] = cscale(Q[e], dsc[e / K]);
    __syncthreads();
    const int rot = *flag_sh, nd = *notdone_sh;
    __syncthreads();
    if (!cleaning && (!rot || !nd)) {
      *converged = 1;
      ++sweep;
      break;
    }
  }
  // work done: per sweep K column norms (4R flops each) and the scale fold (2(R+K) per column), per
  // checked pair one complex inner product (8R), per rotation the scaled update of two columns of
  // X (16R) and of Q (16K)
  if (flops && gl == 0 && (checks | rots)) {
    const double f = 8.0 * R * (double)checks + (16.0 * R + 16.0 * K) * (double)rots;
    atomicAdd(flops, f);
  }
  if (flops && tid == 0) atomicAdd(flops, (4.0 * R * K + 2.0 * (R + K) * K) * (double)sweep);
  return sweep;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(SVD_THREADS) svd_kernel(const SvdArgs p0, size_t stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned long long t_start = global_ns();
  SvdArgs p = p0;   // this CTA's instance
  {
    const size_t io = (size_t)blockIdx.x * stride;
    p.A = ish(p.A, io);
    p.scratch = ish(p.scratch, io);
    p.dims = ish(p.dims, io);
    p.Vs = ish(p.Vs, io);
    p.s = ish(p.s, io);
    p.lam_out = ish(p.lam_out, io);
    p.W = ish(p.W, io);
    p.tape_dims = ish(p.tape_dims, io);
    p.lam_left = ish(p.lam_left, io);
    p.lam_left_copy = ish(p.lam_left_copy, io);
    p.status = ish(p.status, io);
    p.stats = ish(p.stats, io);
  }
  __shared__ double red[SVD_THREADS / 32];
  __shared__ double s_sh[512];
  __shared__ double dsc_sh[512], esc_sh[512];   // column scales of the FP64 sweeps
  __shared__ int flag_sh, conv_sh, k_sh, notdone_sh;
  __shared__ double maxn_sh;
  __shared__ double fro2_sh, smax_sh, nk_sh;
  const int b = p.b;
  const int Dl = p.dims[b], Dr = p.dims[b + 2];
  const int m = 2 * Dl, n = 2 * Dr;
  const bool tall = m >= n;
  const int R = tall ? m : n, K = tall ? n : m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = SVD_THREADS / 32;
  double2* base = p.scratch ? p.scratch : reinterpret_cast<double2*>(smem_raw);
  double2* Q64 = base;                                      // K x K
  double2* X64 = base + (size_t)K * K;                      // R x K
  float2* X32 = reinterpret_cast<float2*>(X64);             // R x K  (inside the X64 region)
  float2* Q32 = X32 + (size_t)R * K;                        // K x K  (inside the X64 region, K <= R)
  const double2* A = p.A;                                   // C~ column-major (m x n)
  auto x0 = [&](int r, int j) -> double2 {                  // element (r, j) of X0
    return tall ? A[(size_t)j * m + r] : conjd(A[(size_t)r * m + j]);
  };
  // ---- FP32 preconditioning sweeps ----
  double f = 0.0;
  for (int e = tid; e < R * K; e += SVD_THREADS) {
    const int j = e / R, r = e % R;
    const double2 v = x0(r, j);
    f += v.x * v.x + v.y * v.y;
    X32[(size_t)j * R + r] = make_float2((float)v.x, (float)v.y);
  }
  for (int e = tid; e < K * K; e += SVD_THREADS) Q32[e] = make_float2((e / K) == (e % K) ? 1.f : 0.f, 0.f);
  f = warp_sum(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    fro2_sh = t;
  }
  __syncthreads();
  int conv = 0;
  const int npairs = (K + (K & 1)) / 2;   // column pairs per round
  // lanes per column pair: the launcher's (tuned) choice, else enough lanes to use all 16 warps
  // in the latency-bound FP32 phase, and 8 unless that would idle an FP64 pipe in the FP64 phase
  const int g32 = p.jg32 > 0 ? p.jg32 : (npairs <= 16 ? 32 : npairs <= 32 ? 16 : 8);
  const int g64 = p.jg64 > 0 ? p.jg64 : (npairs <= 4 ? 32 : npairs <= 8 ? 16 : 8);
  int sweeps32 = 0;
  {
    const float tol32 = 4.f * 1.1920929e-7f * sqrtf((float)R), tiny32 = (float)(1e-30 * fro2_sh) + 1e-37f;
    float* nrm32 = reinterpret_cast<float*>(s_sh);
    double* fl32 = p.stats ? p.stats + 1 : nullptr;
    if (g32 == 32)
      sweeps32 = jacobi_sweeps<float, 32>(X32, Q32, R, K, tol32, tiny32, 30, &flag_sh, &conv, nrm32, fl32);
    else if (g32 == 16)
      sweeps32 = jacobi_sweeps<float, 16>(X32, Q32, R, K, tol32, tiny32, 30, &flag_sh, &conv, nrm32, fl32);
    else
      sweeps32 = jacobi_sweeps<float, 8>(X32, Q32, R, K, tol32, tiny32, 30, &flag_sh, &conv, nrm32, fl32);
  }
  const unsigned long long t_fp32 = global_ns();
  // ---- Q64 = orthonormalised Q32 (modified Gram-Schmidt, FP64) ----
  // A column is handled by a group of 8 lanes (4 columns per warp), so an inner product costs
  // three shuffle-and-add steps shared by four columns rather than five per column: on GB300 each
  // of those adds occupies the FP64 pipe as long as a multiply-add.  Column j + 1 is final once it
  // has been projected against column j; warp 0, which projects it, normalises it in the same
  // step, so each column costs one barrier.
  {
    constexpr int MG = 8;
    const int grp = lane / MG, gl = lane % MG, gpw = 32 / MG;
    for (int e = tid; e < K * K; e += SVD_THREADS) Q64[e] = make_double2((double)Q32[e].x, (double)Q32[e].y);
    __syncthreads();
    if (warp == 0) {   // column 0
      double v = 0.0;
      for (int i = lane; i < K; i += 32) v += Q64[i].x * Q64[i].x + Q64[i].y * Q64[i].y;
      v = warp_sum(v);
      const double inv = rsqrt(v);
      for (int i = lane; i < K; i += 32) Q64[i] = cscale(Q64[i], inv);
    }
    __syncthreads();
    for (int j = 0; j + 1 < K; ++j) {
      const double2* qj = Q64 + (size_t)j * K;
      for (int l0 = j + 1 + warp * gpw; l0 < K; l0 += nwarp * gpw) {   // uniform over the warp
        const int l = l0 + grp;
        const bool live = l < K;
        double2* ql = Q64 + (size_t)(live ? l : j) * K;
        double pr = 0.0, pim = 0.0;
        if (live)
          for (int i = gl; i < K; i += MG) {   // qj^H ql
            const double2 a = qj[i], b = ql[i];
            pr = fma(a.x, b.x, fma(a.y, b.y, pr));
            pim = fma(a.x, b.y, fma(-a.y, b.x, pim));
          }
        pr = group_sum<MG>(pr);
        pim = group_sum<MG>(pim);
        if (live)
          for (int i = gl; i < K; i += MG) {
            const double2 a = qj[i], b = ql[i];
            ql[i] = make_double2(b.x - (pr * a.x - pim * a.y), b.y - (pr * a.y + pim * a.x));
          }
        if (l0 == j + 1) {   // warp 0: normalise column j + 1 (group 0); each lane rescales its own entries
          double v = 0.0;
          if (live)
            for (int i = gl; i < K; i += MG) v += ql[i].x * ql[i].x + ql[i].y * ql[i].y;
          v = group_sum<MG>(v);
          if (grp == 0) {
            const double inv = rsqrt(v);
            for (int i = gl; i < K; i += MG) ql[i] = cscale(ql[i], inv);
          }
        }
      }
      __syncthreads();
    }
  }
  // ---- X64 = X0 Q64 (FP64, from the untouched input) ----
  // A thread forms four columns of one row, so each element of X0 is loaded once per four
  // complex FMAs and the four accumulations are independent.
  {
    constexpr int JB = 4;
    const int nb = (K + JB - 1) / JB;
    for (int e = tid; e < R * nb; e += SVD_THREADS) {
      const int j0 = (e / R) * JB, r = e % R;
      double2 acc[JB];
#pragma unroll
      for (int u = 0; u < JB; ++u) acc[u] = make_double2(0.0, 0.0);
      if (j0 + JB <= K) {
        for (int l = 0; l < K; ++l) {
          const double2 a = x0(r, l);
#pragma unroll
          for (int u = 0; u < JB; ++u) acc[u] = cfma(a, Q64[(size_t)(j0 + u) * K + l], acc[u]);
        }
      } else {
        for (int l = 0; l < K; ++l) {
          const double2 a = x0(r, l);
          for (int u = 0; u < JB && j0 + u < K; ++u) acc[u] = cfma(a, Q64[(size_t)(j0 + u) * K + l], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < JB; ++u)
        if (j0 + u < K) X64[(size_t)(j0 + u) * R + r] = acc[u];
    }
  }
  __syncthreads();
  // ---- FP64 sweeps ----
  const unsigned long long t_reform = global_ns();
  const double tol64 = 4.0 * 2.220446049250313e-16 * sqrt((double)R);
  int sweeps64 = 0;
  {
    const double tiny64 = 1e-30 * fro2_sh, early64 = 100.0 * tol64 * tol64;
    if (g64 == 32)
      sweeps64 = jacobi_sweeps_scaled<32>(X64, Q64, R, K, tol64, tiny64, SVD_MAX_SWEEPS, &flag_sh, &notdone_sh,
                                          &conv_sh, s_sh, dsc_sh, esc_sh, &maxn_sh, p.stats, early64, 1e-5);
    else if (g64 == 16)
      sweeps64 = jacobi_sweeps_scaled<16>(X64, Q64, R, K, tol64, tiny64, SVD_MAX_SWEEPS, &flag_sh, &notdone_sh,
                                          &conv_sh, s_sh, dsc_sh, esc_sh, &maxn_sh, p.stats, early64, 1e-5);
    else
      sweeps64 = jacobi_sweeps_scaled<8>(X64, Q64, R, K, tol64, tiny64, SVD_MAX_SWEEPS, &flag_sh, &notdone_sh,
                                         &conv_sh, s_sh, dsc_sh, esc_sh, &maxn_sh, p.stats, early64, 1e-5);
  }
  const unsigned long long t_fp64 = global_ns();
  // FP64 work outside the sweeps: Gram-Schmidt (~8 K^3) and X = X0 Q (8 R K^2)
  if (p.stats && tid == 0) atomicAdd(p.stats, 8.0 * K * K * (double)K + 8.0 * R * K * (double)K);
  if (tid == 0 && !conv_sh) set_status(p.status, MPS_ENOCONV);
  // ---- singular values, order, outputs ----
  for (int j = warp; j < K; j += nwarp) {
    double v = 0.0;
    for (int i = lane; i < R; i += 32) {
      const double2 x = X64[(size_t)j * R + i];
      v += x.x * x.x + x.y * x.y;
    }
    v = warp_sum(v);
    if (lane == 0) s_sh[j] = sqrt(v);
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int j = 0; j < K; ++j) mx = fmax(mx, s_sh[j]);
    smax_sh = mx;
  }
  __syncthreads();
  // Outputs, sorted descending (stable in the column index):
  //   s[0..K), Vs: K columns of length n (right singular vectors; zero for numerical zeros when
  //   they come from the wide orientation), W: K columns of length m (W_j = C~ v_j; stored as exact
  //   zeros for numerical zeros, s_j <= SVD_NULL_REL s_max).
  for (int j = warp; j < K; j += nwarp) {
    const double sj = s_sh[j];
    int rank = 0;
    for (int i = 0; i < K; ++i) {
      const double si = s_sh[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    const bool null_col = !(sj > SVD_NULL_REL * smax_sh);
    if (lane == 0) p.s[rank] = sj;
    double2* vs = p.Vs + (size_t)rank * n;
    double2* w = p.W ? p.W + (size_t)rank * m : nullptr;
    if (tall) {   // V = Q, W = X
      for (int i = lane; i < n; i += 32) vs[i] = Q64[(size_t)j * K + i];
      if (w)
        for (int i = lane; i < m; i += 32) w[i] = null_col ? make_double2(0, 0) : X64[(size_t)j * R + i];
    } else {      // X = V S, Q = U: v_j = X_j / s_j, W_j = U_j s_j
      const double inv = null_col ? 0.0 : 1.0 / sj;
      for (int i = lane; i < n; i += 32) vs[i] = cscale(X64[(size_t)j * R + i], inv);
      if (w)
        for (int i = lane; i < m; i += 32) w[i] = null_col ? make_double2(0, 0) : cscale(Q64[(size_t)j * K + i], sj);
    }
  }
  __syncthreads();
  if (tid == 0) {
    double n2 = 0.0;
    for (int j = 0; j < K; ++j) n2 += p.s[j] * p.s[j];
    const double nrm = sqrt(n2);
    int cnt = 0;
    if (nrm > 0.0 && isfinite(nrm)) {   // numerical zeros (s <= SVD_NULL_REL s_max) are never kept
      for (int j = 0; j < K; ++j) cnt += (p.s[j] / nrm > p.eps) && (p.s[j] > SVD_NULL_REL * smax_sh);
    } else {
      set_status(p.status, MPS_ENUMERIC);
    }
    int k = cnt < p.D ? cnt : p.D;
    if (k < 1) k = 1;
    double nk2 = 0.0;
    for (int j = 0; j < k; ++j) nk2 += p.s[j] * p.s[j];
    k_sh = k;
    nk_sh = sqrt(nk2);
    if (!(nk_sh > 0.0) || !isfinite(nk_sh)) set_status(p.status, MPS_ENUMERIC);
  }
  __syncthreads();
  const int k = k_sh;
  for (int j = tid; j < k; j += SVD_THREADS) p.lam_out[j] = p.s[j] / nk_sh;
  if (p.lam_left_copy)
    for (int a = tid; a < Dl; a += SVD_THREADS) p.lam_left_copy[a] = p.lam_left[a];
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
    if (p.stats) {   // device-side duration of this launch and of its phases
      const unsigned long long t_end = global_ns();
      atomicAdd(p.stats + 2, (double)(t_end - t_start));
      atomicAdd(p.stats + 3, 1.0);
      atomicAdd(p.stats + 4, (double)(t_fp32 - t_start));
      atomicAdd(p.stats + 5, (double)(t_reform - t_fp32));
      atomicAdd(p.stats + 6, (double)(t_fp64 - t_reform));
      atomicAdd(p.stats + 7, (double)(t_end - t_fp64));
      atomicAdd(p.stats + 8, (double)sweeps32);
      atomicAdd(p.stats + 9, (double)sweeps64);
    }
  }
}

__global__ void vh_rows_kernel(const double2* __restrict__ Vs, const int* __restrict__ dims, int b,
                               double2* Br, size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Vs = ish(Vs, io);
  dims = ish(dims, io);
  Br = ish(Br, io);
  const int k = dims[b + 1], ncol = 2 * dims[b + 2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * ncol) return;
  const int j = t / ncol, r = t % ncol;
  Br[(size_t)j * ncol + r] = conjd(Vs[(size_t)j * ncol + r]);
}

// ---- adjoint pieces -------------------------------------------------------------------------
__global__ void conjT_kernel(const double2* __restrict__ Bbr, const int* __restrict__ td, double2* Vbar,
                             size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Bbr = ish(Bbr, io);
  td = ish(td, io);
  Vbar = ish(Vbar, io);
  const int k = td[3], ncol = 2 * td[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * ncol) return;
  const int r = t / k, j = t % k;                    // Vbar[r][j] = conj(Bbar_r[j][r])
  Vbar[(size_t)r * k + j] = conjd(Bbr[(size_t)j * ncol + r]);
}

__global__ void sbar_kernel(double* lambar, const double* __restrict__ s, const int* __restrict__ td,
                            double* wbar, size_t stride) {
  const size_t io = (size_t)blockIdx.x * stride;
  lambar = ish(lambar, io);
  s = ish(s, io);
  td = ish(td, io);
  wbar = ish(wbar, io);
  const int k = td[3], ncol = td[4];
  __shared__ double nrm_sh, dot_sh;
  if (threadIdx.x == 0) {
    double n2 = 0.0;
    for (int j = 0; j < k; ++j) n2 += s[j] * s[j];
    const double nrm = sqrt(n2);
    double d = 0.0;
    for (int j = 0; j < k; ++j) d += (s[j] / nrm) * lambar[j];
    nrm_sh = nrm;
    dot_sh = d;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
    double w = 0.0;
    if (j < k) {
      const double lam = s[j] / nrm_sh;
      const double sb = (lambar[j] - lam * dot_sh) / nrm_sh;   // d(s/||s||)^T lambar
      w = sb / (2.0 * s[j]);                                  // wbar = sbar / (2 s)
    }
    wbar[j] = w;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) lambar[j] = 0.0;   // old lambda_b is unused
}

__global__ void build_K_kernel(const double2* __restrict__ Y, const double* __restrict__ s,
                               const double* __restrict__ wbar, const int* __restrict__ td, double2* Km,
                               size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Y = ish(Y, io);
  s = ish(s, io);
  wbar = ish(wbar, io);
  td = ish(td, io);
  Km = ish(Km, io);
  const int k = td[3], K = td[4];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * K) return;
  const int i = t / K, j = t % K;
  // numerical zeros (s <= SVD_NULL_REL s_1) enter as exact zeros
  const double wi = s[i] > SVD_NULL_REL * s[0] ? s[i] * s[i] : 0.0;
  const double wj = s[j] > SVD_NULL_REL * s[0] ? s[j] * s[j] : 0.0;
  // F_ij = 1/(w_j - w_i), 0 inside degenerate pairs: |dw| <= SVD_DEGEN_REL max(w), or singular
  // values closer than SVD_DEGEN_ABS s_1 (a computed singular value is known to a few ulps of s_1,
  // so a degenerate pair far below s_1 comes out split by rounding that the relative rule alone
  // would divide by)
  const double dw = wj - wi;
  const double si = wi > 0.0 ? s[i] : 0.0, sj = wj > 0.0 ? s[j] : 0.0;
  const bool split = fabs(dw) > SVD_DEGEN_REL * fmax(wi, wj) && fabs(sj - si) > SVD_DEGEN_ABS * s[0];
  const double F = split ? 1.0 / dw : 0.0;
  double2 v = make_double2(i == j ? wbar[i] : 0.0, 0.0);
  if (i != j) {
    if (j < k) v = cadd(v, cscale(Y[(size_t)i * k + j], F));               // J_ij = F_ij Y_ij
    if (i < k) v = cadd(v, cscale(conjd(Y[(size_t)j * k + i]), -F));       // (J^H)_ij = conj(F_ji Y_ji)
  }
  Km[(size_t)i * K + j] = v;
}

// Z[r][j] /= w_j (j < k): the complement term (W_k diag(1/w_k)) Z^H of the SVD adjoint.  When
// the SVD's K vectors span the whole column space (K = ncol), the complement is empty and Z =
// Vbar - V V^H Vbar is zero.  Computed, it is rounding of size 1e-16 |Vbar|, and 1/w_k of a kept
// value just above the cutoff (w ~ 1e-24 w_1) turns that into a gradient error of many times
// the gradient's norm.  The term is therefore set to exactly zero.
__global__ void zscale_kernel(double2* Z, const double* __restrict__ s, const int* __restrict__ td,
                              size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Z = ish(Z, io);
  s = ish(s, io);
  td = ish(td, io);
  const int k = td[3], n = 2 * td[2], K = td[4];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  if (K >= n) {
    Z[t] = make_double2(0.0, 0.0);
    return;
  }
  const int j = t % k;
  Z[t] = cscale(Z[t], 1.0 / (s[j] * s[j]));
}

__global__ void lam_scale_kernel(double2* Cbar, const double2* __restrict__ Ctbar,
                                 const double2* __restrict__ C, const double* __restrict__ lam_left,
                                 const int* __restrict__ td, double* lambar_left, size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Cbar = ish(Cbar, io);
  Ctbar = ish(Ctbar, io);
  C = ish(C, io);
  lam_left = ish(lam_left, io);
  td = ish(td, io);
  lambar_left = ish(lambar_left, io);
  const int Dl = td[0], ncol = 2 * td[2];
  const int a = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (a >= Dl) return;
  const double la = lam_left[a];
  double acc = 0.0;
  for (int e = lane; e < 2 * ncol; e += 32) {
    const size_t idx = (size_t)(2 * a) * ncol + e;   // rows 2a and 2a+1 are contiguous
    const double2 ct = Ctbar[idx], c = C[idx];
    acc += ct.x * c.x + ct.y * c.y;                  // Re(conj(Ctbar) * C)
    Cbar[idx] = cadd(Cbar[idx], cscale(ct, la));
  }
  acc = warp_sum(acc);
  if (lane == 0 && lambar_left) lambar_left[a] += 2.0 * acc;
}

__global__ void __launch_bounds__(256) gbar_kernel(const double2* __restrict__ Cbar,
                                                   const double2* __restrict__ Th, const int* __restrict__ td,
                                                   const double2* __restrict__ dG, double2* Gbar,
                                                   double* gate_grad, size_t stride) {
  const size_t io = (size_t)blockIdx.x * stride;
  Cbar = ish(Cbar, io);
  Th = ish(Th, io);
  td = ish(td, io);
  dG = ish(dG, io);
  Gbar = ish(Gbar, io);
  gate_grad = ish(gate_grad, io);
  const int Dl = td[0], Dr = td[2], ncol = 2 * Dr;
  double2 acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = make_double2(0, 0);
  for (int t = threadIdx.x; t < Dl * Dr; t += blockDim.x) {
    const int a = t / Dr, c = t % Dr;
    double2 cb[4], th[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const size_t idx = (size_t)(2 * a + (x >> 1)) * ncol + (x & 1) * Dr + c;
      cb[x] = Cbar[idx];
      th[x] = Th[idx];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[4 * x + y] = cadd(acc[4 * x + y], cmulc(cb[x], th[y]));
  }
  // warp shuffles, then a fixed-order sum over warps (deterministic)
  __shared__ double2 sh[8][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    double re = warp_sum(acc[e].x), im = warp_sum(acc[e].y);
    if (lane == 0) sh[warp][e] = make_double2(re, im);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gg = 0.0;
    for (int e = 0; e < 16; ++e) {
      double2 v = make_double2(0, 0);
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = cadd(v, sh[w][e]);
      Gbar[e] = v;
      gg += v.x * dG[e].x + v.y * dG[e].y;   // Re(conj(Gbar) dG)
    }
    *gate_grad = 2.0 * gg;
  }
}

__global__ void thetabar_kernel(const double2* __restrict__ Cbar, const double2* __restrict__ Gm,
                                const int* __restrict__ td, double2* Thbar, size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  Cbar = ish(Cbar, io);
  Gm = ish(Gm, io);
  td = ish(td, io);
  Thbar = ish(Thbar, io);
  const int Dl = td[0], Dr = td[2], ncol = 2 * Dr;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Dl * Dr) return;
  const int a = t / Dr, c = t % Dr;
  double2 cb[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) cb[x] = Cbar[(size_t)(2 * a + (x >> 1)) * ncol + (x & 1) * Dr + c];
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    double2 v = make_double2(0, 0);
#pragma unroll
    for (int x = 0; x < 4; ++x) v = cadd(v, cmul(conjd(Gm[4 * x + y]), cb[x]));   // (G^H)_{yx}
    Thbar[(size_t)(2 * a + (y >> 1)) * ncol + (y & 1) * Dr + c] = v;
  }
}

__global__ void theta_reduce_kernel(const double* __restrict__ gate_grad, const int* __restrict__ off,
                                    const int* __restrict__ gidx, const double* __restrict__ scale,
                                    int n_theta, double* grad, size_t stride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_theta) return;
  const size_t io = (size_t)blockIdx.y * stride;
  gate_grad = ish(gate_grad, io);
  grad = ish(grad, io);
  double acc = 0.0;
  for (int e = off[t]; e < off[t + 1]; ++e) acc += scale[e] * gate_grad[gidx[e]];
  grad[t] = acc;
}

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace


void launch_gate_matrices(const Batch& bt, const void* d_gates, int n_gates, const double* d_theta, int n_theta,
                          double2* G, double2* dG, int* status, cudaStream_t st) {
  if (n_gates <= 0) return;
  gate_matrices_kernel<<<dim3(cdiv(n_gates, 128), bt.n), 128, 0, st>>>((const mps_gate*)d_gates, n_gates, d_theta,
                                                                       n_theta, G, dG, status, bt.stride);
  note_launch();
}

void launch_contract(const Batch& bt, const double2* Bl, const double2* Br, const int* dims, int b,
                     const double2* G, const double* lam_left, double2* C, double2* A, double2* Bl_tape,
                     double2* Br_tape, int max_dl, int max_dr, cudaStream_t st) {
  contract_kernel<<<dim3(cdiv((long long)max_dl * max_dr, 128), bt.n), 128, 0, st>>>(
      Bl, Br, dims, b, G, lam_left, C, A, Bl_tape, Br_tape, bt.stride);
  note_launch();
}

namespace {
__global__ void copy_f64_kernel(double* __restrict__ dst, size_t dst_stride, const double* __restrict__ src,
                                size_t src_stride, size_t n) {
  dst = ish(dst, (size_t)blockIdx.y * dst_stride);
  src = ish(src, (size_t)blockIdx.y * src_stride);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void zero_f64_kernel(double* __restrict__ dst, size_t stride, size_t n) {
  dst = ish(dst, (size_t)blockIdx.y * stride);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = 0.0;
}

// out[0] = first non-zero status over the instances (0 if none), out[1] = that instance;
// every status word is cleared.
__global__ void status_fetch_kernel(int* status, size_t stride, int n_inst, double* out) {
  double code = 0.0, which = -1.0;
  for (int i = 0; i < n_inst; ++i) {
    int* si = ish(status, (size_t)i * stride);
    if (*si != 0 && code == 0.0) {
      code = (double)*si;
      which = (double)i;
    }
    *si = 0;
  }
  out[0] = code;
  out[1] = which;
}
}  // namespace

void launch_copy_f64(const Batch& bt, double* dst, size_t dst_stride, const double* src, size_t src_stride,
                     size_t n, cudaStream_t st) {
  if (n == 0) return;
  const long long blocks = std::min<long long>(cdiv((long long)n, 256), 152LL * 4);
  copy_f64_kernel<<<dim3((unsigned)blocks, bt.n), 256, 0, st>>>(dst, dst_stride, src, src_stride, n);
  note_launch();
}

void launch_zero_f64(const Batch& bt, double* dst, size_t n, cudaStream_t st) {
  if (n == 0) return;
  const long long blocks = std::min<long long>(cdiv((long long)n, 256), 152LL * 4);
  zero_f64_kernel<<<dim3((unsigned)blocks, bt.n), 256, 0, st>>>(dst, bt.stride, n);
  note_launch();
}

void launch_status_fetch(const Batch& bt, int* status, double* out, cudaStream_t st) {
  status_fetch_kernel<<<1, 1, 0, st>>>(status, bt.stride, bt.n, out);
  note_launch();
}

size_t svd_smem_bytes(int m_cap, int n_cap) {
  const size_t R = std::max(m_cap, n_cap), K = std::min(m_cap, n_cap);
  return (K * K + R * K) * sizeof(double2);
}

// Largest dynamic shared memory the SVD kernel may use: the device's opt-in limit per block minus
// the kernel's static shared memory (queried once; 0 if the attribute cannot be raised).
static size_t svd_dynamic_limit_query() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, svd_kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  size_t want = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
  if (cudaFuncSetAttribute(svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want) != cudaSuccess) {
    cudaGetLastError();
    want = 48 * 1024 > fa.sharedSizeBytes ? 48 * 1024 - fa.sharedSizeBytes : 0;
  }
  return want;
}

static size_t svd_dynamic_limit() {
  static const size_t limit = svd_dynamic_limit_query();   // thread-safe one-time initialisation
  return limit;
}

bool svd_fits_smem(int m_cap, int n_cap) { return svd_smem_bytes(m_cap, n_cap) <= svd_dynamic_limit(); }

namespace {
std::mutex g_tiles_mu;
std::map<std::pair<int, int>, std::pair<int, int>> g_tiles;
}  // namespace

void svd_tiles_set(const int* entries, int n) {
  std::lock_guard<std::mutex> lock(g_tiles_mu);
  g_tiles.clear();
  for (int i = 0; i < n; ++i)
    g_tiles[{entries[4 * i], entries[4 * i + 1]}] = {entries[4 * i + 2], entries[4 * i + 3]};
}

void svd_tiles_get(int m_cap, int n_cap, int* jg32, int* jg64) {
  std::lock_guard<std::mutex> lock(g_tiles_mu);
  const auto it = g_tiles.find({m_cap, n_cap});
  *jg32 = it == g_tiles.end() ? 0 : it->second.first;
  *jg64 = it == g_tiles.end() ? 0 : it->second.second;
}

void launch_svd(const Batch& bt, const SvdArgs& a, int m_cap, int n_cap, cudaStream_t st) {
  SvdArgs b = a;
  if (b.jg32 == 0 && b.jg64 == 0) svd_tiles_get(m_cap, n_cap, &b.jg32, &b.jg64);
  size_t smem = 0;
  if (svd_fits_smem(m_cap, n_cap)) {
    b.scratch = nullptr;
    smem = svd_smem_bytes(m_cap, n_cap);
  }
  svd_kernel<<<bt.n, SVD_THREADS, smem, st>>>(b, bt.stride);
  note_launch();
}

void launch_vh_rows(const Batch& bt, const double2* Vs, const int* dims, int b, double2* Br_out, int max_k,
                    int max_ncol, cudaStream_t st) {
  vh_rows_kernel<<<dim3(cdiv((long long)max_k * max_ncol, 256), bt.n), 256, 0, st>>>(Vs, dims, b, Br_out,
                                                                                     bt.stride);
  note_launch();
}

void launch_conjT(const Batch& bt, const double2* Bbar_r, const int* td, double2* Vbar, int max_k, int max_ncol,
                  cudaStream_t st) {
  conjT_kernel<<<dim3(cdiv((long long)max_k * max_ncol, 256), bt.n), 256, 0, st>>>(Bbar_r, td, Vbar, bt.stride);
  note_launch();
}

void launch_sbar(const Batch& bt, double* lambar_slot, const double* s, const int* td, double* wbar,
                 cudaStream_t st) {
  sbar_kernel<<<bt.n, 256, 0, st>>>(lambar_slot, s, td, wbar, bt.stride);
  note_launch();
}

void launch_build_K(const Batch& bt, const double2* Y, const double* s, const double* wbar, const int* td,
                    double2* K, int max_K, cudaStream_t st) {
  build_K_kernel<<<dim3(cdiv((long long)max_K * max_K, 256), bt.n), 256, 0, st>>>(Y, s, wbar, td, K, bt.stride);
  note_launch();
}

void launch_zscale(const Batch& bt, double2* Z, const double* s, const int* td, int max_n, int max_k,
                   cudaStream_t st) {
  zscale_kernel<<<dim3(cdiv((long long)max_n * max_k, 256), bt.n), 256, 0, st>>>(Z, s, td, bt.stride);
  note_launch();
}

void launch_lam_scale(const Batch& bt, double2* Cbar, const double2* Ctbar, const double2* C,
                      const double* lam_left, const int* td, double* lambar_left, int max_dl, cudaStream_t st) {
  lam_scale_kernel<<<dim3(cdiv(max_dl, 8), bt.n), 256, 0, st>>>(Cbar, Ctbar, C, lam_left, td, lambar_left,
                                                                bt.stride);
  note_launch();
}

void launch_gbar(const Batch& bt, const double2* Cbar, const double2* Theta, const int* td, const double2* dG,
                 double2* Gbar, double* gate_grad, cudaStream_t st) {
  gbar_kernel<<<bt.n, 256, 0, st>>>(Cbar, Theta, td, dG, Gbar, gate_grad, bt.stride);
  note_launch();
}

void launch_thetabar(const Batch& bt, const double2* Cbar, const double2* G, const int* td, double2* Thbar,
                     int max_dl, int max_dr, cudaStream_t st) {
  thetabar_kernel<<<dim3(cdiv((long long)max_dl * max_dr, 128), bt.n), 128, 0, st>>>(Cbar, G, td, Thbar,
                                                                                     bt.stride);
  note_launch();
}

void launch_theta_reduce(const Batch& bt, const double* gate_grad, const int* csr_off, const int* csr_gate,
                         const double* csr_scale, int n_theta, double* grad, cudaStream_t st) {
  if (n_theta <= 0) return;
  theta_reduce_kernel<<<dim3(cdiv(n_theta, 128), bt.n), 128, 0, st>>>(gate_grad, csr_off, csr_gate, csr_scale,
                                                                      n_theta, grad, bt.stride);
  note_launch();
}

}  // namespace mpsk
