// Gate application (Sec. 3, two-qubit gate with Hastings' canonical-form update) and the
// custom pieces of its exact adjoint (Sec. 4 / App. A rules), FP64.
#include <cmath>

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
                                     int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_gates) return;
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
                                const double* __restrict__ lam_left, double2* C, double2* A) {
  const int Dl = dims[b], Dm = dims[b + 1], Dr = dims[b + 2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
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

// ---- one-sided Jacobi SVD ------------------------------------------------------------------
constexpr int SVD_THREADS = 256;
constexpr int SVD_MAX_SWEEPS = 60;
constexpr double SVD_NULL_REL = 1e-13;   // numerical-zero singular values (relative to s_max)
constexpr double SVD_DEGEN_REL = 1e-10;  // exactly degenerate pairs of squared singular values

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(SVD_THREADS) svd_kernel(SvdArgs p) {
  const int b = p.b;
  const int Dl = p.dims[b], Dr = p.dims[b + 2];
  const int m = 2 * Dl, K = 2 * Dr;            // A is m x K, orthogonalise its K columns
  const int Kp = K + (K & 1);                  // even count for the round-robin schedule
  double2* A = p.A;
  double2* V = p.Vw;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = SVD_THREADS / 32;
  __shared__ double red[SVD_THREADS / 32];
  __shared__ int rotated;
  __shared__ double s_sh[1024];
  __shared__ double fro2_sh;

  for (int e = tid; e < K * K; e += SVD_THREADS) V[e] = make_double2((e / K) == (e % K) ? 1.0 : 0.0, 0.0);
  // ||A||_F^2 (columns below 1e-15 ||A||_F are treated as numerically zero)
  double f = 0.0;
  for (int e = tid; e < m * K; e += SVD_THREADS) f += A[e].x * A[e].x + A[e].y * A[e].y;
  f = warp_sum(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    fro2_sh = t;
  }
  __syncthreads();
  const double tiny = 1e-30 * fro2_sh;          // (1e-15 ||A||_F)^2
  const double tol = 4.0 * 2.220446049250313e-16 * sqrt((double)m);
  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < Kp - 1; ++r) {
      for (int t = warp; t < Kp / 2; t += nwarp) {
        int pc, qc;
        if (t == 0) {
          pc = r;
          qc = Kp - 1;
        } else {
          pc = (r + t) % (Kp - 1);
          qc = (r - t + Kp - 1) % (Kp - 1);
        }
        if (pc >= K || qc >= K) continue;
        double2* ap = A + (size_t)pc * m;
        double2* aq = A + (size_t)qc * m;
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        for (int i = lane; i < m; i += 32) {
          double2 x = ap[i], y = aq[i];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          gr += x.x * y.x + x.y * y.y;   // conj(x) * y
          gi += x.x * y.y - x.y * y.x;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        if (al < tiny || be < tiny) continue;
        const double g = hypot(gr, gi);
        if (!(g > tol * sqrt(al) * sqrt(be))) continue;
        const double zeta = (be - al) / (2.0 * g);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        const double2 ph = make_double2(gr / g, gi / g);   // e^{i phi}
        // a_p' = c a_p - s e^{-i phi} a_q ; a_q' = s e^{i phi} a_p + c a_q
        const double2 sp = cscale(ph, s), sm = cscale(conjd(ph), s);
        for (int i = lane; i < m; i += 32) {
          double2 x = ap[i], y = aq[i];
          ap[i] = csub(cscale(x, c), cmul(sm, y));
          aq[i] = cadd(cmul(sp, x), cscale(y, c));
        }
        double2* vp = V + (size_t)pc * K;
        double2* vq = V + (size_t)qc * K;
        for (int i = lane; i < K; i += 32) {
          double2 x = vp[i], y = vq[i];
          vp[i] = csub(cscale(x, c), cmul(sm, y));
          vq[i] = cadd(cmul(sp, x), cscale(y, c));
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep >= SVD_MAX_SWEEPS && tid == 0) set_status(p.status, MPS_ENOCONV);
  // column norms -> singular values
  for (int j = warp; j < K; j += nwarp) {
    double v = 0.0;
    for (int i = lane; i < m; i += 32) {
      double2 x = A[(size_t)j * m + i];
      v += x.x * x.x + x.y * x.y;
    }
    v = warp_sum(v);
    if (lane == 0) s_sh[j] = sqrt(v);
  }
  __syncthreads();
  // stable descending rank, then scatter sorted columns; for the tape, columns of A V whose
  // singular value is at most SVD_NULL_REL * s_max are rounding noise of an exactly
  // rank-deficient matrix and are stored as exact zeros (the adjoint relies on it)
  __shared__ double smax_sh;
  if (tid == 0) {
    double mx = 0.0;
    for (int j = 0; j < K; ++j) mx = fmax(mx, s_sh[j]);
    smax_sh = mx;
  }
  __syncthreads();
  for (int j = tid; j < K; j += SVD_THREADS) {
    const double sj = s_sh[j];
    int rank = 0;
    for (int i = 0; i < K; ++i) {
      const double si = s_sh[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    p.s[rank] = sj;
    for (int i = 0; i < K; ++i) p.Vs[(size_t)rank * K + i] = V[(size_t)j * K + i];
    if (p.W) {
      const bool null_col = !(sj > SVD_NULL_REL * smax_sh);
      for (int i = 0; i < m; ++i)
        p.W[(size_t)rank * m + i] = null_col ? make_double2(0.0, 0.0) : A[(size_t)j * m + i];
    }
  }
  __syncthreads();
  __threadfence_block();
  __shared__ int k_sh;
  __shared__ double nk_sh;
  if (tid == 0) {
    double n2 = 0.0;
    for (int j = 0; j < K; ++j) n2 += p.s[j] * p.s[j];
    const double nrm = sqrt(n2);
    int cnt = 0;
    if (nrm > 0.0 && isfinite(nrm)) {
      for (int j = 0; j < K; ++j) cnt += (p.s[j] / nrm > p.eps);
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
    }
    p.dims[b + 1] = k;
  }
}

__global__ void vh_rows_kernel(const double2* __restrict__ Vs, const int* __restrict__ dims, int b,
                               double2* Br) {
  const int k = dims[b + 1], ncol = 2 * dims[b + 2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * ncol) return;
  const int j = t / ncol, r = t % ncol;
  Br[(size_t)j * ncol + r] = conjd(Vs[(size_t)j * ncol + r]);
}

// ---- adjoint pieces -------------------------------------------------------------------------
__global__ void conjT_kernel(const double2* __restrict__ Bbr, const int* __restrict__ td, double2* Vbar) {
  const int k = td[3], ncol = 2 * td[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * ncol) return;
  const int r = t / k, j = t % k;                    // Vbar[r][j] = conj(Bbar_r[j][r])
  Vbar[(size_t)r * k + j] = conjd(Bbr[(size_t)j * ncol + r]);
}

__global__ void sbar_kernel(double* lambar, const double* __restrict__ s, const int* __restrict__ td,
                            double* wbar) {
  const int k = td[3], ncol = 2 * td[2];
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
                               const double* __restrict__ wbar, const int* __restrict__ td, double2* Km) {
  const int k = td[3], ncol = 2 * td[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncol * ncol) return;
  const int i = t / ncol, j = t % ncol;
  // numerical zeros (s <= SVD_NULL_REL s_1) enter as exact zeros
  const double wi = s[i] > SVD_NULL_REL * s[0] ? s[i] * s[i] : 0.0;
  const double wj = s[j] > SVD_NULL_REL * s[0] ? s[j] * s[j] : 0.0;
  // F_ij = 1/(w_j - w_i), 0 inside exactly degenerate pairs (|dw| <= SVD_DEGEN_REL max(w))
  const double dw = wj - wi;
  const double F = fabs(dw) > SVD_DEGEN_REL * fmax(wi, wj) ? 1.0 / dw : 0.0;
  double2 v = make_double2(i == j ? wbar[i] : 0.0, 0.0);
  if (i != j) {
    if (j < k) v = cadd(v, cscale(Y[(size_t)i * k + j], F));               // J_ij = F_ij Y_ij
    if (i < k) v = cadd(v, cscale(conjd(Y[(size_t)j * k + i]), -F));       // (J^H)_ij = conj(F_ji Y_ji)
  }
  Km[(size_t)i * ncol + j] = v;
}

__global__ void lam_scale_kernel(double2* Cbar, const double2* __restrict__ Ctbar,
                                 const double2* __restrict__ C, const double* __restrict__ lam_left,
                                 const int* __restrict__ td, double* lambar_left) {
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
                                                   double* gate_grad) {
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
                                const int* __restrict__ td, double2* Thbar) {
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
                                    int n_theta, double* grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_theta) return;
  double acc = 0.0;
  for (int e = off[t]; e < off[t + 1]; ++e) acc += scale[e] * gate_grad[gidx[e]];
  grad[t] = acc;
}

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

void launch_gate_matrices(const void* d_gates, int n_gates, const double* d_theta, int n_theta, double2* G,
                          double2* dG, int* status, cudaStream_t st) {
  if (n_gates <= 0) return;
  gate_matrices_kernel<<<cdiv(n_gates, 128), 128, 0, st>>>((const mps_gate*)d_gates, n_gates, d_theta, n_theta,
                                                           G, dG, status);
  note_launch();
}

void launch_contract(const double2* Bl, const double2* Br, const int* dims, int b, const double2* G,
                     const double* lam_left, double2* C, double2* A, int max_dl, int max_dr, cudaStream_t st) {
  contract_kernel<<<cdiv((long long)max_dl * max_dr, 128), 128, 0, st>>>(Bl, Br, dims, b, G, lam_left, C, A);
  note_launch();
}

void launch_svd(const SvdArgs& a, cudaStream_t st) {
  svd_kernel<<<1, SVD_THREADS, 0, st>>>(a);
  note_launch();
}

void launch_vh_rows(const double2* Vs, const int* dims, int b, double2* Br_out, int max_k, int max_ncol,
                    cudaStream_t st) {
  vh_rows_kernel<<<cdiv((long long)max_k * max_ncol, 256), 256, 0, st>>>(Vs, dims, b, Br_out);
  note_launch();
}

void launch_conjT(const double2* Bbar_r, const int* td, double2* Vbar, int max_k, int max_ncol, cudaStream_t st) {
  conjT_kernel<<<cdiv((long long)max_k * max_ncol, 256), 256, 0, st>>>(Bbar_r, td, Vbar);
  note_launch();
}

void launch_sbar(double* lambar_slot, const double* s, const int* td, double* wbar, int max_ncol,
                 cudaStream_t st) {
  (void)max_ncol;
  sbar_kernel<<<1, 256, 0, st>>>(lambar_slot, s, td, wbar);
  note_launch();
}

void launch_build_K(const double2* Y, const double* s, const double* wbar, const int* td, double2* K,
                    int max_ncol, cudaStream_t st) {
  build_K_kernel<<<cdiv((long long)max_ncol * max_ncol, 256), 256, 0, st>>>(Y, s, wbar, td, K);
  note_launch();
}

void launch_lam_scale(double2* Cbar, const double2* Ctbar, const double2* C, const double* lam_left,
                      const int* td, double* lambar_left, int max_dl, cudaStream_t st) {
  lam_scale_kernel<<<cdiv(max_dl, 8), 256, 0, st>>>(Cbar, Ctbar, C, lam_left, td, lambar_left);
  note_launch();
}

void launch_gbar(const double2* Cbar, const double2* Theta, const int* td, const double2* dG, double2* Gbar,
                 double* gate_grad, cudaStream_t st) {
  gbar_kernel<<<1, 256, 0, st>>>(Cbar, Theta, td, dG, Gbar, gate_grad);
  note_launch();
}

void launch_thetabar(const double2* Cbar, const double2* G, const int* td, double2* Thbar, int max_dl, int max_dr,
                     cudaStream_t st) {
  thetabar_kernel<<<cdiv((long long)max_dl * max_dr, 128), 128, 0, st>>>(Cbar, G, td, Thbar);
  note_launch();
}

void launch_theta_reduce(const double* gate_grad, const int* csr_off, const int* csr_gate, const double* csr_scale,
                         int n_theta, double* grad, cudaStream_t st) {
  if (n_theta <= 0) return;
  theta_reduce_kernel<<<cdiv(n_theta, 128), 128, 0, st>>>(gate_grad, csr_off, csr_gate, csr_scale, n_theta, grad);
  note_launch();
}

}  // namespace mpsk
