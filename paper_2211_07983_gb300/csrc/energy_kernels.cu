// Pauli-string energy (Sec. 2, Eq. expect-val; Sec. 3, Eq. paulistringexp) and its cotangent
// dE/dB* (Sec. 4, Eq. expecgrad): the element-wise kernels around the batched GEMMs.
#include "../../include/mps.h"
#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// O applied to the physical index of B_s (O = X, Y, Z): the transfer matrix with operator O,
// sum conj(B[a',i',b']) O[i',i] ..., equals the identity transfer with conj(B) replaced by
// conj(O B) (Pauli matrices are Hermitian).
__global__ void apply_paulis_kernel(const double2* __restrict__ B, const size_t* __restrict__ site_off,
                                    const size_t* __restrict__ ob_off, const int* __restrict__ dims,
                                    double2* OB, int n, size_t stride) {
  const int inst = blockIdx.y / n, s = blockIdx.y - inst * n, o = blockIdx.z;
  const size_t io = (size_t)inst * stride;
  B = ish(B, io);
  dims = ish(dims, io);
  OB = ish(OB, io);
  const int Dl = dims[s], Dr = dims[s + 1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Dl * Dr) return;
  const int a = t / Dr, c = t % Dr;
  const double2* src = B + site_off[s];
  double2* dst = OB + ob_off[3 * s + o];
  const double2 b0 = src[(size_t)(2 * a) * Dr + c], b1 = src[(size_t)(2 * a + 1) * Dr + c];
  double2 o0, o1;
  if (o == 0) {          // X
    o0 = b1;
    o1 = b0;
  } else if (o == 1) {   // Y = [[0,-i],[i,0]]
    o0 = make_double2(b1.y, -b1.x);
    o1 = make_double2(-b0.y, b0.x);
  } else {               // Z
    o0 = b0;
    o1 = make_double2(-b1.x, -b1.y);
  }
  dst[(size_t)(2 * a) * Dr + c] = o0;
  dst[(size_t)(2 * a + 1) * Dr + c] = o1;
}

__global__ void env_dots_kernel(const double2* const* __restrict__ Ls, const double2* const* __restrict__ Rs,
                                const int* __restrict__ didx, const int* __restrict__ dims, int count,
                                double2* e, size_t stride) {
  const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (t >= count) return;
  const size_t io = (size_t)blockIdx.y * stride;
  dims = ish(dims, io);
  e = ish(e, io);
  const int D = dims[didx[t]];
  const double2* L = ish(Ls[t], io);
  const double2* R = ish(Rs[t], io);
  double re = 0.0, im = 0.0;
  for (int x = lane; x < D * D; x += 32) {
    const double2 l = L[x], r = R[x];
    re += l.x * r.x - l.y * r.y;
    im += l.x * r.y + l.y * r.x;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) e[t] = make_double2(re, im);
}

// Neumaier (improved Kahan-Babuska) summation, one warp, fixed order: lane l sums terms
// l, l+32, ...; the 32 partial (sum, compensation) pairs are then added by lane 0 in order.
__global__ void energy_sum_kernel(const double2* __restrict__ e, const double* __restrict__ c, int n,
                                  double c0, const double2* __restrict__ Z, double* E_out, double* expect,
                                  int* status, size_t stride) {
  const int lane = threadIdx.x;
  const size_t io = (size_t)blockIdx.x * stride;
  e = ish(e, io);
  Z = ish(Z, io);
  E_out = ish(E_out, io);
  expect = ish(expect, io);
  status = ish(status, io);
  const double z = Z->x;
  double sum = 0.0, comp = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double v = c[k] * e[k].x;
    const double t = sum + v;
    comp += (fabs(sum) >= fabs(v)) ? (sum - t) + v : (v - t) + sum;
    sum = t;
    if (expect) expect[k] = e[k].x / z;
  }
  __shared__ double ps[32], pc[32];
  ps[lane] = sum;
  pc[lane] = comp;
  __syncwarp();
  if (lane == 0) {
    double s2 = c0 * z, c2 = 0.0;   // the identity string contributes c0 <psi|psi>
    for (int l = 0; l < 32; ++l) {
      for (int part = 0; part < 2; ++part) {
        const double v = part ? pc[l] : ps[l];
        const double t = s2 + v;
        c2 += (fabs(s2) >= fabs(v)) ? (s2 - t) + v : (v - t) + s2;
        s2 = t;
      }
    }
    const double E = (s2 + c2) / z;
    if (!isfinite(E) || !(z > 0.0)) set_status(status, MPS_ENUMERIC);
    *E_out = E;
  }
}

__global__ void axpy_lists_kernel(const AxpyList* __restrict__ lists, const double2* const* __restrict__ src,
                                  const double* __restrict__ coef, const int* __restrict__ dims, size_t stride) {
  const AxpyList& L = lists[blockIdx.y];
  const size_t io = (size_t)blockIdx.z * stride;
  dims = ish(dims, io);
  const int D = dims[L.didx];
  const long long ne = (long long)D * D * L.mult;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne) return;
  double2* out = ish(L.out, io);
  double2 v = L.accumulate ? out[t] : make_double2(0.0, 0.0);
  for (int j = L.src_begin; j < L.src_end; ++j) v = cadd(v, cscale(ish(src[j], io)[t], coef[j]));
  out[t] = v;
}

__global__ void seed_assemble_kernel(const SeedSite* __restrict__ sites, const double2* const* __restrict__ Enode,
                                     const int* __restrict__ node_op, const int* __restrict__ dims,
                                     const double2* __restrict__ Z, size_t stride) {
  const SeedSite& S = sites[blockIdx.y];
  const size_t io = (size_t)blockIdx.z * stride;
  dims = ish(dims, io);
  Z = ish(Z, io);
  const int Dl = dims[S.s], Dr = dims[S.s + 1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Dl * Dr) return;
  const int a = t / Dr, c = t % Dr;
  const size_t i0 = (size_t)(2 * a) * Dr + c, i1 = (size_t)(2 * a + 1) * Dr + c;
  const double2* Eid = ish(S.Eid, io);
  double2 v0 = Eid[i0], v1 = Eid[i1];
  for (int nd = S.node_begin; nd < S.node_end; ++nd) {
    const double2* En = ish(Enode[nd], io);
    const double2 e0 = En[i0], e1 = En[i1];
    const int o = node_op[nd];   // out[i'] += sum_i O[i', i] E[i]; 0 I, 1 X, 2 Y, 3 Z
    if (o == 0) {
      v0 = cadd(v0, e0);
      v1 = cadd(v1, e1);
    } else if (o == 1) {
      v0 = cadd(v0, e1);
      v1 = cadd(v1, e0);
    } else if (o == 2) {
      v0 = cadd(v0, make_double2(e1.y, -e1.x));
      v1 = cadd(v1, make_double2(-e0.y, e0.x));
    } else {
      v0 = cadd(v0, e0);
      v1 = csub(v1, e1);
    }
  }
  const double iz = 1.0 / Z->x;
  double2* out = ish(S.out, io);
  out[i0] = cscale(v0, iz);
  out[i1] = cscale(v1, iz);
}

__global__ void rsum_kernel(double2* out, const double2* __restrict__ AR, const double2* __restrict__ RI,
                            double c0, const double* __restrict__ E, const int* __restrict__ dims, int slot,
                            size_t stride) {
  const size_t io = (size_t)blockIdx.y * stride;
  out = ish(out, io);
  AR = ish(AR, io);
  RI = ish(RI, io);
  E = ish(E, io);
  dims = ish(dims, io);
  const int D = dims[slot];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * D) return;
  out[t] = cadd(AR[t], cscale(RI[t], c0 - *E));
}

}  // namespace

void launch_rsum(const Batch& bt, double2* out, const double2* AR, const double2* RI, double c0, const double* E,
                 const int* dims, int slot, int max_elems, cudaStream_t st) {
  rsum_kernel<<<dim3(cdiv(max_elems, 256), bt.n), 256, 0, st>>>(out, AR, RI, c0, E, dims, slot, bt.stride);
  note_launch();
}

void launch_apply_paulis(const Batch& bt, const double2* B, const size_t* site_off, const size_t* ob_off,
                         const int* dims, int n, double2* OB, int max_site, cudaStream_t st) {
  dim3 grid(cdiv(max_site, 128), n * bt.n, 3);
  apply_paulis_kernel<<<grid, 128, 0, st>>>(B, site_off, ob_off, dims, OB, n, bt.stride);
  note_launch();
}

void launch_env_dots(const Batch& bt, const double2* const* Ls, const double2* const* Rs, const int* didx,
                     const int* dims, int count, double2* e, cudaStream_t st) {
  if (count <= 0) return;
  env_dots_kernel<<<dim3(cdiv(count, 8), bt.n), 256, 0, st>>>(Ls, Rs, didx, dims, count, e, bt.stride);
  note_launch();
}

void launch_energy_sum(const Batch& bt, const double2* e, const double* c, int n_terms, double c0,
                       const double2* Z, double* E_out, double* expect, int* status, cudaStream_t st) {
  energy_sum_kernel<<<bt.n, 32, 0, st>>>(e, c, n_terms, c0, Z, E_out, expect, status, bt.stride);
  note_launch();
}

void launch_axpy_lists(const Batch& bt, const AxpyList* lists, int count, const double2* const* src,
                       const double* src_coef, const int* dims, int max_elems, cudaStream_t st) {
  if (count <= 0 || max_elems <= 0) return;
  dim3 grid(cdiv(max_elems, 256), count, bt.n);
  axpy_lists_kernel<<<grid, 256, 0, st>>>(lists, src, src_coef, dims, bt.stride);
  note_launch();
}

void launch_seed_assemble(const Batch& bt, const SeedSite* sites, int n_sites, const double2* const* Enode,
                          const int* node_op, const int* dims, const double2* Z, int max_site, cudaStream_t st) {
  if (n_sites <= 0) return;
  dim3 grid(cdiv(max_site, 128), n_sites, bt.n);
  seed_assemble_kernel<<<grid, 128, 0, st>>>(sites, Enode, node_op, dims, Z, bt.stride);
  note_launch();
}

}  // namespace mpsk
