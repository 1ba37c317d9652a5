// Complex GEMM on the tensor cores in split-TF32 ("3xTF32") arithmetic, for the mixed-precision
// path (MPS_PRECISION_MIXED): same descriptors (GemmDesc), operand ops, dimension expressions and
// instance batching as the FP64 kernels in gemm.cu.
//
// Each real operand x is split into two TF32 numbers, hi = tf32(x) and lo = tf32(x - hi); a real
// product is hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 resolution), accumulated in
// FP32 by mma.sync m16n8k8 TF32 instructions.  A complex product takes four real products
// (re = ArBr - AiBi, im = ArBi + AiBr; no three-multiplication form).  Operands are read in FP64
// and converted while they are staged in shared memory; alpha, beta and the output stay FP64.
// The result is accurate to about FP32 rounding, the precision the mixed path asks of its bond
// contractions and Pauli sweeps.
//
// CTA tile: 32 x 32 outputs, 4 warps (2 x 2), each warp 16 x 16 = two m16n8 tiles; K in steps
// of 8.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

constexpr int TT = 32, TKK = 8, TF_THREADS = 128;

__device__ __forceinline__ double2 ld_op(const double2* X, int ld, int op, int r, int c) {
  switch (op) {   // element (r, c) of op(X)
    case OP_N: return X[(size_t)r * ld + c];
    case OP_T: return X[(size_t)c * ld + r];
    case OP_H: return conjd(X[(size_t)c * ld + r]);
    default: return conjd(X[(size_t)r * ld + c]);
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// hi and lo TF32 parts of a double
__device__ __forceinline__ void split(double v, uint32_t* hi, uint32_t* lo) {
  const float f = (float)v;
  const uint32_t h = to_tf32(f);
  *hi = h;
  *lo = to_tf32(f - __uint_as_float(h));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared tiles: [part][row][k] for A (part: 0 re hi, 1 re lo, 2 im hi, 3 im lo, 4 -im hi, 5 -im lo)
// and [part][k][col] for B (parts 0..3).  +4 padding against bank conflicts.
struct TfSmem {
  uint32_t A[6][TT][TKK + 4];
  uint32_t B[4][TKK][TT + 4];
};

__device__ __forceinline__ void tile_tf32x3(const GemmDesc& d0, int row0, int col0, size_t io, TfSmem& sm) {
  GemmDesc d = d0;
  d.A = ish(d.A, io);
  d.B = ish(d.B, io);
  d.C = ish(d.C, io);
  d.dims = ish(d.dims, io);
  const int M = deval(d.M, d.dims), N = deval(d.N, d.dims), K = deval(d.K, d.dims);
  if (row0 >= M || col0 >= N || M <= 0 || N <= 0) return;
  const int lda = deval(d.lda, d.dims), ldb = deval(d.ldb, d.dims), ldc = deval(d.ldc, d.dims);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 16, wn = (warp & 1) * 16;   // warp's 16 x 16 block in the tile
  const int g = lane >> 2, t4 = lane & 3;
  float accr[2][4], acci[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) accr[j][e] = acci[j][e] = 0.f;
  for (int k0 = 0; k0 < K; k0 += TKK) {
    // stage op(A)[row0.., k0..] (32 x 8) and op(B)[k0.., col0..] (8 x 32): 256 elements each
    for (int e = tid; e < TT * TKK; e += TF_THREADS) {
      const int r = e / TKK, kk = e % TKK;
      const int gr = row0 + r, gk = k0 + kk;
      const double2 v = (gr < M && gk < K) ? ld_op(d.A, lda, d.opA, gr, gk) : make_double2(0.0, 0.0);
      uint32_t h, l;
      split(v.x, &h, &l);
      sm.A[0][r][kk] = h;
      sm.A[1][r][kk] = l;
      split(v.y, &h, &l);
      sm.A[2][r][kk] = h;
      sm.A[3][r][kk] = l;
      sm.A[4][r][kk] = h ^ 0x80000000u;   // -im (sign flip is exact)
      sm.A[5][r][kk] = l ^ 0x80000000u;
    }
    for (int e = tid; e < TKK * TT; e += TF_THREADS) {
      const int kk = e / TT, c = e % TT;
      const int gk = k0 + kk, gc = col0 + c;
      const double2 v = (gk < K && gc < N) ? ld_op(d.B, ldb, d.opB, gk, gc) : make_double2(0.0, 0.0);
      uint32_t h, l;
      split(v.x, &h, &l);
      sm.B[0][kk][c] = h;
      sm.B[1][kk][c] = l;
      split(v.y, &h, &l);
      sm.B[2][kk][c] = h;
      sm.B[3][kk][c] = l;
    }
    __syncthreads();
    // A fragments (16 x 8, row-major): a0 (g, t4), a1 (g+8, t4), a2 (g, t4+4), a3 (g+8, t4+4)
    uint32_t a[6][4];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      a[q][0] = sm.A[q][wm + g][t4];
      a[q][1] = sm.A[q][wm + g + 8][t4];
      a[q][2] = sm.A[q][wm + g][t4 + 4];
      a[q][3] = sm.A[q][wm + g + 8][t4 + 4];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      // B fragments (8 x 8, column-major): b0 (t4, g), b1 (t4+4, g)
      uint32_t b[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        b[q][0] = sm.B[q][t4][wn + 8 * j + g];
        b[q][1] = sm.B[q][t4 + 4][wn + 8 * j + g];
      }
      // re += Ar Br - Ai Bi
      mma_tf32(accr[j], a[0], b[0]);
      mma_tf32(accr[j], a[0], b[1]);
      mma_tf32(accr[j], a[1], b[0]);
      mma_tf32(accr[j], a[4], b[2]);
      mma_tf32(accr[j], a[4], b[3]);
      mma_tf32(accr[j], a[5], b[2]);
      // im += Ar Bi + Ai Br
      mma_tf32(acci[j], a[0], b[2]);
      mma_tf32(acci[j], a[0], b[3]);
      mma_tf32(acci[j], a[1], b[2]);
      mma_tf32(acci[j], a[2], b[0]);
      mma_tf32(acci[j], a[2], b[1]);
      mma_tf32(acci[j], a[3], b[0]);
    }
    __syncthreads();
  }
  const bool zero_beta = (d.beta.x == 0.0 && d.beta.y == 0.0);
  // accumulators: c0 (g, 2 t4), c1 (g, 2 t4 + 1), c2 (g+8, 2 t4), c3 (g+8, 2 t4 + 1)
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = row0 + wm + g + ((e >> 1) << 3);
      const int c = col0 + wn + 8 * j + 2 * t4 + (e & 1);
      if (r >= M || c >= N) continue;
      double2 v = cmul(d.alpha, make_double2((double)accr[j][e], (double)acci[j][e]));
      double2* out = d.C + (size_t)r * ldc + c;
      if (!zero_beta) v = cadd(v, cmul(d.beta, *out));
      *out = v;
    }
}

// grid: x = column tile, y = row tile + tiles_m * instance, z = descriptor
__global__ void __launch_bounds__(TF_THREADS) zgemm_tf32x3_batched_kernel(const GemmDesc* __restrict__ descs,
                                                                          int tiles_m, size_t stride) {
  __shared__ TfSmem sm;
  const int inst = blockIdx.y / tiles_m, tm = blockIdx.y - inst * tiles_m;
  tile_tf32x3(descs[blockIdx.z], tm * TT, blockIdx.x * TT, (size_t)inst * stride, sm);
}

// grid: x = column tile, y = row tile, z = descriptor + count * instance
__global__ void __launch_bounds__(TF_THREADS) zgemm_tf32x3_small_kernel(const GemmBatch batch, size_t stride) {
  __shared__ TfSmem sm;
  const int inst = blockIdx.z / batch.count;
  tile_tf32x3(batch.d[blockIdx.z - inst * batch.count], blockIdx.y * TT, blockIdx.x * TT, (size_t)inst * stride,
              sm);
}

}  // namespace

void launch_zgemm_tf32x3_small(const Batch& bt, const GemmBatch& b, int max_m, int max_n, cudaStream_t st) {
  if (b.count <= 0 || max_m <= 0 || max_n <= 0) return;
  dim3 grid((max_n + TT - 1) / TT, (max_m + TT - 1) / TT, b.count * bt.n);
  zgemm_tf32x3_small_kernel<<<grid, TF_THREADS, 0, st>>>(b, bt.stride);
  note_launch();
}

void launch_zgemm_tf32x3_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n,
                                 cudaStream_t st) {
  if (count <= 0 || max_m <= 0 || max_n <= 0) return;
  const int tiles_m = (max_m + TT - 1) / TT;
  dim3 grid((max_n + TT - 1) / TT, tiles_m * bt.n, count);
  zgemm_tf32x3_batched_kernel<<<grid, TF_THREADS, 0, st>>>(d_descs, tiles_m, bt.stride);
  note_launch();
}

}  // namespace mpsk
