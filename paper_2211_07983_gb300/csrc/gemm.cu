// Batched complex FP64 GEMM driven by device-resident descriptors (see GemmDesc).
//
// Every bond contraction of the FP64 path (the site update B~_n = C V_k, the transfer
// matrices of the Pauli sweeps, the environment contractions of the energy cotangent and
// the GEMMs of the gate adjoints) is expressed as one or more descriptors; one launch
// executes a batch of independent descriptors.  Tiles that fall outside a descriptor's
// run-time M x N exit at once, so a launch can be sized for the bond-dimension caps.
//
// Tile: 64 x 64 outputs per 256-thread CTA, 4 x 4 per thread, K staged through shared
// memory in chunks of 8.  FP64 on GB300 runs at a small fraction of the FP32 rate, so this
// SIMT kernel is bound by the FP64 pipe, not by memory, once a tile is resident.
#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

constexpr int TM = 64, TN = 64, TK = 8;

__device__ __forceinline__ double2 load_op(const double2* X, int ld, int op, int r, int c) {
  // element (r, c) of op(X)
  switch (op) {
    case OP_N: return X[(size_t)r * ld + c];
    case OP_T: return X[(size_t)c * ld + r];
    case OP_H: return conjd(X[(size_t)c * ld + r]);
    default: return conjd(X[(size_t)r * ld + c]);
  }
}

__device__ __forceinline__ void gemm_tile(const GemmDesc& d0, int row0, int col0, size_t io) {
  GemmDesc d = d0;
  d.A = ish(d.A, io);
  d.B = ish(d.B, io);
  d.C = ish(d.C, io);
  d.dims = ish(d.dims, io);
  const int M = deval(d.M, d.dims), N = deval(d.N, d.dims), K = deval(d.K, d.dims);
  if (row0 >= M || col0 >= N || M <= 0 || N <= 0) return;
  const int lda = deval(d.lda, d.dims), ldb = deval(d.ldb, d.dims), ldc = deval(d.ldc, d.dims);
  __shared__ double2 As[TK][TM + 1];
  __shared__ double2 Bs[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      int kk = e / TM, ii = e % TM;
      int r = row0 + ii, c = k0 + kk;
      As[kk][ii] = (r < M && c < K) ? load_op(d.A, lda, d.opA, r, c) : make_double2(0.0, 0.0);
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int kk = e / TN, jj = e % TN;
      int r = k0 + kk, c = col0 + jj;
      Bs[kk][jj] = (r < K && c < N) ? load_op(d.B, ldb, d.opB, r, c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool zero_beta = (d.beta.x == 0.0 && d.beta.y == 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = col0 + tx + 16 * j;
      if (c >= N) continue;
      double2 v = cmul(d.alpha, acc[i][j]);
      double2* out = d.C + (size_t)r * ldc + c;
      if (!zero_beta) v = cadd(v, cmul(d.beta, *out));
      *out = v;
    }
  }
}

// grid: x = column tile, y = row tile + tiles_m * instance, z = descriptor
__global__ void __launch_bounds__(256) zgemm_batched_kernel(const GemmDesc* __restrict__ descs, int tiles_m,
                                                            size_t stride) {
  const int inst = blockIdx.y / tiles_m, tm = blockIdx.y - inst * tiles_m;
  gemm_tile(descs[blockIdx.z], tm * TM, blockIdx.x * TN, (size_t)inst * stride);
}

// Small per-gate GEMMs: 16 x 16 outputs per CTA, one per thread.  FP64 is the bound, so the
// work is spread over as many SMs as the output allows (a 64 x 64 output uses 16 CTAs).
constexpr int SM_T = 16, SK = 16;

// grid: x = column tile, y = row tile, z = descriptor + count * instance
__global__ void __launch_bounds__(256) zgemm_small_kernel(const GemmBatch batch, size_t stride) {
  const int inst = blockIdx.z / batch.count;
  const size_t io = (size_t)inst * stride;
  GemmDesc d = batch.d[blockIdx.z - inst * batch.count];
  d.A = ish(d.A, io);
  d.B = ish(d.B, io);
  d.C = ish(d.C, io);
  d.dims = ish(d.dims, io);
  const int M = deval(d.M, d.dims), N = deval(d.N, d.dims), K = deval(d.K, d.dims);
  const int row0 = blockIdx.y * SM_T, col0 = blockIdx.x * SM_T;
  if (row0 >= M || col0 >= N || M <= 0 || N <= 0) return;
  if (K <= 0 && d.beta.x == 1.0 && d.beta.y == 0.0) return;   // C = 0 + C: nothing to do
  const int lda = deval(d.lda, d.dims), ldb = deval(d.ldb, d.dims), ldc = deval(d.ldc, d.dims);
  __shared__ double2 As[SK][SM_T + 1];
  __shared__ double2 Bs[SK][SM_T + 1];
  const int tx = threadIdx.x % SM_T, ty = threadIdx.x / SM_T;
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += SK) {
    {
      const int kk = threadIdx.x / SM_T, ii = threadIdx.x % SM_T;   // SK x SM_T = 256 loads each
      const int r = row0 + ii, c = k0 + kk;
      As[kk][ii] = (r < M && c < K) ? load_op(d.A, lda, d.opA, r, c) : make_double2(0.0, 0.0);
      const int rb = k0 + kk, cb = col0 + ii;
      Bs[kk][ii] = (rb < K && cb < N) ? load_op(d.B, ldb, d.opB, rb, cb) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK; ++kk) acc = cfma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  const int r = row0 + ty, c = col0 + tx;
  if (r < M && c < N) {
    double2 v = cmul(d.alpha, acc);
    double2* out = d.C + (size_t)r * ldc + c;
    if (!(d.beta.x == 0.0 && d.beta.y == 0.0)) v = cadd(v, cmul(d.beta, *out));
    *out = v;
  }
}

}  // namespace

void launch_zgemm_small(const Batch& bt, const GemmBatch& b, int max_m, int max_n, cudaStream_t st) {
  if (b.count <= 0 || max_m <= 0 || max_n <= 0) return;
  dim3 grid((max_n + SM_T - 1) / SM_T, (max_m + SM_T - 1) / SM_T, b.count * bt.n);
  zgemm_small_kernel<<<grid, 256, 0, st>>>(b, bt.stride);
  note_launch();
}

void launch_zgemm_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n,
                          cudaStream_t st) {
  if (count <= 0 || max_m <= 0 || max_n <= 0) return;
  const int tiles_m = (max_m + TM - 1) / TM;
  dim3 grid((max_n + TN - 1) / TN, tiles_m * bt.n, count);
  zgemm_batched_kernel<<<grid, 256, 0, st>>>(d_descs, tiles_m, bt.stride);
  note_launch();
}

}  // namespace mpsk
