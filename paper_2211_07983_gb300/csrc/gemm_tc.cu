// Complex GEMM on the 5th-generation tensor cores (tcgen05.mma, kind::tf32) in split-TF32
// ("3xTF32") arithmetic, with the accumulators in tensor memory (TMEM).  It serves the same
// descriptors (GemmDesc: operand ops, dimension expressions, instance batching) as the FP64 and
// mma.sync kernels, for the large transfer-matrix contractions of the Pauli sweeps on the
// mixed-precision path (bond dimensions of 64 and more).
//
// Arithmetic.  Every real operand x is split into hi = tf32(x) and lo = tf32(x - hi); a real
// product is hi*hi + hi*lo + lo*hi with FP32 accumulation.  A complex product takes four real
// products accumulated into two TMEM accumulators, D_re += Ar Br - Ai Bi and D_im += Ar Bi + Ai Br
// (the minus sign is the instruction descriptor's negate-A bit), so one k-step of 8 issues
// 4 x 3 = 12 MMAs of 128 x 128 x 8.  The result is accurate to about FP32 rounding.
//
// Tile and pipeline.  One CTA of 8 warps computes a 128 x 128 output tile.  K advances in chunks
// of 16: all threads read the FP64 operands (any op: N, T, H, C), split them and store the hi/lo
// parts of Re and Im in shared memory in the K-major, no-swizzle canonical layout of the MMA
// (8-row x 16-byte core matrices, core matrices adjacent in K 128 bytes apart, adjacent in M/N
// 512 bytes apart); then one thread issues the chunk's 24 MMAs and commits them to the stage's
// mbarrier.  Two stages: the loads of chunk c+1 overlap the MMAs of chunk c.  The epilogue waits
// for the last commit, moves the accumulators TMEM -> registers (tcgen05.ld, each warp its 32
// lanes), and writes alpha D + beta C in FP64.  Every mbarrier wait is bounded (two seconds);
// a wait that gives up records MPS_ETIMEOUT and the CTA skips its store.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mps.h"
#include "common.cuh"
#include "kernels.h"

namespace mpsk {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 16, TC_THREADS = 256, TC_STAGES = 2;
// operand elements each thread stages per chunk (A and B each)
constexpr int TC_PER = TC_M * TC_KC / TC_THREADS;
constexpr int TC_TMEM_COLS = 256;                        // D_re: columns 0..127, D_im: 128..255
// one operand part (128 rows x 16 tf32) = 8 KB; parts per stage: A {re,im} x {hi,lo}, B likewise
constexpr int TC_PART = TC_M * TC_KC * 4;
constexpr int TC_STAGE_BYTES = 8 * TC_PART;              // 64 KB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Element (r, c) of op(X) without the conjugation (applied after the conversion to FP32).
__device__ __forceinline__ double2 ld_raw(const double2* X, int ld, int op, int r, int c) {
  return (op == OP_N || op == OP_C) ? X[(size_t)r * ld + c] : X[(size_t)c * ld + r];
}

// FP64 -> FP32 (round to nearest even) in integer arithmetic.  GB300 runs FP64 instructions,
// conversions included, at 1/64 of the FP32 rate, and every operand element passes through here;
// the integer pipe does it at full rate.  Values below the FP32 normal range become (signed) zero:
// a GEMM operand that small is below the split-TF32 resolution of any product it enters.
__device__ __forceinline__ uint32_t f64_to_f32_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1FFFFFFFu;
  if (e == 0x7FF) return sign | 0x7F800000u | ((mant | rem) ? 0x400000u : 0u);
  const int ef = e - 896;   // rebias 1023 -> 127
  if (ef >= 255) return sign | 0x7F800000u;
  if (ef <= 0) return sign;
  uint32_t f = sign | ((uint32_t)ef << 23) | mant;
  // a carry out of the mantissa moves into the exponent: still the correctly rounded result
  if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) f += 1u;
  return f;
}

// FP32 -> FP64 (exact) in integer arithmetic; denormal inputs take the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float v) {
  const uint32_t f = __float_as_uint(v);
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu, sign = f & 0x80000000u;
  if (e == 0u) return m == 0u ? __longlong_as_double((long long)((unsigned long long)sign << 32)) : (double)v;
  const uint32_t eh = e == 0xFFu ? 0x7FFu : e + 896u;
  const unsigned long long d =
      ((unsigned long long)(sign | (eh << 20) | (m >> 3)) << 32) | ((unsigned long long)(m & 7u) << 29);
  return __longlong_as_double((long long)d);
}

// hi/lo TF32 parts of the real and imaginary part of a complex FP64 operand element
struct Split4 {
  uint32_t rh, rl, ih, il;
};
__device__ __forceinline__ Split4 split_c(double2 v, bool conj) {
  const float fr = __uint_as_float(f64_to_f32_bits(v.x));
  const float fi = __uint_as_float(f64_to_f32_bits(v.y) ^ (conj ? 0x80000000u : 0u));
  Split4 o;
  o.rh = to_tf32(fr);
  o.ih = to_tf32(fi);
  o.rl = to_tf32(fr - __uint_as_float(o.rh));
  o.il = to_tf32(fi - __uint_as_float(o.ih));
  return o;
}

// byte offset of element (row, k) of a 128 x 16 K-major operand part in the canonical
// no-swizzle layout: core matrix (row/8, k/4) at ((row/8)*4 + k/4)*128, row%8 at 16 B, k%4 at 4 B
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((((row >> 3) * (TC_KC / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// shared-memory matrix descriptor: start address, LBO (K direction) = 128 B, SBO (M/N direction)
// = (TC_KC/4)*128 = 512 B, fixed bits 46-48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (TC_KC / 4) * 128;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, K-major both, N = 128, M = 128
__host__ __device__ constexpr uint32_t idesc_tf32(bool neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(TC_N >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = tc_now();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (tc_now() - t0 > TC_WAIT_NS) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One 128 x 128 output tile of descriptor d (instance offset io).  Parts of a stage, in order:
// A re hi, A re lo, A im hi, A im lo, B re hi, B re lo, B im hi, B im lo.
//
// Producer: each thread holds TC_PER elements of A and of B for one chunk in registers.  The
// loads of chunk c+1 are issued right after chunk c is converted into shared memory, so they are
// in flight while the MMAs of chunk c run and while the next stage waits to be free.
__device__ void tc_tile(const GemmDesc& d0, int row0, int col0, size_t io, int* status, unsigned char* smem,
                        uint32_t tmem, uint32_t mbar0) {
  GemmDesc d = d0;
  d.A = ish(d.A, io);
  d.B = ish(d.B, io);
  d.C = ish(d.C, io);
  d.dims = ish(d.dims, io);
  const int M = deval(d.M, d.dims), N = deval(d.N, d.dims), K = deval(d.K, d.dims);
  const int lda = deval(d.lda, d.dims), ldb = deval(d.ldb, d.dims), ldc = deval(d.ldc, d.dims);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunks = (K + TC_KC - 1) / TC_KC;
  const uint32_t sbase = smem_u32(smem);
  uint32_t phase[TC_STAGES] = {0u, 0u};
  bool ok = true;
  // Consecutive threads take consecutive addresses of an operand in memory: along k when its rows
  // are contiguous in k (op N, C for A; op T, H for B), along the other index otherwise.
  const bool a_kfast = (d.opA == OP_N || d.opA == OP_C), b_kfast = !(d.opB == OP_N || d.opB == OP_C);
  const bool a_conj = (d.opA == OP_H || d.opA == OP_C), b_conj = (d.opB == OP_H || d.opB == OP_C);
  double2 ra[TC_PER], rb[TC_PER];
  auto load_chunk = [&](int c) {
    const int k0 = c * TC_KC;
#pragma unroll
    for (int i = 0; i < TC_PER; ++i) {
      const int e = tid + i * TC_THREADS;
      const int r = a_kfast ? e / TC_KC : e % TC_M, k = a_kfast ? e % TC_KC : e / TC_M;
      const int gr = row0 + r, gk = k0 + k;
      ra[i] = (gr < M && gk < K) ? ld_raw(d.A, lda, d.opA, gr, gk) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int i = 0; i < TC_PER; ++i) {
      const int e = tid + i * TC_THREADS;
      const int nn = b_kfast ? e / TC_KC : e % TC_N, k = b_kfast ? e % TC_KC : e / TC_N;
      const int gn = col0 + nn, gk = k0 + k;
      rb[i] = (gn < N && gk < K) ? ld_raw(d.B, ldb, d.opB, gk, gn) : make_double2(0.0, 0.0);
    }
  };
  auto store_chunk = [&](unsigned char* sp) {
#pragma unroll
    for (int i = 0; i < TC_PER; ++i) {
      const int e = tid + i * TC_THREADS;
      const int r = a_kfast ? e / TC_KC : e % TC_M, k = a_kfast ? e % TC_KC : e / TC_M;
      const Split4 q = split_c(ra[i], a_conj);
      const uint32_t o = kmajor_off(r, k);
      *reinterpret_cast<uint32_t*>(sp + 0 * TC_PART + o) = q.rh;
      *reinterpret_cast<uint32_t*>(sp + 1 * TC_PART + o) = q.rl;
      *reinterpret_cast<uint32_t*>(sp + 2 * TC_PART + o) = q.ih;
      *reinterpret_cast<uint32_t*>(sp + 3 * TC_PART + o) = q.il;
    }
#pragma unroll
    for (int i = 0; i < TC_PER; ++i) {
      const int e = tid + i * TC_THREADS;
      const int nn = b_kfast ? e / TC_KC : e % TC_N, k = b_kfast ? e % TC_KC : e / TC_N;
      const Split4 q = split_c(rb[i], b_conj);
      const uint32_t o = kmajor_off(nn, k);
      *reinterpret_cast<uint32_t*>(sp + 4 * TC_PART + o) = q.rh;
      *reinterpret_cast<uint32_t*>(sp + 5 * TC_PART + o) = q.rl;
      *reinterpret_cast<uint32_t*>(sp + 6 * TC_PART + o) = q.ih;
      *reinterpret_cast<uint32_t*>(sp + 7 * TC_PART + o) = q.il;
    }
  };
  if (nchunks > 0) load_chunk(0);
  for (int c = 0; c < nchunks; ++c) {
    const int st = c % TC_STAGES;
    unsigned char* sp = smem + st * TC_STAGE_BYTES;
    if (c >= TC_STAGES) {   // the MMAs of chunk c - STAGES read this stage: wait for their commit
      if (!mbar_wait(mbar0 + 8 * st, phase[st])) ok = false;
      phase[st] ^= 1u;
    }
    store_chunk(sp);
    if (c + 1 < nchunks) load_chunk(c + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = sbase + st * TC_STAGE_BYTES;
      const uint32_t dre = tmem, dim = tmem + TC_N;
      const uint32_t id_pos = idesc_tf32(false), id_neg = idesc_tf32(true);
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {   // k-steps of 8 = two core matrices = 256 bytes
        const uint32_t ko = kk * 256;
        const uint64_t arh = smem_desc(a0 + 0 * TC_PART + ko), arl = smem_desc(a0 + 1 * TC_PART + ko);
        const uint64_t aih = smem_desc(a0 + 2 * TC_PART + ko), ail = smem_desc(a0 + 3 * TC_PART + ko);
        const uint64_t brh = smem_desc(a0 + 4 * TC_PART + ko), brl = smem_desc(a0 + 5 * TC_PART + ko);
        const uint64_t bih = smem_desc(a0 + 6 * TC_PART + ko), bil = smem_desc(a0 + 7 * TC_PART + ko);
        const uint32_t first = (c == 0 && kk == 0) ? 0u : 1u;
        // D_re += Ar Br - Ai Bi
        mma_tf32(dre, arh, brh, id_pos, first);
        mma_tf32(dre, arh, brl, id_pos, 1u);
        mma_tf32(dre, arl, brh, id_pos, 1u);
        mma_tf32(dre, aih, bih, id_neg, 1u);
        mma_tf32(dre, aih, bil, id_neg, 1u);
        mma_tf32(dre, ail, bih, id_neg, 1u);
        // D_im += Ar Bi + Ai Br
        mma_tf32(dim, arh, bih, id_pos, first);
        mma_tf32(dim, arh, bil, id_pos, 1u);
        mma_tf32(dim, arl, bih, id_pos, 1u);
        mma_tf32(dim, aih, brh, id_pos, 1u);
        mma_tf32(dim, aih, brl, id_pos, 1u);
        mma_tf32(dim, ail, brh, id_pos, 1u);
      }
      mma_commit(mbar0 + 8 * st);
    }
  }
  // wait for the last commit of each stage that was used
  for (int st = 0; st < TC_STAGES && st < nchunks; ++st) {
    if (!mbar_wait(mbar0 + 8 * st, phase[st])) ok = false;
    phase[st] ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) set_status(status, MPS_ETIMEOUT);
    return;
  }
  // epilogue: warp w reads accumulator rows (TMEM lanes) 32 (w % 4) .. + 31 and the column half
  // w / 4 of each accumulator
  const int q4 = warp & 3, half = warp >> 2;
  const int r = row0 + q4 * 32 + lane;
  const bool zero_beta = (d.beta.x == 0.0 && d.beta.y == 0.0);
  const bool unit_alpha = (d.alpha.x == 1.0 && d.alpha.y == 0.0);
  const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
#pragma unroll 1
  for (int cb = half * (TC_N / 2); cb < (half + 1) * (TC_N / 2); cb += 16) {
    float vr[16], vi[16];
    tmem_ld16(lane_base + cb, vr);
    tmem_ld16(lane_base + TC_N + cb, vi);
    if (r < M && nchunks > 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int cc = col0 + cb + j;
        if (cc >= N) break;
        double2 v = make_double2(f32_to_f64(vr[j]), f32_to_f64(vi[j]));
        double2* out = d.C + (size_t)r * ldc + cc;
        if (!unit_alpha) v = cmul(d.alpha, v);
        if (!zero_beta) v = cadd(v, cmul(d.beta, *out));
        *out = v;
      }
    }
  }
}

// grid: x = column tile, y = row tile + tiles_m * instance, z = descriptor
__global__ void __launch_bounds__(TC_THREADS, 1) zgemm_tc_kernel(const GemmDesc* __restrict__ descs, int tiles_m,
                                                                  size_t stride, int* status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar[TC_STAGES];
  __shared__ uint32_t tmem_slot;
  const int inst = blockIdx.y / tiles_m, tm = blockIdx.y - inst * tiles_m;
  const GemmDesc& d = descs[blockIdx.z];
  const size_t io = (size_t)inst * stride;
  // tiles outside the descriptor's run-time size exit before touching TMEM
  {
    const int* dims = ish(d.dims, io);
    const int M = deval(d.M, dims), N = deval(d.N, dims);
    if (tm * TC_M >= M || (int)blockIdx.x * TC_N >= N || M <= 0 || N <= 0) return;
  }
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(smem_u32(&mbar[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  tc_tile(d, tm * TC_M, blockIdx.x * TC_N, io, ish(status, io), smem, tmem, smem_u32(&mbar[0]));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

bool tc_configured() {
  static const bool ok = [] {
    cudaError_t e = cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess;
  }();
  return ok;
}

}  // namespace

bool zgemm_tc_available() { return tc_configured(); }

void launch_zgemm_tc_batched(const Batch& bt, const GemmDesc* d_descs, int count, int max_m, int max_n, int* status,
                             cudaStream_t st) {
  if (count <= 0 || max_m <= 0 || max_n <= 0) return;
  const int tiles_m = (max_m + TC_M - 1) / TC_M;
  dim3 grid((max_n + TC_N - 1) / TC_N, tiles_m * bt.n, count);
  zgemm_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(d_descs, tiles_m, bt.stride, status);
  note_launch();
}

}  // namespace mpsk
