// Arithmetic peak microbenchmarks of the GPU this library runs on (libpeaks.so, C ABI).
//
// The roofline denominators of the benchmark: the FP64 and FP32 FMA pipes (SIMT), the TF32
// tensor-core rate of the legacy warp-level mma.sync path, and the TF32 rate of the 5th-generation
// tensor cores (tcgen05.mma kind::tf32, 128 x 256 x 8 per instruction, accumulator in tensor
// memory, operands in shared memory).  Each kernel keeps every operand in
// registers (no memory traffic inside the timed loop), runs many independent accumulation chains
// per thread so that latency is hidden, and writes one value per thread at the end so that the
// compiler keeps the work.  The host side times a launch of one CTA wave over every SM with CUDA
// events after a warm-up launch and returns the rate in flop/s (an FMA counts 2 flops; an
// m16n8k8 TF32 mma counts 2*16*8*8).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int CHAINS = 8;

template <class T>
__global__ void fma_kernel(T* out, int iters, T a, T b) {
  T acc[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void mma_tf32_kernel(float* out, int iters, uint32_t av, uint32_t bv) {
  float d[CHAINS][4];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) d[c][q] = 0.f;
  const uint32_t a0 = av ^ threadIdx.x, a1 = av, a2 = av, a3 = av ^ 1u, b0 = bv, b1 = bv ^ threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// tcgen05: one thread per CTA issues `iters` MMAs of 128 x 256 x 8 (TF32, F32 accumulation) on
// operand tiles in shared memory (no-swizzle K-major layout: A 128 x 8 = 4 KB, B 256 x 8 = 8 KB),
// commits them to an mbarrier and waits (bounded), then reads one accumulator value.
__device__ __forceinline__ uint32_t pk_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t pk_desc(uint32_t addr) {
  // LBO 128 B (the two core matrices along K), SBO 256 B (8-row groups), fixed bits 46-48 = 0b001
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

__global__ void __launch_bounds__(128, 1) tc_tf32_kernel(float* out, int iters) {
  __shared__ __align__(1024) uint32_t opnd[(128 + 256) * 8];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  for (int i = threadIdx.x; i < (128 + 256) * 8; i += blockDim.x) opnd[i] = 0x3f800000u ^ (i & 1);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pk_smem(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(pk_smem(&tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  int ok = 1;
  if (threadIdx.x == 0) {
    const uint64_t a = pk_desc(pk_smem(opnd)), b = pk_desc(pk_smem(opnd + 128 * 8));
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
    for (int i = 0; i < iters; ++i) {
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(a), "l"(b), "r"(idesc), "r"(i > 0 ? 1 : 0));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(pk_smem(&mbar))
                 : "memory");
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
      uint32_t done;
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(pk_smem(&mbar))
          : "memory");
      if (done) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) {
        ok = 0;
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(tmem));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (threadIdx.x == 0) out[blockIdx.x] = ok ? __uint_as_float(r) : -1.f;
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

template <class K>
double time_launch(K launch, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms * 1e-3 / reps;
}

}  // namespace

extern "C" {

// out[0] = TF32 rate of tcgen05.mma (flop/s; one CTA per SM issuing back-to-back 128 x 256 x 8
// MMAs), out[1] = the accumulator value it read (a check that the MMAs ran: with A = B = ones-ish
// it is the sum over 8 x iters products).  Returns 0, or the CUDA error code.
int peaks_measure_tcgen05(double* out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float* buf = nullptr;
  if (cudaMalloc(&buf, sms * sizeof(float)) != cudaSuccess) return 2;
  const int iters = 20000;
  const double t = time_launch([&] { tc_tf32_kernel<<<sms, 128>>>(buf, iters); }, 3);
  float v = 0.f;
  cudaMemcpy(&v, buf, sizeof(float), cudaMemcpyDeviceToHost);
  out[0] = 2.0 * 128 * 256 * 8 * (double)iters * sms / t;
  out[1] = v;
  cudaFree(buf);
  return (int)cudaGetLastError();
}

// out[0] = FP64 FMA rate, out[1] = FP32 FMA rate, out[2] = TF32 mma.sync rate (flop/s),
// out[3] = SM count.  Returns 0, or the CUDA error code.
int peaks_measure(double* out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return 2;
  const int it64 = 2048, it32 = 8192, itm = 2048;
  const double t64 = time_launch([&] { fma_kernel<double><<<blocks, threads>>>((double*)buf, it64, 1.0000001, 1e-9); }, 5);
  const double t32 =
      time_launch([&] { fma_kernel<float><<<blocks, threads>>>((float*)buf, it32, 1.0000001f, 1e-9f); }, 5);
  const double tm = time_launch([&] { mma_tf32_kernel<<<blocks, threads>>>((float*)buf, itm, 0x3f800000u, 0x3f000000u); }, 5);
  const double nthr = (double)blocks * threads;
  out[0] = 2.0 * CHAINS * it64 * nthr / t64;
  out[1] = 2.0 * CHAINS * it32 * nthr / t32;
  out[2] = 2.0 * 16 * 8 * 8 * CHAINS * (double)itm * (nthr / 32.0) / tm;
  out[3] = sms;
  cudaFree(buf);
  return (int)cudaGetLastError();
}

}  // extern "C"
