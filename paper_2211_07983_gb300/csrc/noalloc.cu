// The gate SVD for callers that must not allocate device memory (see mps_svd_noalloc in
// include/mps.h).  Its scratch is one file-scope __device__ array of fixed size that every GPU
// loading the library keeps until the process exits; nothing here calls cudaMalloc, cudaFree or
// any other allocating routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mps.h"
#include "kernels.h"
#include "mps_internal.h"

using namespace mpsk;

namespace {

constexpr int NA_MAX = 128;                                     // largest m and ncol accepted
constexpr size_t NA_SQ = (size_t)NA_MAX * NA_MAX;
// layout in complex doubles: A column-major | SVD work (K^2 + R K <= 2 MAX^2) | V | W |
// then doubles s, lambda, ones and the ints dims[3], status
constexpr size_t NA_A = 0, NA_WORK = NA_SQ, NA_V = 3 * NA_SQ, NA_W = 4 * NA_SQ, NA_CPLX = 5 * NA_SQ;
constexpr size_t NA_BYTES = NA_CPLX * sizeof(double2) + 3 * NA_MAX * sizeof(double) + 256;

__device__ __align__(256) unsigned char g_svd_scratch[NA_BYTES];

std::mutex g_mu;
void* g_base[128] = {};   // device address of g_svd_scratch, per device ordinal

struct View {
  double2* A;
  double2* work;
  double2* V;
  double2* W;
  double* s;
  double* lam;
  double* ones;
  int* dims;
  int* status;
};

View view_of(void* base) {
  char* p = static_cast<char*>(base);
  View v;
  v.A = reinterpret_cast<double2*>(p) + NA_A;
  v.work = reinterpret_cast<double2*>(p) + NA_WORK;
  v.V = reinterpret_cast<double2*>(p) + NA_V;
  v.W = reinterpret_cast<double2*>(p) + NA_W;
  double* d = reinterpret_cast<double*>(p + NA_CPLX * sizeof(double2));
  v.s = d;
  v.lam = d + NA_MAX;
  v.ones = d + 2 * NA_MAX;
  v.dims = reinterpret_cast<int*>(d + 3 * NA_MAX);
  v.status = v.dims + 4;
  return v;
}

// First call on a device: resolve the array's device address with that device current.
mps_status scratch_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mpsi::fail(MPS_ECUDA, std::string("mps_svd_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess || !p)
      return mpsi::fail(MPS_ECUDA, std::string("mps_svd_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return MPS_OK;
}

// device (or managed) memory that the current device may use; memory of another GPU is refused
bool on_device(const void* p) { return mpsi::ptr_location(p) == mpsi::PTR_DEVICE; }

// row-major input -> column-major working copy; dims, lambda_left = 1, status = 0
__global__ void na_prepare(const double2* __restrict__ A, int m, int n, View v) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m * n) {
    const int r = t / n, c = t % n;
    v.A[(size_t)c * m + r] = A[t];
  }
  if (t < m / 2) v.ones[t] = 1.0;
  if (t == 0) {
    v.dims[0] = m / 2;
    v.dims[1] = 1;
    v.dims[2] = n / 2;
    *v.status = 0;
  }
}

// column-major V (K columns of length n) and W (K columns of length m) -> row-major outputs
__global__ void na_finish(View v, int m, int n, double* s_out, double2* V_out, double2* W_out, int* k_out) {
  const int K = m < n ? m : n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * K) {
    const int r = t / K, j = t % K;
    V_out[t] = v.V[(size_t)j * n + r];
  }
  if (t < m * K) {
    const int r = t / K, j = t % K;
    W_out[t] = v.W[(size_t)j * m + r];
  }
  if (t < K) s_out[t] = v.s[t];
  if (t == 0) *k_out = v.dims[1];
}

}  // namespace

extern "C" mps_status mps_svd_noalloc(int32_t m, int32_t ncol, const double* A, int32_t D, double eps,
                                      double* s_out, double* V_out, double* W_out, int32_t* k_out,
                                      void* cuda_stream) {
  mpsi::clear_error();
  if (!A || !s_out || !V_out || !W_out || !k_out) return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: NULL argument");
  if (m < 2 || ncol < 2 || (m & 1) || (ncol & 1))
    return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: m and ncol must be even and >= 2");
  if (m > NA_MAX || ncol > NA_MAX)
    return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: m and ncol must not exceed " + std::to_string(NA_MAX) +
                                      " (size of the library's fixed scratch array)");
  if (D < 1 || !(eps >= 0.0)) return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: bad D or eps");
  if (!on_device(A) || !on_device(s_out) || !on_device(V_out) || !on_device(W_out) || !on_device(k_out))
    return mpsi::fail(MPS_EINVAL, "mps_svd_noalloc: every array must be device memory of the current device");
  void* base = nullptr;
  mps_status st = scratch_base(&base);
  if (st != MPS_OK) return st;
  const View v = view_of(base);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int total = m * ncol;
  na_prepare<<<(total + 255) / 256, 256, 0, stream>>>(reinterpret_cast<const double2*>(A), m, ncol, v);
  SvdArgs a{};
  a.A = v.A;
  a.scratch = v.work;   // used only when shared memory cannot hold the working matrices
  a.dims = v.dims;
  a.b = 0;
  a.D = D;
  a.eps = eps;
  a.Vs = v.V;
  a.s = v.s;
  a.lam_out = v.lam;
  a.W = v.W;
  a.tape_dims = nullptr;
  a.lam_left = v.ones;
  a.lam_left_copy = nullptr;
  a.status = v.status;
  a.stats = nullptr;
  launch_svd(Batch{1, 0}, a, m, ncol, stream);
  const int K = m < ncol ? m : ncol;
  const int outs = (ncol > m ? ncol : m) * K;
  na_finish<<<(outs + 255) / 256, 256, 0, stream>>>(v, m, ncol, s_out, reinterpret_cast<double2*>(V_out),
                                                    reinterpret_cast<double2*>(W_out), k_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mpsi::fail(MPS_ECUDA, std::string("mps_svd_noalloc: launch: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return mpsi::fail(MPS_ECUDA, std::string("mps_svd_noalloc: ") + cudaGetErrorString(e));
  int code = 0;
  e = cudaMemcpy(&code, v.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return mpsi::fail(MPS_ECUDA, std::string("mps_svd_noalloc: ") + cudaGetErrorString(e));
  if (code != 0) return mpsi::fail((mps_status)code, "mps_svd_noalloc: the SVD reported a device-side error");
  return MPS_OK;
}
