// Device-side helpers shared by the kernels of libmps (FP64 complex path).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mpsk {

// ---- complex double ---------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
// a * conj(b)
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// ---- instance batching ------------------------------------------------------------------------
// A state may hold n instances (independent evaluations of the same circuit shape).  They are
// replicas of one address layout, `stride` bytes apart: instance i's copy of any per-instance
// byte sits i*stride bytes after instance 0's.  Every kernel takes its instance from one grid
// dimension and shifts each per-instance pointer by i*stride, both its arguments and the
// pointers it reads from descriptor tables.  Shared read-only tables (the gate list, Hamiltonian
// coefficients, offset tables, the descriptor tables themselves) are not shifted.
struct Batch {
  int n;           // instances per launch
  size_t stride;   // bytes between instances
};

template <class T>
__host__ __device__ __forceinline__ T* ish(T* p, size_t off) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + off) : p;
}

// ---- device status word -----------------------------------------------------------------
// First error wins; the host reads it after the stream work of a call completes.
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---- dimension expressions ----------------------------------------------------------------
// value = add + mul * dims[idx]  (idx < 0: just `add`).  Bond dimensions live on the device, so
// every contraction reads its sizes at run time and no host synchronisation is needed when a
// truncation changes a bond dimension.
struct DimExpr {
  int32_t add;
  int16_t mul;
  int16_t idx;
};

__host__ __device__ __forceinline__ DimExpr dconst(int v) { return DimExpr{v, 0, -1}; }
__host__ __device__ __forceinline__ DimExpr dref(int idx, int mul = 1, int add = 0) {
  return DimExpr{add, (int16_t)mul, (int16_t)idx};
}
__device__ __forceinline__ int deval(DimExpr e, const int* dims) {
  return e.idx < 0 ? e.add : e.add + e.mul * dims[e.idx];
}

enum Op : int { OP_N = 0, OP_T = 1, OP_H = 2, OP_C = 3 };

// C[M x N] = alpha * op(A) * op(B) + beta * C, row-major with leading dimensions.
// op(A) is M x K: N -> A[i*lda+k], T -> A[k*lda+i], H -> conj(A[k*lda+i]), C -> conj(A[i*lda+k]).
struct GemmDesc {
  const double2* A;
  const double2* B;
  double2* C;
  const int* dims;
  DimExpr M, N, K, lda, ldb, ldc;
  int32_t opA, opB;
  double2 alpha, beta;
};

}  // namespace mpsk
