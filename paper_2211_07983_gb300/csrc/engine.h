// Host-side engine of libmps: state layout, device buffers and the three passes
// (forward gates, energy + cotangent, checkpointed reverse).  Internal header.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mps.h"
#include "kernels.h"
#include "mps_internal.h"

namespace mpsi {

using mpsk::DimExpr;
using mpsk::GemmDesc;

#define MPS_CU(call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return ::mpsi::fail(MPS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define MPS_TRY(expr)                  \
  do {                                 \
    mps_status s_ = (expr);            \
    if (s_ != MPS_OK) return s_;       \
  } while (0)

mps_status legacy_fence();

// Device memory of a state's instances: n copies of one address layout, `stride` bytes apart
// (instance i's copy of a byte at address a is at a + i*stride).  The layout grows on demand:
// alloc() hands out a zero-filled range in every copy, mapping physical memory as needed.
// Ranges are released only with the arena.
struct Arena {
  long long uid = 0;   // unique per arena (keys plans built against it)
  int n = 1, dev = 0;
  size_t stride = 0, gran = 0;
  uintptr_t base = 0;
  size_t used = 0, mapped = 0;   // per instance
  struct Mapping {
    uintptr_t at;
    size_t bytes;
    unsigned long long handle;
  };
  std::vector<Mapping> maps;
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena();
  mps_status init(int n_inst);
  mps_status alloc(size_t nbytes, void** out);
  mpsk::Batch batch() const { return mpsk::Batch{n, stride}; }

 private:
  mps_status grow(size_t need);
};

// Device allocation: owned (cudaMalloc) or, when `arena` is set, a per-instance range of that
// arena (released with the arena).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Arena* arena = nullptr;
  DevBuf() = default;
  explicit DevBuf(Arena* a) : arena(a) {}
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p && !arena) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  mps_status alloc(size_t nbytes);       // exact size, zero-filled
  mps_status ensure(size_t nbytes);      // grow-only
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// Bond-dimension caps and buffer offsets of an n-site MPS with bond cap D.
struct Layout {
  int n = 0, D = 0;
  std::vector<int> cap;          // cap[i], i = 0..n: bond left of site i
  std::vector<size_t> site_off;  // n+1 prefix offsets (complex elements)
  std::vector<size_t> lam_off;   // n+2 prefix offsets (doubles), slots 0..n
  int max_cap = 1;
  bool one_cta_svd = false;      // policy: never the cooperative SVD (mps_set_svd_policy)
  void build(int n_, int D_);
  size_t site_cap(int s) const { return site_off[s + 1] - site_off[s]; }
  size_t site_elems() const { return site_off[n]; }
  size_t lam_elems() const { return lam_off[n + 1]; }
};

// Device storage of one MPS (tensors, Schmidt vectors, bond dims), per instance.
struct StateBuf {
  DevBuf mem;
  double2* B = nullptr;
  double* lam = nullptr;
  int* dims = nullptr;
  explicit StateBuf(Arena* a = nullptr) : mem(a) {}
  mps_status alloc(const Layout& L);
  mps_status copy_from(const StateBuf& o, const Layout& L, cudaStream_t st);
};

struct Workspace;

}  // namespace mpsi

struct mps_state {
  long long uid = 0;     // unique per created state (keys the energy plan)
  mpsi::Layout L;
  mps_config cfg{};
  cudaStream_t st = nullptr;
  std::unique_ptr<mpsi::Arena> arena;   // declared first: released after every buffer below
  mpsi::StateBuf buf;
  mpsi::DevBuf status;   // one int per instance
  std::unique_ptr<mpsi::Workspace> ws;
  int n_inst() const { return arena->n; }
  mpsk::Batch batch() const { return arena->batch(); }
};

struct mps_circuit {
  long long uid = 0;      // unique per created circuit (keys captured graphs)
  int n = 0, n_gates = 0, max_theta_idx = -1;
  std::vector<mps_gate> host;
  mpsi::DevBuf gates;     // mps_gate array
  // theta index -> (gate, scale) CSR, built for every theta index < max_theta_idx+1
  mpsi::DevBuf csr_off, csr_gate, csr_scale;
};

namespace mpsi {
struct EnergyCache;
long long next_uid();
}

struct mps_hamiltonian_dev {
  long long uid = 0;      // unique per created Hamiltonian (keys captured graphs)
  int n = 0;
  double c0 = 0.0;                         // identity-string coefficient
  std::vector<uint64_t> x, z;              // canonical order, identity excluded
  std::vector<double> c;
  // sweep trie: nodes sorted by site; parent = -1 means the identity environment L^I_{site-1}
  std::vector<int> node_site, node_op, node_parent;
  std::vector<double> node_end_coeff;      // coefficient of the string ending at the node (or 0)
  std::vector<int> node_is_end;
  std::vector<int> term_node;              // leaf node of each term
  std::vector<int> site_begin;             // n+1
  std::vector<int> child_off, child_idx;   // children CSR
  mpsi::DevBuf d_coeff;
  std::unique_ptr<mpsi::EnergyCache> cache;
  ~mps_hamiltonian_dev();
};

