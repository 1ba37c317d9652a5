// Replicated device memory for the instances of a batched state (see Arena in engine.h).
//
// One virtual address range holds n copies of a layout that grows on demand; physical memory is
// mapped into every copy of a range when the layout reaches it.  The driver's virtual-memory
// calls are looked up through the runtime (cudaGetDriverEntryPointByVersion), so the library
// does not link the driver library itself.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "engine.h"

namespace mpsi {

namespace {

using PfnReserve = CUresult (*)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long);
using PfnFree = CUresult (*)(CUdeviceptr, size_t);
using PfnCreate = CUresult (*)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*,
                               unsigned long long);
using PfnRelease = CUresult (*)(CUmemGenericAllocationHandle);
using PfnMap = CUresult (*)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long);
using PfnUnmap = CUresult (*)(CUdeviceptr, size_t);
using PfnSetAccess = CUresult (*)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t);
using PfnGranularity = CUresult (*)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags);

struct Vmm {
  PfnReserve reserve = nullptr;
  PfnFree free = nullptr;
  PfnCreate create = nullptr;
  PfnRelease release = nullptr;
  PfnMap map = nullptr;
  PfnUnmap unmap = nullptr;
  PfnSetAccess set_access = nullptr;
  PfnGranularity granularity = nullptr;
  bool ok = false;
  std::string err;
};

template <class F>
bool lookup(const char* name, F* out, std::string* err) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    *err = std::string("driver entry point ") + name + " is unavailable";
    return false;
  }
  *out = reinterpret_cast<F>(fn);
  return true;
}

const Vmm& vmm() {
  static Vmm v;
  static std::once_flag once;
  std::call_once(once, [] {
    v.ok = lookup("cuMemAddressReserve", &v.reserve, &v.err) && lookup("cuMemAddressFree", &v.free, &v.err) &&
           lookup("cuMemCreate", &v.create, &v.err) && lookup("cuMemRelease", &v.release, &v.err) &&
           lookup("cuMemMap", &v.map, &v.err) && lookup("cuMemUnmap", &v.unmap, &v.err) &&
           lookup("cuMemSetAccess", &v.set_access, &v.err) &&
           lookup("cuMemGetAllocationGranularity", &v.granularity, &v.err);
  });
  return v;
}

CUmemAllocationProp device_prop(int dev) {
  CUmemAllocationProp prop{};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = dev;
  return prop;
}

size_t round_up(size_t x, size_t g) { return (x + g - 1) / g * g; }

constexpr size_t kChunk = size_t(64) << 20;   // physical growth step per instance

}  // namespace

mps_status Arena::init(int n_inst) {
  const Vmm& v = vmm();
  if (!v.ok) return fail(MPS_ECUDA, "device memory arena: " + v.err);
  if (n_inst < 1) return fail(MPS_EINVAL, "device memory arena: n_inst < 1");
  MPS_CU(cudaGetDevice(&dev));
  uid = next_uid();
  const CUmemAllocationProp prop = device_prop(dev);
  if (v.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || gran == 0)
    return fail(MPS_ECUDA, "device memory arena: cuMemGetAllocationGranularity failed");
  size_t fr = 0, tot = 0;
  MPS_CU(cudaMemGetInfo(&fr, &tot));
  n = n_inst;
  // One instance can never use more than the whole device, so its copy of the layout reserves
  // that much address space (address space only; nothing is committed).  Smaller strides are
  // tried if the reservation is refused.
  for (size_t want = round_up(tot, gran); want >= (size_t(1) << 30); want = round_up(want / 2, gran)) {
    CUdeviceptr p = 0;
    if (v.reserve(&p, want * (size_t)n, gran, 0, 0) == CUDA_SUCCESS) {
      base = (uintptr_t)p;
      stride = want;
      return MPS_OK;
    }
  }
  return fail(MPS_ENOMEM, "device memory arena: cannot reserve address space for " + std::to_string(n) +
                              " instances");
}

mps_status Arena::grow(size_t need) {
  const Vmm& v = vmm();
  const size_t add = round_up(need - mapped, kChunk);
  if (mapped + add > stride) return fail(MPS_ENOMEM, "device memory arena: instance layout exceeds its stride");
  const CUmemAllocationProp prop = device_prop(dev);
  CUmemAccessDesc acc{};
  acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  acc.location.id = dev;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  for (int i = 0; i < n; ++i) {
    const CUdeviceptr at = (CUdeviceptr)(base + (size_t)i * stride + mapped);
    CUmemGenericAllocationHandle h = 0;
    if (v.create(&h, add, &prop, 0) != CUDA_SUCCESS)
      return fail(MPS_ENOMEM, "device memory arena: cuMemCreate(" + std::to_string(add) + " bytes) failed");
    if (v.map(at, add, 0, h, 0) != CUDA_SUCCESS) {
      v.release(h);
      return fail(MPS_ECUDA, "device memory arena: cuMemMap failed");
    }
    maps.push_back({(uintptr_t)at, add, (unsigned long long)h});
    if (v.set_access(at, add, &acc, 1) != CUDA_SUCCESS) return fail(MPS_ECUDA, "device memory arena: cuMemSetAccess failed");
  }
  mapped += add;
  return MPS_OK;
}

mps_status Arena::alloc(size_t nbytes, void** out) {
  const size_t off = round_up(used, 256);
  const size_t end = off + round_up(nbytes == 0 ? 16 : nbytes, 256);
  if (end > mapped) MPS_TRY(grow(end));
  used = end;
  // zero every instance's copy (the legacy stream, then the fence)
  for (int i = 0; i < n; ++i) MPS_CU(cudaMemsetAsync((void*)(base + (size_t)i * stride + off), 0, end - off, 0));
  MPS_TRY(legacy_fence());
  *out = (void*)(base + off);
  return MPS_OK;
}

Arena::~Arena() {
  const Vmm& v = vmm();
  if (!base) return;   // the owner has synchronised its stream: no kernel uses the ranges
  for (const Mapping& m : maps) {
    v.unmap((CUdeviceptr)m.at, m.bytes);
    v.release((CUmemGenericAllocationHandle)m.handle);
  }
  v.free((CUdeviceptr)base, stride * (size_t)n);
}

}  // namespace mpsi
