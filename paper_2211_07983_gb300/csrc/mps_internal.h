// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>

#include "../../include/mps.h"

namespace mpsi {

// Records the thread-local error text and returns the status (for `return fail(...)`).
mps_status fail(mps_status st, const std::string& msg);
void clear_error();

// Where a caller's pointer lives: PTR_HOST (host memory, registered or not), PTR_DEVICE (device
// or managed memory usable by the current device), PTR_OTHER_DEVICE (device memory of another
// GPU, which the library's kernels on the current device must not be given).
enum PtrLocation { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
PtrLocation ptr_location(const void* p);

}  // namespace mpsi
