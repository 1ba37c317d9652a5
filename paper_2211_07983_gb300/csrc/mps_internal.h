// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>

#include "../../include/mps.h"

namespace mpsi {

// Records the thread-local error text and returns the status (for `return fail(...)`).
mps_status fail(mps_status st, const std::string& msg);
void clear_error();

}  // namespace mpsi
