// api_internal.h -- helpers the C ABI's source files share (not exported):
// the per-thread error message and the checks of a matrix descriptor.
#pragma once
#include "../../include/sfhe.h"

namespace sfhe {

// records a formatted message for sfhe_last_error() and returns st
sfhe_status set_error(sfhe_status st, const char* fmt, ...);
// shape, encoding and structure arrays of a descriptor (host side only)
sfhe_status validate_view(const sfhe_matrix_view& m, const char* name);
// the device the context was created on
int ctx_device(const sfhe_ctx* c);

}  // namespace sfhe
