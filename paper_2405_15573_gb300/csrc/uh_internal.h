// Internal declarations shared by the host side and the CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace uh {

// Records a message for uh_last_error() (calling thread) and returns `code`.
int set_error(int code, const char* fmt, ...);

}  // namespace uh
