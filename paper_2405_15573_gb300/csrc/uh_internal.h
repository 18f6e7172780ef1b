// Internal declarations shared by the host side and the CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace uh {

// Records a message for uh_last_error() (calling thread) and returns `code`.
int set_error(int code, const char* fmt, ...);

}  // namespace uh

struct uh_op;

namespace uh {

// Right-hand sides per pass of the op's CUDA-core multi-RHS product (uh_reserve), 0 if none.
int multi_rhs_width(const uh_op* op);
// y0 = A x0 and y1 = A x1 in one pass over the operator (complex64 vectors of n values anywhere in
// device memory, outputs disjoint from everything else); each result is bitwise that of uh_matvec.
// Needs multi_rhs_width(op) >= 2. Ordered with the op's other calls like uh_matvec.
int matvec_pair(uh_op* op, const void* x0, const void* x1, void* y0, void* y1, void* stream);

}  // namespace uh
