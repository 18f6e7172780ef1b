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
// ys[r] = A xs[r] for r < nr (2 or 4) in one pass over the operator (complex64 vectors of n values
// anywhere in device memory, outputs disjoint from everything else); each result is bitwise that
// of uh_matvec. Needs multi_rhs_width(op) >= nr. Ordered with the op's other calls like uh_matvec.
int matvec_group(uh_op* op, int nr, const void* const* xs, void* const* ys, void* stream);

}  // namespace uh
