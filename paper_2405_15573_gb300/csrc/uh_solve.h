// FP64 vector kernels of the GMRES solves (uh_solve.cu). Vectors are complex128 unless named
// otherwise; a basis V holds cnt vectors of length n back to back. Each call launches on `s` and
// returns UH_OK or UH_ECUDA (launch error).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace uh {

// Blocks of the partial sums of dot products and norms for vectors of length n (<= 152).
int solve_partials(int64_t n);

int vec_d2f(const void* a, void* b, int64_t n, cudaStream_t s);  // complex128 -> complex64
int vec_f2d(const void* a, void* b, int64_t n, cudaStream_t s);  // complex64 -> complex128
// r = b - y (y complex64 if y_c64, else complex128).
int vec_residual(const void* b, const void* y, bool y_c64, void* r, int64_t n, cudaStream_t s);
// h[i] = sum_k conj(V_i[k]) w[k] for i < cnt (h[i] += ... if accumulate); part holds
// cnt * solve_partials(n) complex128 partial sums. cnt <= 64.
int vec_dots(const void* V, int64_t n, int cnt, const void* w, void* part, void* h, bool accumulate, cudaStream_t s);
// w[k] += sign * sum_{i < cnt} V_i[k] c[i]; c on the device, cnt <= 64.
int vec_combine(const void* V, int64_t n, int cnt, const void* c, double sign, void* w, cudaStream_t s);
// out[0] = ||w||_2, out[1] = 1 / out[0] (0 for a zero vector), both on the device; if hcol is not
// null, *hcol = out[0] as a complex128. part holds solve_partials(n) doubles.
int vec_norm(const void* w, int64_t n, void* part, double* out, void* hcol, cudaStream_t s);
// v = w * scale[1].
int vec_scale(const void* w, const double* scale, void* v, int64_t n, cudaStream_t s);
// v = w * scale[1] and v32 = complex64(v) (v32 may be null).
int vec_scale_f(const void* w, const double* scale, void* v, void* v32, int64_t n, cudaStream_t s);
// As vec_dots (no accumulation) with w given as complex64 y; also writes w = complex128(y).
int vec_dots_f(const void* V, int64_t n, int cnt, const void* y, void* w, void* part, void* h, cudaStream_t s);

}  // namespace uh
