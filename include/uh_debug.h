/*
 * uh_debug.h - host-only checks of the device program (no CUDA call; for tests), and device
 * probes used by the benchmark.
 *
 * uh_create / h_create pack a product into a device program (work items, chunks, input runs and
 * their dependency flags, one item list per CTA of the persistent kernel) and check every
 * address the kernel will derive from it before anything is uploaded. These entry points run
 * the same validation, packing and check for a chosen number of CTAs without touching a GPU,
 * and return UH_OK, or UH_EINVAL with the first violation in uh_last_error().
 */
#ifndef UH_DEBUG_H
#define UH_DEBUG_H

#include "uh.h"

#ifdef __cplusplus
extern "C" {
#endif

int uh_pack_check(const uh_desc* desc, int32_t precision, int32_t ncta);
int h_pack_check(const h_desc* desc, int32_t precision, int32_t ncta);
int uh_batch_pack_check(const uh_desc* const* descs, int32_t count, int32_t precision, int32_t ncta);
int uh_batch_pack_check_ex(const uh_desc* const* descs, int32_t count, int32_t precision,
                           const uh_pack_params* params, int32_t ncta);
/* uh_pack_check with packing parameters (as uh_create_ex); ncta = SMs x params->ctas_per_sm. */
int uh_pack_check_ex(const uh_desc* desc, int32_t precision, const uh_pack_params* params, int32_t ncta);

/*
 * Runs one uh_matvec whose dependency waits look for an epoch that no chunk ever publishes, so
 * every such wait runs out after timeout_cycles (1e3 .. 4e9 SM cycles): the kernel records the
 * timeout in the op's status word, lets its copies in flight land and returns. y is then
 * undefined; uh_check reports UH_ETIMEOUT once, and later products of the op are unaffected.
 * For testing the bounded-wait path without hanging or faulting the GPU.
 */
int uh_debug_stalled_matvec(uh_op* op, const void* x, void* y, long long timeout_cycles, void* stream);

/*
 * Measures the FP64 fused multiply-add rate of the current device: one launch of 4 resident
 * CTAs per SM, each thread running 8 independent chains of `iters` dependent DFMAs (the
 * instruction mix of the complex128 product's inner loop, without its loads), timed with CUDA
 * events on `stream`; blocks until done. *tflops = 2 * FMAs / time / 1e12. The ceiling that the
 * complex128 product (8 flops per 16-byte element) is compared with. UH_EINVAL for
 * iters < 1000 or a null pointer, UH_ECUDA on a CUDA error.
 */
int uh_debug_dfma_rate(int32_t iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UH_DEBUG_H */
