/*
 * uh_debug.h - host-only checks of the device program (no CUDA call; for tests).
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

/*
 * Runs one uh_matvec whose dependency waits look for an epoch that no chunk ever publishes, so
 * every such wait runs out after timeout_cycles (1e3 .. 4e9 SM cycles): the kernel records the
 * timeout in the op's status word, lets its copies in flight land and returns. y is then
 * undefined; uh_check reports UH_ETIMEOUT once, and later products of the op are unaffected.
 * For testing the bounded-wait path without hanging or faulting the GPU.
 */
int uh_debug_stalled_matvec(uh_op* op, const void* x, void* y, long long timeout_cycles, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UH_DEBUG_H */
