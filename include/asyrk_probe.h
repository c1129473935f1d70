/*
 * asyrk_probe.h -- measurement probes of libasyrk.so (not part of the method).
 *
 * Every thread keeps 8 independent operations in flight per loop trip.
 * They time, with CUDA events on the legacy default stream, the memory
 * operations the projection kernel is made of, so that its throughput can be
 * put against rates measured on the same GPU:
 *   ASYRK_PROBE_RED_F32    red.relaxed.gpu.global.add.f32 to uniformly random
 *                          elements of an n-element float array (L2-resident
 *                          for n * 4 B well below the L2 size);
 *   ASYRK_PROBE_GATHER_F32 ld.global.cg of uniformly random elements;
 *   ASYRK_PROBE_GATHER_RED gathers of 8 random elements, their sum, then a
 *                          red.add to each of the same 8 (the projection's
 *                          pattern); one operation = one gather + one red;
 *   ASYRK_PROBE_STREAM     16-byte streaming loads of an n-element float array
 *                          (HBM read bandwidth when n * 4 B exceeds the L2).
 * The probe allocates and frees its own array.  `ops` is the number of
 * operations (elements, for STREAM); *ms receives the kernel time.
 * Errors: EINVAL (unknown kind, n < 1, ops < 1), ENOMEM, ECUDA.
 */
#ifndef ASYRK_PROBE_H
#define ASYRK_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ASYRK_PROBE_RED_F32 = 0,
    ASYRK_PROBE_GATHER_F32 = 1,
    ASYRK_PROBE_GATHER_RED = 2,
    ASYRK_PROBE_STREAM = 3
};

int asyrk_probe(int kind, int64_t n, int64_t ops, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* ASYRK_PROBE_H */
