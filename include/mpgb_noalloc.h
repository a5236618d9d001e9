/*
 * mpgb_noalloc.h — allocation-free decode entry point of the GB300 Matching
 * Pursuit library.  The paper has no counterpart to this entry point: it
 * exists for callers that cannot allocate GPU memory.
 */
#ifndef MPGB_NOALLOC_H
#define MPGB_NOALLOC_H

#include "mpgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Decode one signal like mp_recover, without a plan and without allocating
 * anything: no cudaMalloc, cudaFree, pinned-host allocation or allocating
 * library call.  It is meant for callers that cannot allocate GPU memory,
 * for example code that must run inside a memory budget fixed by its host
 * application, a plugin that only receives buffers, or a loop that may not
 * call the allocator.
 *
 *  psi      : device pointer, 16-byte aligned, the dictionary atom-major:
 *             M rows of `ld` floats, row m holds psi_m in its first N
 *             entries and zeros in the remaining ld - N.  Caller-owned; the
 *             unit-norm precondition is the caller's to meet (no check).
 *  ld       : row stride in floats, >= N and a multiple of 4.
 *  y        : device pointer, N floats.
 *  x        : device pointer, M floats; receives x~.
 *  stop     : eps (finite, >= 0) and T (>= 0).
 *  trace    : optional per-iteration trace (device pointers), as for
 *             mp_recover; may be NULL.
 *  host_out : required; the call synchronises `stream` and fills it.
 *  stream   : a stream of the current device (NULL = legacy default stream).
 * With the dictionary stored at the stride a plan would use (N rounded up
 * to a multiple of 32, MP_Q_LD_FP32), the result equals mp_recover's bit
 * for bit; another stride changes the order of the FP32 sums.
 *
 * Scratch: the kernel's scratch (argmax key slots, grid-barrier counter,
 * error word, result record; 256 bytes at most, independent of N and M)
 * lives in a static device array inside the library, present on every GPU
 * that loads the library until the process exits.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress), so
 * make that first call before any stream capture.  With lazy module loading
 * that first call (or the first use of any entry point) also loads the
 * library's device code, and the driver allocates memory for that module;
 * a caller with a fixed memory budget should make the first call before it
 * fills the budget.  The looked-up address is kept per device and is not
 * valid after a cudaDeviceReset of that device.  Every call shares the
 * one array and the call clears it before its kernel starts: calls whose
 * work overlaps on the GPU (different streams, threads, or an unsynchronised
 * call in flight) race on it; serialise them.
 *
 * Errors: MP_ERR_INVALID (NULL pointers, ld, alignment, stop, a stream of
 * another device),
 * MP_ERR_UNSUPPORTED (N too large for the on-chip residual), MP_ERR_CUDA,
 * MP_ERR_TIMEOUT, MP_ERR_NONFINITE (non-finite y). */
MPGB_API mp_status mp_recover_noalloc(const float* psi, int N, int M, int ld, const float* y, float* x,
                                      const mp_stop* stop, const mp_trace* trace, mp_result* host_out,
                                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPGB_NOALLOC_H */
