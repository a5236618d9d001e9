/*
 * mpgb_server.h — continuous-batching decode server of the GB300 Matching
 * Pursuit library.
 *
 * The paper decodes one signal at a time against a dictionary shared by
 * encoder and decoder (Sec. 2; Sec. 4 notes that the dictionary is moved to
 * the device once and signals afterwards).  The server keeps several such
 * dictionaries resident and decodes requests for them as they arrive: each
 * dictionary gets a table of device decode slots, sized from an HBM budget,
 * and requests join the running batch between MP steps (Sec. 3, Eqs. 9-12)
 * while others are mid-decode.  Results are the same as a lone decode of the
 * request through mp_recover_batched with B = 1.
 */
#ifndef MPGB_SERVER_H
#define MPGB_SERVER_H

#include "mpgb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    long long submitted;       /* requests accepted by mp_server_submit               */
    long long rejected;        /* submits refused with MP_ERR_BUSY (queue full)       */
    long long admitted;        /* requests that got a device slot                     */
    long long completed;       /* requests whose result is ready                      */
    long long queued;          /* waiting for a slot now                              */
    long long active;          /* holding a slot now                                  */
    double latency_p50_s;      /* submit -> result ready, completed requests          */
    double latency_p99_s;
    double latency_mean_s;
    double latency_max_s;
    size_t hbm_bytes;          /* device memory the server's dictionaries use         */
    long long chunks;          /* step chunks launched (each: k steps + retire)       */
    long long retired;         /* results handed back by the retire step              */
} mp_server_stats;

/* Create a server on the current device.
 *  hbm_budget_bytes : device memory the dictionaries and their slot tables
 *                     may use (plans included); slots are sized from it.
 *  max_slots        : upper bound on decode slots per dictionary (>= 1).
 *  max_queue        : requests that may wait for a slot per dictionary;
 *                     a submit beyond it returns MP_ERR_BUSY.
 * Errors: MP_ERR_INVALID, MP_ERR_NOMEM. */
MPGB_API mp_status mp_server_create(mp_server_t* out, size_t hbm_budget_bytes, int max_slots, int max_queue);

/* Make a plan's dictionary resident for serving at `prec` (MP_PREC_BF16 or
 * MP_PREC_FP8E4M3; the plan must hold that copy).  The plan stays owned by
 * the caller and must outlive the server.  Only before the first submit.
 * With the plan's MP_OPT_BATCH_GRAM set (BF16, a period that is a multiple
 * of the 16 steps of a chunk) the dictionary is served in the Gram mode:
 * the plan's Gram matrix (4 M^2 bytes) is built here and counts against
 * the budget, and each slot keeps an FP32 correlation row (4 M bytes).
 *  dict_id : receives the id to submit against.
 * Errors: MP_ERR_INVALID, MP_ERR_UNSUPPORTED, MP_ERR_BUSY (HBM budget
 * exhausted), MP_ERR_NOMEM, MP_ERR_CUDA. */
MPGB_API mp_status mp_server_add_dictionary(mp_server_t srv, mp_plan_t plan, int prec, int* dict_id);

/* Number of decode slots the budget gave dictionary `dict_id`. */
MPGB_API mp_status mp_server_dictionary_slots(mp_server_t srv, int dict_id, int* slots);

/* Queue one request.  y_host (N floats of that dictionary) is copied before
 * the call returns.  *ticket identifies the request for mp_server_poll.
 * Thread-safe.  Errors: MP_ERR_INVALID, MP_ERR_NOT_FOUND (dictionary),
 * MP_ERR_BUSY (queue full), MP_ERR_NOMEM, MP_ERR_CUDA (the server hit a
 * CUDA error earlier). */
MPGB_API mp_status mp_server_submit(mp_server_t srv, int dict_id, const float* y_host, const mp_stop* stop,
                                    uint64_t* ticket);

/* MP_PENDING while the request runs; MP_OK once finished, after copying x~
 * (M floats) to x_host_out (may be NULL) and the result to *out (may be
 * NULL).  A ticket is released by the MP_OK poll.  Thread-safe.
 * Errors: MP_ERR_NOT_FOUND (unknown or released ticket), MP_ERR_CUDA. */
MPGB_API mp_status mp_server_poll(mp_server_t srv, uint64_t ticket, float* x_host_out, mp_result* out);

/* Counters and latency percentiles since creation or the last reset. */
MPGB_API mp_status mp_server_get_stats(mp_server_t srv, mp_server_stats* out);
MPGB_API mp_status mp_server_reset_stats(mp_server_t srv);

/* Stop the scheduler, wait for the device, free everything (tickets not yet
 * polled are dropped).  NULL is accepted. */
MPGB_API mp_status mp_server_destroy(mp_server_t srv);

#ifdef __cplusplus
}
#endif

#endif /* MPGB_SERVER_H */
