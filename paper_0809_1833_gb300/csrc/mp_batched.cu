// Batched decode of B signals sharing one dictionary.
#include <cmath>
#include <cstring>
#include <vector>

#include "mp_internal.h"

namespace mpgb {

struct BatchEngine {};

void batch_destroy(BatchEngine* b) { delete b; }

}  // namespace mpgb

using namespace mpgb;

extern "C" {

mp_status mp_recover_batched(mp_plan_t plan, int prec, const float* Y, float* X, int B, const mp_stop* stops,
                             int n_stops, mp_result* host_out, void* stream) {
    clear_error();
    if (!plan || !Y || !X || !stops || !host_out) return fail(MP_ERR_INVALID, "mp_recover_batched: NULL argument");
    if (B < 0) return fail(MP_ERR_INVALID, "mp_recover_batched: B < 0");
    if (n_stops != 1 && n_stops != B) return fail(MP_ERR_INVALID, "mp_recover_batched: n_stops must be 1 or B");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_FP32 && prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_recover_batched: unknown precision");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_recover_batched: the plan holds no copy for this precision");
    if (prec != MP_PREC_FP32)
        return fail(MP_ERR_UNSUPPORTED, "mp_recover_batched: low-precision path not available");
    mp_status worst = MP_OK;
    for (int b = 0; b < B; ++b) {
        const mp_stop* sb = &stops[n_stops == 1 ? 0 : b];
        mp_status s = mp_recover(plan, Y + static_cast<size_t>(b) * p->N, X + static_cast<size_t>(b) * p->M, sb,
                                 nullptr, &host_out[b], stream);
        if (s < 0 && worst == MP_OK) worst = s;
    }
    return worst;
}

}  // extern "C"
