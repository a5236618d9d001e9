// One decode with the atoms split across devices (ranks): each rank's plan
// holds a contiguous shard of Psi, atoms [atom_offset, atom_offset + M).
// Per MP iteration (Sec. 3, Eqs. 9-12):
//   local  : c = <r, psi_m> for the shard's atoms, the shard's best packed
//            key (|c|, ~global index, sign), and a record carrying that key
//            and the atom's FP32 row                       (mp_shard_step_local)
//   gather : the caller all-gathers the records of every rank (one exchange
//            per iteration: 16 + 4 ldN bytes per rank)
//   apply  : every rank picks the largest key (ties to the smallest global
//            index, as Sec. 4), updates its copy of r with the winner's
//            row, the FP64 energy and the stop test; the owner adds c to its
//            x~ slice                                       (mp_shard_step_apply)
// Every rank applies the same arithmetic to the same r, so the copies stay
// bit-identical; the correlation and energy orders are those of the
// persistent kernel, so one shard reproduces mp_recover bit for bit.
#include <cmath>
#include <cstring>

#include "mp_device.cuh"
#include "mp_dot.cuh"
#include "mp_internal.h"

namespace mpgb {

constexpr int kShardThreads = 256;
constexpr int kShardChains = 128;     // FP64 energy: the persistent kernel's 128 chains

struct ShardRecordHead {
    unsigned long long key;           // packed (|c|, ~global atom, sign); 0 = none
    int atom;                         // global atom index (-1 = none)
    float coef;
};
static_assert(sizeof(ShardRecordHead) == 16, "record head is 16 bytes");

// c for every local atom, one warp per 4 atoms at a time (the persistent
// kernel's dot4/dot1 orders), folded into one global atomic max key.
__global__ void __launch_bounds__(kShardThreads) shard_best_kernel(const float* __restrict__ psi, int M, int ldN,
                                                                    int offset, const float* __restrict__ r,
                                                                    unsigned long long* key) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long best = 0ull;
    for (int j = 4 * gw; j < M; j += 4 * nw) {
        const float* p = psi + static_cast<size_t>(j) * ldN;
        if (j + 4 <= M) {
            float c[4];
            dot4(p, r, ldN, lane, c);
#pragma unroll
            for (int i = 0; i < 4; ++i) best = umax64(best, pack_key(c[i], offset + j + i));
        } else {
            for (int q = j; q < M; ++q)
                best = umax64(best, pack_key(dot1(psi + static_cast<size_t>(q) * ldN, r, ldN, lane), offset + q));
        }
    }
    __shared__ unsigned long long wk[kShardThreads / 32];
    if (lane == 0) wk[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0ull;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) b = umax64(b, wk[w]);
        if (b) atomicMax(key, b);
    }
}

// Complete the record: the winner's global index, coefficient and FP32 row.
__global__ void __launch_bounds__(kShardThreads) shard_fill_kernel(const float* __restrict__ psi, int ldN, int offset,
                                                                    unsigned char* rec) {
    ShardRecordHead* h = reinterpret_cast<ShardRecordHead*>(rec);
    float* row = reinterpret_cast<float*>(rec + sizeof(ShardRecordHead));
    const unsigned long long k = h->key;
    const int m = k ? key_index(k) : -1;
    if (threadIdx.x == 0) {
        h->atom = m;
        h->coef = k ? key_coef(k) : 0.f;
    }
    const float4* src = m >= 0 ? reinterpret_cast<const float4*>(psi + static_cast<size_t>(m - offset) * ldN) : nullptr;
    float4* dst = reinterpret_cast<float4*>(row);
    for (int i = threadIdx.x; i < ldN / 4; i += blockDim.x)
        dst[i] = src ? __ldg(src + i) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// r <- y (zero padded), x~ slice <- 0, e0 and the stop state.
__global__ void __launch_bounds__(kShardThreads) shard_init_kernel(const float* __restrict__ y, int N, int ldN,
                                                                    float* r, float* x, int M, double eps2, int T,
                                                                    mp_shard_state* s) {
    __shared__ double ws[kShardThreads / 32];
    for (int i = threadIdx.x; i < ldN; i += blockDim.x) r[i] = i < N ? y[i] : 0.f;
    for (int i = threadIdx.x; i < M; i += blockDim.x) x[i] = 0.f;
    __syncthreads();
    const float4* r4 = reinterpret_cast<const float4*>(r);
    double acc = 0.0;
    if (threadIdx.x < kShardChains)
        for (int k = threadIdx.x; k < ldN / 4; k += kShardChains) {
            const float4 v = r4[k];
            acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
            acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
            acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
            acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
        }
    acc = warp_sum_f64(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < kShardChains / 32; ++w) e += ws[w];
        s->e0 = e;
        s->e = e;
        s->thr2 = eps2 * e;
        s->audit = 0.0;
        s->t = 0;
        s->T = T;
        s->status = isfinite(e) ? MP_OK : MP_ERR_NONFINITE;
        s->stopped = !(isfinite(e) && e > s->thr2 && T > 0);
        s->stop_reason = e == 0.0 ? MP_STOP_ZERO_Y : (e <= s->thr2 ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS);
    }
}

// Pick the winner among n records, update r, the energy and the state; the
// owner of the atom adds c to its x~ slice.  One CTA; a no-op once stopped.
__global__ void __launch_bounds__(kShardThreads) shard_apply_kernel(const unsigned char* __restrict__ recs, int n,
                                                                     size_t rec_bytes, int offset, int M, int ldN,
                                                                     float* r, float* x, mp_shard_state* s,
                                                                     int* trace_atoms, float* trace_coefs,
                                                                     int trace_cap) {
    __shared__ double ws[kShardThreads / 32];
    __shared__ int win;
    if (s->stopped) return;
    if (threadIdx.x == 0) {
        unsigned long long b = 0ull;
        int w = -1;
        for (int i = 0; i < n; ++i) {
            const unsigned long long k = reinterpret_cast<const ShardRecordHead*>(recs + i * rec_bytes)->key;
            if (k > b) {
                b = k;
                w = i;
            }
        }
        win = w;
    }
    __syncthreads();
    if (win < 0) {   // no candidate anywhere: nothing can be selected
        if (threadIdx.x == 0) {
            s->status = MP_ERR_INVALID;
            s->stopped = 1;
        }
        return;
    }
    const ShardRecordHead* h = reinterpret_cast<const ShardRecordHead*>(recs + win * rec_bytes);
    const float4* p4 = reinterpret_cast<const float4*>(recs + win * rec_bytes + sizeof(ShardRecordHead));
    const float c = h->coef;
    const int m = h->atom;
    float4* r4 = reinterpret_cast<float4*>(r);
    for (int k = threadIdx.x; k < ldN / 4; k += blockDim.x) {
        const float4 p = p4[k];
        float4 v = r4[k];
        v.x = fmaf(-c, p.x, v.x);
        v.y = fmaf(-c, p.y, v.y);
        v.z = fmaf(-c, p.z, v.z);
        v.w = fmaf(-c, p.w, v.w);
        r4[k] = v;
    }
    __syncthreads();
    double acc = 0.0;
    if (threadIdx.x < kShardChains)
        for (int k = threadIdx.x; k < ldN / 4; k += kShardChains) {
            const float4 v = r4[k];
            acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
            acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
            acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
            acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
        }
    acc = warp_sum_f64(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < kShardChains / 32; ++w) e += ws[w];
        if (m >= offset && m < offset + M) x[m - offset] += c;   // Eq. 10 on the owner
        const int t = s->t;
        if (t < trace_cap) {
            if (trace_atoms) trace_atoms[t] = m;
            if (trace_coefs) trace_coefs[t] = c;
        }
        const double cc = static_cast<double>(c);
        s->audit = fmax(s->audit, fabs(e - (s->e - cc * cc)) / s->e0);
        s->e = e;
        s->t = t + 1;   // Eq. 12
        if (!(e > s->thr2 && s->t < s->T)) {
            s->stopped = 1;
            s->stop_reason = e <= s->thr2 ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS;
        }
    }
}

static size_t record_bytes(const PlanImpl* p) {
    return sizeof(ShardRecordHead) + static_cast<size_t>(p->ldN) * sizeof(float);
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

size_t mp_shard_record_bytes(mp_plan_t plan) { return plan ? record_bytes(&plan->impl) : 0; }

mp_status mp_shard_init(mp_plan_t plan, const float* y, float* r, float* x, const mp_stop* stop,
                        mp_shard_state* state, void* stream) {
    clear_error();
    if (!plan || !y || !r || !x || !stop || !state) return fail(MP_ERR_INVALID, "mp_shard_init: NULL argument");
    if (!(stop->eps >= 0.0) || !std::isfinite(stop->eps) || stop->max_iters < 0 || stop->reserved)
        return fail(MP_ERR_INVALID, "mp_shard_init: bad stop");
    PlanImpl* p = &plan->impl;
    shard_init_kernel<<<1, kShardThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        y, p->N, p->ldN, r, x, p->M, stop->eps * stop->eps, stop->max_iters, state);
    MP_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return MP_OK;
}

mp_status mp_shard_step_local(mp_plan_t plan, int atom_offset, const float* r, void* record, void* stream) {
    clear_error();
    if (!plan || !r || !record) return fail(MP_ERR_INVALID, "mp_shard_step_local: NULL argument");
    if (atom_offset < 0) return fail(MP_ERR_INVALID, "mp_shard_step_local: atom_offset < 0");
    PlanImpl* p = &plan->impl;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* rec = static_cast<unsigned char*>(record);
    MP_CUDA_TRY(cudaMemsetAsync(rec, 0, sizeof(unsigned long long), st));
    const int warps_needed = (p->M + 3) / 4;
    const int blocks = std::max(1, std::min(4 * p->sm_count, (warps_needed + kShardThreads / 32 - 1) / (kShardThreads / 32)));
    shard_best_kernel<<<blocks, kShardThreads, 0, st>>>(p->psi32, p->M, p->ldN, atom_offset, r,
                                                         reinterpret_cast<unsigned long long*>(rec));
    MP_CUDA_TRY(cudaGetLastError());
    shard_fill_kernel<<<1, kShardThreads, 0, st>>>(p->psi32, p->ldN, atom_offset, rec);
    MP_CUDA_TRY(cudaGetLastError());
    p->launches += 2;
    return MP_OK;
}

mp_status mp_shard_step_apply(mp_plan_t plan, int atom_offset, const void* records, int n_records, float* r,
                              float* x, mp_shard_state* state, const mp_trace* trace, void* stream) {
    clear_error();
    if (!plan || !records || !r || !x || !state || n_records < 1)
        return fail(MP_ERR_INVALID, "mp_shard_step_apply: NULL argument or n_records < 1");
    PlanImpl* p = &plan->impl;
    shard_apply_kernel<<<1, kShardThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const unsigned char*>(records), n_records, record_bytes(p), atom_offset, p->M, p->ldN, r, x,
        state, trace ? trace->atoms : nullptr, trace ? trace->coefs : nullptr, trace ? trace->capacity : 0);
    MP_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return MP_OK;
}

}  // extern "C"
