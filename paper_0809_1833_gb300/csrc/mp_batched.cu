// Batched Matching Pursuit: B signals share one dictionary (Sec. 2), and
// each step performs one MP iteration (Sec. 3, Eqs. 9-12) for every signal
// that is still active.
//
// One step is two kernels:
//   corr_top8   (mp_corr.cu) C = Rq * Psiq^T on the tensor cores; per signal
//               and per atom tile the 8 largest |c| (FP8: times the atom scale).
//   select      per signal: merge the sorted per-tile candidate lists into the
//               top 8, rescore those atoms in FP32 from the FP32 atoms
//               (<r, psi_m>, Eq. 9), commit the best (ties to the smallest
//               index): x~_m += c (Eq. 10), r -= c psi_m in FP32 (Eq. 11),
//               e = sum r^2 in FP64, t += 1 (Eq. 12), stop test; a signal
//               that runs on takes the next row of the other half of the
//               double-buffered GEMM operand (one atomic) and writes its
//               requantised residual there, so the next step's rows are
//               compact.  A signal's arithmetic does not depend on its row,
//               so results are the same alone, in any batch and in any row
//               order.
// After an admission, fixup (one CTA) drops the newly admitted signals that
// need no iteration, filling their rows from the tail.
// Signals stop independently; the steps are captured in a CUDA graph and
// replayed until no signal is active.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mp_batch.cuh"
#include "mp_device.cuh"
#include "mp_dot.cuh"
#include "mp_internal.h"

namespace mpgb {

constexpr int kSelThreads = 256;
// select/update: one CTA per signal (8 warps, or 4 in engines of 512 slots
// and more; see launch_step).  The FP64
// energy always runs in the persistent kernel's order (128 chains over
// float4s, then warp sums in warp order), so energies and stop decisions
// equal the plain decode's bit for bit whenever the selected atoms do.
constexpr int kSumChains = 128;
constexpr int kWideSelectCap = 512;   // engines with fewer slots run the 8-warp select
constexpr int kFixThreads = 1024;
constexpr int kStepsPerGraph = 16;   // even: every graph starts and ends on operand half 0

// ------------------------------------------------------------------ block helpers
// The FP64 sum of the energy chains (threads 0..kSumChains-1; the other
// threads hold zeros): warp butterflies, then the chain warps' sums in warp
// order (adding the other warps' +0.0 would not change a bit, and FP64 adds
// are slow on this part, so they are left out).
MP_DEV double block_sum_f64(double v, double* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum_f64(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < kSumChains / 32; ++w) s += red[w];
    return s;
}
MP_DEV float block_max_f32(float v, float* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    return m;
}
// Exclusive prefix of `flag` over the block's threads in thread order;
// *total receives the block sum.  red: 32 ints.
MP_DEV int block_scan_flag(int flag, int* red, int* total) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(b & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) red[warp] = __popc(b);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
        if (w < warp) before += red[w];
        tot += red[w];
    }
    *total = tot;
    return before + in_warp;
}

// Exclusive block scan of small non-negative counts (their total < 2^31).
MP_DEV int block_scan_count(int v, int* red, int* total) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = x;
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
        if (w < warp) before += red[w];
        tot += red[w];
    }
    *total = tot;
    return before + x - v;
}

// Quantise one residual row (ldN floats) into a GEMM operand row of ldq
// elements (BF16) or bytes (E4M3, per-row scale max|r| / 448).  Whole block.
// Returns the row scale (1 for BF16).
MP_DEV float block_quantize(const float* r, int ldN, void* dst, int ldq, int fp8, float* red) {
    if (!fp8) {
        __nv_bfloat16* q = static_cast<__nv_bfloat16*>(dst);
        for (int n = threadIdx.x; n < ldq; n += blockDim.x) q[n] = __float2bfloat16_rn(n < ldN ? r[n] : 0.f);
        return 1.f;
    }
    float mx = 0.f;
    for (int n = threadIdx.x; n < ldN; n += blockDim.x) mx = fmaxf(mx, fabsf(r[n]));
    const float amax = block_max_f32(mx, red);
    const float inv = amax > 0.f ? 448.f / amax : 1.f;
    __nv_fp8_storage_t* q = static_cast<__nv_fp8_storage_t*>(dst);
    for (int n = threadIdx.x; n < ldq; n += blockDim.x)
        q[n] = __nv_cvt_float_to_fp8(n < ldN ? r[n] * inv : 0.f, __NV_SATFINITE, __NV_E4M3);
    return amax > 0.f ? amax / 448.f : 1.f;
}

// ------------------------------------------------------------------ admission (Eq. 8)
// New signal k takes slot slots[k] (k when slots == NULL) and GEMM row
// *n_act + k of operand half 0; signals that need no iteration are marked
// done and leave at the fixup that follows.  *n_extra = n_new tells the
// fixup how many rows were added.
struct AdmitArgs {
    const float* Y;         // n_new x N
    int n_new, N, ldN, M;
    const int* slots;
    const double* eps2;     // per new signal
    const int* T;
    float* R32;
    const BatchIO* io;
    SlotState* st;
    void* Rq;
    int ldq, fp8;
    float* rscale;          // optional: FP8 row scales (diagnostic)
    int* act;
    int* done;
    const int* n_act;
    int* n_extra;
    int* fin_count;         // signals that need no iteration are reported here
    int* fin_list;
};

__global__ void __launch_bounds__(kSelThreads) admit_kernel(const AdmitArgs a) {
    __shared__ double redd[kSelThreads / 32];
    __shared__ float redf[kSelThreads / 32];
    const int k = blockIdx.x;
    const int slot = a.slots ? a.slots[k] : k;
    const int row = *a.n_act + k;
    const float* y = a.Y + static_cast<size_t>(k) * a.N;
    float* r = a.R32 + static_cast<size_t>(slot) * a.ldN;
    for (int n = threadIdx.x; n < a.ldN; n += blockDim.x) r[n] = n < a.N ? y[n] : 0.f;
    if (a.io->X) {
        float* x = a.io->X + static_cast<size_t>(slot) * a.io->ldx;
        for (int m = threadIdx.x; m < a.M; m += blockDim.x) x[m] = 0.f;
    }
    __syncthreads();
    // e0 in the persistent kernel's order: 128 chains over float4s, warp
    // sums in warp order (threads 128.. contribute zeros)
    double acc = 0.0;
    if (threadIdx.x < kSumChains) {
        const float4* r4 = reinterpret_cast<const float4*>(r);
        for (int q = threadIdx.x; q < a.ldN / 4; q += kSumChains) {
            const float4 v = r4[q];
            acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
            acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
            acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
            acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
        }
    }
    const double e0 = block_sum_f64(acc, redd);   // also orders the r writes before the quantise
    const float sc = block_quantize(r, a.ldN, static_cast<char*>(a.Rq) + static_cast<size_t>(row) * a.ldq * (a.fp8 ? 1 : 2),
                                    a.ldq, a.fp8, redf);
    if (threadIdx.x == 0) {
        SlotState s;
        s.e0 = e0;
        s.e = e0;
        s.thr2 = a.eps2[k] * e0;
        s.audit = 0.0;
        s.t = 0;
        s.T = a.T[k];
        const bool finite = isfinite(e0);
        s.status = finite ? MP_OK : MP_ERR_NONFINITE;
        const bool run = finite && e0 > s.thr2 && s.T > 0;
        s.stop_reason = e0 == 0.0 ? MP_STOP_ZERO_Y : (e0 <= s.thr2 ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS);
        a.st[slot] = s;
        a.act[row] = slot;
        a.done[row] = run ? 0 : 1;
        if (a.rscale) a.rscale[row] = sc;
        if (!run && a.fin_list) a.fin_list[atomicAdd(a.fin_count, 1)] = slot;
        if (k == 0) *a.n_extra = a.n_new;
    }
}

// ------------------------------------------------------------------ select / rescore / update
struct SelArgs {
    const int* n_act;       // rows of this step's half
    const int* act;         // this half's slot ids by row
    int* n_next;            // survivors take rows of the other half:
    int* act_next;          //   its row count, slot ids
    void* Rq_next;          //   and quantised operand rows
    const uint2* cand;
    const int* n_at;        // sorted candidate lists per row (atom tiles of the step's GEMM)
    const float* psi32;
    int ldN, N, M;
    float* R32;
    const BatchIO* io;
    SlotState* st;
    int ldq, fp8;
    int* fin_count;         // optional: slots that stopped this step are appended here
    int* fin_list;
    // Gram mode
    float* Cg;              // per-slot correlations, ldC floats apart
    int ldC;
    const float* G;         // Psi^T Psi, ldG floats per row
    int ldG;
    unsigned long long* gtop;   // per-slot 8 largest |c| of Cg (keys as cand_key), sorted
    int* n_act_w;           // Gram mode: this half's count, cleared by the step's last CTA
    int* done_ctr;          //   CTAs of the step that finished (NULL: not cleared here)
    int* err;               // Gram mode: a bounded wait gave up (MP_ERR_TIMEOUT)
    unsigned long long lim; //   the waits' limit, ns
};

// Gram mode: the step's last CTA clears the count it read, after every CTA
// of the step has read it, so the next step's survivors (a select kernel,
// not a GEMM that would clear it) append from 0.
MP_DEV void step_done(const SelArgs& a) {
    if (threadIdx.x == 0 && a.done_ctr) {
        if (atomicAdd(a.done_ctr, 1) == static_cast<int>(gridDim.x) - 1) {
            *a.n_act_w = 0;
            *a.done_ctr = 0;
        }
    }
}

// Asynchronous 16-byte global -> shared copies (completed by cp_async_wait_all
// in the issuing thread, made visible to the block by a barrier after it).
MP_DEV void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
MP_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
MP_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// A candidate entry (score bits, atom) as a key ordering larger scores
// first, then smaller atoms; 0 for an empty entry (atom >= M).
MP_DEV unsigned long long cand_key(uint32_t score_bits, uint32_t atom, int M) {
    return atom < static_cast<uint32_t>(M)
               ? (static_cast<unsigned long long>(score_bits) << 32) | (0xffffffffu - atom)
               : 0ull;
}
// after it a >= b
MP_DEV void cex64(unsigned long long& a, unsigned long long& b) {
    const unsigned long long hi = umax64(a, b);
    b = a ^ b ^ hi;
    a = hi;
}
// t <- the best 8 of (t, c), both sorted descending: the elementwise max of
// t and reversed c is a bitonic sequence holding them; a bitonic merge
// network (12 exchanges) sorts it
MP_DEV void merge_top8_u64(unsigned long long (&t)[kTop], const unsigned long long (&c)[kTop]) {
#pragma unroll
    for (int i = 0; i < kTop; ++i) t[i] = umax64(t[i], c[kTop - 1 - i]);
    cex64(t[0], t[4]); cex64(t[1], t[5]); cex64(t[2], t[6]); cex64(t[3], t[7]);
    cex64(t[0], t[2]); cex64(t[1], t[3]); cex64(t[4], t[6]); cex64(t[5], t[7]);
    cex64(t[0], t[1]); cex64(t[2], t[3]); cex64(t[4], t[5]); cex64(t[6], t[7]);
}
// Two FP32 correlations with r at once, each in exactly dot1's order (four
// chains over the lane's float4s in increasing offset, ((x + y) + (z + w)),
// then the warp butterfly), so both atoms' loads are in flight together.
MP_DEV void dot1_pair(const float* __restrict__ p0, const float* __restrict__ p1, const float* __restrict__ r,
                      int ldN, int lane, float& d0, float& d1) {
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f, bx = 0.f, by = 0.f, bz = 0.f, bw = 0.f;
#pragma unroll 4
    for (int off = lane * 4; off < ldN; off += 128) {
        const float4 q = *reinterpret_cast<const float4*>(r + off);
        const float4 v = *reinterpret_cast<const float4*>(p0 + off);
        const float4 u = *reinterpret_cast<const float4*>(p1 + off);
        ax = fmaf(v.x, q.x, ax);
        ay = fmaf(v.y, q.y, ay);
        az = fmaf(v.z, q.z, az);
        aw = fmaf(v.w, q.w, aw);
        bx = fmaf(u.x, q.x, bx);
        by = fmaf(u.y, q.y, by);
        bz = fmaf(u.z, q.z, bz);
        bw = fmaf(u.w, q.w, bw);
    }
    d0 = warp_sum_f32((ax + ay) + (az + aw));
    d1 = warp_sum_f32((bx + by) + (bz + bw));
}

// One FP32 correlation in exactly dot1's order, with the atom's loads of U
// consecutive lane steps issued before their FMAs, so that U float4s per
// lane are in flight at once (a long row is otherwise one L2 round trip per
// few elements).  The tail steps run one at a time in the same order.
template <int U>
MP_DEV float dot1_deep(const float* __restrict__ p, const float* __restrict__ r, int ldN, int lane) {
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
    int off = lane * 4;
    for (; off + 128 * (U - 1) < ldN; off += 128 * U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(reinterpret_cast<const float4*>(p + off + 128 * u));
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 q = *reinterpret_cast<const float4*>(r + off + 128 * u);
            ax = fmaf(v[u].x, q.x, ax);
            ay = fmaf(v[u].y, q.y, ay);
            az = fmaf(v[u].z, q.z, az);
            aw = fmaf(v[u].w, q.w, aw);
        }
    }
    for (; off < ldN; off += 128) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + off));
        const float4 q = *reinterpret_cast<const float4*>(r + off);
        ax = fmaf(v.x, q.x, ax);
        ay = fmaf(v.y, q.y, ay);
        az = fmaf(v.z, q.z, az);
        aw = fmaf(v.w, q.w, aw);
    }
    return warp_sum_f32((ax + ay) + (az + aw));
}

// Insert key k into the sorted (descending) top 8 t.
MP_DEV void top8_insert(unsigned long long (&t)[kTop], unsigned long long k) {
    if (k <= t[kTop - 1]) return;
    t[kTop - 1] = k;
#pragma unroll
    for (int i = kTop - 1; i > 0; --i) {
        const unsigned long long hi = umax64(t[i - 1], t[i]);
        t[i] = t[i - 1] ^ t[i] ^ hi;
        t[i - 1] = hi;
    }
}

// Score of the 8th (smallest) key of a sorted top 8 as a float (0 while the
// list is not full): an |c| below it cannot enter, so the key is not built.
MP_DEV float top8_floor(const unsigned long long (&t)[kTop]) {
    return __uint_as_float(static_cast<uint32_t>(t[kTop - 1] >> 32));
}
// Offer |c| of atom j to the sorted top 8 t (thr: top8_floor(t), kept).
MP_DEV void top8_offer(unsigned long long (&t)[kTop], float& thr, float c, int j, int M) {
    const float s = fabsf(c);
    if (s >= thr && j < M) {
        top8_insert(t, cand_key(__float_as_uint(s), static_cast<uint32_t>(j), M));
        thr = top8_floor(t);
    }
}


// Block-wide best 8 of the threads' sorted lists lk (a butterfly of the
// bitonic top-8 merge inside each warp, then warp 0 over the warps' lists,
// through w, a THREADS / 32 x 8 shared array); thread 0 stores them to out.
template <int THREADS>
MP_DEV void block_top8_store(unsigned long long (&lk)[kTop], unsigned long long (*w)[kTop], unsigned long long* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other[kTop];
#pragma unroll
        for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
        merge_top8_u64(lk, other);
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kTop; ++k) w[warp][k] = lk[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < kTop; ++k) lk[k] = lane < THREADS / 32 ? w[lane][k] : 0ull;
#pragma unroll
        for (int o = 1; o < THREADS / 32; o <<= 1) {
            unsigned long long other[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
            merge_top8_u64(lk, other);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < kTop; ++k) out[k] = lk[k];
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == kSumChains ? 6 : (THREADS == 2 * kSumChains ? 2 : 1))
    select_update_kernel(const SelArgs a) {
    extern __shared__ float4 r_sh4[];
    float* r = reinterpret_cast<float*>(r_sh4);
    __shared__ double redd[THREADS / 32];
    __shared__ float redf[THREADS / 32];
    __shared__ int top[kTop];
    __shared__ unsigned long long rkey[kTop];
    const int i = blockIdx.x;
    if (i >= *a.n_act) {
        step_done(a);
        return;
    }
    const int slot = a.act[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* rs4 = reinterpret_cast<float4*>(r);
    float4* rg4 = reinterpret_cast<float4*>(a.R32 + static_cast<size_t>(slot) * a.ldN);
    const int n4 = a.ldN / 4;
    SlotState s = a.st[slot];   // loaded now, used after the rescore
    // r streams into shared memory while the candidate lists are merged
    for (int k = threadIdx.x; k < n4; k += blockDim.x) cp_async16(rs4 + k, rg4 + k);
    cp_async_commit();

    // merge the sorted per-tile lists: keys (score bits, ~atom) order by
    // score, then by the smaller atom.  Thread t folds lists t, t + THREADS,
    // ... into its sorted best 8 (a bitonic top-8 merge per list); a
    // butterfly of the same merge gives lane 0 of every warp the warp's best
    // 8, and warp 0 merges those.  Candidate sets are disjoint at every merge,
    // so the result is the set of the 8 largest keys, whatever the split.
    {
        __shared__ unsigned long long wtop[THREADS / 32][kTop];
        unsigned long long lk[kTop];
#pragma unroll
        for (int k = 0; k < kTop; ++k) lk[k] = 0ull;
        const int n_at = *a.n_at;
        const uint2* cd = a.cand + static_cast<size_t>(i) * n_at * kTop;
        for (int t = threadIdx.x; t < n_at; t += THREADS) {
            // the whole list in one go (64 bytes): no chain of dependent loads
            unsigned long long lst[kTop];
            const uint4* l4 = reinterpret_cast<const uint4*>(cd + static_cast<size_t>(t) * kTop);
#pragma unroll
            for (int u = 0; u < kTop / 2; ++u) {
                const uint4 q = l4[u];
                lst[2 * u] = cand_key(q.x, q.y, a.M);
                lst[2 * u + 1] = cand_key(q.z, q.w, a.M);
            }
            merge_top8_u64(lk, lst);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
            merge_top8_u64(lk, other);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < kTop; ++k) wtop[warp][k] = lk[k];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < kTop; ++k) lk[k] = lane < THREADS / 32 ? wtop[lane][k] : 0ull;
#pragma unroll
            for (int o = 1; o < THREADS / 32; o <<= 1) {
                unsigned long long other[kTop];
#pragma unroll
                for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
                merge_top8_u64(lk, other);
            }
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < kTop; ++k)
                    top[k] = lk[k] ? static_cast<int>(0xffffffffu - static_cast<uint32_t>(lk[k])) : -1;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // rescore the candidates in FP32 from the FP32 atoms (Eq. 9), in the
    // plain kernel's correlation order; a warp takes candidates w and
    // w + THREADS / 32 together so their loads are in flight at once
    if constexpr (THREADS / 32 >= kTop) {
        if (warp < kTop) {
            const int m0 = top[warp];
            unsigned long long key = 0ull;
            if (m0 >= 0) key = pack_key(dot1_deep<16>(a.psi32 + static_cast<size_t>(m0) * a.ldN, r, a.ldN, lane), m0);
            if (lane == 0) rkey[warp] = key;
        }
    } else
    for (int cnd = warp; cnd < kTop; cnd += 2 * (THREADS / 32)) {
        const int c2 = cnd + THREADS / 32;
        const int m0 = top[cnd];
        const int m1 = c2 < kTop ? top[c2] : -1;
        const float* p0 = a.psi32 + static_cast<size_t>(m0 < 0 ? 0 : m0) * a.ldN;
        const float* p1 = m1 < 0 ? p0 : a.psi32 + static_cast<size_t>(m1) * a.ldN;
        float d0, d1;
        dot1_pair(p0, p1, r, a.ldN, lane, d0, d1);
        if (lane == 0) {
            rkey[cnd] = m0 >= 0 ? pack_key(d0, m0) : 0ull;
            if (c2 < kTop) rkey[c2] = m1 >= 0 ? pack_key(d1, m1) : 0ull;
        }
    }
    __syncthreads();
    unsigned long long kbest = 0ull;
    for (int w = 0; w < kTop; ++w) kbest = umax64(kbest, rkey[w]);
    if (kbest == 0ull) {   // no candidate: nothing can be selected; the signal leaves
        if (threadIdx.x == 0) {
            s.status = MP_ERR_INVALID;
            a.st[slot] = s;
            if (a.fin_list) a.fin_list[atomicAdd(a.fin_count, 1)] = slot;
        }
        step_done(a);
        return;
    }
    const int m = key_index(kbest);
    const float c = key_coef(kbest);
    // thread 0 updates x~[m] at the end: fetch the old value now
    BatchIO io;
    float xm = 0.f;
    if (threadIdx.x == 0) {
        io = *a.io;
        xm = io.X[static_cast<size_t>(slot) * io.ldx + m];
    }
    // Eq. 11 in FP32, the FP64 energy, then the requantised row of a signal
    // that runs on
    const float4* pm = reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(m) * a.ldN);
    {
        // the thread's first kUpd vectors of psi_m are loaded together, so
        // their latencies overlap, then applied; any rest in a plain loop
        constexpr int kUpd = 4;
        float4 p[kUpd];
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
            const int k = threadIdx.x + u * THREADS;
            if (k < n4) p[u] = __ldg(pm + k);
        }
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
            const int k = threadIdx.x + u * THREADS;
            if (k < n4) {
                float4 v = rs4[k];
                v.x = fmaf(-c, p[u].x, v.x);
                v.y = fmaf(-c, p[u].y, v.y);
                v.z = fmaf(-c, p[u].z, v.z);
                v.w = fmaf(-c, p[u].w, v.w);
                rg4[k] = v;
                rs4[k] = v;
            }
        }
        for (int k = threadIdx.x + kUpd * THREADS; k < n4; k += THREADS) {
            const float4 q = __ldg(pm + k);
            float4 v = rs4[k];
            v.x = fmaf(-c, q.x, v.x);
            v.y = fmaf(-c, q.y, v.y);
            v.z = fmaf(-c, q.z, v.z);
            v.w = fmaf(-c, q.w, v.w);
            rg4[k] = v;
            rs4[k] = v;
        }
    }
    if (THREADS != kSumChains) __syncthreads();   // the chains read other threads' updates
    double acc = 0.0;
    if (threadIdx.x < kSumChains)
        for (int k = threadIdx.x; k < n4; k += kSumChains) {
            const float4 v = rs4[k];
            acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
            acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
            acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
            acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
        }
    const double e = block_sum_f64(acc, redd);   // also orders the smem r writes
    __shared__ int next_row;
    if (threadIdx.x == 0) {
        io.X[static_cast<size_t>(slot) * io.ldx + m] = xm + c;   // Eq. 10
        if (io.tr_atoms && s.t < io.tr_cap) io.tr_atoms[static_cast<size_t>(slot) * io.tr_cap + s.t] = m;
        if (io.tr_coefs && s.t < io.tr_cap) io.tr_coefs[static_cast<size_t>(slot) * io.tr_cap + s.t] = c;
        if (io.tr_energy && s.t < io.tr_cap) io.tr_energy[static_cast<size_t>(slot) * io.tr_cap + s.t] = e;
        const double cc = static_cast<double>(c);
        s.audit = fmax(s.audit, fabs(e - (s.e - cc * cc)));   // divided by e0 when reported
        s.e = e;
        s.t += 1;   // Eq. 12
        const bool conv = !(e > s.thr2);
        const bool stop = conv || s.t >= s.T;
        if (stop) s.stop_reason = conv ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS;
        a.st[slot] = s;
        int row = -1;
        if (!stop) {
            row = atomicAdd(a.n_next, 1);
            a.act_next[row] = slot;
        } else if (a.fin_list) {
            a.fin_list[atomicAdd(a.fin_count, 1)] = slot;
        }
        next_row = row;
    }
    __syncthreads();
    const int row = next_row;
    if (row < 0) {
        step_done(a);
        return;
    }
    char* qrow = static_cast<char*>(a.Rq_next) + static_cast<size_t>(row) * a.ldq * (a.fp8 ? 1 : 2);
    if (a.fp8) {
        block_quantize(r, a.ldN, qrow, a.ldq, 1, redf);
    } else {
        // the first ldN elements; the row's padding up to ldq holds zeros (the
        // operand is zeroed when allocated, and admission and compaction,
        // which write whole rows, write zeros there)
        for (int k = threadIdx.x; k < n4; k += THREADS) {
            const float4 v = rs4[k];
            __nv_bfloat162* q2 = reinterpret_cast<__nv_bfloat162*>(qrow) + 2 * k;
            q2[0] = __floats2bfloat162_rn(v.x, v.y);
            q2[1] = __floats2bfloat162_rn(v.z, v.w);
        }
    }
    step_done(a);
}

// ------------------------------------------------------------------ Gram-mode step (one kernel)
// One MP step of one signal in the Gram mode.  The candidates are the slot's
// carried 8 largest |c|; they are rescored in FP32 from the FP32 atoms in
// the plain kernel's correlation order and the best is committed (Eq. 10),
// r -= c psi_m in FP32 (Eq. 11).  Then two warp groups run at once:
//   warps 0..3   the FP64 energy in the plain kernel's 128-chain order, the
//                stop test (Eq. 8) and the slot's bookkeeping;
//   warps 4..15  the Gram update of the slot's correlations,
//                c_j -= c G[m][j] (one FP32 FMA per entry), and their 8
//                largest |c| for the next step (keys as cand_key): each
//                thread keeps the largest |c| of its entries; a warp sort of
//                those gives, over the group's warps, a threshold that at
//                least 8 entries reach, so the 8 largest are among the few
//                entries at or above it, which are ranked exactly.
// The update runs whether or not the signal stops (a stopped slot's row is
// not read again).  The same 8 keys as a full ranking of the row, so the
// same results bit for bit.
constexpr int kGramThreads = 512;                       // threads of an SM's Gram-step CTAs together
constexpr int kGramGroup0 = kSumChains;                // energy group: threads 0..127
constexpr int kGramList = 256;                          // entries at or above the threshold kept

MP_DEV float warp_kth_largest(float v, int k) {
    // descending bitonic sort of the warp's 32 values; lane k-1 then holds
    // the k-th largest
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 2; s <= 32; s <<= 1)
#pragma unroll
        for (int j = s >> 1; j > 0; j >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool desc = (lane & s) == 0 || s == 32;
            const bool low = (lane & j) == 0;
            v = (low == desc) ? fmaxf(v, o) : fminf(v, o);
        }
    return __shfl_sync(0xffffffffu, v, k - 1);
}

// The row's 8 largest keys from the kept entries (list, n entries): with at
// most 32, one warp ranks each by counting the larger keys (keys are
// distinct); with more, each lane folds its share into a sorted top 8 and
// a butterfly merges them.  Lane 0's results go to out.
MP_DEV void list_top8_store(const unsigned long long* list, int n, unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    if (n <= 32) {
        const unsigned long long k = lane < n ? list[lane] : 0ull;
        int rank = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) rank += __shfl_sync(0xffffffffu, k, j) > k ? 1 : 0;
        if (lane < n && rank < kTop) out[rank] = k;
        if (lane >= n && lane < kTop) out[lane] = 0ull;   // fewer than 8 entries: empty keys
        return;
    }
    unsigned long long lk[kTop];
#pragma unroll
    for (int k = 0; k < kTop; ++k) lk[k] = 0ull;
    for (int t = lane; t < n; t += 32) top8_insert(lk, list[t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other[kTop];
#pragma unroll
        for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
        merge_top8_u64(lk, other);
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kTop; ++k) out[k] = lk[k];
}

// SM: the slot's correlation row and the selected atom's row of G are
// brought into shared memory by bulk copies (issued as soon as their
// addresses are known, landing while the step rescores and updates r);
// otherwise they are read from global memory.  CTA = 256 (two CTAs per SM:
// two signals' chains of dependent phases at once) when two fit in an SM's
// shared memory, else 512 (one CTA per SM, 12 warps on each long row); the
// grid has kGramThreads / CTA CTAs per SM; each CTA takes rows blockIdx.x,
// blockIdx.x + gridDim.x, ...
template <bool SM, int CTA>
__global__ void __launch_bounds__(CTA, kGramThreads / CTA) gram_select_kernel(const SelArgs a) {
    extern __shared__ float4 dsm[];
    float* r = reinterpret_cast<float*>(dsm);
    float4* rs4 = dsm;
    const int n4 = a.ldN / 4;
    const int nq = a.ldC / 4;
    float4* cs4 = dsm + n4;          // SM: the correlation row
    float4* gs4 = dsm + n4 + nq;     //     the row of G
    __shared__ double redd[kGramGroup0 / 32];
    __shared__ int top[kTop];
    __shared__ unsigned long long rkey[kTop];
    __shared__ float wthr[CTA / 32];
    __shared__ unsigned long long list[kGramList];
    __shared__ int list_n;
    __shared__ unsigned long long gtw[CTA / 32][kTop];
    __shared__ uint64_t bar_c, bar_g;
    __shared__ int abort_flag;
    __shared__ int spec_m;   // SM: the row of G whose copy started with the signal (-1: none)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the first row's slot is fetched with the row count, not after it (the
    // grid never exceeds the slot table, so the index is in range)
    const int slot0 = a.act[blockIdx.x];
    const int n_act = *a.n_act;
    if (SM && threadIdx.x == 0) {
        mbar_init(&bar_c, 1);
        mbar_init(&bar_g, 1);
        fence_mbar_init();
    }
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    // parity of bar_g's next phase: it completes once per signal, or twice
    // when the speculative row of G was not the selected one
    uint32_t gph = 0;
    for (int i = blockIdx.x, it = 0; i < n_act && !abort_flag; i += gridDim.x, ++it) {
        const uint32_t ph = static_cast<uint32_t>(it & 1);
        const int slot = it == 0 ? slot0 : a.act[i];
        float4* rg4 = reinterpret_cast<float4*>(a.R32 + static_cast<size_t>(slot) * a.ldN);
        float4* cr4 = reinterpret_cast<float4*>(a.Cg + static_cast<size_t>(slot) * a.ldC);
        if (SM && threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar_c, static_cast<uint32_t>(a.ldC) * 4u);
            bulk_g2s(cs4, cr4, static_cast<uint32_t>(a.ldC) * 4u, &bar_c);
            // the carried best candidate is nearly always the one the rescore
            // selects: its row of G starts coming in with the correlations
            const unsigned long long k0 = a.gtop[static_cast<size_t>(slot) * kTop];
            const int mg = k0 ? static_cast<int>(0xffffffffu - static_cast<uint32_t>(k0)) : -1;
            spec_m = mg;
            if (mg >= 0) {
                mbar_arrive_expect_tx(&bar_g, static_cast<uint32_t>(a.ldG) * 4u);
                bulk_g2s(gs4, a.G + static_cast<size_t>(mg) * a.ldG, static_cast<uint32_t>(a.ldG) * 4u, &bar_g);
            }
        }
        SlotState s = a.st[slot];
        BatchIO io;
        if (threadIdx.x == 0) io = *a.io;
        for (int k = threadIdx.x; k < n4; k += CTA) cp_async16(rs4 + k, rg4 + k);
        cp_async_commit();
        if (!SM)
            for (int q = threadIdx.x * 8; q < nq; q += CTA * 8) prefetch_line_l2(cr4 + q);
        if (threadIdx.x < kTop) {
            const unsigned long long k = a.gtop[static_cast<size_t>(slot) * kTop + threadIdx.x];
            top[threadIdx.x] = k ? static_cast<int>(0xffffffffu - static_cast<uint32_t>(k)) : -1;
        }
        if (threadIdx.x == 0) list_n = 0;
        cp_async_wait_all();
        __syncthreads();
        // rescore in FP32 (Eq. 9), one candidate per warp
        if (warp < kTop) {
            const int m0 = top[warp];
            unsigned long long key = 0ull;
            if (m0 >= 0) key = pack_key(dot1_deep<16>(a.psi32 + static_cast<size_t>(m0) * a.ldN, r, a.ldN, lane), m0);
            if (lane == 0) rkey[warp] = key;
        }
        __syncthreads();
        unsigned long long kbest = 0ull;
#pragma unroll
        for (int w = 0; w < kTop; ++w) kbest = umax64(kbest, rkey[w]);
        const int m = kbest ? key_index(kbest) : 0;
        const float c = kbest ? key_coef(kbest) : 0.f;
        const float4* gr4 = reinterpret_cast<const float4*>(a.G + static_cast<size_t>(m) * a.ldG);
        const int mg = SM ? spec_m : -1;
        const bool g_miss = SM && kbest && mg >= 0 && mg != m;   // the same in every thread
        if (kbest && SM && threadIdx.x == 0) {
            bool issue = mg < 0;
            if (g_miss) {
                // the guessed row lands first (the buffer is not written twice
                // at once), then the selected row comes in
                issue = mbar_wait_bounded(&bar_g, gph, a.lim);
                if (!issue) {
                    atomicCAS(a.err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                    abort_flag = 1;
                    mbar_wait_bounded(&bar_g, gph, a.lim);   // the copy in flight, once more
                }
            }
            if (issue) {
                mbar_arrive_expect_tx(&bar_g, static_cast<uint32_t>(a.ldG) * 4u);
                bulk_g2s(gs4, gr4, static_cast<uint32_t>(a.ldG) * 4u, &bar_g);
            }
        }
        // the phase the row update waits for; bar_g completes one phase for
        // this signal, two after a missed guess
        const uint32_t gwait = g_miss ? (gph ^ 1u) : gph;
        if (!g_miss) gph ^= 1u;
        if (kbest == 0ull) {   // no candidate: nothing can be selected; the signal leaves
            if (threadIdx.x == 0) {
                s.status = MP_ERR_INVALID;
                a.st[slot] = s;
                if (a.fin_list) a.fin_list[atomicAdd(a.fin_count, 1)] = slot;
                if (SM && !mbar_wait_bounded(&bar_c, ph, a.lim)) {
                    atomicCAS(a.err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                    abort_flag = 1;
                    mbar_wait_bounded(&bar_c, ph, a.lim);   // the copy in flight, once more
                }
                // a speculative row of G lands before its buffer is reused
                if (SM && mg >= 0 && !mbar_wait_bounded(&bar_g, gwait, a.lim)) {
                    atomicCAS(a.err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                    abort_flag = 1;
                    mbar_wait_bounded(&bar_g, gwait, a.lim);
                }
            }
            __syncthreads();
            if (SM && mg < 0 && !abort_flag && threadIdx.x == 0) {
                // no row of G was copied: complete its phase by hand
                mbar_arrive(&bar_g);
            }
            __syncthreads();
            continue;
        }
        if (!SM)
            for (int q = threadIdx.x * 8; q < nq; q += CTA * 8) prefetch_line_l2(gr4 + q);
        float xm = 0.f;
        if (threadIdx.x == 0) xm = io.X[static_cast<size_t>(slot) * io.ldx + m];
        // Eq. 11 in FP32
        const float4* pm = reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(m) * a.ldN);
        for (int k = threadIdx.x; k < n4; k += CTA) {
            const float4 p = __ldg(pm + k);
            float4 v = rs4[k];
            v.x = fmaf(-c, p.x, v.x);
            v.y = fmaf(-c, p.y, v.y);
            v.z = fmaf(-c, p.z, v.z);
            v.w = fmaf(-c, p.w, v.w);
            rg4[k] = v;
            rs4[k] = v;
        }
        __syncthreads();
        if (threadIdx.x < kGramGroup0) {
            // ---- energy group: e = sum r^2 in FP64 in the plain kernel's order
            double acc = 0.0;
            for (int k = threadIdx.x; k < n4; k += kSumChains) {
                const float4 v = rs4[k];
                acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
                acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
                acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
                acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
            }
            acc = warp_sum_f64(acc);
            if (lane == 0) redd[warp] = acc;
            named_bar_sync(1, kGramGroup0);
            if (threadIdx.x == 0) {
                double e = 0.0;
#pragma unroll
                for (int w = 0; w < kGramGroup0 / 32; ++w) e += redd[w];
                io.X[static_cast<size_t>(slot) * io.ldx + m] = xm + c;   // Eq. 10
                if (io.tr_atoms && s.t < io.tr_cap) io.tr_atoms[static_cast<size_t>(slot) * io.tr_cap + s.t] = m;
                if (io.tr_coefs && s.t < io.tr_cap) io.tr_coefs[static_cast<size_t>(slot) * io.tr_cap + s.t] = c;
                if (io.tr_energy && s.t < io.tr_cap) io.tr_energy[static_cast<size_t>(slot) * io.tr_cap + s.t] = e;
                const double cc = static_cast<double>(c);
                s.audit = fmax(s.audit, fabs(e - (s.e - cc * cc)));   // divided by e0 when reported
                s.e = e;
                s.t += 1;   // Eq. 12
                const bool conv = !(e > s.thr2);
                const bool stop = conv || s.t >= s.T;
                if (stop) s.stop_reason = conv ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS;
                a.st[slot] = s;
                if (!stop) {
                    const int row = atomicAdd(a.n_next, 1);
                    a.act_next[row] = slot;
                } else if (a.fin_list) {
                    a.fin_list[atomicAdd(a.fin_count, 1)] = slot;
                }
            }
        } else {
            // ---- Gram group: c_j -= c G[m][j] and the row's 8 largest |c|
            constexpr int GT = CTA - kGramGroup0;
            const int gt = threadIdx.x - kGramGroup0, gw = warp - kGramGroup0 / 32;
            bool ok = true;
            if (SM) {
                // both rows in shared memory (bounded waits; every thread
                // of the group sees the same outcome)
                if (gt == 0) {
                    const bool okc = mbar_wait_bounded(&bar_c, ph, a.lim);
                    const bool okg = mbar_wait_bounded(&bar_g, gwait, a.lim);
                    if (!(okc && okg)) {
                        atomicCAS(a.err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                        abort_flag = 1;
                        // let any copy still in flight land before the
                        // buffers are left (bounded again)
                        if (!okc) mbar_wait_bounded(&bar_c, ph, a.lim);
                        if (!okg) mbar_wait_bounded(&bar_g, gwait, a.lim);
                    }
                }
                named_bar_sync(2, GT);
                ok = !abort_flag;
                if (ok) {
                    // every thread passes its own wait (the phase is complete)
                    mbar_try_wait(&bar_c, ph);
                    mbar_try_wait(&bar_g, gwait);
                }
            }
            float mx = 0.f;
            if (ok) {
                constexpr int U = SM ? 4 : 8;   // shared memory needs fewer loads in flight
                for (int q0 = gt; q0 < nq; q0 += U * GT) {
                    float4 g[U], v[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int q = q0 + u * GT;
                        if (q < nq) {
                            g[u] = SM ? gs4[q] : __ldg(gr4 + q);
                            v[u] = SM ? cs4[q] : cr4[q];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int q = q0 + u * GT;
                        if (q >= nq) break;
                        v[u].x = fmaf(-c, g[u].x, v[u].x);
                        v[u].y = fmaf(-c, g[u].y, v[u].y);
                        v[u].z = fmaf(-c, g[u].z, v[u].z);
                        v[u].w = fmaf(-c, g[u].w, v[u].w);
                        cr4[q] = v[u];
                        if (SM) cs4[q] = v[u];
                        // entries past M (the row's padding) never rank
                        const int j0 = 4 * q;
                        if (j0 + 0 < a.M) mx = fmaxf(mx, fabsf(v[u].x));
                        if (j0 + 1 < a.M) mx = fmaxf(mx, fabsf(v[u].y));
                        if (j0 + 2 < a.M) mx = fmaxf(mx, fabsf(v[u].z));
                        if (j0 + 3 < a.M) mx = fmaxf(mx, fabsf(v[u].w));
                    }
                }
            }
            // the warp's 8th largest thread maximum: 8 entries of the warp
            // reach it, so the row's 8th largest |c| does too; the largest
            // such value over the group's warps is the threshold
            const float w8 = warp_kth_largest(mx, kTop);
            if (lane == 0) wthr[gw] = w8;
            named_bar_sync(2, GT);
            float thr = 0.f;
#pragma unroll
            for (int w = 0; w < GT / 32; ++w) thr = fmaxf(thr, wthr[w]);
            // entries at or above the threshold (only threads whose
            // maximum reaches it look at their entries again)
            if (ok && mx >= thr) {
                for (int q = gt; q < nq; q += GT) {
                    const float4 v = SM ? cs4[q] : cr4[q];
                    const float e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = 4 * q + u;
                        const float sc = fabsf(e4[u]);
                        if (j < a.M && sc >= thr) {
                            const int at = atomicAdd(&list_n, 1);
                            if (at < kGramList) list[at] = cand_key(__float_as_uint(sc), static_cast<uint32_t>(j), a.M);
                        }
                    }
                }
            }
            named_bar_sync(2, GT);
            const int ln = list_n;
            unsigned long long* out = a.gtop + static_cast<size_t>(slot) * kTop;
            if (!ok) {
                // no update (a wait gave up): nothing to rank
            } else if (ln <= kGramList) {
                if (gw == 0) list_top8_store(list, ln, out);
            } else {
                // more entries tie at the threshold than the list holds: rank
                // the whole row (every thread its own entries, then the group)
                unsigned long long lk[kTop];
#pragma unroll
                for (int k = 0; k < kTop; ++k) lk[k] = 0ull;
                float t8 = 0.f;
                for (int q = gt; q < nq; q += GT) {
                    const float4 v = SM ? cs4[q] : cr4[q];
                    top8_offer(lk, t8, v.x, 4 * q + 0, a.M);
                    top8_offer(lk, t8, v.y, 4 * q + 1, a.M);
                    top8_offer(lk, t8, v.z, 4 * q + 2, a.M);
                    top8_offer(lk, t8, v.w, 4 * q + 3, a.M);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    unsigned long long other[kTop];
#pragma unroll
                    for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
                    merge_top8_u64(lk, other);
                }
                if (lane == 0)
#pragma unroll
                    for (int k = 0; k < kTop; ++k) gtw[gw][k] = lk[k];
                named_bar_sync(2, GT);
                if (gw == 0) {
#pragma unroll
                    for (int k = 0; k < kTop; ++k) lk[k] = lane < GT / 32 ? gtw[lane][k] : 0ull;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        unsigned long long other[kTop];
#pragma unroll
                        for (int k = 0; k < kTop; ++k) other[k] = __shfl_xor_sync(0xffffffffu, lk[k], o);
                        merge_top8_u64(lk, other);
                    }
                    if (lane == 0)
#pragma unroll
                        for (int k = 0; k < kTop; ++k) out[k] = lk[k];
                }
            }
        }
        // the next row reuses the buffers (its bulk copies write where this
        // row's threads wrote) and the barriers
        if (SM) fence_proxy_async_smem();
        __syncthreads();
    }
    step_done(a);
}

// ------------------------------------------------------------------ Gram mode: direct FP32 correlations
// c = Psi^T r (Eq. 9) in FP32 for listed slots, written to their correlation
// rows: at admission (r = y) and, in the graph, for the active slots whose
// own step count reached a multiple of the refresh period (bounding the
// recurrence's drift).  A CTA stages up to kCorrRows residual rows in shared
// memory and its warps run over a block of kCorrAtoms atoms, each atom read
// once from HBM for all the staged rows; float4 loads, 8 in flight per lane.
constexpr int kCorrRows = 8;
constexpr int kCorrAtoms = 64;
constexpr int kCorrThreads = 256;
constexpr int kCorrSmem = 200 * 1024;   // shared memory for the staged rows, at most

static int corr_rows_per_cta(const PlanImpl* p) {
    return std::max(1, std::min(kCorrRows, kCorrSmem / (p->ldN * static_cast<int>(sizeof(float)))));
}

struct CorrRowsArgs {
    const float* psi32;
    int ldN, M;
    const float* R32;       // residual rows by slot (ldN floats)
    const int* rows;        // slot of listed row k (NULL: slot k)
    const int* n_ptr;       // number of listed rows on the device (NULL: n)
    int n;
    const SlotState* st;    // R > 0: only slots with st.t a positive multiple of R
    int R;
    float* Cg;
    int ldC;
    int rpc;                // rows staged per CTA (<= kCorrRows, by the row length)
};

MP_DEV bool corr_row_wanted(const CorrRowsArgs& a, int slot) {
    if (a.R <= 0) return true;
    const int t = a.st[slot].t;
    return t > 0 && t % a.R == 0;
}

__global__ void __launch_bounds__(kCorrThreads) corr_rows_kernel(const CorrRowsArgs a) {
    extern __shared__ float4 rsh[];           // a.rpc rows of ldN floats
    __shared__ int slots[kCorrRows];
    __shared__ int want[kCorrRows];
    const int n = a.n_ptr ? *a.n_ptr : a.n;
    const int n4 = a.ldN / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int W = kCorrThreads / 32;
    const int m_end = min(a.M, (blockIdx.x + 1) * kCorrAtoms);
    // the CTA's block of atoms against every group of listed rows with a
    // row to compute (groups without one cost a look at their flags)
    for (int g0 = 0; g0 < n; g0 += a.rpc) {
        const int nr = min(a.rpc, n - g0);
        __syncthreads();   // the previous group's rows are no longer read
        if (threadIdx.x < kCorrRows) {
            int sl = -1, w = 0;
            if (static_cast<int>(threadIdx.x) < nr) {
                sl = a.rows ? a.rows[g0 + threadIdx.x] : g0 + static_cast<int>(threadIdx.x);
                w = corr_row_wanted(a, sl) ? 1 : 0;
            }
            slots[threadIdx.x] = sl;
            want[threadIdx.x] = w;
        }
        __syncthreads();
        int any = 0;
#pragma unroll
        for (int j = 0; j < kCorrRows; ++j) any |= want[j];
        if (!any) continue;
        for (int j = 0; j < nr; ++j) {
            const float4* src = reinterpret_cast<const float4*>(a.R32 + static_cast<size_t>(slots[j]) * a.ldN);
            for (int k = threadIdx.x; k < n4; k += kCorrThreads) rsh[j * n4 + k] = src[k];
        }
        __syncthreads();
        // two atoms per warp at a time, 8 float4 loads of each in flight
        for (int m0 = blockIdx.x * kCorrAtoms + warp; m0 < m_end; m0 += 2 * W) {
            const int m1 = m0 + W;
            const bool two = m1 < m_end;
            const float4* p0 = reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(m0) * a.ldN);
            const float4* p1 = reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(two ? m1 : m0) * a.ldN);
            float acc0[kCorrRows], acc1[kCorrRows];
#pragma unroll
            for (int j = 0; j < kCorrRows; ++j) acc0[j] = acc1[j] = 0.f;
            constexpr int U = 8;
            for (int k0 = lane; k0 < n4; k0 += 32 * U) {
                float4 v0[U], v1[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (k0 + 32 * u < n4) {
                        v0[u] = __ldg(p0 + k0 + 32 * u);
                        v1[u] = __ldg(p1 + k0 + 32 * u);
                    }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int k = k0 + 32 * u;
                    if (k >= n4) break;
#pragma unroll
                    for (int j = 0; j < kCorrRows; ++j) {
                        if (j >= nr) break;
                        const float4 q = rsh[j * n4 + k];
                        acc0[j] = fmaf(v0[u].x, q.x, fmaf(v0[u].y, q.y, fmaf(v0[u].z, q.z, fmaf(v0[u].w, q.w, acc0[j]))));
                        acc1[j] = fmaf(v1[u].x, q.x, fmaf(v1[u].y, q.y, fmaf(v1[u].z, q.z, fmaf(v1[u].w, q.w, acc1[j]))));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kCorrRows; ++j) {
                if (j >= nr) break;
                const float c0 = warp_sum_f32(acc0[j]);
                const float c1 = warp_sum_f32(acc1[j]);
                if (lane == 0 && want[j]) {
                    a.Cg[static_cast<size_t>(slots[j]) * a.ldC + m0] = c0;
                    if (two) a.Cg[static_cast<size_t>(slots[j]) * a.ldC + m1] = c1;
                }
            }
        }
    }
}

// The same correlations as a register-tiled FP32 GEMM, for refreshes whose
// listed rows are all due together (every row, or rows that share one step
// count, as in a batched decode where every active signal has taken the same
// number of steps): C[i][j] = sum_n r_slot(i)[n] psi_j[n], a 128-row x
// 128-atom output tile per CTA, 8 x 8 per thread, 16-deep slices of both
// operands staged transposed in shared memory; each entry is one FP32 FMA
// chain in increasing n.  A CTA whose tile holds no due row (or lies past
// the device's row count) leaves at once.
constexpr int kTileC = 128;
constexpr int kTileK = 16;
// below this many listed rows a 128-row tile computes mostly padding: the
// row-group kernel (one pass over the atoms per 8 rows) is cheaper
constexpr int kTiledMinRows = 64;

__global__ void __launch_bounds__(256) corr_tile_kernel(const CorrRowsArgs a) {
    __shared__ __align__(16) float As[kTileK][kTileC + 4];
    __shared__ __align__(16) float Bs[kTileK][kTileC + 4];
    __shared__ int slots[kTileC];
    __shared__ int any_due;
    const int n = a.n_ptr ? *a.n_ptr : a.n;
    const int i0 = blockIdx.y * kTileC, j0 = blockIdx.x * kTileC;
    if (i0 >= n) return;   // the same for every thread of the CTA
    const int tid = threadIdx.x;
    if (tid == 0) any_due = 0;
    __syncthreads();
    if (tid < kTileC) {
        int sl = -1;
        if (i0 + tid < n) {
            sl = a.rows ? a.rows[i0 + tid] : i0 + tid;
            if (corr_row_wanted(a, sl)) any_due = 1;
            else sl = -1;
        }
        slots[tid] = sl;
    }
    __syncthreads();
    if (!any_due) return;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    // each thread stages 2 float4 of each operand per slice: tile row
    // q >> 2, K offset 4 (q & 3), for q = tid and tid + 256
    for (int k0 = 0; k0 < a.ldN; k0 += kTileK) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = tid + 256 * h;
            const int row = q >> 2, kk = 4 * (q & 3);
            const int sl = slots[row], jb = j0 + row;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (sl >= 0) va = *reinterpret_cast<const float4*>(a.R32 + static_cast<size_t>(sl) * a.ldN + k0 + kk);
            if (jb < a.M) vb = __ldg(reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(jb) * a.ldN + k0 + kk));
            As[kk + 0][row] = va.x;
            As[kk + 1][row] = va.y;
            As[kk + 2][row] = va.z;
            As[kk + 3][row] = va.w;
            Bs[kk + 0][row] = vb.x;
            Bs[kk + 1][row] = vb.y;
            Bs[kk + 2][row] = vb.z;
            Bs[kk + 3][row] = vb.w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTileK; ++k) {
            float x[8], w[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8 + 4]);
            x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
            x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
            w[0] = b0.x; w[1] = b0.y; w[2] = b0.z; w[3] = b0.w;
            w[4] = b1.x; w[5] = b1.y; w[6] = b1.z; w[7] = b1.w;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(x[u], w[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int sl = slots[ty * 8 + u];
        if (sl < 0) continue;
        float* crow = a.Cg + static_cast<size_t>(sl) * a.ldC;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int j = j0 + tx * 8 + v;
            if (j < a.M) crow[j] = acc[u][v];
        }
    }
}

// The 8 largest |c| (keys as cand_key) of each listed slot's correlation
// row, for its next step; one CTA per listed row, the same filter as above.
__global__ void __launch_bounds__(kCorrThreads) gram_scan_kernel(const CorrRowsArgs a, unsigned long long* gtop) {
    __shared__ unsigned long long w[kCorrThreads / 32][kTop];
    const int n = a.n_ptr ? *a.n_ptr : a.n;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int slot = a.rows ? a.rows[k] : k;
        if (!corr_row_wanted(a, slot)) continue;   // the same for every thread of the CTA
        const float4* cr4 = reinterpret_cast<const float4*>(a.Cg + static_cast<size_t>(slot) * a.ldC);
        unsigned long long lk[kTop];
#pragma unroll
        for (int j = 0; j < kTop; ++j) lk[j] = 0ull;
        float thr = 0.f;
        for (int q = threadIdx.x; q < a.ldC / 4; q += kCorrThreads) {
            const float4 v = cr4[q];
            const int j0 = 4 * q;
            top8_offer(lk, thr, v.x, j0 + 0, a.M);
            top8_offer(lk, thr, v.y, j0 + 1, a.M);
            top8_offer(lk, thr, v.z, j0 + 2, a.M);
            top8_offer(lk, thr, v.w, j0 + 3, a.M);
        }
        block_top8_store<kCorrThreads>(lk, w, gtop + static_cast<size_t>(slot) * kTop);
        __syncthreads();   // w is reused by the next row
    }
}

// ------------------------------------------------------------------ fixup (one CTA)
// After an admission, on operand half 0 (between steps the select kernel
// keeps the rows compact itself).  Rows 0..n-1 with n = *n_act + *n_extra;
// rows with done set leave.  Holes below the new count n' are filled, in
// order, with the surviving rows at or above n' (moving the slot id and the
// quantised GEMM row).
struct FixupArgs {
    int* n_act;
    int* n_extra;
    int* act;
    int* done;
    char* Rq;
    int ldq_bytes;
    int* holes;             // scratch, capacity rows
    int* surv;
};

__global__ void __launch_bounds__(kFixThreads) fixup_kernel(const FixupArgs a) {
    __shared__ int red[32];
    const int n = *a.n_act + *a.n_extra;
    if (n <= static_cast<int>(blockDim.x)) {
        // one row per thread: the flag stays in a register, one count and one
        // packed scan (holes in the low half, survivors in the high half)
        // place every move, and the lists live in shared memory
        __shared__ int sh_holes[kFixThreads], sh_surv[kFixThreads];
        const int p = threadIdx.x;
        const int f = p < n ? a.done[p] : 0;
        int cnt;
        block_scan_flag(p < n && f, red, &cnt);
        const int n_new = n - cnt;
        const int hole = p < n_new && f;
        const int sv = p >= n_new && p < n && !f;
        int tot;
        const int rk = block_scan_count(hole | (sv << 16), red, &tot);
        if (hole) sh_holes[rk & 0xffff] = p;
        if (sv) sh_surv[rk >> 16] = p;
        __syncthreads();
        const int nh = tot & 0xffff;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int k = warp; k < nh; k += blockDim.x >> 5) {
            const int ph = sh_holes[k], q = sh_surv[k];
            if (lane == 0) a.act[ph] = a.act[q];
            const uint4* src = reinterpret_cast<const uint4*>(a.Rq + static_cast<size_t>(q) * a.ldq_bytes);
            uint4* dst = reinterpret_cast<uint4*>(a.Rq + static_cast<size_t>(ph) * a.ldq_bytes);
            for (int o = lane; o < a.ldq_bytes / 16; o += 32) dst[o] = src[o];
        }
        if (p < n_new) a.done[p] = 0;
        if (threadIdx.x == 0) {
            *a.n_act = n_new;
            *a.n_extra = 0;
        }
        return;
    }
    int tot = 0, cnt = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int p = base + threadIdx.x;
        int t;
        block_scan_flag(p < n && a.done[p], red, &t);
        cnt += t;
    }
    const int n_new = n - cnt;
    int nh = 0;
    for (int base = 0; base < n_new; base += blockDim.x) {
        const int p = base + threadIdx.x;
        const int f = p < n_new && a.done[p];
        const int rk = block_scan_flag(f, red, &tot);
        if (f) a.holes[nh + rk] = p;
        nh += tot;
    }
    int ns = 0;
    for (int base = n_new; base < n; base += blockDim.x) {
        const int q = base + threadIdx.x;
        const int f = q < n && !a.done[q];
        const int rk = block_scan_flag(f, red, &tot);
        if (f) a.surv[ns + rk] = q;
        ns += tot;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k < nh; k += blockDim.x >> 5) {
        const int p = a.holes[k], q = a.surv[k];
        if (lane == 0) a.act[p] = a.act[q];
        const uint4* src = reinterpret_cast<const uint4*>(a.Rq + static_cast<size_t>(q) * a.ldq_bytes);
        uint4* dst = reinterpret_cast<uint4*>(a.Rq + static_cast<size_t>(p) * a.ldq_bytes);
        for (int o = lane; o < a.ldq_bytes / 16; o += 32) dst[o] = src[o];
    }
    // every remaining row is active: clear the flags (a filled hole still
    // holds its old flag, and the steps never write them, so the next
    // admission's fixup reads these rows as running)
    for (int k = threadIdx.x; k < n_new; k += blockDim.x) a.done[k] = 0;
    if (threadIdx.x == 0) {
        *a.n_act = n_new;
        *a.n_extra = 0;
    }
}

// ------------------------------------------------------------------ retire
// Copy the results of the slots that stopped since the last retire (x~ row
// and state, by slot) and their list to the caller's buffers (host-mapped
// memory in the server), so the host learns about them without a copy.
struct RetireArgs {
    const int* fin_count;
    const int* fin_list;
    const SlotState* st;
    const BatchIO* io;
    int M;
    float* out_x;           // slot s at out_x + s * M
    SlotState* out_state;   // by slot
    int* out_list;
    int* out_count;
};

__global__ void __launch_bounds__(kSelThreads) retire_kernel(const RetireArgs a) {
    const int n = *a.fin_count;
    const int k = blockIdx.x;
    if (k == 0 && threadIdx.x == 0) *a.out_count = n;
    if (k >= n) return;
    const int slot = a.fin_list[k];
    if (threadIdx.x == 0) {
        a.out_list[k] = slot;
        a.out_state[slot] = a.st[slot];
    }
    const float* x = a.io->X + static_cast<size_t>(slot) * a.io->ldx;
    float* o = a.out_x + static_cast<size_t>(slot) * a.M;
    for (int m = threadIdx.x; m < a.M; m += blockDim.x) o[m] = x[m];
}

// ------------------------------------------------------------------ host engine
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// rows x row_elems matrix (row stride row_elems elements); box = box_rows
// rows x 128 bytes, 128-byte swizzle (the UMMA K-major layout)
static mp_status make_map(CUtensorMap* map, void* base, bool fp8, long long rows, long long row_elems, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int esize = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(row_elems), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_elems * esize)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / esize), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return MP_OK;
}

// The same matrix as a 3-D view: K slices of 128 bytes (x), rows (y), slice
// index (z, stride 128 bytes); box = 128 rows x 2 slices, 128-byte swizzle.
// The box lands in shared memory as two slices of 128 rows one after the
// other, each in the layout of a 2-D box of make_map.
static mp_status make_map3(CUtensorMap* map, void* base, bool fp8, long long rows, long long row_elems) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int esize = fp8 ? 1 : 2;
    const long long ke = kRowBytes / esize;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(ke), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(row_elems / ke)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(row_elems * esize), static_cast<cuuint64_t>(kRowBytes)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(ke), static_cast<cuuint32_t>(kBM), 2u};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string(r) + ")");
    return MP_OK;
}

void engine_free(BatchEngine* e) {
    if (!e) return;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->graph_g) cudaGraphExecDestroy(e->graph_g);
    if (e->graph_gn) cudaGraphExecDestroy(e->graph_gn);
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    for (cudaEvent_t ev : e->cnt_ready)
        if (ev) cudaEventDestroy(ev);
    void* dev[] = {e->R32, e->Rq, e->st, e->act, e->counters, e->done, e->holes, e->surv, e->cand,
                   e->eps2, e->T, e->err, e->io, e->rscale, e->fin_list, e->Cg, e->gtop};
    for (void* p : dev) cudaFree(p);
    void* host[] = {e->h_st, e->h_cnt, e->h_eps2, e->h_T, e->h_io, e->h_err};
    for (void* p : host) cudaFreeHost(p);
    *e = BatchEngine();
}

void batch_destroy(BatchEngine* b) {
    engine_free(b);
    delete b;
}

size_t engine_slot_bytes(const PlanImpl* p, int prec, bool with_x, int gram_R) {
    const bool fp8 = prec == MP_PREC_FP8E4M3;
    const size_t TN = 128;   // the narrowest tile the shape choice may pick (most candidate lists)
    const size_t n_at = (p->M + TN - 1) / TN;
    const size_t gram = gram_R > 0 ? sizeof(float) * ((p->M + 3) / 4 * 4) + sizeof(unsigned long long) * kTop : 0;
    return sizeof(float) * p->ldN + 2 * (fp8 ? p->ldK8 : 2 * p->ldK16) + sizeof(uint2) * n_at * kTop +
           sizeof(SlotState) + 7 * sizeof(int) + sizeof(double) + sizeof(float) + (with_x ? sizeof(float) * p->M : 0) +
           gram;
}

mp_status autotune(PlanImpl* p, int prec, int B, const float* R_dev, cudaStream_t st, GemmShape* out, int lo_rows = 0);

mp_status batch_shape(PlanImpl* p, int prec, int B, const float* R, cudaStream_t st, GemmShape* shape, int lo_rows) {
    const int rt = (B + kBM - 1) / kBM;
    GemmShape g;
    g.tn = 256;
    g.tm = rt >= 2 ? 256 : 128;
    g.pair = p->batch_pair == 2 ? 1 : 0;
    if (g.pair) g.tm = 256;
    if (p->batch_autotune && !p->batch_tile_n && !p->batch_tile_m && p->batch_pair == 0) {
        mp_status s = autotune(p, prec, B, R, st, &g, lo_rows);
        if (s != MP_OK) return s;
    }
    if (p->batch_tile_n) g.tn = p->batch_tile_n;
    if (p->batch_tile_m && !g.pair) g.tm = p->batch_tile_m;
    *shape = g;
    return MP_OK;
}

static mp_status engine_prepare(PlanImpl* p, int prec, int cap, const GemmShape& g, int gram_R = 0,
                                int gram_below = 0) {
    BatchEngine* e = p->batch;
    if (e && e->prec == prec && e->cap >= cap && e->TM == g.tm && e->TN == g.tn && e->pair == g.pair &&
        e->gram_R == gram_R && e->gram_below == gram_below)
        return MP_OK;
    if (!e) e = p->batch = new BatchEngine();
    return engine_alloc(e, p, prec, std::max(cap, e->cap), g, gram_R, gram_below);
}

mp_status engine_alloc(BatchEngine* e, PlanImpl* p, int prec, int newcap, const GemmShape& g, int gram_R,
                       int gram_below) {
    engine_free(e);
    if (gram_R > 0 && !p->gram)
        return fail(MP_ERR_UNSUPPORTED, "batched Gram mode: the plan's Gram matrix is not built");
    if (gram_below < 0 || (gram_below > 0 && gram_R <= 0))
        return fail(MP_ERR_INVALID, "batched switched mode: needs a Gram period");
    const int TN = g.tn;
    if (g.pair ? g.tm != 256 : (g.tm != 128 && g.tm != 256)) return fail(MP_ERR_INVALID, "batched GEMM: unsupported tile shape");
    if (TN < 128 || TN > 256 || TN % 32)
        return fail(MP_ERR_INVALID, "batched GEMM: unsupported tile shape");
    e->pair = g.pair;
    e->gram_R = gram_R;
    e->gram_below = gram_below;
    e->cap = newcap;
    e->cap_pad = (newcap + kBM - 1) / kBM * kBM;
    e->prec = prec;
    e->TM = g.tm;
    e->TN = TN;
    e->n_at = (p->M + TN - 1) / TN;
    const bool fp8 = prec == MP_PREC_FP8E4M3;
    e->ldq = fp8 ? p->ldK8 : p->ldK16;
    const size_t qbytes = static_cast<size_t>(e->cap_pad) * e->ldq * (fp8 ? 1 : 2);
    const size_t C = static_cast<size_t>(e->cap);
    cudaError_t r = cudaSuccess;
    auto A = [&](auto** ptr, size_t b) {
        if (r != cudaSuccess) return;
        e->bytes += b;
        r = cudaMalloc(reinterpret_cast<void**>(ptr), b);
    };
    A(&e->R32, sizeof(float) * C * p->ldN);
    A(reinterpret_cast<char**>(&e->Rq), 2 * qbytes);
    A(&e->st, sizeof(SlotState) * C);
    A(&e->act, 2 * sizeof(int) * C);
    A(&e->counters, sizeof(int) * 8);
    A(&e->done, sizeof(int) * C);
    A(&e->holes, sizeof(int) * C);
    A(&e->surv, sizeof(int) * C);
    // room for the lists of half-width tiles (taken by the GEMM when few row
    // blocks are active)
    const bool half_ok = TN == 256 && !g.pair;
    const size_t n_at_max = half_ok ? (p->M + TN / 2 - 1) / (TN / 2) : e->n_at;
    A(&e->cand, sizeof(uint2) * C * n_at_max * kTop);
    A(&e->eps2, sizeof(double) * C);
    A(&e->T, sizeof(int) * C);
    A(&e->err, sizeof(int));
    A(&e->io, sizeof(BatchIO));
    A(&e->rscale, sizeof(float) * C);
    A(&e->fin_list, sizeof(int) * C);
    if (gram_R > 0) {
        e->ldC = (p->M + 3) / 4 * 4;
        A(&e->Cg, sizeof(float) * C * e->ldC);
        A(&e->gtop, sizeof(unsigned long long) * C * kTop);
        const int sm = corr_rows_per_cta(p) * p->ldN * static_cast<int>(sizeof(float));
        if (r == cudaSuccess && sm > 48 * 1024)
            r = cudaFuncSetAttribute(corr_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_st, sizeof(SlotState) * C);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_cnt, sizeof(int) * 8);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_eps2, sizeof(double) * C);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_T, sizeof(int) * C);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_io, sizeof(BatchIO));
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_err, sizeof(int));
    if (r == cudaSuccess) r = cudaMemset(e->Rq, 0, 2 * qbytes);
    if (r == cudaSuccess) r = cudaMemset(e->counters, 0, sizeof(int) * 8);
    if (r != cudaSuccess) {
        engine_free(e);
        return cuda_fail(r, "batched engine allocation");
    }
    mp_status s = make_map(&e->tmA, e->Rq, fp8, e->cap_pad, e->ldq, kBM);
    if (s == MP_OK) s = make_map(&e->tmA1, static_cast<char*>(e->Rq) + qbytes, fp8, e->cap_pad, e->ldq, kBM);
    if (s == MP_OK) s = make_map(&e->tmB, fp8 ? p->psi8 : p->psi16, fp8, p->M, e->ldq, TN);
    if (s == MP_OK) s = make_map(&e->tmBh, fp8 ? p->psi8 : p->psi16, fp8, p->M, e->ldq, half_ok ? TN / 2 : TN);
    if (s == MP_OK && g.pair) s = make_map(&e->tmBp, fp8 ? p->psi8 : p->psi16, fp8, p->M, e->ldq, TN / 2);
    if (s == MP_OK) s = make_map3(&e->tmA3, e->Rq, fp8, e->cap_pad, e->ldq);
    if (s == MP_OK) s = make_map3(&e->tmA1_3, static_cast<char*>(e->Rq) + qbytes, fp8, e->cap_pad, e->ldq);
    if (s == MP_OK) s = make_map3(&e->tmB3, fp8 ? p->psi8 : p->psi16, fp8, p->M, e->ldq);
    if (s != MP_OK) {
        engine_free(e);
        return s;
    }
    return MP_OK;
}

static CorrArgs corr_args(PlanImpl* p, BatchEngine* e) {
    const bool fp8 = e->prec == MP_PREC_FP8E4M3;
    CorrArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.n_act = e->counters;
    ca.TN = e->TN;
    ca.RM = e->TM / kBM;
    // two accumulator buffers (the epilogue of one tile overlaps the MMAs of
    // the next) when they fit in TMEM's 512 columns, else one
    const int nbuf = (ca.RM == 1 || 2 * ca.RM * e->TN <= 512 || e->pair) ? 2 : 1;
    ca.n_at = e->n_at;
    ca.half_ok = e->TN == 256 && !e->pair ? 1 : 0;
    ca.M = p->M;
    ca.nk = (fp8 ? p->ldK8 : p->ldK16 * 2) / kRowBytes;
    ca.fp8 = fp8 ? 1 : 0;
    // allocations are powers of two >= 32; a two-SM tile keeps 128 rows x TN
    // columns per SM, two buffers
    const int cols = e->pair ? 2 * e->TN : nbuf * ca.RM * e->TN;
    ca.tmem_cols = cols > 256 ? 512 : (cols > 128 ? 256 : 128);
    ca.stages = e->pair ? corr_stages(kBM, e->TN / 2) : corr_stages(e->TM, e->TN);
    ca.colscale = p->scale8;
    ca.ks2_ok = e->pair ? 0 : 1;
    ca.cand = e->cand;
    ca.watchdog_ns = static_cast<unsigned long long>(p->watchdog_ns);
    ca.err = e->err;
    return ca;
}

// The step's GEMM on operand half `half` (single-CTA or two-SM tiles).
static cudaError_t launch_gemm(const BatchEngine* e, const CorrArgs& ca, int half, int max_rows, cudaStream_t st) {
    const CUtensorMap& tA = half ? e->tmA1 : e->tmA;
    if (e->pair) return launch_corr_pair(tA, e->tmBp, ca, max_rows, st);
    return launch_corr_top8(tA, e->tmB, e->tmBh, half ? e->tmA1_3 : e->tmA3, e->tmB3, ca, max_rows, st);
}

static cudaError_t launch_fixup(PlanImpl* p, BatchEngine* e, cudaStream_t st) {
    FixupArgs fa;
    fa.n_act = e->counters;
    fa.n_extra = e->counters + 1;
    fa.act = e->act;
    fa.done = e->done;
    fa.Rq = static_cast<char*>(e->Rq);
    fa.ldq_bytes = e->ldq * (e->prec == MP_PREC_FP8E4M3 ? 1 : 2);
    fa.holes = e->holes;
    fa.surv = e->surv;
    fixup_kernel<<<1, kFixThreads, 0, st>>>(fa);
    p->launches++;
    return cudaGetLastError();
}

// Gram-step kernel's dynamic shared memory: r, and with `rows` the slot's
// correlation row and a row of G.
static size_t gram_smem_bytes(const PlanImpl* p, const BatchEngine* e, bool rows) {
    return sizeof(float) * (static_cast<size_t>(p->ldN) + (rows ? 2 * static_cast<size_t>(e->ldC) : 0));
}
static bool gram_rows_in_smem(const PlanImpl* p, const BatchEngine* e) {
    return gram_smem_bytes(p, e, true) <= 200u * 1024u;
}
// threads per Gram-step CTA: 256 when the rows are staged in shared memory
// and two such CTAs fit in an SM's (with the static part and the per-CTA
// reserve), else 512: rows read from global memory are long, and 12 warps
// on each row's update beat a second CTA (measured on M = 32768)
static int gram_cta(const PlanImpl* p, const BatchEngine* e) {
    if (!gram_rows_in_smem(p, e)) return 512;
    const size_t per_cta = gram_smem_bytes(p, e, true) + 4096u;
    return 2u * per_cta <= static_cast<size_t>(p->smem_per_sm) ? 256 : 512;
}

// One step on operand half `half`: GEMM + top-8, then select / rescore /
// update, which moves the signals that run on into the other half.  In the
// Gram mode a step is the select kernel alone: its candidates are each
// slot's carried top 8, and it updates the slot's correlation row from G.
// Adds the kernels launched to *kernels.
// gram: a Gram-updated step (select kernel only) instead of a direct one
// (GEMM, then select)
static cudaError_t launch_step(PlanImpl* p, BatchEngine* e, int half, bool gram, cudaStream_t st, int* kernels) {
    int* fin_count = e->counters + 2;
    int* fin_list = e->fin_list;
    int* cnt[2] = {e->counters, e->counters + 3};
    const size_t qbytes = static_cast<size_t>(e->cap_pad) * e->ldq * (e->prec == MP_PREC_FP8E4M3 ? 1 : 2);
    cudaError_t r = cudaSuccess;
    if (!gram) {
        CorrArgs ca = corr_args(p, e);
        ca.n_act = cnt[half];
        ca.zero_next = cnt[1 - half];
        ca.n_at_out = e->counters + 4;
        r = launch_gemm(e, ca, half, e->cap_pad, st);
        ++*kernels;
    }
    if (r != cudaSuccess) return r;
    SelArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.n_act = cnt[half];
    sa.act = e->act + static_cast<size_t>(half) * e->cap;
    sa.n_next = cnt[1 - half];
    sa.act_next = e->act + static_cast<size_t>(1 - half) * e->cap;
    sa.Rq_next = static_cast<char*>(e->Rq) + (1 - half) * qbytes;
    sa.cand = e->cand;
    sa.n_at = e->counters + 4;   // written by the step's GEMM
    sa.psi32 = p->psi32;
    sa.ldN = p->ldN;
    sa.N = p->N;
    sa.M = p->M;
    sa.R32 = e->R32;
    sa.io = e->io;
    sa.st = e->st;
    sa.ldq = e->ldq;
    sa.fp8 = e->prec == MP_PREC_FP8E4M3 ? 1 : 0;
    sa.fin_count = fin_count;
    sa.fin_list = fin_list;
    sa.Cg = e->Cg;
    sa.ldC = e->ldC;
    sa.G = p->gram;
    sa.ldG = p->ldG;
    sa.gtop = e->gtop;
    // in the Gram mode a select step follows a select step with no GEMM
    // between them to clear the count its survivors append to: each select
    // kernel clears the count it read once all its CTAs have read it
    sa.n_act_w = cnt[half];
    sa.done_ctr = gram ? e->counters + 5 : nullptr;
    // direct step, small engines: 8 warps, each rescoring one candidate
    // with 16 loads per lane in flight (with few signals the rescore is a
    // latency chain of L2 / HBM reads); engines of 512 slots and more: 4
    // warps, two candidates each, so more signals' CTAs fit on an SM at a
    // full batch.  Gram mode: the Gram-step kernel (8 or 16 warps per CTA,
    // gram_cta).
    sa.err = e->err;
    sa.lim = static_cast<unsigned long long>(p->watchdog_ns);
    const size_t sm = p->ldN * sizeof(float);
    if (gram) {
        const int cta = gram_cta(p, e);
        const int per_sm = kGramThreads / cta;
        const int ctas = std::max(1, std::min(e->cap, p->sm_count > 0 ? per_sm * p->sm_count : e->cap));
        const bool rows_sm = gram_rows_in_smem(p, e);
        const size_t gsm = gram_smem_bytes(p, e, rows_sm);
        if (cta == 256) {
            if (rows_sm) gram_select_kernel<true, 256><<<ctas, 256, gsm, st>>>(sa);
            else gram_select_kernel<false, 256><<<ctas, 256, gsm, st>>>(sa);
        } else {
            if (rows_sm) gram_select_kernel<true, 512><<<ctas, 512, gsm, st>>>(sa);
            else gram_select_kernel<false, 512><<<ctas, 512, gsm, st>>>(sa);
        }
    } else if (e->cap < kWideSelectCap) select_update_kernel<2 * kSumChains><<<e->cap, 2 * kSumChains, sm, st>>>(sa);
    else select_update_kernel<kSumChains><<<e->cap, kSumChains, sm, st>>>(sa);
    ++*kernels;
    return cudaGetLastError();
}

// Gram mode: direct FP32 correlations and their top 8 for listed slots
// (rows == NULL: slots 0..n_max-1; n_ptr: the device's row count; R > 0:
// only the slots whose step count is a positive multiple of R).  `tiled`:
// the listed rows are all due together (R = 0, or one shared step count),
// so the register-tiled GEMM computes them; otherwise (a server's slots at
// different steps) the row-group kernel looks at each row's own count.
static cudaError_t launch_gram_refresh(PlanImpl* p, BatchEngine* e, const int* rows, const int* n_ptr, int n_max, int R,
                                       bool tiled, cudaStream_t st, int* kernels) {
    if (n_max <= 0) return cudaSuccess;
    CorrRowsArgs a;
    a.psi32 = p->psi32;
    a.ldN = p->ldN;
    a.M = p->M;
    a.R32 = e->R32;
    a.rows = rows;
    a.n_ptr = n_ptr;
    a.n = n_max;
    a.st = e->st;
    a.R = R;
    a.Cg = e->Cg;
    a.ldC = e->ldC;
    // a host-known row count (admission) stages no more rows than listed:
    // less shared memory per CTA, more CTAs per SM, more loads in flight
    a.rpc = n_ptr ? corr_rows_per_cta(p) : std::min(corr_rows_per_cta(p), n_max);
    // one CTA per block of atoms (each runs over the row groups); the scan
    // at most two CTAs per SM over the rows
    const int sms = p->sm_count > 0 ? p->sm_count : 132;
    if (tiled)
        corr_tile_kernel<<<dim3((p->M + kTileC - 1) / kTileC, (n_max + kTileC - 1) / kTileC), 256, 0, st>>>(a);
    else
        corr_rows_kernel<<<(p->M + kCorrAtoms - 1) / kCorrAtoms, kCorrThreads,
                           static_cast<size_t>(a.rpc) * p->ldN * sizeof(float), st>>>(a);
    gram_scan_kernel<<<std::min(n_max, 2 * sms), kCorrThreads, 0, st>>>(a, e->gtop);
    *kernels += 2;
    return cudaGetLastError();
}

// Capture `steps` steps of one kind (direct or Gram-updated), optionally
// followed by the retire copy, and instantiate them into *out.
static mp_status capture_steps(PlanImpl* p, BatchEngine* e, int steps, bool gram, bool retire, float* out_x,
                               SlotState* out_state, int* out_list, int* out_count, cudaGraphExec_t* out,
                               int* out_kernels, bool refresh = true) {
    MP_CUDA_TRY(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t r = cudaSuccess;
    int kernels = 0;
    // Gram steps: a replay starts with every active slot's step count a
    // multiple of `steps` (signals join between replays and each step moves
    // every active signal by one); the slots at a multiple of the period get
    // their correlations recomputed directly.  A batched decode's active
    // signals have all taken the same number of steps (they start together),
    // a server's (retire) have not; a small batch's refreshes stay with the
    // row-group kernel (a 128-row tile would compute mostly padding).
    if (gram && refresh)
        r = launch_gram_refresh(p, e, e->act, e->counters, e->cap, e->gram_R, !retire && e->cap >= kTiledMinRows,
                                e->cap_stream, &kernels);
    for (int s = 0; s < steps && r == cudaSuccess; ++s) r = launch_step(p, e, s & 1, gram, e->cap_stream, &kernels);
    if (retire && r == cudaSuccess) {
        RetireArgs ra;
        ra.fin_count = e->counters + 2;
        ra.fin_list = e->fin_list;
        ra.st = e->st;
        ra.io = e->io;
        ra.M = p->M;
        ra.out_x = out_x;
        ra.out_state = out_state;
        ra.out_list = out_list;
        ra.out_count = out_count;
        retire_kernel<<<e->cap, kSelThreads, 0, e->cap_stream>>>(ra);
        ++kernels;
        r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaMemsetAsync(e->counters + 2, 0, sizeof(int), e->cap_stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t r2 = cudaStreamEndCapture(e->cap_stream, &g);
    if (r != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(r, "batched step capture");
    }
    if (r2 != cudaSuccess) return cuda_fail(r2, "cudaStreamEndCapture");
    r = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (r != cudaSuccess) return cuda_fail(r, "cudaGraphInstantiate");
    *out_kernels = kernels;
    return MP_OK;
}

mp_status engine_build_graph(PlanImpl* p, BatchEngine* e, int steps, bool retire, float* out_x, SlotState* out_state,
                             int* out_list, int* out_count) {
    if (steps <= 0 || steps % 2) return fail(MP_ERR_INVALID, "batched step graph: an even number of steps");
    if (e->graph && e->graph_steps == steps && e->graph_retire == retire) return MP_OK;
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    if (e->graph_g) {
        cudaGraphExecDestroy(e->graph_g);
        e->graph_g = nullptr;
    }
    if (e->graph_gn) {
        cudaGraphExecDestroy(e->graph_gn);
        e->graph_gn = nullptr;
    }
    if (e->gram_below > 0 && retire)
        return fail(MP_ERR_UNSUPPORTED, "batched step graph: the switched mode has no retiring graph");
    if (!e->cap_stream) MP_CUDA_TRY(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
    MP_CUDA_TRY(corr_prepare());
    MP_CUDA_TRY(pair_prepare());
    if (p->ldN * 4 > 48 * 1024) {
        const int b = p->ldN * 4;
        MP_CUDA_TRY(cudaFuncSetAttribute(select_update_kernel<2 * kSumChains>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MP_CUDA_TRY(cudaFuncSetAttribute(select_update_kernel<kSumChains>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, b));

    }
    if (e->gram_R > 0) {
        // only the variant launch_step will take (rows in shared memory
        // when they fit; a long row may not fit any CTA's shared memory)
        const bool rows_sm = gram_rows_in_smem(p, e);
        const int gsm = static_cast<int>(gram_smem_bytes(p, e, rows_sm));
        const bool two = gram_cta(p, e) == 256;
        MP_CUDA_TRY(cudaFuncSetAttribute(rows_sm ? (two ? gram_select_kernel<true, 256> : gram_select_kernel<true, 512>)
                                                 : (two ? gram_select_kernel<false, 256> : gram_select_kernel<false, 512>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, gsm));
    }
    if (e->gram_R > 0 && (e->gram_R % steps || !p->gram))
        return fail(MP_ERR_INVALID, "batched step graph: the Gram period must be a multiple of the steps per graph");
    // the main graph: Gram steps in the Gram mode, direct steps otherwise
    // (the switched mode starts direct); the switched mode's Gram steps in
    // a second graph
    const bool gram_main = e->gram_R > 0 && e->gram_below == 0;
    mp_status s = capture_steps(p, e, steps, gram_main, retire, out_x, out_state, out_list, out_count, &e->graph,
                                &e->graph_kernels);
    if (s == MP_OK && e->gram_below > 0)
        s = capture_steps(p, e, steps, true, false, nullptr, nullptr, nullptr, nullptr, &e->graph_g,
                          &e->graph_g_kernels);
    // a batched decode's Gram steps without the refresh (replays that do not
    // start at a multiple of the period)
    if (s == MP_OK && e->gram_R > 0 && !retire)
        s = capture_steps(p, e, steps, true, false, nullptr, nullptr, nullptr, nullptr, &e->graph_gn,
                          &e->graph_gn_kernels, false);
    if (s != MP_OK) {
        for (cudaGraphExec_t* gp : {&e->graph, &e->graph_g, &e->graph_gn})
            if (*gp) {
                cudaGraphExecDestroy(*gp);
                *gp = nullptr;
            }
        return s;
    }
    e->graph_steps = steps;
    e->graph_retire = retire;
    return MP_OK;
}

static AdmitArgs admit_args(PlanImpl* p, BatchEngine* e, const float* Y, int n_new, const int* slots) {
    AdmitArgs aa;
    aa.Y = Y;
    aa.n_new = n_new;
    aa.N = p->N;
    aa.ldN = p->ldN;
    aa.M = p->M;
    aa.slots = slots;
    aa.eps2 = e->eps2;
    aa.T = e->T;
    aa.R32 = e->R32;
    aa.io = e->io;
    aa.st = e->st;
    aa.Rq = e->Rq;
    aa.ldq = e->ldq;
    aa.fp8 = e->prec == MP_PREC_FP8E4M3 ? 1 : 0;
    aa.rscale = nullptr;
    aa.act = e->act;
    aa.done = e->done;
    aa.n_act = e->counters;
    aa.n_extra = e->counters + 1;
    aa.fin_count = e->counters + 2;
    aa.fin_list = e->fin_list;
    return aa;
}

cudaError_t engine_admit(PlanImpl* p, BatchEngine* e, const float* Y, int n, const int* slots_dev, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    admit_kernel<<<n, kSelThreads, 0, st>>>(admit_args(p, e, Y, n, slots_dev));
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    p->launches++;
    if (e->gram_R > 0 && e->gram_below == 0) {
        // the Gram mode starts every signal from its direct FP32 correlations
        // (the switched mode computes them when it switches)
        int k = 0;
        r = launch_gram_refresh(p, e, slots_dev, nullptr, n, 0, n >= kTiledMinRows, st, &k);
        p->launches += k;
        if (r != cudaSuccess) return r;
    }
    return launch_fixup(p, e, st);
}

static mp_status batched_run(PlanImpl* p, int prec, const float* Y, float* X, long long ldx, int B, const mp_stop* stops,
                             int n_stops, const mp_trace* trace, mp_result* out, cudaStream_t st) {
    GemmShape g;
    // the switched mode's GEMMs see more than the threshold's active rows
    const int sw = p->batch_gram > 0 ? p->batch_gram_below : 0;
    mp_status s = batch_shape(p, prec, B, Y, st, &g, sw > 0 && B > sw ? sw + 1 : 0);
    if (s != MP_OK) return s;
    if (p->batch_gram > 0) {
        // Gram steps use the FP32 atoms only (the precision's copy serves the
        // switched mode's direct steps and the operand rows)
        s = gram_prepare(p, st);
        if (s != MP_OK) return s;
    }
    const int gram_below = p->batch_gram > 0 ? p->batch_gram_below : 0;
    s = engine_prepare(p, prec, B, g, p->batch_gram, gram_below);
    if (s != MP_OK) return s;
    BatchEngine* e = p->batch;
    s = engine_build_graph(p, e, kStepsPerGraph, false, nullptr, nullptr, nullptr, nullptr);
    if (s != MP_OK) return s;
    int maxT = 0;
    for (int b = 0; b < B; ++b) {
        const mp_stop& sb = stops[n_stops == 1 ? 0 : b];
        e->h_eps2[b] = sb.eps * sb.eps;
        e->h_T[b] = sb.max_iters;
        maxT = std::max(maxT, sb.max_iters);
    }
    BatchIO io;
    std::memset(&io, 0, sizeof(io));
    io.X = X;
    io.ldx = ldx;
    if (trace) {
        io.tr_atoms = trace->atoms;
        io.tr_coefs = trace->coefs;
        io.tr_energy = trace->energies;
        io.tr_cap = std::max(0, trace->capacity);
    }
    *e->h_io = io;
    MP_CUDA_TRY(cudaMemcpyAsync(e->eps2, e->h_eps2, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->T, e->h_T, sizeof(int) * B, cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->io, e->h_io, sizeof(BatchIO), cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemsetAsync(e->err, 0, sizeof(int), st));
    MP_CUDA_TRY(cudaMemsetAsync(e->counters, 0, sizeof(int) * 8, st));
    // signal b -> slot b, GEMM row b; then drop those that need no iteration
    MP_CUDA_TRY(engine_admit(p, e, Y, B, nullptr, st));
    // Switched mode: from direct steps to Gram-updated ones.  Between
    // replays the active rows are half 0's (count counters[0]); every active
    // signal gets its correlations computed directly from the FP32 atoms
    // (and its 8 largest), and the count the first Gram step's survivors
    // append to (half 1's, left over from the last direct step, which a GEMM
    // would have cleared) is cleared.
    bool gram_steps = false;
    // n_rows: the active count last seen (at least the count at the switch)
    auto switch_to_gram = [&](int n_rows) -> mp_status {
        MP_CUDA_TRY(cudaMemsetAsync(e->counters + 3, 0, sizeof(int), st));
        int k = 0;
        MP_CUDA_TRY(launch_gram_refresh(p, e, e->act, e->counters, e->cap, 0, n_rows >= kTiledMinRows, st, &k));
        p->launches += k;
        gram_steps = true;
        return MP_OK;
    };
    // a batch no larger than the threshold starts with Gram steps
    if (gram_below > 0 && B <= gram_below) {
        s = switch_to_gram(B);
        if (s != MP_OK) return s;
    }
    // replay the captured steps until no signal is active (each step moves
    // every active signal by one iteration, so maxT steps always suffice).
    // Replay k is queued before the active count after replay k - 1 is
    // known, so the GPU never waits for the host's read; the replay queued
    // after the last signal stopped runs empty steps (every CTA exits at once)
    for (int j = 0; j < 2; ++j)
        if (!e->cnt_ready[j]) MP_CUDA_TRY(cudaEventCreateWithFlags(&e->cnt_ready[j], cudaEventDisableTiming));
    const long long max_replays = (static_cast<long long>(maxT) + kStepsPerGraph - 1) / kStepsPerGraph + 1;
    // every active signal has taken kStepsPerGraph * k steps when replay k
    // starts; a Gram replay refreshes them only when that is a positive
    // multiple of the period, and runs without the refresh launches otherwise
    const bool pure_gram = e->gram_R > 0 && gram_below == 0;
    for (long long k = 0; k < max_replays; ++k) {
        cudaGraphExec_t g = e->graph;
        int gk = e->graph_kernels;
        if (pure_gram || gram_steps) {
            const long long t0 = static_cast<long long>(kStepsPerGraph) * k;
            if (t0 > 0 && t0 % e->gram_R == 0) {
                if (gram_steps) {
                    g = e->graph_g;
                    gk = e->graph_g_kernels;
                }
            } else {
                g = e->graph_gn;
                gk = e->graph_gn_kernels;
            }
        }
        MP_CUDA_TRY(cudaGraphLaunch(g, st));
        p->launches += gk;
        MP_CUDA_TRY(cudaMemcpyAsync(e->h_cnt + (k & 1), e->counters, sizeof(int), cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaEventRecord(e->cnt_ready[k & 1], st));
        if (k > 0) {
            MP_CUDA_TRY(cudaEventSynchronize(e->cnt_ready[(k - 1) & 1]));
            const int n_left = e->h_cnt[(k - 1) & 1];
            if (n_left == 0) break;
            // the count after replay k - 1 reached the threshold: switch
            // after replay k (already queued; it holds at most that many)
            if (gram_below > 0 && !gram_steps && n_left <= gram_below) {
                s = switch_to_gram(n_left);
                if (s != MP_OK) return s;
            }
        }
    }
    // each signal's final FP32 residual (slot b = signal b), for callers that
    // check the drift of this path's own arithmetic
    if (trace && trace->residual)
        MP_CUDA_TRY(cudaMemcpy2DAsync(trace->residual, sizeof(float) * p->N, e->R32, sizeof(float) * p->ldN,
                                      sizeof(float) * p->N, B, cudaMemcpyDeviceToDevice, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->h_st, e->st, sizeof(SlotState) * B, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->h_err, e->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    mp_status worst = MP_OK;
    for (int b = 0; b < B; ++b) {
        const SlotState& ss = e->h_st[b];
        mp_result& o = out[b];
        std::memset(&o, 0, sizeof(o));
        o.iters = ss.t;
        o.stop_reason = ss.stop_reason;
        o.status = *e->h_err ? *e->h_err : ss.status;
        o.rel_residual = ss.e0 > 0.0 ? std::sqrt(ss.e / ss.e0) : 0.0;
        o.energy_audit_max = ss.e0 > 0.0 ? ss.audit / ss.e0 : 0.0;
        if (o.status < 0 && worst == MP_OK) worst = static_cast<mp_status>(o.status);
    }
    if (worst == MP_ERR_TIMEOUT) set_error("a device-side wait in the batched step exceeded the watchdog limit");
    else if (worst == MP_ERR_NONFINITE) set_error("a signal has a non-finite entry");
    return worst;
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

mp_status mp_recover_batched(mp_plan_t plan, int prec, const float* Y, float* X, int B, const mp_stop* stops,
                             int n_stops, const mp_trace* trace, mp_result* host_out, void* stream) {
    clear_error();
    if (!plan || !Y || !X || !stops || !host_out) return fail(MP_ERR_INVALID, "mp_recover_batched: NULL argument");
    if (B < 0) return fail(MP_ERR_INVALID, "mp_recover_batched: B < 0");
    if (n_stops != 1 && n_stops != B) return fail(MP_ERR_INVALID, "mp_recover_batched: n_stops must be 1 or B");
    for (int i = 0; i < n_stops; ++i)
        if (!(stops[i].eps >= 0.0) || !std::isfinite(stops[i].eps) || stops[i].max_iters < 0 || stops[i].reserved)
            return fail(MP_ERR_INVALID, "mp_recover_batched: bad stop entry " + std::to_string(i));
    PlanImpl* p = &plan->impl;
    if (prec == MP_PREC_FP64)
        return fail(MP_ERR_UNSUPPORTED, "mp_recover_batched: FP64 decodes run one signal at a time (mp_recover_f64)");
    if (prec != MP_PREC_FP32 && prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_recover_batched: unknown precision");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_recover_batched: the plan holds no copy for this precision");
    if (B == 0) return MP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == MP_PREC_FP32) {
        mp_status worst = MP_OK;
        for (int b = 0; b < B; ++b) {
            const mp_stop* sb = &stops[n_stops == 1 ? 0 : b];
            mp_trace tb;
            const mp_trace* tp = nullptr;
            if (trace) {
                tb = *trace;
                const size_t off = static_cast<size_t>(b) * std::max(0, trace->capacity);
                tb.atoms = trace->atoms ? trace->atoms + off : nullptr;
                tb.coefs = trace->coefs ? trace->coefs + off : nullptr;
                tb.energies = trace->energies ? trace->energies + off : nullptr;
                tb.residual = trace->residual ? trace->residual + static_cast<size_t>(b) * p->N : nullptr;
                tp = &tb;
            }
            mp_status s = mp_recover(plan, Y + static_cast<size_t>(b) * p->N, X + static_cast<size_t>(b) * p->M, sb, tp,
                                     &host_out[b], stream);
            if (s < 0 && worst == MP_OK) worst = s;
        }
        return worst;
    }
    return batched_run(p, prec, Y, X, p->M, B, stops, n_stops, trace, host_out, st);
}

mp_status mp_debug_correlations(mp_plan_t plan, int prec, const float* R, int B, float* C, void* stream) {
    clear_error();
    if (!plan || !R || !C || B < 1) return fail(MP_ERR_INVALID, "mp_debug_correlations: bad argument");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_debug_correlations: precision must be BF16 or FP8");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_debug_correlations: the plan holds no copy for this precision");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GemmShape g;
    mp_status s = batch_shape(p, prec, B, R, st, &g);
    if (s != MP_OK) return s;
    s = engine_prepare(p, prec, B, g);
    if (s != MP_OK) return s;
    BatchEngine* e = p->batch;
    MP_CUDA_TRY(corr_prepare());
    MP_CUDA_TRY(pair_prepare());
    for (int b = 0; b < B; ++b) {
        e->h_eps2[b] = 0.0;
        e->h_T[b] = 1;
    }
    BatchIO io;
    std::memset(&io, 0, sizeof(io));
    *e->h_io = io;
    MP_CUDA_TRY(cudaMemcpyAsync(e->eps2, e->h_eps2, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->T, e->h_T, sizeof(int) * B, cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemcpyAsync(e->io, e->h_io, sizeof(BatchIO), cudaMemcpyHostToDevice, st));
    MP_CUDA_TRY(cudaMemsetAsync(e->err, 0, sizeof(int), st));
    MP_CUDA_TRY(cudaMemsetAsync(e->counters, 0, sizeof(int) * 8, st));
    // rows 0..B-1 hold R (quantised); the row count is set directly so that
    // zero rows are kept too
    AdmitArgs aa = admit_args(p, e, R, B, nullptr);
    aa.rscale = e->rscale;
    admit_kernel<<<B, kSelThreads, 0, st>>>(aa);
    MP_CUDA_TRY(cudaMemcpyAsync(e->counters, &B, sizeof(int), cudaMemcpyHostToDevice, st));
    CorrArgs ca = corr_args(p, e);
    ca.dump = C;
    ca.rscale = e->rscale;
    MP_CUDA_TRY(launch_gemm(e, ca, 0, B, st));
    p->launches += 2;
    MP_CUDA_TRY(cudaMemcpyAsync(e->h_err, e->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (*e->h_err) return fail(static_cast<mp_status>(*e->h_err), "mp_debug_correlations: device wait timed out");
    return MP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace mpgb {

// Deterministic pseudo-random rows in [-1, 1) (splitmix-style hash of the
// element index): stand-in residuals for timing the GEMM.
__global__ void fill_rows_kernel(float* R, int B, int N, unsigned seed) {
    const size_t n = static_cast<size_t>(B) * N;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull + seed;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        R[i] = static_cast<float>(static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

static int batch_bucket(int B) {
    int b = 128;
    while (b < B) b *= 2;
    return b;
}

// Time the correlation GEMM for B active rows with tile shape g: mean of
// `reps` launches after 2 warm-up launches; returns microseconds per launch
// (or a negative value on failure).
static double time_gemm(PlanImpl* p, int prec, int B, const GemmShape& g, const float* R, cudaStream_t st,
                        int reps = 5) {
    BatchEngine e;
    double us = -1.0;
    if (engine_alloc(&e, p, prec, B, g) == MP_OK && corr_prepare() == cudaSuccess && pair_prepare() == cudaSuccess) {
        for (int b = 0; b < B; ++b) {
            e.h_eps2[b] = 0.0;
            e.h_T[b] = 1;
        }
        BatchIO io;
        std::memset(&io, 0, sizeof(io));
        *e.h_io = io;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t r = cudaMemcpyAsync(e.eps2, e.h_eps2, sizeof(double) * B, cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaMemcpyAsync(e.T, e.h_T, sizeof(int) * B, cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaMemcpyAsync(e.io, e.h_io, sizeof(BatchIO), cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaMemsetAsync(e.counters, 0, sizeof(int) * 8, st);
        if (r == cudaSuccess) {
            admit_kernel<<<B, kSelThreads, 0, st>>>(admit_args(p, &e, R, B, nullptr));
            r = cudaGetLastError();
        }
        if (r == cudaSuccess) r = cudaMemcpyAsync(e.counters, &B, sizeof(int), cudaMemcpyHostToDevice, st);
        if (r == cudaSuccess) r = cudaEventCreate(&e0);
        if (r == cudaSuccess) r = cudaEventCreate(&e1);
        const CorrArgs ca = corr_args(p, &e);
        for (int it = 0; it < 2 && r == cudaSuccess; ++it) r = launch_gemm(&e, ca, 0, B, st);
        if (r == cudaSuccess) r = cudaEventRecord(e0, st);
        for (int it = 0; it < reps && r == cudaSuccess; ++it) r = launch_gemm(&e, ca, 0, B, st);
        if (r == cudaSuccess) r = cudaEventRecord(e1, st);
        if (r == cudaSuccess) r = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (r == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) us = 1e3 * ms / reps;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(st);
        cudaGetLastError();
        p->launches += 2 + reps + 1;
    }
    engine_free(&e);
    return us;
}

mp_status autotune(PlanImpl* p, int prec, int B, const float* R_dev, cudaStream_t st, GemmShape* out, int lo_rows) {
    const int bucket = batch_bucket(B);
    const int lo = lo_rows > 0 ? std::min(lo_rows, B) : 0;
    for (const TuneEntry& t : p->tuned)
        if (t.prec == prec && t.bucket == bucket && t.lo == lo) {
            *out = t.shape;
            return MP_OK;
        }
    float* R = nullptr;
    if (!R_dev) {
        MP_CUDA_TRY(cudaMallocAsync(&R, sizeof(float) * static_cast<size_t>(B) * p->N, st));
        fill_rows_kernel<<<256, 256, 0, st>>>(R, B, p->N, 12345u);
        MP_CUDA_TRY(cudaGetLastError());
        p->launches++;
    }
    double best = -1.0;
    GemmShape best_g;
    const int rt = (B + kBM - 1) / kBM;
    // a shape is timed on the full batch and on a quarter of it: a batch
    // drains as its signals stop, and a shape that only wins when full can
    // lose the decode (a decode that switches to Gram steps below a count
    // runs no GEMM under it: the shapes are timed at that count instead)
    const int Bq = lo > 0 ? lo : std::max(1, B / 4);
    auto consider = [&](const GemmShape& g) {
        const double u1 = time_gemm(p, prec, B, g, R_dev ? R_dev : R, st);
        const double u2 = u1 > 0.0 ? time_gemm(p, prec, Bq, g, R_dev ? R_dev : R, st) : -1.0;
        const double us = u2 > 0.0 ? u1 + u2 : -1.0;
        if (us > 0.0 && (best < 0.0 || us < best)) {
            best = us;
            best_g = g;
        }
    };
    for (int tm : {128, 256}) {
        if (tm == 256 && rt < 2) continue;      // one row block: the same work as 128
        for (int tn : {256, 224, 128}) {
            GemmShape g;
            g.tm = tm;
            g.tn = tn;
            consider(g);
        }
    }
    // two-SM tiles, unless switched off: widths that spread the tiles over
    // the clusters in whole rounds differently
    if (rt >= 2 && p->batch_pair != 1)
        for (int tn : {256, 224, 192}) {
            GemmShape g;
            g.tm = 256;
            g.tn = tn;
            g.pair = 1;
            consider(g);
        }
    if (R) cudaFreeAsync(R, st);
    if (best < 0.0) return fail(MP_ERR_CUDA, "autotune: no tile shape could be timed");
    cudaStreamSynchronize(st);
    p->tuned.push_back(TuneEntry{prec, bucket, best_g, best, lo});
    *out = best_g;
    return MP_OK;
}

}  // namespace mpgb

extern "C" {

mp_status mp_plan_autotune_shape(mp_plan_t plan, int prec, int B, int* tile_n, int* tile_m, int* pair) {
    clear_error();
    if (!plan || B < 1) return fail(MP_ERR_INVALID, "mp_plan_autotune: bad argument");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_plan_autotune: precision must be BF16 or FP8");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_plan_autotune: the plan holds no copy for this precision");
    MP_CUDA_TRY(corr_prepare());
    MP_CUDA_TRY(pair_prepare());
    GemmShape g;
    mp_status s = autotune(p, prec, B, nullptr, nullptr, &g);
    if (s != MP_OK) return s;
    if (tile_n) *tile_n = g.tn;
    if (tile_m) *tile_m = g.tm;
    if (pair) *pair = g.pair;
    return MP_OK;
}

mp_status mp_plan_autotune(mp_plan_t plan, int prec, int B, int* tile_n, int* tile_m) {
    return mp_plan_autotune_shape(plan, prec, B, tile_n, tile_m, nullptr);
}

mp_status mp_debug_time_gemm(mp_plan_t plan, int prec, int B, int tile_m, int tile_n, int reps,
                             double* us) {
    return mp_debug_time_gemm_pair(plan, prec, B, tile_m, tile_n, 0, reps, us);
}

mp_status mp_debug_time_gemm_pair(mp_plan_t plan, int prec, int B, int tile_m, int tile_n, int pair, int reps,
                                  double* us) {
    clear_error();
    if (!plan || B < 1 || reps < 1 || !us) return fail(MP_ERR_INVALID, "mp_debug_time_gemm: bad argument");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_debug_time_gemm: precision must be BF16 or FP8");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_debug_time_gemm: the plan holds no copy for this precision");
    GemmShape g;
    if (tile_m || tile_n || pair) {
        const bool tn_ok = tile_n >= 128 && tile_n <= 256 && tile_n % 32 == 0;
        const bool ok = tn_ok && (pair == 1 ? tile_m == 256 : (pair == 0 && (tile_m == 128 || tile_m == 256)));
        if (!ok) return fail(MP_ERR_INVALID, "mp_debug_time_gemm: bad tile shape");
        g.tm = tile_m;
        g.tn = tile_n;
        g.pair = pair;
    } else {
        mp_status s = batch_shape(p, prec, B, nullptr, nullptr, &g);
        if (s != MP_OK) return s;
    }
    float* R = nullptr;
    MP_CUDA_TRY(cudaMalloc(&R, sizeof(float) * static_cast<size_t>(B) * p->N));
    fill_rows_kernel<<<256, 256>>>(R, B, p->N, 12345u);
    p->launches++;
    cudaError_t r = cudaGetLastError();
    const double t = r == cudaSuccess ? time_gemm(p, prec, B, g, R, nullptr, reps) : -1.0;
    cudaFree(R);
    if (t < 0.0) return fail(MP_ERR_CUDA, "mp_debug_time_gemm: the GEMM could not be timed");
    *us = t;
    return MP_OK;
}

}  // extern "C"
