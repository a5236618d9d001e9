// Batched Matching Pursuit: B signals share one dictionary (Sec. 2), and
// each step performs one MP iteration (Sec. 3, Eqs. 9-12) for every signal
// that is still active.
//
// One step is three kernels:
//   corr_top8   C = Rq * Psiq^T on the tensor cores (tcgen05, BF16 or FP8-E4M3
//               operands, FP32 accumulation in TMEM); the epilogue keeps, per
//               signal and per tile of atoms, the 8 largest |c| (FP8: times the
//               atom's scale), so C is never written to memory.
//   select      per signal: merge the per-tile candidates into the top 8,
//               rescore those 8 atoms in FP32 from the FP32 atoms
//               (<r, psi_m>, Eq. 9), commit the best (ties to the smallest
//               index), x~_m += c (Eq. 10), r -= c psi_m in FP32 (Eq. 11),
//               e = sum r^2 in FP64, t += 1 (Eq. 12), stop test.
//   compact     order-preserving compaction of the still-active signals and
//               requantisation of their residuals into the GEMM operand.
// Signals stop independently; finished signals leave the GEMM.  The steps
// are captured in a CUDA graph and replayed until no signal is active.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mp_device.cuh"
#include "mp_dot.cuh"
#include "mp_internal.h"
#include "mp_tcgen05.cuh"

namespace mpgb {

constexpr int kBM = 128;            // signals per tile = TMEM lanes = UMMA M
constexpr int kRowBytes = 128;      // bytes of K per operand row per stage (one swizzle row)
constexpr int kStages = 4;
constexpr int kTop = 8;
constexpr int kGemmThreads = 192;   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kSelThreads = 256;
constexpr int kStepsPerGraph = 16;  // even: the active-list parity returns to 0

struct SlotState {
    double e0, e, thr2, audit;
    int t, T, status, stop_reason;
};

// Per-call outputs, read by the kernels through one device pointer so the
// captured graph does not depend on the caller's buffers.
struct BatchIO {
    float* X;              // row b at X + b * ldx
    long long ldx;
    int* tr_atoms;         // row b at tr_atoms + b * tr_cap (optional)
    float* tr_coefs;
    double* tr_energy;
    int tr_cap;
    int pad;
};

// ------------------------------------------------------------------ GEMM + top-8
struct CorrArgs {
    const int* n_act;       // active rows this step
    int TN;                 // atoms per tile
    int n_at;               // atom tiles
    int M;
    int nk;                 // K blocks of 128 bytes
    int fp8;
    int tmem_cols;
    const float* colscale;  // FP8 per-atom scale
    uint2* cand;            // [row][n_at][8] = (score bits, atom)
    unsigned long long watchdog_ns;
    int* err;
    float* dump;            // diagnostic: full correlation rows (row * M + m), or NULL
    const float* rscale;    // diagnostic FP8: per-row scale of the quantised residual
};

struct CorrShared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

MP_DEV void corr_timeout(int* err, CorrShared* sh) {
    atomicCAS(err, 0, static_cast<int>(MP_ERR_TIMEOUT));
    *reinterpret_cast<volatile int*>(&sh->abort) = 1;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    corr_top8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const CorrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // operand tiles need 1024-byte alignment for the 128-byte swizzle atoms
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    const int TN = a.TN;
    const uint32_t a_bytes = kBM * kRowBytes;
    const uint32_t b_bytes = static_cast<uint32_t>(TN) * kRowBytes;
    uint8_t* tilesA = smem;
    uint8_t* tilesB = smem + kStages * a_bytes;
    CorrShared* sh = reinterpret_cast<CorrShared*>(tilesB + kStages * b_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_act = *a.n_act;
    const int n_rt = (n_act + kBM - 1) / kBM;
    const int n_tiles = n_rt * a.n_at;
    if (static_cast<int>(blockIdx.x) >= n_tiles) return;   // uniform across the CTA

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->tfull[b], 1);
            mbar_init(&sh->tempty[b], 4 * 32);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) tmem_alloc(&sh->tmem_base, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    const uint64_t lim = a.watchdog_ns;

    if (warp == 0) {
        // ---------------- TMA producer (one thread)
        if (lane == 0) {
            long long g = 0;
            const int kelems = a.fp8 ? kRowBytes : kRowBytes / 2;
            bool stop = false;
            for (int tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x) {
                const int rt = tile % n_rt, at = tile / n_rt;
                for (int kb = 0; kb < a.nk; ++kb) {
                    const int s = static_cast<int>(g % kStages);
                    const long long use = g / kStages;
                    if (use > 0 && !mbar_wait_bounded(&sh->empty[s], static_cast<uint32_t>((use - 1) & 1), lim)) {
                        corr_timeout(a.err, sh);
                        stop = true;
                        break;
                    }
                    if (*reinterpret_cast<volatile int*>(&sh->abort)) {
                        stop = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->full[s], a_bytes + b_bytes);
                    tma_load_2d(tilesA + s * a_bytes, &tmA, kb * kelems, rt * kBM, &sh->full[s]);
                    tma_load_2d(tilesB + s * b_bytes, &tmB, kb * kelems, at * TN, &sh->full[s]);
                    ++g;
                }
            }
            // every issued load lands before the CTA may exit: the only load
            // that can be in flight in stage s is the last one issued to it
            for (int s = 0; s < kStages && s < g; ++s) {
                const long long last = g - 1 - ((g - 1 - s) % kStages);
                mbar_wait_bounded(&sh->full[s], static_cast<uint32_t>((last / kStages) & 1), lim);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = make_idesc(kBM, TN, a.fp8 ? 0u : 1u);
            long long g = 0;
            int li = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++li) {
                const int buf = li & 1, useb = li >> 1;
                if (useb > 0 && !mbar_wait_bounded(&sh->tempty[buf], static_cast<uint32_t>((useb - 1) & 1), lim)) {
                    corr_timeout(a.err, sh);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * TN);
                for (int kb = 0; kb < a.nk; ++kb, ++g) {
                    const int s = static_cast<int>(g % kStages);
                    if (!mbar_wait_bounded(&sh->full[s], static_cast<uint32_t>((g / kStages) & 1), lim) ||
                        *reinterpret_cast<volatile int*>(&sh->abort)) {
                        corr_timeout(a.err, sh);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tilesA + s * a_bytes);
                    const uint32_t sb = smem_u32(tilesB + s * b_bytes);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // 32 bytes of K per instruction: 16 BF16 or 32 E4M3 values
                        const uint64_t ad = sw128_kmajor_desc(sa + 32u * k);
                        const uint64_t bd = sw128_kmajor_desc(sb + 32u * k);
                        const uint32_t acc = (kb | k) ? 1u : 0u;
                        if (a.fp8) mma_fp8(d, ad, bd, idesc, acc);
                        else mma_bf16(d, ad, bd, idesc, acc);
                    }
                    mma_commit(&sh->empty[s]);   // stage reusable once these MMAs finish
                }
                if (ok) mma_commit(&sh->tfull[buf]);
            }
            // no MMA may still write TMEM when it is freed: this commit
            // arrives once every MMA issued above has completed
            mma_commit(&sh->drain);
            mbar_wait_bounded(&sh->drain, 0u, lim);
        }
    } else {
        // ---------------- epilogue: one TMEM lane (= one signal row) per thread
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        int li = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++li) {
            const int rt = tile % n_rt, at = tile / n_rt;
            const int buf = li & 1, useb = li >> 1;
            bool ok = mbar_wait_bounded(&sh->tfull[buf], static_cast<uint32_t>(useb & 1), lim) &&
                      !*reinterpret_cast<volatile int*>(&sh->abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) corr_timeout(a.err, sh);
                break;
            }
            tc_fence_after();
            const int row = rt * kBM + q * 32 + lane;
            float ts[kTop];
            int ti[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) {
                ts[k] = -1.f;
                ti[k] = 0x7fffffff;
            }
            const int m0 = at * TN;
            for (int c = 0; c < TN / 32; ++c) {
                float v[32];
                tmem_ld_32cols(tmem + (static_cast<uint32_t>(q * 32) << 16) +
                                   static_cast<uint32_t>(buf * TN + c * 32),
                               v);
                if (a.dump && row < n_act) {
                    const float rsc = a.fp8 ? a.rscale[row] : 1.f;
                    for (int j = 0; j < 32; ++j) {
                        const int m = m0 + c * 32 + j;
                        if (m < a.M) a.dump[static_cast<size_t>(row) * a.M + m] = v[j] * (a.fp8 ? a.colscale[m] * rsc : 1.f);
                    }
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int m = m0 + c * 32 + j;
                    if (m >= a.M) continue;
                    float s = fabsf(v[j]);
                    if (a.fp8) s *= __ldg(a.colscale + m);
                    // strict: an equal score keeps the earlier (smaller) atom
                    if (s > ts[kTop - 1]) {
                        ts[kTop - 1] = s;
                        ti[kTop - 1] = m;
#pragma unroll
                        for (int k = kTop - 1; k > 0; --k) {
                            if (ts[k] > ts[k - 1]) {
                                const float f = ts[k];
                                ts[k] = ts[k - 1];
                                ts[k - 1] = f;
                                const int ii = ti[k];
                                ti[k] = ti[k - 1];
                                ti[k - 1] = ii;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&sh->tempty[buf]);
            if (row < n_act) {
                uint2* o = a.cand + (static_cast<size_t>(row) * a.n_at + at) * kTop;
#pragma unroll
                for (int k = 0; k < kTop; ++k) o[k] = make_uint2(__float_as_uint(ts[k]), static_cast<uint32_t>(ti[k]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
    }
}

// ------------------------------------------------------------------ block helpers
MP_DEV double block_sum_f64(double v, double* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_sum_f64(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    return s;
}
MP_DEV unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    v = warp_max_u64(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long m = 0ull;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) m = umax64(m, red[w]);
    return m;
}
MP_DEV int block_sum_i32(int v, int* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// ------------------------------------------------------------------ init
struct InitArgs {
    const float* Y;         // B x N
    int B, N, ldN, M;
    float* R32;             // slot b row at R32 + b * ldN
    const BatchIO* io;
    const double* eps2;     // per slot
    const int* T;           // per slot
    SlotState* st;
    int* act;               // list written here (all slots, in order)
    int* n_act;
    int* done;
};

__global__ void __launch_bounds__(kSelThreads) batch_init_kernel(const InitArgs a) {
    __shared__ double red[kSelThreads / 32];
    const int b = blockIdx.x;
    const float* y = a.Y + static_cast<size_t>(b) * a.N;
    float* r = a.R32 + static_cast<size_t>(b) * a.ldN;
    double acc = 0.0;
    for (int n = threadIdx.x; n < a.ldN; n += blockDim.x) {
        const float v = n < a.N ? y[n] : 0.f;
        r[n] = v;
        acc = fma(static_cast<double>(v), static_cast<double>(v), acc);
    }
    float* x = a.io->X + static_cast<size_t>(b) * a.io->ldx;
    for (int m = threadIdx.x; m < a.M; m += blockDim.x) x[m] = 0.f;
    const double e0 = block_sum_f64(acc, red);
    if (threadIdx.x == 0) {
        SlotState s;
        s.e0 = e0;
        s.e = e0;
        s.thr2 = a.eps2[b] * e0;
        s.audit = 0.0;
        s.t = 0;
        s.T = a.T[b];
        const bool finite = isfinite(e0);
        s.status = finite ? MP_OK : MP_ERR_NONFINITE;
        const bool run = finite && e0 > s.thr2 && s.T > 0;
        s.stop_reason = e0 == 0.0 ? MP_STOP_ZERO_Y : (e0 <= s.thr2 ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS);
        a.st[b] = s;
        a.act[b] = b;
        a.done[b] = run ? 0 : 1;
        if (b == 0) *a.n_act = a.B;
    }
}

// ------------------------------------------------------------------ select / rescore / update
struct SelArgs {
    const int* n_act;
    const int* act;
    int* done;              // by position in the active list
    const uint2* cand;
    int n_at;
    const float* psi32;
    int ldN, N, M;
    float* R32;
    const BatchIO* io;
    SlotState* st;
};

__global__ void __launch_bounds__(kSelThreads) select_update_kernel(const SelArgs a) {
    extern __shared__ float4 r_sh4[];
    float* r = reinterpret_cast<float*>(r_sh4);
    __shared__ unsigned long long redk[kSelThreads / 32];
    __shared__ double redd[kSelThreads / 32];
    __shared__ int top[kTop];
    __shared__ unsigned long long rkey[kTop];
    const int i = blockIdx.x;
    if (i >= *a.n_act) return;
    const int slot = a.act[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* rs4 = reinterpret_cast<float4*>(r);
    const float4* rg4 = reinterpret_cast<const float4*>(a.R32 + static_cast<size_t>(slot) * a.ldN);
    const int n4 = a.ldN / 4;
    for (int k = threadIdx.x; k < n4; k += blockDim.x) rs4[k] = rg4[k];

    // merge: 8 rounds, each the largest (score, -atom) key below the previous
    const int nc = a.n_at * kTop;
    const uint2* cd = a.cand + static_cast<size_t>(i) * nc;
    unsigned long long prev = ~0ull;
    for (int round = 0; round < kTop; ++round) {
        unsigned long long best = 0ull;
        for (int k = threadIdx.x; k < nc; k += blockDim.x) {
            const uint2 c = cd[k];
            if (c.y >= static_cast<uint32_t>(a.M)) continue;
            const unsigned long long key = (static_cast<unsigned long long>(c.x) << 32) | (0xffffffffu - c.y);
            if (key < prev && key > best) best = key;
        }
        best = block_max_u64(best, redk);
        if (threadIdx.x == 0) top[round] = best ? static_cast<int>(0xffffffffu - static_cast<uint32_t>(best)) : -1;
        prev = best ? best : 0ull;
    }
    __syncthreads();
    // rescore the candidates in FP32 from the FP32 atoms (Eq. 9)
    if (warp < kTop) {
        const int m = top[warp];
        unsigned long long key = 0ull;
        if (m >= 0) key = pack_key(dot1(a.psi32 + static_cast<size_t>(m) * a.ldN, r, a.ldN, lane), m);
        if (lane == 0) rkey[warp] = key;
    }
    __syncthreads();
    unsigned long long kbest = 0ull;
    for (int w = 0; w < kTop; ++w) kbest = umax64(kbest, rkey[w]);
    const int m = key_index(kbest);
    const float c = key_coef(kbest);
    SlotState s = a.st[slot];
    if (kbest == 0ull) {   // no candidate: nothing to select
        if (threadIdx.x == 0) {
            s.status = MP_ERR_INVALID;
            a.st[slot] = s;
            a.done[i] = 1;
        }
        return;
    }
    // Eq. 11 in FP32 and the FP64 energy
    const float4* pm = reinterpret_cast<const float4*>(a.psi32 + static_cast<size_t>(m) * a.ldN);
    float4* rw4 = reinterpret_cast<float4*>(a.R32 + static_cast<size_t>(slot) * a.ldN);
    double acc = 0.0;
    for (int k = threadIdx.x; k < n4; k += blockDim.x) {
        const float4 p = __ldg(pm + k);
        float4 v = rs4[k];
        v.x = fmaf(-c, p.x, v.x);
        v.y = fmaf(-c, p.y, v.y);
        v.z = fmaf(-c, p.z, v.z);
        v.w = fmaf(-c, p.w, v.w);
        rw4[k] = v;
        acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
        acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
        acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
        acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
    }
    const double e = block_sum_f64(acc, redd);
    if (threadIdx.x == 0) {
        const BatchIO& io = *a.io;
        io.X[static_cast<size_t>(slot) * io.ldx + m] += c;   // Eq. 10
        if (io.tr_atoms && s.t < io.tr_cap) io.tr_atoms[static_cast<size_t>(slot) * io.tr_cap + s.t] = m;
        if (io.tr_coefs && s.t < io.tr_cap) io.tr_coefs[static_cast<size_t>(slot) * io.tr_cap + s.t] = c;
        if (io.tr_energy && s.t < io.tr_cap) io.tr_energy[static_cast<size_t>(slot) * io.tr_cap + s.t] = e;
        const double cc = static_cast<double>(c);
        s.audit = fmax(s.audit, fabs(e - (s.e - cc * cc)) / s.e0);
        s.e = e;
        s.t += 1;   // Eq. 12
        const bool conv = !(e > s.thr2);
        const bool stop = conv || s.t >= s.T;
        if (stop) s.stop_reason = conv ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS;
        a.st[slot] = s;
        a.done[i] = stop ? 1 : 0;
    }
}

// ------------------------------------------------------------------ compact / requantise
struct CompactArgs {
    const int* n_old;
    const int* act_old;
    const int* done;
    int* n_new;
    int* act_new;
    const float* R32;
    int ldN, N;
    void* Rq;               // BF16 (ldq elements per row) or E4M3 (ldq bytes per row)
    int ldq;
    int fp8;
    float* rscale;          // FP8: per-row scale written here (optional)
};

__global__ void __launch_bounds__(kSelThreads) compact_requant_kernel(const CompactArgs a) {
    __shared__ int redi[kSelThreads / 32];
    __shared__ float redf[kSelThreads / 32];
    const int i = blockIdx.x;
    const int n_old = *a.n_old;
    if (i == 0) {
        int cnt = 0;
        for (int k = threadIdx.x; k < n_old; k += blockDim.x) cnt += a.done[k] ? 0 : 1;
        cnt = block_sum_i32(cnt, redi);
        if (threadIdx.x == 0) *a.n_new = cnt;
    }
    if (i >= n_old || a.done[i]) return;
    int before = 0;
    for (int k = threadIdx.x; k < i; k += blockDim.x) before += a.done[k] ? 0 : 1;
    before = block_sum_i32(before, redi);
    const int slot = a.act_old[i];
    if (threadIdx.x == 0) a.act_new[before] = slot;
    const float* r = a.R32 + static_cast<size_t>(slot) * a.ldN;
    if (!a.fp8) {
        __nv_bfloat16* q = static_cast<__nv_bfloat16*>(a.Rq) + static_cast<size_t>(before) * a.ldq;
        for (int n = threadIdx.x; n < a.ldq; n += blockDim.x) q[n] = __float2bfloat16_rn(n < a.ldN ? r[n] : 0.f);
    } else {
        // per-signal scale max|r| / 448 maps r onto the E4M3 range; one
        // positive factor per row leaves the row's ranking unchanged
        float mx = 0.f;
        for (int n = threadIdx.x; n < a.ldN; n += blockDim.x) mx = fmaxf(mx, fabsf(r[n]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = mx;
        __syncthreads();
        float amax = 0.f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) amax = fmaxf(amax, redf[w]);
        const float inv = amax > 0.f ? 448.f / amax : 1.f;
        if (a.rscale && threadIdx.x == 0) a.rscale[before] = amax > 0.f ? amax / 448.f : 1.f;
        __nv_fp8_storage_t* q = static_cast<__nv_fp8_storage_t*>(a.Rq) + static_cast<size_t>(before) * a.ldq;
        for (int n = threadIdx.x; n < a.ldq; n += blockDim.x)
            q[n] = __nv_cvt_float_to_fp8(n < a.ldN ? r[n] * inv : 0.f, __NV_SATFINITE, __NV_E4M3);
    }
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

// rows x row_bytes matrix (row stride = row_bytes), box of box_rows rows x 128 bytes
static mp_status make_map(CUtensorMap* map, void* base, bool fp8, long long rows, long long row_elems,
                          int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const int esize = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(row_elems), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_elems * esize)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / esize), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MP_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return MP_OK;
}

struct BatchEngine {
    int cap = 0;            // slots
    int cap_pad = 0;        // rows of the GEMM operand (multiple of 128)
    int prec = -1;
    int TN = 0;
    int n_at = 0;
    float* R32 = nullptr;
    void* Rq = nullptr;
    SlotState* st = nullptr;
    int* act = nullptr;     // 2 x cap
    int* n_act = nullptr;   // 2
    int* done = nullptr;
    uint2* cand = nullptr;
    double* eps2 = nullptr;
    int* T = nullptr;
    int* err = nullptr;
    BatchIO* io = nullptr;
    float* rscale = nullptr;   // diagnostic FP8 row scales
    // pinned host mirrors
    SlotState* h_st = nullptr;
    int* h_nact = nullptr;
    double* h_eps2 = nullptr;
    int* h_T = nullptr;
    BatchIO* h_io = nullptr;
    int* h_err = nullptr;
    CUtensorMap tmA, tmB;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    size_t bytes = 0;
};

static void engine_free(BatchEngine* e) {
    if (!e) return;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    cudaFree(e->R32);
    cudaFree(e->Rq);
    cudaFree(e->st);
    cudaFree(e->act);
    cudaFree(e->n_act);
    cudaFree(e->done);
    cudaFree(e->cand);
    cudaFree(e->eps2);
    cudaFree(e->T);
    cudaFree(e->err);
    cudaFree(e->io);
    cudaFree(e->rscale);
    cudaFreeHost(e->h_st);
    cudaFreeHost(e->h_nact);
    cudaFreeHost(e->h_eps2);
    cudaFreeHost(e->h_T);
    cudaFreeHost(e->h_io);
    cudaFreeHost(e->h_err);
    *e = BatchEngine();
}

void batch_destroy(BatchEngine* b) {
    engine_free(b);
    delete b;
}

static int gemm_smem_bytes(int TN) {
    return 1024 + kStages * (kBM * kRowBytes + TN * kRowBytes) + static_cast<int>(sizeof(CorrShared));
}

// (Re)build the engine for `cap` slots at precision `prec`.
static mp_status engine_prepare(PlanImpl* p, int prec, int cap) {
    BatchEngine* e = p->batch;
    const int TN = p->batch_tile_n ? p->batch_tile_n : 256;
    if (e && e->prec == prec && e->cap >= cap && e->TN == TN) return MP_OK;
    if (!e) e = p->batch = new BatchEngine();
    const int newcap = std::max(cap, e->cap);
    engine_free(e);
    e->cap = newcap;
    e->cap_pad = (newcap + kBM - 1) / kBM * kBM;
    e->prec = prec;
    e->TN = TN;
    e->n_at = (p->M + TN - 1) / TN;
    const bool fp8 = prec == MP_PREC_FP8E4M3;
    const int ldq = fp8 ? p->ldK8 : p->ldK16;
    const size_t qbytes = static_cast<size_t>(e->cap_pad) * ldq * (fp8 ? 1 : 2);
    auto A = [&](void** ptr, size_t b) {
        e->bytes += b;
        return cudaMalloc(ptr, b);
    };
    cudaError_t r = cudaSuccess;
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->R32), sizeof(float) * e->cap * static_cast<size_t>(p->ldN));
    if (r == cudaSuccess) r = A(&e->Rq, qbytes);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->st), sizeof(SlotState) * e->cap);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->act), sizeof(int) * 2 * e->cap);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->n_act), sizeof(int) * 2);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->done), sizeof(int) * e->cap);
    if (r == cudaSuccess)
        r = A(reinterpret_cast<void**>(&e->cand), sizeof(uint2) * static_cast<size_t>(e->cap) * e->n_at * kTop);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->eps2), sizeof(double) * e->cap);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->T), sizeof(int) * e->cap);
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->err), sizeof(int));
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->io), sizeof(BatchIO));
    if (r == cudaSuccess) r = A(reinterpret_cast<void**>(&e->rscale), sizeof(float) * e->cap);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_st, sizeof(SlotState) * e->cap);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_nact, sizeof(int) * 2);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_eps2, sizeof(double) * e->cap);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_T, sizeof(int) * e->cap);
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_io, sizeof(BatchIO));
    if (r == cudaSuccess) r = cudaMallocHost(&e->h_err, sizeof(int));
    if (r == cudaSuccess) r = cudaMemset(e->Rq, 0, qbytes);
    if (r != cudaSuccess) {
        engine_free(e);
        return cuda_fail(r, "batched engine allocation");
    }
    mp_status s = make_map(&e->tmA, e->Rq, fp8, e->cap_pad, ldq, kBM);
    if (s == MP_OK) s = make_map(&e->tmB, fp8 ? p->psi8 : p->psi16, fp8, p->M, ldq, TN);
    if (s != MP_OK) {
        engine_free(e);
        return s;
    }
    return MP_OK;
}

// Launch one step (GEMM, select, compact) with active-list parity `par`.
static cudaError_t launch_step(PlanImpl* p, BatchEngine* e, int par, cudaStream_t st) {
    const bool fp8 = e->prec == MP_PREC_FP8E4M3;
    int* act_cur = e->act + par * e->cap;
    int* act_new = e->act + (1 - par) * e->cap;
    const int* n_cur = e->n_act + par;
    int* n_new = e->n_act + (1 - par);
    CorrArgs ca;
    ca.n_act = n_cur;
    ca.TN = e->TN;
    ca.n_at = e->n_at;
    ca.M = p->M;
    ca.nk = (fp8 ? p->ldK8 : p->ldK16 * 2) / kRowBytes;
    ca.fp8 = fp8 ? 1 : 0;
    ca.tmem_cols = 2 * e->TN >= 512 ? 512 : (2 * e->TN >= 256 ? 256 : 128);
    ca.colscale = p->scale8;
    ca.cand = e->cand;
    ca.watchdog_ns = static_cast<unsigned long long>(p->watchdog_ns);
    ca.err = e->err;
    ca.dump = nullptr;
    ca.rscale = nullptr;
    const int max_tiles = (e->cap_pad / kBM) * e->n_at;
    const int grid = std::max(1, std::min(max_tiles, p->sm_count));
    corr_top8_kernel<<<grid, kGemmThreads, gemm_smem_bytes(e->TN), st>>>(e->tmA, e->tmB, ca);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    SelArgs sa;
    sa.n_act = n_cur;
    sa.act = act_cur;
    sa.done = e->done;
    sa.cand = e->cand;
    sa.n_at = e->n_at;
    sa.psi32 = p->psi32;
    sa.ldN = p->ldN;
    sa.N = p->N;
    sa.M = p->M;
    sa.R32 = e->R32;
    sa.io = e->io;
    sa.st = e->st;
    select_update_kernel<<<e->cap, kSelThreads, p->ldN * sizeof(float), st>>>(sa);
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    CompactArgs cp;
    cp.n_old = n_cur;
    cp.act_old = act_cur;
    cp.done = e->done;
    cp.n_new = n_new;
    cp.act_new = act_new;
    cp.R32 = e->R32;
    cp.ldN = p->ldN;
    cp.N = p->N;
    cp.Rq = e->Rq;
    cp.ldq = fp8 ? p->ldK8 : p->ldK16;
    cp.fp8 = fp8 ? 1 : 0;
    cp.rscale = nullptr;
    compact_requant_kernel<<<e->cap, kSelThreads, 0, st>>>(cp);
    return cudaGetLastError();
}

static mp_status build_graph(PlanImpl* p, BatchEngine* e) {
    if (e->graph) return MP_OK;
    if (!e->cap_stream) MP_CUDA_TRY(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
    static bool attr = false;
    if (!attr) {
        MP_CUDA_TRY(cudaFuncSetAttribute(corr_top8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         gemm_smem_bytes(256)));
        attr = true;
    }
    MP_CUDA_TRY(cudaFuncSetAttribute(select_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     std::max(p->ldN * 4, 48 * 1024)));
    MP_CUDA_TRY(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t r = cudaSuccess;
    for (int s = 0; s < kStepsPerGraph && r == cudaSuccess; ++s) r = launch_step(p, e, s & 1, e->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t r2 = cudaStreamEndCapture(e->cap_stream, &g);
    if (r != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(r, "batched step capture");
    }
    if (r2 != cudaSuccess) return cuda_fail(r2, "cudaStreamEndCapture");
    r = cudaGraphInstantiate(&e->graph, g, 0);
    cudaGraphDestroy(g);
    if (r != cudaSuccess) return cuda_fail(r, "cudaGraphInstantiate");
    return MP_OK;
}

static mp_status batched_run(PlanImpl* p, int prec, const float* Y, float* X, long long ldx, int B,
                             const mp_stop* stops, int n_stops, const mp_trace* trace, mp_result* out,
                             cudaStream_t st) {
    mp_status s = engine_prepare(p, prec, B);
    if (s != MP_OK) return s;
    BatchEngine* e = p->batch;
    s = build_graph(p, e);
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
    InitArgs ia;
    ia.Y = Y;
    ia.B = B;
    ia.N = p->N;
    ia.ldN = p->ldN;
    ia.M = p->M;
    ia.R32 = e->R32;
    ia.io = e->io;
    ia.eps2 = e->eps2;
    ia.T = e->T;
    ia.st = e->st;
    ia.act = e->act + e->cap;      // list 1, compacted into list 0 below
    ia.n_act = e->n_act + 1;
    ia.done = e->done;
    batch_init_kernel<<<B, kSelThreads, 0, st>>>(ia);
    MP_CUDA_TRY(cudaGetLastError());
    // slots beyond B never enter the list; compact list 1 into list 0
    CompactArgs cp;
    cp.n_old = e->n_act + 1;
    cp.act_old = e->act + e->cap;
    cp.done = e->done;
    cp.n_new = e->n_act;
    cp.act_new = e->act;
    cp.R32 = e->R32;
    cp.ldN = p->ldN;
    cp.N = p->N;
    cp.Rq = e->Rq;
    const bool fp8 = prec == MP_PREC_FP8E4M3;
    cp.ldq = fp8 ? p->ldK8 : p->ldK16;
    cp.fp8 = fp8 ? 1 : 0;
    cp.rscale = nullptr;
    compact_requant_kernel<<<B, kSelThreads, 0, st>>>(cp);
    MP_CUDA_TRY(cudaGetLastError());
    p->launches += 2;
    // replay the captured steps until no signal is active (each step moves
    // every active signal by one iteration, so maxT + 1 steps always suffice)
    const long long max_replays = (static_cast<long long>(maxT) + kStepsPerGraph) / kStepsPerGraph + 1;
    for (long long k = 0; k < max_replays; ++k) {
        MP_CUDA_TRY(cudaMemcpyAsync(e->h_nact, e->n_act, sizeof(int), cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        if (*e->h_nact == 0) break;
        MP_CUDA_TRY(cudaGraphLaunch(e->graph, st));
        p->launches += 3 * kStepsPerGraph;
    }
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
        o.energy_audit_max = ss.audit;
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
                tb.residual = nullptr;
                tp = &tb;
            }
            mp_status s = mp_recover(plan, Y + static_cast<size_t>(b) * p->N, X + static_cast<size_t>(b) * p->M, sb,
                                     tp, &host_out[b], stream);
            if (s < 0 && worst == MP_OK) worst = s;
        }
        return worst;
    }
    return batched_run(p, prec, Y, X, p->M, B, stops, n_stops, trace, host_out, st);
}

}  // extern "C"

namespace mpgb {

// Diagnostic: load B residuals as active rows 0..B-1 (slot b = row b).
__global__ void debug_load_kernel(const float* R, int B, int N, int ldN, float* R32, int* act, int* n_act,
                                  int* done) {
    const int b = blockIdx.x;
    for (int n = threadIdx.x; n < ldN; n += blockDim.x)
        R32[static_cast<size_t>(b) * ldN + n] = n < N ? R[static_cast<size_t>(b) * N + n] : 0.f;
    if (threadIdx.x == 0) {
        act[b] = b;
        done[b] = 0;
        if (b == 0) *n_act = B;
    }
}

}  // namespace mpgb

extern "C" {

mp_status mp_debug_correlations(mp_plan_t plan, int prec, const float* R, int B, float* C, void* stream) {
    clear_error();
    if (!plan || !R || !C || B < 1) return fail(MP_ERR_INVALID, "mp_debug_correlations: bad argument");
    PlanImpl* p = &plan->impl;
    if (prec != MP_PREC_BF16 && prec != MP_PREC_FP8E4M3)
        return fail(MP_ERR_INVALID, "mp_debug_correlations: precision must be BF16 or FP8");
    if (!(p->prec_mask & (1u << prec)))
        return fail(MP_ERR_UNSUPPORTED, "mp_debug_correlations: the plan holds no copy for this precision");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mp_status s = engine_prepare(p, prec, B);
    if (s != MP_OK) return s;
    BatchEngine* e = p->batch;
    MP_CUDA_TRY(cudaFuncSetAttribute(corr_top8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     gemm_smem_bytes(256)));
    MP_CUDA_TRY(cudaMemsetAsync(e->err, 0, sizeof(int), st));
    debug_load_kernel<<<B, 256, 0, st>>>(R, B, p->N, p->ldN, e->R32, e->act + e->cap, e->n_act + 1, e->done);
    const bool fp8 = prec == MP_PREC_FP8E4M3;
    CompactArgs cp;
    cp.n_old = e->n_act + 1;
    cp.act_old = e->act + e->cap;
    cp.done = e->done;
    cp.n_new = e->n_act;
    cp.act_new = e->act;
    cp.R32 = e->R32;
    cp.ldN = p->ldN;
    cp.N = p->N;
    cp.Rq = e->Rq;
    cp.ldq = fp8 ? p->ldK8 : p->ldK16;
    cp.fp8 = fp8 ? 1 : 0;
    cp.rscale = e->rscale;
    compact_requant_kernel<<<B, kSelThreads, 0, st>>>(cp);
    CorrArgs ca;
    ca.n_act = e->n_act;
    ca.TN = e->TN;
    ca.n_at = e->n_at;
    ca.M = p->M;
    ca.nk = (fp8 ? p->ldK8 : p->ldK16 * 2) / kRowBytes;
    ca.fp8 = fp8 ? 1 : 0;
    ca.tmem_cols = 2 * e->TN >= 512 ? 512 : (2 * e->TN >= 256 ? 256 : 128);
    ca.colscale = p->scale8;
    ca.cand = e->cand;
    ca.watchdog_ns = static_cast<unsigned long long>(p->watchdog_ns);
    ca.err = e->err;
    ca.dump = C;
    ca.rscale = e->rscale;
    const int tiles = ((B + kBM - 1) / kBM) * e->n_at;
    corr_top8_kernel<<<std::max(1, std::min(tiles, p->sm_count)), kGemmThreads, gemm_smem_bytes(e->TN), st>>>(
        e->tmA, e->tmB, ca);
    MP_CUDA_TRY(cudaGetLastError());
    p->launches += 3;
    MP_CUDA_TRY(cudaMemcpyAsync(e->h_err, e->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (*e->h_err) return fail(static_cast<mp_status>(*e->h_err), "mp_debug_correlations: device wait timed out");
    return MP_OK;
}

}  // extern "C"
