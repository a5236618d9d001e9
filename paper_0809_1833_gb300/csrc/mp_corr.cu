// Batched correlation GEMM with a segmented top-8 epilogue (Sec. 3 Eq. 9 for
// many signals at once): C = Rq * Psiq^T on the tcgen05 tensor cores, BF16
// (kind::f16) or FP8-E4M3 (kind::f8f6f4) operands staged by TMA with
// 128-byte swizzling, FP32 accumulators in TMEM, and per signal row the 8
// largest |c| of each atom tile kept in registers and written out, so the
// correlation matrix itself is never stored.
//
// Operand reuse: a cluster of CL CTAs takes CL consecutive 128-signal row
// tiles of one atom tile.  Each CTA loads its own rows of R, but only 1/CL of
// the atom tile, and multicasts that slice to every CTA of the cluster; a
// stage is refilled only after all CL CTAs released it (their MMA commits are
// multicast to every CTA's "empty" barrier).  The atom operand, the larger
// one, then crosses from L2 once per cluster instead of once per CTA.
#include <cuda.h>

#include <algorithm>

#include "mp_batch.cuh"
#include "mp_device.cuh"
#include "mp_tcgen05.cuh"

namespace mpgb {

// ---------------------------------------------------------------- top-8
// Candidate order: larger score first, equal scores by the smaller atom.
// A non-negative float's bits order like its value, so (score bits, ~atom)
// packed in 64 bits orders as one unsigned integer.
MP_DEV unsigned long long score_key(float s, int m) {
    return (static_cast<unsigned long long>(__float_as_uint(s)) << 32) | (0xffffffffu - static_cast<uint32_t>(m));
}
// after it a >= b
MP_DEV void cex(unsigned long long& a, unsigned long long& b) {
    const unsigned long long hi = umax64(a, b);
    b = a ^ b ^ hi;
    a = hi;
}
// descending sort of 8 keys: Batcher's odd-even merge network (19 exchanges)
MP_DEV void sort8_desc(unsigned long long (&x)[8]) {
    cex(x[0], x[1]); cex(x[2], x[3]); cex(x[4], x[5]); cex(x[6], x[7]);
    cex(x[0], x[2]); cex(x[1], x[3]); cex(x[4], x[6]); cex(x[5], x[7]);
    cex(x[1], x[2]); cex(x[5], x[6]);
    cex(x[0], x[4]); cex(x[1], x[5]); cex(x[2], x[6]); cex(x[3], x[7]);
    cex(x[2], x[4]); cex(x[3], x[5]);
    cex(x[1], x[2]); cex(x[3], x[4]); cex(x[5], x[6]);
}
// t <- the best 8 of (t, c), both sorted descending: the elementwise max
// of t and reversed c is a bitonic sequence holding them; a bitonic merge
// network (12 exchanges) sorts it
MP_DEV void merge_top8(unsigned long long (&t)[8], const unsigned long long (&c)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = umax64(t[i], c[7 - i]);
    cex(t[0], t[4]); cex(t[1], t[5]); cex(t[2], t[6]); cex(t[3], t[7]);
    cex(t[0], t[2]); cex(t[1], t[3]); cex(t[4], t[6]); cex(t[5], t[7]);
    cex(t[0], t[1]); cex(t[2], t[3]); cex(t[4], t[5]); cex(t[6], t[7]);
}

struct CorrShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
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

template <int CL>
__global__ void __launch_bounds__(kGemmThreads, 1)
    corr_top8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const CorrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // operand tiles need 1024-byte alignment for the 128-byte swizzle atoms
    // (the same offset in every CTA, as multicast writes the same offsets)
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    const int TN = a.TN;
    const uint32_t a_bytes = kBM * kRowBytes;
    const uint32_t b_bytes = static_cast<uint32_t>(TN) * kRowBytes;
    const uint32_t slice_bytes = b_bytes / CL;   // this CTA's share of the atom tile
    uint8_t* tilesA = smem;
    uint8_t* tilesB = smem + a.stages * a_bytes;
    CorrShared* sh = reinterpret_cast<CorrShared*>(tilesB + a.stages * b_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = CL > 1 ? static_cast<int>(cluster_ctarank()) : 0;     // rank in the cluster
    const int cid = static_cast<int>(blockIdx.x) / CL;
    const int n_clusters = static_cast<int>(gridDim.x) / CL;
    const int n_act = *a.n_act;
    const int n_rt = (n_act + kBM - 1) / kBM;
    const int n_rg = (n_rt + CL - 1) / CL;         // groups of CL row tiles
    const int n_ct = n_rg * a.n_at;                 // cluster tiles
    if (cid >= n_ct) return;                        // uniform across the cluster
    const uint16_t all = static_cast<uint16_t>((1u << CL) - 1u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], CL);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->tfull[b], 1);
            mbar_init(&sh->tempty[b], 4 * 32 * kEpiGroups);
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
    if (CL > 1) cluster_sync_all();   // every CTA's barriers exist before any multicast
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    const uint64_t lim = a.watchdog_ns;

    if (warp == 0) {
        // ---------------- TMA producer (one thread)
        if (lane == 0) {
            long long g = 0;
            const int kelems = a.fp8 ? kRowBytes : kRowBytes / 2;
            bool stop = false;
            for (int ct = cid; ct < n_ct && !stop; ct += n_clusters) {
                const int rt = (ct % n_rg) * CL + q, at = ct / n_rg;
                for (int kb = 0; kb < a.nk; ++kb) {
                    const int s = static_cast<int>(g % a.stages);
                    const long long use = g / a.stages;
                    // all CL CTAs released the stage's previous use
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
                    if (CL == 1)
                        tma_load_2d(tilesB + s * b_bytes, &tmB, kb * kelems, at * TN, &sh->full[s]);
                    else
                        tma_load_2d_multicast(tilesB + s * b_bytes + q * slice_bytes, &tmB, kb * kelems,
                                              at * TN + q * (TN / CL), &sh->full[s], all);
                    ++g;
                }
            }
            // before the CTA may exit: its own loads have landed (the only one
            // that can be in flight in stage s is the last one issued to it),
            // and every CTA of the cluster released the stages' last uses, so
            // no peer still writes into this CTA or arrives on its barriers
            for (int s = 0; s < a.stages && s < g; ++s) {
                const long long last = g - 1 - ((g - 1 - s) % a.stages);
                mbar_wait_bounded(&sh->full[s], static_cast<uint32_t>((last / a.stages) & 1), lim);
                mbar_wait_bounded(&sh->empty[s], static_cast<uint32_t>((last / a.stages) & 1), lim);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = make_idesc(kBM, TN, a.fp8 ? 0u : 1u);
            long long g = 0;
            int li = 0;
            bool ok = true;
            for (int ct = cid; ct < n_ct && ok; ct += n_clusters, ++li) {
                const int buf = li & 1, useb = li >> 1;
                if (useb > 0 && !mbar_wait_bounded(&sh->tempty[buf], static_cast<uint32_t>((useb - 1) & 1), lim)) {
                    corr_timeout(a.err, sh);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * TN);
                for (int kb = 0; kb < a.nk; ++kb, ++g) {
                    const int s = static_cast<int>(g % a.stages);
                    if (!mbar_wait_bounded(&sh->full[s], static_cast<uint32_t>((g / a.stages) & 1), lim) ||
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
                    // stage reusable once these MMAs finish (in every CTA that
                    // will refill it with a multicast)
                    if (CL == 1) mma_commit(&sh->empty[s]);
                    else mma_commit_multicast(&sh->empty[s], all);
                }
                if (ok) mma_commit(&sh->tfull[buf]);
            }
            // no MMA may still write TMEM when it is freed: this commit
            // arrives once every MMA issued above has completed
            mma_commit(&sh->drain);
            mbar_wait_bounded(&sh->drain, 0u, lim);
        }
    } else {
        // ---------------- epilogue: kEpiGroups threads per signal row; a warp
        // reads the TMEM lane quadrant warp % 4 (the quadrant a warp may
        // access), and warp group grp scans atom columns [grp, grp+1) * TN/kEpiGroups
        const int quad = warp & 3;
        const int grp = (warp - 2) >> 2;
        const int cols = TN / kEpiGroups;
        int li = 0;
        for (int ct = cid; ct < n_ct; ct += n_clusters, ++li) {
            const int rt = (ct % n_rg) * CL + q, at = ct / n_rg;
            const int buf = li & 1, useb = li >> 1;
            bool ok = mbar_wait_bounded(&sh->tfull[buf], static_cast<uint32_t>(useb & 1), lim) &&
                      !*reinterpret_cast<volatile int*>(&sh->abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) corr_timeout(a.err, sh);
                break;
            }
            tc_fence_after();
            const int row = rt * kBM + quad * 32 + lane;
            // the thread's best 8 as packed keys (score bits, ~atom): larger
            // score first, then the smaller atom; 0 = empty
            unsigned long long tk[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) tk[k] = 0ull;
            const int m0 = at * TN + grp * cols;
            for (int c = 0; c < cols / 32; ++c) {
                float v[32];
                tmem_ld_32cols(tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                                   static_cast<uint32_t>(buf * TN + grp * cols + c * 32),
                               v);
                if (a.dump && row < n_act) {
                    const float rsc = a.fp8 ? a.rscale[row] : 1.f;
                    for (int j = 0; j < 32; ++j) {
                        const int m = m0 + c * 32 + j;
                        if (m < a.M) a.dump[static_cast<size_t>(row) * a.M + m] = v[j] * (a.fp8 ? a.colscale[m] * rsc : 1.f);
                    }
                }
                // branch-free: sort each group of 8 keys, then keep the best
                // 8 of (list, group) -- every lane does the same work
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    unsigned long long ck[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int m = m0 + c * 32 + h * 8 + j;
                        float sc = fabsf(v[h * 8 + j]);
                        if (a.fp8) sc *= m < a.M ? __ldg(a.colscale + m) : 0.f;
                        ck[j] = (m < a.M && sc <= 3.0e38f) ? score_key(sc, m) : 0ull;
                    }
                    sort8_desc(ck);
                    merge_top8(tk, ck);
                }
            }
            tc_fence_before();
            mbar_arrive(&sh->tempty[buf]);
            if (row < n_act) {
                uint2* o = a.cand + ((static_cast<size_t>(row) * a.n_at + at) * kEpiGroups + grp) * kTop;
#pragma unroll
                for (int k = 0; k < kTop; ++k)
                    o[k] = make_uint2(static_cast<uint32_t>(tk[k] >> 32), 0xffffffffu - static_cast<uint32_t>(tk[k]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
    }
    if (CL > 1) cluster_sync_all();   // no CTA leaves while a peer may still address it
}

int corr_smem_bytes(int TN) {
    return 1024 + corr_stages(TN) * (kBM * kRowBytes + TN * kRowBytes) + static_cast<int>(sizeof(CorrShared));
}

template <int CL>
static cudaError_t set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(corr_top8_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         std::max(corr_smem_bytes(128), corr_smem_bytes(256)));
    return e;
}

cudaError_t corr_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = set_attrs<1>();
    if (e == cudaSuccess) e = set_attrs<2>();
    if (e == cudaSuccess) e = set_attrs<4>();
    if (e == cudaSuccess) done = true;
    return e;
}

// Largest number of CL-CTA clusters that can be resident at once.
int corr_max_clusters(int CL, int TN) {
    static int cache[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
    const int ci = CL == 1 ? 0 : (CL == 2 ? 1 : 2), ti = TN == 256 ? 1 : 0;
    if (cache[ci][ti] >= 0) return cache[ci][ti];
    int sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    int n = sm / CL;
    if (CL > 1 && corr_prepare() == cudaSuccess) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(CL);
        lc.blockDim = dim3(kGemmThreads);
        lc.dynamicSmemBytes = corr_smem_bytes(TN);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int k = 0;
        cudaError_t e = CL == 2 ? cudaOccupancyMaxActiveClusters(&k, corr_top8_kernel<2>, &lc)
                                : cudaOccupancyMaxActiveClusters(&k, corr_top8_kernel<4>, &lc);
        if (e == cudaSuccess && k > 0) n = std::min(n, k);
        cudaGetLastError();
    }
    cache[ci][ti] = n;
    return n;
}

cudaError_t launch_corr_top8(const CUtensorMap& tmA, const CUtensorMap& tmB, const CorrArgs& a, int max_row_tiles,
                             int CL, cudaStream_t st) {
    // enough clusters for the largest tile count this launch can see
    const int max_ct = ((max_row_tiles + CL - 1) / CL) * a.n_at;
    const int clusters = std::max(1, std::min(max_ct, corr_max_clusters(CL, a.TN)));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(clusters * CL);
    lc.blockDim = dim3(kGemmThreads);
    lc.dynamicSmemBytes = corr_smem_bytes(a.TN);
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    switch (CL) {
        case 1: return cudaLaunchKernelEx(&lc, corr_top8_kernel<1>, tmA, tmB, a);
        case 2: return cudaLaunchKernelEx(&lc, corr_top8_kernel<2>, tmA, tmB, a);
        case 4: return cudaLaunchKernelEx(&lc, corr_top8_kernel<4>, tmA, tmB, a);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mpgb
