// Batched correlation GEMM with a segmented top-8 epilogue (Sec. 3 Eq. 9 for
// many signals at once): C = Rq * Psiq^T on the tcgen05 tensor cores, BF16
// (kind::f16) or FP8-E4M3 (kind::f8f6f4) operands staged by TMA with
// 128-byte swizzling, FP32 accumulators in TMEM, and per signal row the 8
// largest |c| of each atom tile kept in registers and written out, so the
// correlation matrix itself is never stored.
//
// Operand reuse: a tile of 256 signal rows is two 128-row MMAs per K slice
// reading the same staged atom slice, so each atom byte brought into the SM
// feeds 256 rows (and each signal byte TN atoms).  Every CTA loads its own
// operand tiles; no shared memory is written by another CTA.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "mp_batch.cuh"
#include "mp_device.cuh"
#include "mp_tcgen05.cuh"

namespace mpgb {

// ---------------------------------------------------------------- top-8
// Candidate order: larger score first, equal scores by the smaller atom.
// A non-negative float's bits order like its value, so one 32-bit key
// holds the score's top 24 bits (sign, exponent, 15 mantissa bits: far
// finer than the BF16 / FP8 products' own rounding) and, in the low byte,
// 255 - the atom's column in the tile, plus 0x100 so that no candidate's
// key is 0 (0 = empty).  Keys order as unsigned integers; a compare-
// exchange is one max and one min.  The candidates only pick which 8
// atoms are rescored in FP32, so the truncation never decides a selection
// by itself.
MP_DEV uint32_t score_key(float s, int col) {
    return ((__float_as_uint(s) | 0xffu) - static_cast<uint32_t>(col)) + 0x100u;
}
MP_DEV uint32_t key_score_bits(uint32_t k) { return (k - 0x100u) & 0xffffff00u; }
MP_DEV int key_col(uint32_t k) { return 255 - static_cast<int>(k & 0xffu); }
// after it a >= b
MP_DEV void cex(uint32_t& a, uint32_t& b) {
    const uint32_t hi = max(a, b);
    b = min(a, b);
    a = hi;
}
// descending sort of 8 keys: Batcher's odd-even merge network (19 exchanges)
MP_DEV void sort8_desc(uint32_t (&x)[8]) {
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
MP_DEV void merge_top8(uint32_t (&t)[8], const uint32_t (&c)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = max(t[i], c[7 - i]);
    cex(t[0], t[4]); cex(t[1], t[5]); cex(t[2], t[6]); cex(t[3], t[7]);
    cex(t[0], t[2]); cex(t[1], t[3]); cex(t[4], t[6]); cex(t[5], t[7]);
    cex(t[0], t[1]); cex(t[2], t[3]); cex(t[4], t[5]); cex(t[6], t[7]);
}

// The MMAs of one 128-byte K slice of a stage: 4 steps of 32 bytes of K
// (16 BF16 or 32 E4M3 values), each one MMA per row block of the tile, all
// reading the stage's atom tile.  a0, b0: descriptors of the stage's signal
// and atom tiles; a step of 32 bytes adds 2 to the start-address field
// (address >> 4), a row block of 128 rows 1024.  Row block mb accumulates
// in TMEM columns [mb * TN, (mb + 1) * TN) from d; `first` starts the
// accumulation (the tile's first slice).
template <int RM, bool FP8>
MP_DEV void issue_kblock(uint32_t d, uint64_t a0, uint64_t b0, uint32_t idesc, int nmb, int TN, bool first) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t acc = (first && k == 0) ? 0u : 1u;
        const uint64_t bd = b0 + static_cast<uint64_t>(2 * k);
#pragma unroll
        for (int mb = 0; mb < RM; ++mb) {
            if (mb >= nmb) break;
            const uint64_t ad = a0 + static_cast<uint64_t>(2 * k + mb * ((kBM * kRowBytes) >> 4));
            const uint32_t dm = d + static_cast<uint32_t>(mb * TN);
            if (FP8) mma_fp8(dm, ad, bd, idesc, acc);
            else mma_bf16(dm, ad, bd, idesc, acc);
        }
    }
}

// 3-D tiled load: box {x.., y.., z..} at (x, y, z) (the operands' 3-D view:
// 128-byte K slice, rows, slice index), completion counted on `bar`.
MP_DEV void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// FP8: the per-atom scales of atoms m .. m+7 (0 for atoms past M), as two
// 16-byte loads where all 8 exist (m is a multiple of 8, so they are
// aligned), else one by one.
MP_DEV void colscale8(const float* __restrict__ cs, int m, int M, float (&out)[8]) {
    if (m + 8 <= M) {
        const float4 c0 = __ldg(reinterpret_cast<const float4*>(cs + m));
        const float4 c1 = __ldg(reinterpret_cast<const float4*>(cs + m + 4));
        out[0] = c0.x; out[1] = c0.y; out[2] = c0.z; out[3] = c0.w;
        out[4] = c1.x; out[5] = c1.y; out[6] = c1.z; out[7] = c1.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] = m + j < M ? __ldg(cs + m + j) : 0.f;
    }
}

// The running top 8 (keys tk) of one signal row over `ncols` accumulator
// columns (a multiple of 8) at TMEM address taddr: tile columns col0..,
// atoms m0...  Optionally dumps the correlations (diagnostic).
template <bool FP8>
MP_DEV void offer8(const float* v, int col, int m, const CorrArgs& a, int row, bool dump_row, uint32_t (&tk)[8]) {
    uint32_t ck[8];
    float cs8[8];
    if (FP8) colscale8(a.colscale, m, a.M, cs8);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool in = m + j < a.M;
        float sc = fabsf(v[j]);
        if (FP8) sc *= cs8[j];
        ck[j] = (in && sc <= 3.0e38f) ? score_key(sc, col + j) : 0u;
        if (dump_row && in)
            a.dump[static_cast<size_t>(row) * a.M + m + j] = v[j] * (FP8 ? a.colscale[m + j] * a.rscale[row] : 1.f);
    }
    sort8_desc(ck);
    merge_top8(tk, ck);
}
template <bool FP8>
MP_DEV void scan_top8(uint32_t taddr, int ncols, int col0, int m0, const CorrArgs& a, int row, bool dump_row,
                      uint32_t (&tk)[8]) {
    int c = 0;
    for (; c + 32 <= ncols; c += 32) {
        float v[32];
        tmem_ld_32cols(taddr + static_cast<uint32_t>(c), v);
#pragma unroll
        for (int h = 0; h < 4; ++h) offer8<FP8>(v + 8 * h, col0 + c + 8 * h, m0 + c + 8 * h, a, row, dump_row, tk);
    }
    if (c + 16 <= ncols) {
        float v[16];
        tmem_ld_16cols(taddr + static_cast<uint32_t>(c), v);
#pragma unroll
        for (int h = 0; h < 2; ++h) offer8<FP8>(v + 8 * h, col0 + c + 8 * h, m0 + c + 8 * h, a, row, dump_row, tk);
        c += 16;
    }
    if (c + 8 <= ncols) {
        float v[8];
        tmem_ld_8cols(taddr + static_cast<uint32_t>(c), v);
        offer8<FP8>(v, col0 + c, m0 + c, a, row, dump_row, tk);
    }
}

struct CorrShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t xfull[4];       // per lane quadrant: column groups 1-3 wrote their lists
    uint64_t xempty[4];      // per lane quadrant: group 0 has read them
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    // exchange of the epilogue's per-group lists: [group 1..3][key][row of the block]
    uint32_t xk[(kEpiGroups - 1) * kTop * kBM];
};

MP_DEV void corr_timeout(int* err, CorrShared* sh) {
    atomicCAS(err, 0, static_cast<int>(MP_ERR_TIMEOUT));
    *reinterpret_cast<volatile int*>(&sh->abort) = 1;
}

// Per-CTA state the three roles share (set up by the kernel).
struct CorrCtx {
    uint8_t* tilesA;       // A stages, as_stride bytes apart (1024-byte aligned)
    uint8_t* tilesB;       // B stages
    CorrShared* sh;
    uint32_t tmem;
    uint32_t as_stride;    // bytes of one K slice's A region (room for the launch's tile)
    int n_act, n_blk;      // active rows, 128-row blocks holding them
    int n_rt, n_ct;        // row tiles and tiles (for this launch's RM)
    int tn, n_at;          // atoms per tile and atom tiles of this launch
    int stages;            // ring depth for this launch's tile
    int ks;                // K slices per stage: 1, or 2 (one 3-D box per operand)
    uint32_t b_stride;     // bytes of one K slice's B region
    int warp, lane;
    uint64_t lim;          // watchdog, ns
};

// The producer, MMA and epilogue roles over this CTA's tiles of RM 128-row
// blocks x TN atoms.
template <int RM, int KS, bool TAIL>
MP_DEV void corr_roles(const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmA3,
                       const CUtensorMap* tmB3, const CorrArgs& a, const CorrCtx& x) {
    const int TN = a.TN;      // stage and accumulator strides
    const int tn = x.tn;      // atoms per tile in this launch: TN, or TN / 2
    // TMEM accumulator buffers: two unless one tile fills the 512 columns
    const int nbuf = (RM == 1 || RM * TN * 2 <= 512) ? 2 : 1;
    const uint32_t a_bytes = kBM * kRowBytes;        // one row block of a stage
    const uint32_t as_bytes = x.as_stride;
    const uint32_t b_bytes = x.b_stride;         // one stage's B region (tn atom rows)
    const int stages = x.stages;
    // a stage holds ks K slices (slice-major: [slice][rows]); with ks = 2
    // each operand's two slices come in one 3-D box
    constexpr int ks = KS;   // the launch's x.ks
    const int n_st = (a.nk + ks - 1) / ks;     // stages per tile
    const uint32_t ast_bytes = static_cast<uint32_t>(ks) * as_bytes, bst_bytes = static_cast<uint32_t>(ks) * b_bytes;
    uint8_t* tilesA = x.tilesA;
    uint8_t* tilesB = x.tilesB;
    CorrShared* sh = x.sh;
    const uint32_t tmem = x.tmem;
    const int n_act = x.n_act, n_blk = x.n_blk, n_rt = x.n_rt, n_ct = x.n_ct;
    (void)n_blk;
    const int cid = static_cast<int>(blockIdx.x), n_ctas = static_cast<int>(gridDim.x);
    const int warp = x.warp, lane = x.lane;
    const uint64_t lim = x.lim;

    if (warp == 0) {
        // ---------------- TMA producer (one thread)
        if (lane == 0) {
            // ring position: stage s, its use count parity ph, loads issued g
            // (kept incrementally: a division per K slice would stall this
            // single thread for hundreds of cycles)
            long long g = 0;
            int s = 0;
            uint32_t ph = 0;
            const int kelems = a.fp8 ? kRowBytes : kRowBytes / 2;
            bool stop = false;
            for (int ct = cid; ct < n_ct && !stop; ct += n_ctas) {
                const int rt = ct % n_rt, at = ct / n_rt;
                // row blocks of this tile with active rows
                const int nmb = RM == 1 ? 1 : min(RM, n_blk - rt * RM);
                // a partial row block is loaded whole, as one 128-row box: an
                // SM completes TMA boxes at a fixed rate whatever their size,
                // so one box costs less than several small ones (the rows past
                // the active ones hold stale finite data of the operand, and
                // their accumulators are never read)
                const uint32_t tx =
                    static_cast<uint32_t>(ks) * (static_cast<uint32_t>(tn) + static_cast<uint32_t>(nmb) * kBM) * kRowBytes;
                for (int kb = 0; kb < n_st; ++kb) {
                    // the MMAs released the stage's previous use
                    if (g >= stages && !mbar_wait_bounded(&sh->empty[s], ph ^ 1u, lim)) {
                        corr_timeout(a.err, sh);
                        stop = true;
                        break;
                    }
                    if (*reinterpret_cast<volatile int*>(&sh->abort)) {
                        stop = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->full[s], tx);
                    if constexpr (KS == 2) {
                        // one row block (RM = 1 launches only), slices 2kb and
                        // 2kb + 1 (past the last one: zero fill, not multiplied)
                        tma_load_3d(tilesA + s * ast_bytes, tmA3, 0, rt * kBM, 2 * kb, &sh->full[s]);
                        tma_load_3d(tilesB + s * bst_bytes, tmB3, 0, at * tn, 2 * kb, &sh->full[s]);
                    } else {
#pragma unroll
                        for (int mb = 0; mb < RM; ++mb) {
                            if (mb >= nmb) break;
                            uint8_t* dst = tilesA + s * as_bytes + mb * a_bytes;
                            tma_load_2d(dst, tmA, kb * kelems, (rt * RM + mb) * kBM, &sh->full[s]);
                        }
                        tma_load_2d(tilesB + s * b_bytes, tmB, kb * kelems, at * tn, &sh->full[s]);
                    }
                    ++g;
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // before the CTA may exit: its own loads have landed (the only one
            // that can be in flight in stage s is the last one issued to it),
            // and the MMAs released the stages' last uses
            for (int t = 0; t < stages && t < g; ++t) {
                const long long last = g - 1 - ((g - 1 - t) % stages);
                mbar_wait_bounded(&sh->full[t], static_cast<uint32_t>((last / stages) & 1), lim);
                mbar_wait_bounded(&sh->empty[t], static_cast<uint32_t>((last / stages) & 1), lim);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = make_idesc(kBM, tn, a.fp8 ? 0u : 1u);
            // ring stage s and its phase ph; accumulator buffer buf and its
            // phase bph (all incremental: no division in the issue loop)
            int s = 0, buf = 0, li = 0;
            uint32_t ph = 0, bph = 0;
            bool ok = true;
            for (int ct = cid; ct < n_ct && ok; ct += n_ctas, ++li) {
                const int rt = ct % n_rt;
                const int nmb = RM == 1 ? 1 : min(RM, n_blk - rt * RM);
                if (li >= nbuf && !mbar_wait_bounded(&sh->tempty[buf], bph ^ 1u, lim)) {
                    corr_timeout(a.err, sh);
                    break;
                }
                tc_fence_after();
                // row block mb accumulates in columns [mb * TN, (mb + 1) * TN) of the buffer
                const uint32_t d = tmem + static_cast<uint32_t>(buf * RM * TN);
                for (int kb = 0; kb < n_st; ++kb) {
                    if (!mbar_wait_bounded(&sh->full[s], ph, lim) || *reinterpret_cast<volatile int*>(&sh->abort)) {
                        corr_timeout(a.err, sh);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors of the stage's slices; a step of 32 bytes
                    // along K adds 2 to the start-address field (address >> 4)
                    const uint64_t a0 = sw128_kmajor_desc(smem_u32(tilesA + s * ast_bytes));
                    const uint64_t b0 = sw128_kmajor_desc(smem_u32(tilesB + s * bst_bytes));
                    if (a.fp8) issue_kblock<RM, true>(d, a0, b0, idesc, nmb, TN, kb == 0);
                    else issue_kblock<RM, false>(d, a0, b0, idesc, nmb, TN, kb == 0);
                    if (KS == 2 && 2 * kb + 1 < a.nk) {
                        // the stage's second slice: as_bytes / b_bytes further
                        // (address >> 4 in the descriptors' start field)
                        const uint64_t a1 = a0 + (as_bytes >> 4), b1 = b0 + (b_bytes >> 4);
                        if (a.fp8) issue_kblock<RM, true>(d, a1, b1, idesc, nmb, TN, false);
                        else issue_kblock<RM, false>(d, a1, b1, idesc, nmb, TN, false);
                    }
                    // stage reusable once these MMAs finish
                    mma_commit(&sh->empty[s]);
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit(&sh->tfull[buf]);
                if (++buf == nbuf) {
                    buf = 0;
                    bph ^= 1u;
                }
            }
            // no MMA may still write TMEM when it is freed: this commit
            // arrives once every MMA issued above has completed
            mma_commit(&sh->drain);
            mbar_wait_bounded(&sh->drain, 0u, lim);
        }
    } else {
        // ---------------- epilogue: kEpiGroups threads per signal row; a warp
        // reads the TMEM lane quadrant warp % 4 (the quadrant a warp may
        // access), and warp group grp scans atom columns [grp, grp+1) * TN/kEpiGroups.
        // Groups 1-3 then hand their sorted lists to group 0 through shared
        // memory (bounded mbarrier waits per quadrant and round), which
        // merges them into the tile's one list of 8 per row.
        const int quad = warp & 3;
        const int grp = (warp - 2) >> 2;
        const int cols = tn / kEpiGroups;
        int buf = 0;
        uint32_t bph = 0;
        uint32_t xround = 0;          // exchange rounds of this quadrant so far
        bool alive = true;
        for (int ct = cid; ct < n_ct && alive; ct += n_ctas) {
            const int rt = ct % n_rt, at = ct / n_rt;
            const int nmb = RM == 1 ? 1 : min(RM, n_blk - rt * RM);
            bool ok = mbar_wait_bounded(&sh->tfull[buf], bph, lim) &&
                      !*reinterpret_cast<volatile int*>(&sh->abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) corr_timeout(a.err, sh);
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int mb = 0; mb < RM; ++mb) {
                if (mb >= nmb) break;
                const int row = (rt * RM + mb) * kBM + quad * 32 + lane;
                // the thread's best 8 as keys (score_key): larger score
                // first, then the smaller atom; 0 = empty
                uint32_t tk[kTop];
#pragma unroll
                for (int k = 0; k < kTop; ++k) tk[k] = 0u;
                const int m0 = at * tn + grp * cols;
                // a warp whose 32 rows are all past the active ones has
                // nothing to rank (uniform across the warp)
                const int c_end = (rt * RM + mb) * kBM + quad * 32 < n_act ? cols / 32 : 0;
                for (int c = 0; c < c_end; ++c) {
                    float v[32];
                    tmem_ld_32cols(tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                                       static_cast<uint32_t>((buf * RM + mb) * TN + grp * cols + c * 32),
                                   v);
                    if (a.dump && row < n_act) {
                        const float rsc = a.fp8 ? a.rscale[row] : 1.f;
                        for (int j = 0; j < 32; ++j) {
                            const int m = m0 + c * 32 + j;
                            if (m < a.M)
                                a.dump[static_cast<size_t>(row) * a.M + m] = v[j] * (a.fp8 ? a.colscale[m] * rsc : 1.f);
                        }
                    }
                    // branch-free: sort each group of 8 keys, then keep the best
                    // 8 of (list, group) -- every lane does the same work
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        uint32_t ck[8];
                        float cs8[8];
                        if (a.fp8) colscale8(a.colscale, m0 + c * 32 + h * 8, a.M, cs8);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = grp * cols + c * 32 + h * 8 + j;   // column in the tile
                            const int m = m0 + c * 32 + h * 8 + j;
                            float sc = fabsf(v[h * 8 + j]);
                            if (a.fp8) sc *= cs8[j];
                            ck[j] = (m < a.M && sc <= 3.0e38f) ? score_key(sc, col) : 0u;
                        }
                        sort8_desc(ck);
                        merge_top8(tk, ck);
                    }
                }
                // column groups that are not whole 32-column chunks (TN = 160
                // or 224, the TAIL instantiation): their last 16 and / or 8
                // columns
                if (TAIL && c_end > 0 && (cols & 31)) {
                    const int c0 = (cols / 32) * 32;
                    const uint32_t taddr = tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                                           static_cast<uint32_t>((buf * RM + mb) * TN + grp * cols + c0);
                    const bool dump_row = a.dump && row < n_act;
                    if (a.fp8) scan_top8<true>(taddr, cols - c0, grp * cols + c0, m0 + c0, a, row, dump_row, tk);
                    else scan_top8<false>(taddr, cols - c0, grp * cols + c0, m0 + c0, a, row, dump_row, tk);
                }
                if (mb == nmb - 1) {
                    // the buffer's last columns are in registers: the MMAs may reuse it
                    tc_fence_before();
                    mbar_arrive(&sh->tempty[buf]);
                }
                const int rr = quad * 32 + lane;      // row within the block
                if (grp != 0) {
                    // the slots are free once group 0 read the previous round
                    bool okx = xround == 0 || mbar_wait_bounded(&sh->xempty[quad], (xround - 1u) & 1u, lim);
                    okx = __all_sync(0xffffffffu, okx);
                    if (!okx) {
                        if (lane == 0) corr_timeout(a.err, sh);
                        alive = false;
                        break;
                    }
#pragma unroll
                    for (int k = 0; k < kTop; ++k) sh->xk[((grp - 1) * kTop + k) * kBM + rr] = tk[k];
                    mbar_arrive(&sh->xfull[quad]);
                } else {
                    bool okx = mbar_wait_bounded(&sh->xfull[quad], xround & 1u, lim);
                    okx = __all_sync(0xffffffffu, okx);
                    if (!okx) {
                        if (lane == 0) corr_timeout(a.err, sh);
                        alive = false;
                        break;
                    }
#pragma unroll
                    for (int g = 0; g < kEpiGroups - 1; ++g) {
                        uint32_t ck[kTop];
#pragma unroll
                        for (int k = 0; k < kTop; ++k) ck[k] = sh->xk[(g * kTop + k) * kBM + rr];
                        merge_top8(tk, ck);
                    }
                    mbar_arrive(&sh->xempty[quad]);
                    if (row < n_act) {
                        uint2* o = a.cand + (static_cast<size_t>(row) * x.n_at + at) * kTop;
#pragma unroll
                        for (int k = 0; k < kTop; ++k) {
                            const uint32_t m = static_cast<uint32_t>(at * tn + key_col(tk[k]));
                            o[k] = tk[k] ? make_uint2(key_score_bits(tk[k]), m) : make_uint2(0u, 0xffffffffu);
                        }
                    }
                }
                ++xround;
            }
            if (++buf == nbuf) {
                buf = 0;
                bph ^= 1u;
            }
        }
    }
}

// RM = 2: 256-row tiles while the batch has more 128-row tiles than the
// grid has CTAs, 128-row tiles once it has drained below that (the choice
// is made per launch from the active row count, the same in every CTA).
template <int RM, bool TAIL>
__global__ void __launch_bounds__(kGemmThreads, 1)
    corr_top8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmA3,
                     const __grid_constant__ CUtensorMap tmB3,
                     const CorrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    // operand tiles need 1024-byte alignment for the 128-byte swizzle atoms
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    CorrCtx x;
    // the ring the launch allocated (a.stages stages of RM row blocks and TN
    // atoms), then the barriers and the epilogue's exchange lists
    const uint32_t ring_bytes = static_cast<uint32_t>(a.stages) * (RM * kBM + a.TN) * kRowBytes;
    CorrShared* sh = reinterpret_cast<CorrShared*>(smem + ring_bytes);
    x.sh = sh;
    x.warp = threadIdx.x >> 5;
    x.lane = threadIdx.x & 31;
    const int warp = x.warp;
    // the step's select kernel appends its survivors to the other half; its
    // count was last read by the previous step, which has completed
    if (a.zero_next && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_next = 0;
    x.n_act = *a.n_act;
    x.n_blk = (x.n_act + kBM - 1) / kBM;     // 128-row blocks holding active rows
    const int rm = (RM == 2 && x.n_blk * a.n_at > static_cast<int>(gridDim.x)) ? 2 : 1;
    x.n_rt = (x.n_blk + rm - 1) / rm;        // row tiles of rm blocks
    // with few row blocks the grid has SMs to spare: tiles of TN / 2 atoms
    // double the tiles and give each SM 2/3 of the bytes of a TN-atom tile,
    // as long as they all still fit in one wave.  The candidate set each row
    // ends with is the same (its best 8 keys are in their tiles' lists)
    x.tn = a.TN;
    x.n_at = a.n_at;
    if (rm == 1 && a.half_ok) {
        const int n_at_h = (a.M + a.TN / 2 - 1) / (a.TN / 2);
        if (x.n_blk * n_at_h <= static_cast<int>(gridDim.x)) {
            x.tn = a.TN / 2;
            x.n_at = n_at_h;
        }
    }
    if (a.n_at_out && blockIdx.x == 0 && threadIdx.x == 0) *a.n_at_out = x.n_at;
    // the ring re-cut into stages of this launch's tile (rm row blocks, tn
    // atoms): a smaller tile gets a deeper ring, so that as many bytes stay
    // in flight per SM as with the largest one (up to kMaxStages stages).
    // Offsets stay 1024-byte aligned.
    x.as_stride = static_cast<uint32_t>(rm) * kBM * kRowBytes;
    x.b_stride = static_cast<uint32_t>(x.tn) * kRowBytes;
    // two K slices per stage (one 3-D box per operand) when the tile is one
    // row block by 128 atoms and the ring still holds 3 such stages: an SM
    // completes TMA boxes at a fixed rate, so bigger boxes feed it faster
    x.ks = (a.ks2_ok && rm == 1 && x.tn == 128 && ring_bytes / (2u * (x.as_stride + x.b_stride)) >= 3u) ? 2 : 1;
    x.stages = min(kMaxStages, static_cast<int>(ring_bytes / (static_cast<uint32_t>(x.ks) * (x.as_stride + x.b_stride))));
    x.tilesA = smem;
    x.tilesB = smem + x.stages * x.ks * x.as_stride;
    x.n_ct = x.n_rt * x.n_at;                       // tiles
    if (static_cast<int>(blockIdx.x) >= x.n_ct) return;   // a CTA with no tile
    x.lim = a.watchdog_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < x.stages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->tfull[b], 1);
            mbar_init(&sh->tempty[b], 4 * 32 * kEpiGroups);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(&sh->xfull[b], 32 * (kEpiGroups - 1));
            mbar_init(&sh->xempty[b], 32);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(x.tn == a.TN ? &tmB : &tmBh);
        if (x.ks == 2) {
            tma_prefetch_desc(&tmA3);
            tma_prefetch_desc(&tmB3);
        }
    }
    if (warp == 1) tmem_alloc(&sh->tmem_base, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    x.tmem = sh->tmem_base;
    const uint32_t tmem = x.tmem;

    const CUtensorMap* mb = x.tn == a.TN ? &tmB : &tmBh;
    if constexpr (RM == 2) {
        if (rm == 2) corr_roles<2, 1, TAIL>(&tmA, mb, &tmA3, &tmB3, a, x);
        else if (x.ks == 2) corr_roles<1, 2, false>(&tmA, mb, &tmA3, &tmB3, a, x);
        else corr_roles<1, 1, TAIL>(&tmA, mb, &tmA3, &tmB3, a, x);
    } else {
        if (x.ks == 2) corr_roles<1, 2, false>(&tmA, mb, &tmA3, &tmB3, a, x);
        else corr_roles<1, 1, TAIL>(&tmA, mb, &tmA3, &tmB3, a, x);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, static_cast<uint32_t>(a.tmem_cols));
    }
}

// ---------------------------------------------------------------- CTA pairs
// The same GEMM and epilogue on a two-SM tile: a cluster of two CTAs takes
// 256 signal rows (128 per CTA) x TN atoms, and the even CTA issues M = 256
// MMAs (cta_group::2) that read each CTA's own 128 rows and its half of the
// TN atom rows from the same shared-memory offsets.  Each SM then holds a
// 128 x TN accumulator, so TMEM keeps two of them: the epilogue of one tile
// runs under the MMAs of the next, at the bytes per flop of a 256 x 256
// single-CTA tile.  Tiles are ordered row pair fastest, so the clusters
// running at one time share the atom tile they stream.

// Per-CTA state of the paired kernel.
struct PairCtx {
    uint8_t* tilesA;     // A stages (128 rows each)
    uint8_t* tilesB;     // B stages (TN / 2 atom rows each)
    CorrShared* sh;
    uint32_t tmem;
    uint32_t rank;       // 0: the CTA that issues the MMAs, 1: its peer
    int n_act, n_rp, n_pt;   // active rows, row pairs (256-row tiles), tiles
    int warp, lane;
    uint64_t lim;
};

// cluster address of `p` (a shared variable of this CTA) in CTA `rank`
MP_DEV uint32_t in_cta(const void* p, uint32_t rank) { return mapa_shared(smem_u32(p), rank); }

// Bytes one CTA loads for its 128-row block of a stage (rows: its active
// rows): the whole block as one box if any row is active, else nothing.
MP_DEV uint32_t pair_a_bytes(int rows) { return rows > 0 ? static_cast<uint32_t>(kBM) * kRowBytes : 0u; }

template <bool FP8>
MP_DEV void pair_roles(const CUtensorMap* tmA, const CUtensorMap* tmB, const CorrArgs& a,
                       const PairCtx& x) {
    const int TN = a.TN;
    const int half = TN / 2;
    const uint32_t as_bytes = kBM * kRowBytes;
    const uint32_t bs_bytes = static_cast<uint32_t>(half) * kRowBytes;
    const int stages = a.stages;
    CorrShared* sh = x.sh;
    const int n_act = x.n_act, n_rp = x.n_rp, n_pt = x.n_pt;
    const int cl = static_cast<int>(blockIdx.x >> 1), n_cl = static_cast<int>(gridDim.x >> 1);
    const int warp = x.warp, lane = x.lane;
    const uint64_t lim = x.lim;
    const uint32_t rank = x.rank;
    const int kelems = FP8 ? kRowBytes : kRowBytes / 2;

    if (warp == 0) {
        // ---------------- TMA producer of this CTA (one thread).  Its loads
        // complete on the even CTA's `full` barrier, whose expected bytes
        // the even CTA's producer sets for both.
        if (lane == 0) {
            const uint32_t full0 = in_cta(&sh->full[0], 0);
            long long g = 0;
            int s = 0;
            uint32_t ph = 0;
            bool stop = false;
            for (int pt = cl; pt < n_pt && !stop; pt += n_cl) {
                const int rp = pt % n_rp, at = pt / n_rp;
                const int row0 = (rp * 2 + static_cast<int>(rank)) * kBM;
                const bool rows = n_act > row0;   // this CTA's block has active rows
                const uint32_t tx = pair_a_bytes(n_act - rp * 2 * kBM) + pair_a_bytes(n_act - (rp * 2 + 1) * kBM) +
                                    2u * bs_bytes;
                for (int kb = 0; kb < a.nk; ++kb) {
                    if (g >= stages && !mbar_wait_bounded(&sh->empty[s], ph ^ 1u, lim)) {
                        corr_timeout(a.err, sh);
                        stop = true;
                        break;
                    }
                    if (*reinterpret_cast<volatile int*>(&sh->abort)) {
                        stop = true;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&sh->full[s], tx);
                    const uint32_t bar = full0 + static_cast<uint32_t>(s) * 8u;
                    uint8_t* dst = x.tilesA + s * as_bytes;
                    if (rows) tma_load_2d_pair(dst, tmA, kb * kelems, row0, bar);
                    tma_load_2d_pair(x.tilesB + s * bs_bytes, tmB, kb * kelems, at * TN + static_cast<int>(rank) * half,
                                     bar);
                    ++g;
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // before the CTA may exit: the MMAs released every stage's last
            // use (so this CTA's loads into it have landed and been read)
            for (int t = 0; t < stages && t < g; ++t) {
                const long long last = g - 1 - ((g - 1 - t) % stages);
                mbar_wait_bounded(&sh->empty[t], static_cast<uint32_t>((last / stages) & 1), lim);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: one thread of the even CTA
        if (lane == 0 && rank == 0) {
            const uint32_t idesc = make_idesc(2 * kBM, TN, FP8 ? 0u : 1u);
            int s = 0, buf = 0, li = 0;
            uint32_t ph = 0, bph = 0;
            bool ok = true;
            for (int pt = cl; pt < n_pt && ok; pt += n_cl, ++li) {
                if (li >= 2 && !mbar_wait_bounded(&sh->tempty[buf], bph ^ 1u, lim)) {
                    corr_timeout(a.err, sh);
                    break;
                }
                tc_fence_after();
                const uint32_t d = x.tmem + static_cast<uint32_t>(buf * TN);
                for (int kb = 0; kb < a.nk; ++kb) {
                    if (!mbar_wait_bounded(&sh->full[s], ph, lim) || *reinterpret_cast<volatile int*>(&sh->abort)) {
                        corr_timeout(a.err, sh);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t a0 = sw128_kmajor_desc(smem_u32(x.tilesA + s * as_bytes));
                    const uint64_t b0 = sw128_kmajor_desc(smem_u32(x.tilesB + s * bs_bytes));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = (kb == 0 && k == 0) ? 0u : 1u;
                        if (FP8) mma_fp8_pair(d, a0 + 2 * k, b0 + 2 * k, idesc, acc);
                        else mma_bf16_pair(d, a0 + 2 * k, b0 + 2 * k, idesc, acc);
                    }
                    // both CTAs' copies of the stage are free once these finish
                    mma_commit_pair(in_cta(&sh->empty[s], 0));
                    mma_commit_pair(in_cta(&sh->empty[s], 1));
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) {
                    mma_commit_pair(in_cta(&sh->tfull[buf], 0));
                    mma_commit_pair(in_cta(&sh->tfull[buf], 1));
                }
                if (++buf == 2) {
                    buf = 0;
                    bph ^= 1u;
                }
            }
            // no MMA may still write TMEM when it is freed
            mma_commit_pair(in_cta(&sh->drain, 0));
            mbar_wait_bounded(&sh->drain, 0u, lim);
        }
    } else {
        // ---------------- epilogue of this CTA's 128 rows (as corr_roles:
        // warp w reads TMEM lane quadrant w % 4, column group (w - 2) / 4)
        const int quad = warp & 3;
        const int grp = (warp - 2) >> 2;
        const int cols = TN / kEpiGroups;
        const uint32_t tempty0 = in_cta(&sh->tempty[0], 0);
        int buf = 0;
        uint32_t bph = 0, xround = 0;
        bool alive = true;
        for (int pt = cl; pt < n_pt && alive; pt += n_cl) {
            const int rp = pt % n_rp, at = pt / n_rp;
            bool ok = mbar_wait_bounded(&sh->tfull[buf], bph, lim) && !*reinterpret_cast<volatile int*>(&sh->abort);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) corr_timeout(a.err, sh);
                break;
            }
            tc_fence_after();
            const int blk0 = (rp * 2 + static_cast<int>(rank)) * kBM;
            const int row = blk0 + quad * 32 + lane;
            uint32_t tk[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) tk[k] = 0u;
            // a warp whose 32 rows are all past the active ones has nothing to rank
            if (blk0 + quad * 32 < n_act) {
                const uint32_t taddr = x.tmem + (static_cast<uint32_t>(quad * 32) << 16) +
                                       static_cast<uint32_t>(buf * TN + grp * cols);
                const bool dump_row = a.dump && row < n_act;
                scan_top8<FP8>(taddr, cols, grp * cols, at * TN + grp * cols, a, row, dump_row, tk);
            }
            // the accumulator buffer is in registers: the MMAs may reuse it
            // (one arrival per warp of each CTA on the even CTA's barrier)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) mbar_arrive(&sh->tempty[buf]);
                else mbar_arrive_remote(tempty0 + static_cast<uint32_t>(buf) * 8u);
            }
            const int rr = quad * 32 + lane;
            if (grp != 0) {
                bool okx = xround == 0 || mbar_wait_bounded(&sh->xempty[quad], (xround - 1u) & 1u, lim);
                okx = __all_sync(0xffffffffu, okx);
                if (!okx) {
                    if (lane == 0) corr_timeout(a.err, sh);
                    alive = false;
                    break;
                }
#pragma unroll
                for (int k = 0; k < kTop; ++k) sh->xk[((grp - 1) * kTop + k) * kBM + rr] = tk[k];
                mbar_arrive(&sh->xfull[quad]);
            } else {
                bool okx = mbar_wait_bounded(&sh->xfull[quad], xround & 1u, lim);
                okx = __all_sync(0xffffffffu, okx);
                if (!okx) {
                    if (lane == 0) corr_timeout(a.err, sh);
                    alive = false;
                    break;
                }
#pragma unroll
                for (int g = 0; g < kEpiGroups - 1; ++g) {
                    uint32_t ck[kTop];
#pragma unroll
                    for (int k = 0; k < kTop; ++k) ck[k] = sh->xk[(g * kTop + k) * kBM + rr];
                    merge_top8(tk, ck);
                }
                mbar_arrive(&sh->xempty[quad]);
                if (row < n_act) {
                    uint2* o = a.cand + (static_cast<size_t>(row) * a.n_at + at) * kTop;
#pragma unroll
                    for (int k = 0; k < kTop; ++k) {
                        const uint32_t m = static_cast<uint32_t>(at * TN + key_col(tk[k]));
                        o[k] = tk[k] ? make_uint2(key_score_bits(tk[k]), m) : make_uint2(0u, 0xffffffffu);
                    }
                }
            }
            ++xround;
            if (++buf == 2) {
                buf = 0;
                bph ^= 1u;
            }
        }
    }
}

// Two CTAs (a cluster) per tile of 256 signal rows x a.TN atoms; a.stages
// is corr_stages(128, a.TN / 2), a.tmem_cols 2 * a.TN rounded up to a power
// of two.  tmB's box is a.TN / 2 atom rows.
template <bool FP8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGemmThreads, 1)
    corr_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const CorrArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_u32 = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
    const uint32_t as_bytes = kBM * kRowBytes;
    const uint32_t bs_bytes = static_cast<uint32_t>(a.TN / 2) * kRowBytes;
    PairCtx x;
    x.tilesA = smem;
    x.tilesB = smem + a.stages * as_bytes;
    CorrShared* sh = reinterpret_cast<CorrShared*>(x.tilesB + a.stages * bs_bytes);
    x.sh = sh;
    x.warp = static_cast<int>(threadIdx.x >> 5);
    x.lane = static_cast<int>(threadIdx.x & 31);
    x.rank = cluster_ctarank();
    if (a.zero_next && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_next = 0;
    if (a.n_at_out && blockIdx.x == 0 && threadIdx.x == 0) *a.n_at_out = a.n_at;
    x.n_act = *a.n_act;
    const int n_blk = (x.n_act + kBM - 1) / kBM;
    x.n_rp = (n_blk + 1) / 2;
    x.n_pt = x.n_rp * a.n_at;
    // both CTAs of a cluster leave together, before any barrier or TMEM use
    if (static_cast<int>(blockIdx.x >> 1) >= x.n_pt) return;
    x.lim = a.watchdog_ns;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->tfull[b], 1);
            mbar_init(&sh->tempty[b], 2 * 4 * kEpiGroups);   // one arrival per epilogue warp of both CTAs
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(&sh->xfull[b], 32 * (kEpiGroups - 1));
            mbar_init(&sh->xempty[b], 32);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (x.warp == 1) tmem_alloc_pair(&sh->tmem_base, static_cast<uint32_t>(a.tmem_cols));
    tc_fence_before();
    __syncthreads();
    // the peer's barriers are initialised before either CTA signals them
    cluster_sync_all();
    tc_fence_after();
    x.tmem = sh->tmem_base;
    pair_roles<FP8>(&tmA, &tmB, a, x);
    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still signal its barriers or
    // the MMAs read its shared memory
    cluster_sync_all();
    if (x.warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(x.tmem, static_cast<uint32_t>(a.tmem_cols));
    }
}

int corr_smem_bytes(int TM, int TN) {
    return 1024 + corr_stages(TM, TN) * (TM * kRowBytes + TN * kRowBytes) + static_cast<int>(sizeof(CorrShared));
}

template <int RM, bool TAIL>
static cudaError_t set_attrs() {
    int most = 0;
    for (int tn = 128; tn <= 256; tn += 32) most = std::max(most, corr_smem_bytes(kBM * RM, tn));
    return cudaFuncSetAttribute(corr_top8_kernel<RM, TAIL>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
}

cudaError_t corr_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = set_attrs<1, false>();
    if (e == cudaSuccess) e = set_attrs<2, false>();
    if (e == cudaSuccess) e = set_attrs<1, true>();
    if (e == cudaSuccess) e = set_attrs<2, true>();
    if (e == cudaSuccess) done = true;
    return e;
}

// CTAs that can be resident at once (one per SM: each takes most of the
// SM's shared memory).
int corr_max_ctas() {
    static int cache = -1;
    if (cache >= 0) return cache;
    int sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm < 1) {
        cudaGetLastError();
        return 1;
    }
    cache = sm;
    return cache;
}

cudaError_t launch_corr_top8(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmBh,
                             const CUtensorMap& tmA3, const CUtensorMap& tmB3, const CorrArgs& a, int max_rows,
                             cudaStream_t st) {
    const int nbuf = (a.RM == 1 || a.RM * a.TN * 2 <= 512) ? 2 : 1;   // as the kernel computes it
    if ((a.RM != 1 && a.RM != 2) || a.TN < 128 || a.TN > 256 || a.TN % 32 || nbuf * a.RM * a.TN > a.tmem_cols ||
        a.stages != corr_stages(kBM * a.RM, a.TN) || (a.half_ok && a.TN != 256))
        return cudaErrorInvalidValue;
    // enough CTAs for the largest tile count this launch can see (with
    // RM = 2 the kernel takes 128-row tiles whenever they fit the grid, so
    // the grid is sized by those)
    const int max_rt = (max_rows + kBM - 1) / kBM;
    int max_ct = max_rt * a.n_at;
    if (a.half_ok)   // room for the half-width tiles of one or two row blocks
        max_ct = std::max(max_ct, std::min(max_rt, 2) * ((a.M + a.TN / 2 - 1) / (a.TN / 2)));
    const int ctas = std::max(1, std::min(max_ct, corr_max_ctas()));
    const int smem = corr_smem_bytes(kBM * a.RM, a.TN);
    // column groups of TN / 4 that are not whole 32-column chunks need the
    // tail scan (TN = 160, 224)
    const bool tail = (a.TN / kEpiGroups) % 32 != 0;
    if (a.RM == 2) {
        if (tail) corr_top8_kernel<2, true><<<ctas, kGemmThreads, smem, st>>>(tmA, tmB, tmBh, tmA3, tmB3, a);
        else corr_top8_kernel<2, false><<<ctas, kGemmThreads, smem, st>>>(tmA, tmB, tmBh, tmA3, tmB3, a);
    } else {
        if (tail) corr_top8_kernel<1, true><<<ctas, kGemmThreads, smem, st>>>(tmA, tmB, tmBh, tmA3, tmB3, a);
        else corr_top8_kernel<1, false><<<ctas, kGemmThreads, smem, st>>>(tmA, tmB, tmBh, tmA3, tmB3, a);
    }
    return cudaGetLastError();
}

int pair_smem_bytes(int TN) { return corr_smem_bytes(kBM, TN / 2); }

cudaError_t pair_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    int most = 0;
    for (int tn = 128; tn <= 256; tn += 32) most = std::max(most, pair_smem_bytes(tn));
    cudaError_t e = cudaFuncSetAttribute(corr_pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(corr_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess) done = true;
    return e;
}

// Clusters of two that can be resident at once for a tile of TN atoms
// (at most half the SMs; fewer when the GPCs cannot all be paired).
int pair_max_clusters(int TN, bool fp8) {
    static int cache[2][9] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1, -1, -1, -1}};
    const int slot = (TN - 128) / 16;
    if (TN < 128 || TN > 256 || TN % 16) return 1;
    int& c = cache[fp8 ? 1 : 0][slot];
    if (c >= 0) return c;
    const int half = std::max(1, corr_max_ctas() / 2);
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2 * half, 1, 1);
    cfg.blockDim = dim3(kGemmThreads, 1, 1);
    cfg.dynamicSmemBytes = pair_smem_bytes(TN);
    int n = 0;
    const cudaError_t e =
        fp8 ? cudaOccupancyMaxActiveClusters(&n, reinterpret_cast<const void*>(corr_pair_kernel<true>), &cfg)
            : cudaOccupancyMaxActiveClusters(&n, reinterpret_cast<const void*>(corr_pair_kernel<false>), &cfg);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = half;
    }
    c = std::min(n, half);
    return c;
}

cudaError_t launch_corr_pair(const CUtensorMap& tmA, const CUtensorMap& tmBp,
                             const CorrArgs& a, int max_rows, cudaStream_t st) {
    if (a.TN < 128 || a.TN > 256 || a.TN % 32 || 2 * a.TN > a.tmem_cols || a.stages != corr_stages(kBM, a.TN / 2) ||
        a.half_ok)
        return cudaErrorInvalidValue;
    const int max_rp = ((max_rows + kBM - 1) / kBM + 1) / 2;
    const int clusters = std::max(1, std::min(max_rp * a.n_at, pair_max_clusters(a.TN, a.fp8 != 0)));
    const int smem = pair_smem_bytes(a.TN);
    if (a.fp8) corr_pair_kernel<true><<<2 * clusters, kGemmThreads, smem, st>>>(tmA, tmBp, a);
    else corr_pair_kernel<false><<<2 * clusters, kGemmThreads, smem, st>>>(tmA, tmBp, a);
    return cudaGetLastError();
}

}  // namespace mpgb
