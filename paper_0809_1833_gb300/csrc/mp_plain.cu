// Persistent FP32 Matching Pursuit kernel (Sec. 3, Eqs. 8-12): one launch
// runs every iteration of one decode on the device.
//
// Each CTA owns a contiguous slice of atoms and keeps a full copy of the
// residual r in shared memory.  Per iteration:
//   1. correlate  c_m = <r, psi_m> for the CTA's atoms       (Eq. 9)
//   2. select     the CTA's best packed key (|c|, -m, sign)  (Eq. 9, Sec. 4 ties)
//   3. exchange   the grid-wide max key (a hardware cluster barrier, then every
//                 warp reads all of the cluster's warp keys over DSMEM; or
//                 global atomics and a bounded grid barrier)
//   4. update     every CTA applies r -= c psi_m* to its own copy of r
//                 (identical arithmetic in every CTA, so all copies stay
//                 bit-identical) and reduces e = sum r^2 in FP64   (Eq. 11)
//   5. CTA 0 adds c to x~_m*                                  (Eq. 10)
//   6. every CTA evaluates the same stop test e <= eps^2 e0 or t = T.
//
// Launch shapes (chosen per plan from N, M and shared-memory capacity):
//   mode 1  one cluster of up to 16 CTAs, the whole dictionary resident in
//           the cluster's shared memory (small dictionaries: latency bound)
//   mode 2  one CTA per SM, the dictionary resident across the grid
//   mode 3  one CTA per SM; a producer warp streams the CTA's atoms from HBM
//           through a ring of shared-memory stages with 1-D bulk copies and
//           mbarriers, running ahead across iteration boundaries so that the
//           exchange/update bubble overlaps the next pass's loads.  Consumer
//           warps own whole-atom slots; in FP64 with large atoms, groups of 4
//           warps share each stage instead (one class of segments per warp)
//           and an atom streams as several stages.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mp_device.cuh"
#include "mp_dot.cuh"
#include "mp_internal.h"

namespace mpgb {

constexpr int kMaxWarps = 32;
constexpr int kMaxStages = 64;
constexpr int kResidentThreads = 256;
constexpr int kMaxClusterCtas = 16;
// mode 1: every warp key of the cluster, in every CTA
constexpr int kClusterKeys = kMaxClusterCtas * (kResidentThreads / 32);
// FP64 streaming with shared stages: a producer warp and two groups of four
// consumer warps (two warps per SM sub-partition keep its FP64 pipe fed)
constexpr int kCoopGroups = 2;
constexpr int kMaxPlainThreads = 32 * (1 + 4 * kCoopGroups);
// FP64 sums of squares (the energy, OMP's ||w||^2) run as kSumChains FMA
// chains (chain i takes the elements i, i + kSumChains, ...), then warp sums
// in warp order: the same bits for every launch shape, whatever its thread
// count (each shape has at least kSumChains compute threads).
constexpr int kSumChains = 128;

// Per-precision types: the argmax key and the 16-byte vector the residual
// and the atoms are read in.
template <typename T>
struct PlainTraits;
template <>
struct PlainTraits<float> {
    using Key = unsigned long long;
    using V = float4;
};
template <>
struct PlainTraits<double> {
    using Key = Key128;
    using V = double2;
};

// FP64 grid streaming with atoms too large for two ring slots per warp:
// every warp computes its class of each atom's sum (see dot1 for double)
// into these partials, kept for a window of kCoopWindow atoms and double-
// buffered by the window's parity; after the window's barrier each warp
// combines a quarter of its atoms.
constexpr int kCoopWindow = 8;
template <typename T>
struct CoopPartials {};
template <>
struct CoopPartials<double> {
    double part[2][kCoopWindow][4][32];
    int abort[2];
};

template <typename T>
struct PlainShared {
    using Key = typename PlainTraits<T>::Key;
    CoopPartials<T> coop;
    Key wkeys[2][kClusterKeys];          // mode 1: the cluster's warp keys (CTA-major), two-slot ring
    Key wkey[kMaxWarps];                 // per compute warp best key
    double wsum[kMaxWarps];              // per compute warp energy partial
    Key key;                             // selected key broadcast
    int abort;
    int done;
    uint64_t full[kMaxStages];           // mode 3 ring barriers
    uint64_t empty[kMaxStages];
};

template <typename T>
struct PlainArgs {
    const T* psi;          // M x ldN atom-major, zero padded
    const T* y;            // N
    T* x;                  // M
    int N, ldN, M, T_max;
    double eps2;
    int stage_atoms, stages;
    int stage_elems;       // mode 3: elements per ring stage (its stride in the ring)
    int pieces;            // mode 3: stages per atom (> 1: one atom streams as pieces)
    int prefetch;          // mode 3: L2 prefetch distance in stages (0 = off)
    int evict_first;       // mode 3: evict-first L2 hint on the streamed atoms
    int l2_keep_atoms;     // mode 3: the CTA's first atoms loaded evict-last (kept in L2)
    int off_sh, off_data;
    PlainWorkspace* ws;
    Key128* slots;         // FP64 grid exchange: two rings of one key per CTA
    const T* G;            // mode 4: Gram matrix, row stride ldG
    int ldG;
    int gram_period;       // mode 4: direct correlations every gram_period steps
    // modes 5, 6 (OMP): orthonormal basis Q of the selected atoms (kmax rows
    // of ldN), R = Q^T Psi_S by packed columns (column k at k(k+1)/2),
    // alpha = Q^T y, the selected atoms, Gram-Schmidt scratch, per-CTA norm
    // partials and the solution of R x_S = alpha
    T* Q;
    T* Rc;
    T* alpha;
    int* sel;
    T* h;
    T* h2;
    T* w;
    T* w2;
    T* wpart;              // 4 x ldN partial sums of the Gram-Schmidt update
    double* nrm;
    T* xs;
    int kmax;
    int coop;              // FP64 streaming: four warps share every stage (CoopPartials)
    int piece_elems;       // coop: elements per piece (whole 4-segment groups)
    int* tr_atoms;
    T* tr_coefs;
    double* tr_energy;
    T* tr_resid;
    int tr_cap;
    unsigned long long watchdog_ns;
    int skip_cta;
};

// ------------------------------------------------------------------ vectors
MP_DEV double sq_acc(const float4 v, double acc) {
    acc = fma(static_cast<double>(v.x), static_cast<double>(v.x), acc);
    acc = fma(static_cast<double>(v.y), static_cast<double>(v.y), acc);
    acc = fma(static_cast<double>(v.z), static_cast<double>(v.z), acc);
    acc = fma(static_cast<double>(v.w), static_cast<double>(v.w), acc);
    return acc;
}
MP_DEV double sq_acc(const double2 v, double acc) {
    acc = fma(v.x, v.x, acc);
    acc = fma(v.y, v.y, acc);
    return acc;
}
// v - c p, elementwise
MP_DEV float4 sub_scaled(float c, const float4 p, float4 v) {
    v.x = fmaf(-c, p.x, v.x);
    v.y = fmaf(-c, p.y, v.y);
    v.z = fmaf(-c, p.z, v.z);
    v.w = fmaf(-c, p.w, v.w);
    return v;
}
MP_DEV double2 sub_scaled(double c, const double2 p, double2 v) {
    v.x = fma(-c, p.x, v.x);
    v.y = fma(-c, p.y, v.y);
    return v;
}
MP_DEV float4 scale_vec(const float4 v, float s) { return make_float4(v.x * s, v.y * s, v.z * s, v.w * s); }
MP_DEV double2 scale_vec(const double2 v, double s) { return make_double2(v.x * s, v.y * s); }
MP_DEV void dsmem_ld(uint32_t addr, float4* v) { *v = dsmem_ld_f32x4(addr); }
MP_DEV void dsmem_ld(uint32_t addr, double2* v) { *v = dsmem_ld_f64x2(addr); }
MP_DEV void dsmem_ld(uint32_t addr, unsigned long long* k) { *k = dsmem_ld_u64(addr); }
MP_DEV void dsmem_ld(uint32_t addr, Key128* k) {
    k->hi = dsmem_ld_u64(addr);
    k->lo = dsmem_ld_u64(addr + 8u);
}
MP_DEV void dsmem_st(uint32_t addr, unsigned long long k) { dsmem_st_u64(addr, k); }
MP_DEV void dsmem_st(uint32_t addr, const Key128& k) {
    dsmem_st_u64(addr, k.hi);
    dsmem_st_u64(addr + 8u, k.lo);
}

// ------------------------------------------------------------------ dots
// Scan `n` consecutive atoms at p (first index m0) and fold into `best`.
template <typename T, typename Key>
MP_DEV Key scan_atoms(const T* __restrict__ p, const T* __restrict__ r, int ldN, int n, int m0, int lane, Key best) {
    int q = 0;
    for (; q + 4 <= n; q += 4) {
        T c[4];
        dot4(p + static_cast<size_t>(q) * ldN, r, ldN, lane, c);
#pragma unroll
        for (int i = 0; i < 4; ++i) best = kmax(best, pack_key(c[i], m0 + q + i));
    }
    for (; q < n; ++q) best = kmax(best, pack_key(dot1(p + static_cast<size_t>(q) * ldN, r, ldN, lane), m0 + q));
    return best;
}

// ------------------------------------------------------------------ grid barrier
// Wait (bounded) until all G CTAs arrived at barrier t.
MP_DEV bool grid_wait(PlainWorkspace* ws, unsigned long long target, unsigned long long limit_ns) {
    if (ld_acquire_u64(&ws->count) < target) {
        const uint64_t deadline = globaltimer_ns() + limit_ns;
        while (ld_acquire_u64(&ws->count) < target) {
            if (ld_volatile_i32(&ws->err) != 0 || globaltimer_ns() > deadline) {
                atomicCAS(&ws->err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                return false;
            }
        }
    }
    return true;
}

// FP32 (one thread): fold the CTA's key into the iteration's slot with a
// 64-bit atomic max, arrive at grid barrier `bar`, wait, read the max.
MP_DEV bool grid_exchange(const PlainArgs<float>& a, int cta, int G, int t, int bar, unsigned long long k,
                          unsigned long long* out) {
    PlainWorkspace* ws = a.ws;
    atomicMax(&ws->keys[t % 3], k);
    if (!(cta == a.skip_cta && t == 0)) red_release_add_u64(&ws->count, 1ull);
    if (!grid_wait(ws, static_cast<unsigned long long>(bar + 1) * G, a.watchdog_ns)) return false;
    *out = ld_relaxed_u64(&ws->keys[t % 3]);
    // slot (t+2)%3 was last read at iteration t-1, before every CTA arrived
    // at this barrier; it is next written at iteration t+2, after the next one.
    if (cta == 0) st_relaxed_u64(&ws->keys[(t + 2) % 3], 0ull);
    return true;
}

// FP64 (one warp): the 128-bit key has no atomic max, so each CTA writes its
// key to its own slot of ring t&1, arrives, and after the barrier every lane
// reads a share of the G slots; a warp max gives the grid's key.  Ring t&1
// is rewritten at iteration t+2, after barrier t+1, which every CTA reaches
// only after finishing its reads of iteration t.
MP_DEV bool grid_exchange(const PlainArgs<double>& a, int cta, int G, int t, Key128 k, int lane, Key128* out) {
    PlainWorkspace* ws = a.ws;
    Key128* ring = a.slots + (t & 1) * G;
    if (lane == 0) {
        st_relaxed_u64(&ring[cta].hi, k.hi);
        st_relaxed_u64(&ring[cta].lo, k.lo);
        if (!(cta == a.skip_cta && t == 0)) red_release_add_u64(&ws->count, 1ull);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, grid_wait(ws, static_cast<unsigned long long>(t + 1) * G,
                                                      a.watchdog_ns));
    if (!ok) return false;
    Key128 best = {0ull, 0ull};
    for (int i = lane; i < G; i += 32) {
        Key128 v;
        v.hi = ld_relaxed_u64(&ring[i].hi);
        v.lo = ld_relaxed_u64(&ring[i].lo);
        best = kmax(best, v);
    }
    *out = warp_max_key(best);
    return true;
}

// Every compute thread of every CTA: grid barrier `bar` (the CTA's writes
// before it are visible to every CTA after it).  False when the wait ran
// out (the error word is set; the CTA's abort flag too).
template <typename T>
MP_DEV bool cta_grid_sync(const PlainArgs<T>& a, PlainShared<T>* sh, int G, int bar, int ct, int nct) {
    named_bar_sync(1, nct);
    if (ct == 0) {
        red_release_add_u64(&a.ws->count, 1ull);
        if (!grid_wait(a.ws, static_cast<unsigned long long>(bar + 1) * G, a.watchdog_ns))
            *reinterpret_cast<volatile int*>(&sh->abort) = 1;
    }
    named_bar_sync(1, nct);
    return *reinterpret_cast<volatile int*>(&sh->abort) == 0;
}

// <q, r> with q = s w elementwise, in dot1's order (one warp).
MP_DEV float dot1_scaled(const float* __restrict__ w, float s, const float* __restrict__ r, int ldN, int lane) {
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
    for (int off = lane * 4; off < ldN; off += 128) {
        const float4 q = *reinterpret_cast<const float4*>(r + off);
        const float4 v = *reinterpret_cast<const float4*>(w + off);
        ax = fmaf(v.x * s, q.x, ax);
        ay = fmaf(v.y * s, q.y, ay);
        az = fmaf(v.z * s, q.z, az);
        aw = fmaf(v.w * s, q.w, aw);
    }
    return warp_sum_f32((ax + ay) + (az + aw));
}

// ------------------------------------------------------------------ producer
template <typename T>
MP_DEV void plain_producer(const PlainArgs<T>& a, PlainShared<T>* sh, T* ring, int a0, int na) {
    const int A = a.stage_atoms, D = a.stages, ldN = a.ldN;
    const int S = (na + A - 1) / A;
    if (S == 0) return;
    const size_t stage_elems = static_cast<size_t>(A) * ldN;
    const uint64_t pol = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    volatile int* vdone = &sh->done;
    long long seq = 0;
    while (true) {
        const int slot = static_cast<int>(seq % D);
        if (seq >= D) {
            const uint32_t par = static_cast<uint32_t>(((seq / D) - 1) & 1);
            bool ok = mbar_try_wait(&sh->empty[slot], par);
            uint64_t deadline = 0;
            while (!ok) {
                if (*vdone) break;
                const uint64_t now = globaltimer_ns();
                if (deadline == 0) {
                    deadline = now + a.watchdog_ns;
                } else if (now > deadline) {
                    atomicCAS(&a.ws->err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                    *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                    break;
                }
                ok = mbar_try_wait(&sh->empty[slot], par);
            }
            if (!ok) break;
        }
        if (*vdone) break;
        const int j = static_cast<int>(seq % S);
        const int atom0 = a0 + j * A;
        const int nat = min(A, na - j * A);
        const uint32_t bytes = static_cast<uint32_t>(nat) * ldN * static_cast<uint32_t>(sizeof(T));
        mbar_arrive_expect_tx(&sh->full[slot], bytes);
        // the first l2_keep_atoms atoms of the slice stay in L2 from pass to
        // pass (evict-last); the rest streams through it (evict-first)
        if (j * A < a.l2_keep_atoms)
            bulk_g2s_hint(ring + slot * stage_elems, a.psi + static_cast<size_t>(atom0) * ldN, bytes,
                          &sh->full[slot], pol_keep);
        else if (a.evict_first)
            bulk_g2s_hint(ring + slot * stage_elems, a.psi + static_cast<size_t>(atom0) * ldN, bytes,
                          &sh->full[slot], pol);
        else
            bulk_g2s(ring + slot * stage_elems, a.psi + static_cast<size_t>(atom0) * ldN, bytes, &sh->full[slot]);
        // L2 as a deeper window than the shared-memory ring: pull the stage
        // `prefetch` positions ahead into L2 now, so HBM keeps streaming
        // while the ring is full during the per-iteration exchange.
        if (a.prefetch > 0) {
            const int jp = static_cast<int>((seq + a.prefetch) % S);
            const int np = min(A, na - jp * A);
            prefetch_l2(a.psi + static_cast<size_t>(a0 + jp * A) * ldN,
                        static_cast<uint32_t>(np) * ldN * static_cast<uint32_t>(sizeof(T)));
        }
        ++seq;
    }
    // Wait for every copy still in flight before the CTA may exit: the only
    // outstanding copy of slot k is the last one issued into it.
    const long long issued = seq;
    for (int k = 0; k < D && k < issued; ++k) {
        const long long last = issued - 1 - ((issued - 1 - k) % D);
        mbar_wait_bounded(&sh->full[k], static_cast<uint32_t>((last / D) & 1), a.watchdog_ns);
    }
}

// The same for the FP64 shared-stage shape: stage j of a pass is piece
// j % np of atom j / np (np >= 1), stages piece_elems elements apart.
template <typename T>
MP_DEV void plain_producer_shared(const PlainArgs<T>& a, PlainShared<T>* sh, T* ring, int a0, int na) {
    const int D = a.stages, ldN = a.ldN, np = a.pieces;
    if (na == 0) return;
    const size_t stage_elems = static_cast<size_t>(a.stage_elems);
    const uint64_t pol = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    volatile int* vdone = &sh->done;
    // ring position (slot, parity of its use count) and stage (atom, piece),
    // kept incrementally
    long long seq = 0;
    int slot = 0, ja = 0, jp = 0;
    uint32_t upar = 0;
    while (true) {
        if (seq >= D) {
            const uint32_t par = upar ^ 1u;
            bool ok = mbar_try_wait(&sh->empty[slot], par);
            uint64_t deadline = 0;
            while (!ok) {
                if (*vdone) break;
                const uint64_t now = globaltimer_ns();
                if (deadline == 0) {
                    deadline = now + a.watchdog_ns;
                } else if (now > deadline) {
                    atomicCAS(&a.ws->err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                    *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                    break;
                }
                ok = mbar_try_wait(&sh->empty[slot], par);
            }
            if (!ok) break;
        }
        if (*vdone) break;
        // this stage: piece jp of atom ja
        const int atom0 = a0 + ja;
        const size_t off = static_cast<size_t>(jp) * a.piece_elems;
        const int nel = min(a.piece_elems, ldN - jp * a.piece_elems);
        const uint32_t bytes = static_cast<uint32_t>(nel) * static_cast<uint32_t>(sizeof(T));
        const T* src = a.psi + static_cast<size_t>(atom0) * ldN + off;
        mbar_arrive_expect_tx(&sh->full[slot], bytes);
        // the first l2_keep_atoms atoms of the slice stay in L2 from pass to
        // pass (evict-last); the rest streams through it (evict-first)
        if (atom0 - a0 < a.l2_keep_atoms)
            bulk_g2s_hint(ring + slot * stage_elems, src, bytes, &sh->full[slot], pol_keep);
        else if (a.evict_first)
            bulk_g2s_hint(ring + slot * stage_elems, src, bytes, &sh->full[slot], pol);
        else
            bulk_g2s(ring + slot * stage_elems, src, bytes, &sh->full[slot]);
        ++seq;
        if (++slot == D) {
            slot = 0;
            upar ^= 1u;
        }
        if (++jp == np) {
            jp = 0;
            if (++ja == na) ja = 0;
        }
    }
    // Wait for every copy still in flight before the CTA may exit: the only
    // outstanding copy of slot k is the last one issued into it.
    const long long issued = seq;
    for (int k = 0; k < D && k < issued; ++k) {
        const long long last = issued - 1 - ((issued - 1 - k) % D);
        mbar_wait_bounded(&sh->full[k], static_cast<uint32_t>((last / D) & 1), a.watchdog_ns);
    }
}

// ------------------------------------------------------------------ kernel
// T = float: the FP32 decode; T = double: the same iteration in FP64 (the
// paper's double-precision runs).
template <typename T, int MODE>
__global__ void __launch_bounds__(kMaxPlainThreads, 1) mp_plain_kernel(const PlainArgs<T> a) {
    using Key = typename PlainTraits<T>::Key;
    using V = typename PlainTraits<T>::V;
    constexpr bool OMP = MODE >= 5;       // 5 grid-resident, 6 grid-streaming
    constexpr bool STREAM = MODE == 3 || MODE == 6;
    constexpr bool CLUSTER = MODE == 1;
    constexpr bool GRAM = MODE == 4;
    constexpr bool FP64 = sizeof(T) == 8;
    constexpr int NB = OMP ? 5 : 1;       // grid barriers per iteration
    constexpr int kV = 16 / sizeof(T);
    extern __shared__ __align__(128) unsigned char smem[];
    T* r = reinterpret_cast<T*>(smem);
    PlainShared<T>* sh = reinterpret_cast<PlainShared<T>*>(smem + a.off_sh);
    T* data = reinterpret_cast<T*>(smem + a.off_data);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = STREAM ? static_cast<int>(blockDim.x >> 5) - 1 : static_cast<int>(blockDim.x >> 5);
    const int nct = ncw * 32;
    const int cw = STREAM ? warp - 1 : warp;
    const int ct = cw * 32 + lane;
    const int cta = CLUSTER ? static_cast<int>(cluster_ctarank()) : static_cast<int>(blockIdx.x);
    const int G = CLUSTER ? static_cast<int>(cluster_nctarank()) : static_cast<int>(gridDim.x);
    const int ldN = a.ldN;
    const int base = a.M / G, rem = a.M % G;
    const int a0 = cta * base + min(cta, rem);
    const int na = base + (cta < rem ? 1 : 0);
    const Key kzero = {};

    if (threadIdx.x == 0) {
        for (int w = 0; w < kClusterKeys; ++w) sh->wkeys[0][w] = sh->wkeys[1][w] = kzero;
        if constexpr (FP64) sh->coop.abort[0] = sh->coop.abort[1] = 0;
        sh->abort = 0;
        sh->done = 0;
        if (STREAM) {
            for (int s = 0; s < a.stages; ++s) {
                mbar_init(&sh->full[s], 1);
                // shared stages are released by every consumer warp
                mbar_init(&sh->empty[s], a.coop ? kSumChains / 32 : 1);
            }
            fence_mbar_init();
        }
    }
    __syncthreads();

    if (STREAM && warp == 0) {
        if (lane == 0) {
            if (a.coop) plain_producer_shared(a, sh, data, a0, na);
            else plain_producer(a, sh, data, a0, na);
        }
        return;
    }

    // ---- Eq. 8: r <- y (zero padded), x~ <- 0 (own slice), resident atoms
    for (int i = ct; i < ldN; i += nct) r[i] = i < a.N ? a.y[i] : T(0);
    for (int i = ct; i < na; i += nct) a.x[a0 + i] = T(0);
    if (!STREAM && !GRAM) {
        const float4* src = reinterpret_cast<const float4*>(a.psi + static_cast<size_t>(a0) * ldN);
        float4* dst = reinterpret_cast<float4*>(data);
        const int n16 = na * (ldN / kV);
        for (int i = ct; i < n16; i += nct) dst[i] = __ldg(src + i);
    }
    named_bar_sync(1, nct);

    V* rv = reinterpret_cast<V*>(r);
    const int nvr = ldN / kV;
    double acc = 0.0;
    if (ct < kSumChains)
        for (int k = ct; k < nvr; k += kSumChains) acc = sq_acc(rv[k], acc);
    acc = warp_sum_f64(acc);
    if (lane == 0) sh->wsum[cw] = acc;
    named_bar_sync(1, nct);
    // warp sums in warp order; only the kSumChains / 32 chain warps carry a
    // partial (the others hold exact zeros)
    double e = 0.0;
    for (int w = 0; w < kSumChains / 32; ++w) e += sh->wsum[w];
    const double e0 = e;
    const double thr2 = a.eps2 * e0;
    const bool finite0 = isfinite(e0);
    // cluster shape: every CTA of the cluster has started (and initialised
    // its key ring) before any CTA stores into another's shared memory
    if (CLUSTER) cluster_sync_all();

    int t = 0;
    double audit = 0.0;    // max |e_t - (e_{t-1} - c^2)|, divided by e0 once at the end
    bool aborted = false;
    bool rank_stop = false;   // OMP: the selected atom lies in the span of those selected
    const int A = a.stage_atoms, D = a.stages;
    int m_prev = 0;        // mode 4: the previous step's atom and coefficient
    T c_prev = T(0);
    while (finite0 && e > thr2 && t < a.T_max) {
        // ---- Eq. 9: correlations of this CTA's atoms, best packed key
        Key best = kzero;
        if constexpr (GRAM) {
            // the CTA's correlations live in shared memory: recomputed from
            // the atoms (same order as the other shapes) every gram_period
            // steps, otherwise updated by c_m -= c_prev G[m_prev][m]
            T* cs = data;
            if (t % a.gram_period == 0) {
                for (int j = 4 * cw; j < na; j += 4 * ncw) {
                    if (j + 4 <= na) {
                        T c4[4];
                        dot4(a.psi + static_cast<size_t>(a0 + j) * ldN, r, ldN, lane, c4);
                        if (lane == 0)
                            for (int i = 0; i < 4; ++i) cs[j + i] = c4[i];
                    } else {
                        for (int q = j; q < na; ++q) {
                            const T v = dot1(a.psi + static_cast<size_t>(a0 + q) * ldN, r, ldN, lane);
                            if (lane == 0) cs[q] = v;
                        }
                    }
                }
            } else {
                const T* g = a.G + static_cast<size_t>(m_prev) * a.ldG + a0;
                for (int j = ct; j < na; j += nct) cs[j] = fmaf(-c_prev, __ldg(g + j), cs[j]);
            }
            named_bar_sync(1, nct);
            for (int j = ct; j < na; j += nct) best = kmax(best, pack_key(cs[j], a0 + j));
            best = warp_max_key(best);
        } else if (!STREAM) {
            for (int j = 4 * cw; j < na; j += 4 * ncw)
                best = scan_atoms(data + static_cast<size_t>(j) * ldN, r, ldN, min(4, na - j), a0 + j, lane, best);
        } else {
            const int np = a.pieces;
            const int S = np > 1 ? na * np : (na + A - 1) / A;
            const long long seq0 = static_cast<long long>(t) * S;
            int slot = static_cast<int>(seq0 % D);
            uint32_t par = static_cast<uint32_t>((seq0 / D) & 1);
            bool shared_stages = false;
            if constexpr (FP64) {
                if (a.coop) {
                    // every warp takes its class of each atom.  An atom
                    // streams as np stages of whole 4-segment groups; the
                    // warp's two chains run on across them in dot1's order,
                    // and the warp releases a stage as soon as its class of
                    // it is summed.  The lane partials of a window of atoms
                    // (and the abort word) go to shared memory, double-
                    // buffered by the window's parity: written only before
                    // that window's barrier and read only after it,
                    // rewritten two windows later -- so every warp reads the
                    // same abort word and leaves at the same window
                    // With ng = ncw / 4 groups of 4 warps (1 or 2), group g
                    // takes the atoms in slots s with (s / np) % ng == g:
                    // the ring holds a multiple of ng np stages, so a slot
                    // always belongs to the same group, which consumes its
                    // uses in order.
                    shared_stages = true;
                    const int ng = ncw >> 2;
                    const int cls = cw & 3, grp = cw >> 2;    // class of segments, group
                    const int spp = a.piece_elems / 64;       // segments per piece, a multiple of 4
                    const int nseg = (ldN + 63) / 64;
                    const int nfull = ldN / 64;               // segments with all 64 elements
                    const double2* r2 = reinterpret_cast<const double2*>(r);
                    double ax = 0.0, ay = 0.0;
                    bool failed = false;
                    int jp = 0, ja = 0, wa = 0, wpar = 0;     // piece, atom, atom in window, window parity
                    int sgrp = (slot / np) % ng;              // group of the current slot
                    int sin = slot % np;                      // position of the slot in its group of np
                    for (int j = 0; j < S; ++j) {
                        const bool mine = sgrp == grp;
                        if (mine && !failed) {
                            const bool ok =
                                __all_sync(0xffffffffu, mbar_wait_bounded(&sh->full[slot], par, a.watchdog_ns));
                            if (ok) {
                                const int s0 = jp * spp, s1 = min(s0 + spp, nseg), s1f = min(s1, nfull);
                                // st2: the stage's element pairs, the piece's first at 0
                                const double2* st2 =
                                    reinterpret_cast<const double2*>(data + static_cast<size_t>(slot) * a.stage_elems);
                                const int pb = s0 * 32;                   // the piece's first element pair
                                int sg = s0 + cls;
#pragma unroll 4
                                for (; sg < s1f; sg += 4) {
                                    const int e2 = sg * 32 + lane;    // element pair in the atom
                                    const double2 u = r2[e2];
                                    const double2 v = st2[e2 - pb];
                                    ax = fma(v.x, u.x, ax);
                                    ay = fma(v.y, u.y, ay);
                                }
                                if (sg < s1 && sg * 64 + lane * 2 < ldN) {   // the partial last segment
                                    const int e2 = sg * 32 + lane;
                                    const double2 u = r2[e2];
                                    const double2 v = st2[e2 - pb];
                                    ax = fma(v.x, u.x, ax);
                                    ay = fma(v.y, u.y, ay);
                                }
                                __syncwarp();
                                if (lane == 0) mbar_arrive(&sh->empty[slot]);
                            } else {
                                failed = true;
                                if (lane == 0) {
                                    atomicCAS(&a.ws->err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                                    sh->coop.abort[wpar] = 1;
                                    *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                                }
                            }
                        }
                        if (jp == np - 1) {
                            if (mine) sh->coop.part[wpar][wa][cls][lane] = failed ? 0.0 : ax + ay;
                            ax = ay = 0.0;
                            if (wa == kCoopWindow - 1 || ja == na - 1) {
                                named_bar_sync(2, nct);
                                if (sh->coop.abort[wpar]) break;
                                const int wbase = ja - wa;
                                for (int k = cw; k <= wa; k += ncw) {
                                    const double(&pp)[4][32] = sh->coop.part[wpar][k];
                                    const double tot = (pp[0][lane] + pp[1][lane]) + (pp[2][lane] + pp[3][lane]);
                                    best = kmax(best, pack_key(warp_sum_f64(tot), a0 + wbase + k));
                                }
                                wa = 0;
                                wpar ^= 1;
                            } else {
                                ++wa;
                            }
                        }
                        if (++jp == np) {
                            jp = 0;
                            ++ja;
                        }
                        if (++slot == D) {
                            slot = 0;
                            par ^= 1u;
                        }
                        if (++sin == np) {
                            sin = 0;
                            if (++sgrp == ng) sgrp = 0;
                        }
                    }
                }
            }
            // otherwise slot s belongs to warp s % ncw, which consumes the
            // slot's uses in order (so it never waits two phases ahead on a
            // barrier)
            if (!shared_stages) {
                for (int j = 0; j < S; ++j, slot = slot + 1 == D ? (par ^= 1u, 0) : slot + 1) {
                    if (slot % ncw != cw) continue;
                    if (!mbar_wait_bounded(&sh->full[slot], par, a.watchdog_ns)) {
                        if (lane == 0) {
                            atomicCAS(&a.ws->err, 0, static_cast<int>(MP_ERR_TIMEOUT));
                            *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                        }
                        break;
                    }
                    const T* st = data + static_cast<size_t>(slot) * a.stage_elems;
                    best = scan_atoms(st, r, ldN, min(A, na - j * A), a0 + j * A, lane, best);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh->empty[slot]);
                }
            }
        }
        // ---- CTA max, then grid max
        Key key;
        if (CLUSTER) {
            // every warp's best (the same in all its lanes) goes to entry
            // cta * ncw + cw of a two-slot ring in every CTA of the cluster:
            // lane q stores it into CTA q over DSMEM before the barrier,
            // whose release / acquire makes the stores visible.  After it
            // every warp reads the cluster's keys from its own shared memory
            // and their max is the cluster's key, the same in every warp of
            // every CTA.  A slot is rewritten only at iteration t+2, after
            // every warp of the cluster has passed barrier t+1 and so
            // finished its reads of iteration t
            if (lane < G)
                dsmem_st(mapa_shared(smem_u32(&sh->wkeys[t & 1][cta * ncw + cw]), static_cast<uint32_t>(lane)), best);
            cluster_sync_all();
            Key v = kzero;
            for (int j = lane; j < G * ncw; j += 32) v = kmax(v, sh->wkeys[t & 1][j]);
            key = warp_max_key(v);
        } else {
            if (lane == 0) sh->wkey[cw] = best;
            named_bar_sync(1, nct);
            if constexpr (!FP64) {
                if (ct == 0) {
                    unsigned long long k = 0ull;
                    for (int w = 0; w < ncw; ++w) k = umax64(k, sh->wkey[w]);
                    unsigned long long g = 0ull;
                    // the grid's winner is one of the CTAs' local bests: start
                    // pulling this one into L2 for the residual update
                    if (k != 0ull) prefetch_l2(a.psi + static_cast<size_t>(key_index(k)) * ldN, ldN * 4u);
                    if (!grid_exchange(a, cta, G, t, t * NB, k, &g)) *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                    sh->key = g;
                }
            } else {
                if (cw == 0) {
                    const Key k = warp_max_key(lane < ncw ? sh->wkey[lane] : kzero);
                    if (lane == 0 && k.hi != 0ull)
                        prefetch_l2(a.psi + static_cast<size_t>(key_index(k)) * ldN, ldN * 8u);
                    Key g = kzero;
                    const bool ok = grid_exchange(a, cta, G, t, k, lane, &g);
                    if (lane == 0) {
                        if (!ok) *reinterpret_cast<volatile int*>(&sh->abort) = 1;
                        sh->key = g;
                    }
                }
            }
            named_bar_sync(1, nct);
            if (*reinterpret_cast<volatile int*>(&sh->abort)) {
                aborted = true;
                break;
            }
            key = sh->key;
        }
        const int m = key_index(key);
        const T c = key_coef(key);
        if constexpr (GRAM) {
            // the next step reads this CTA's slice of row m of G (from HBM):
            // start pulling it into L2 now, behind the residual update
            // (16-byte aligned cover of [a0, a0 + na); rows are padded to 4)
            if (ct == 0 && na > 0) {
                const int g0 = a0 & ~3, g1 = (a0 + na + 3) & ~3;
                prefetch_l2(a.G + static_cast<size_t>(m) * a.ldG + g0, static_cast<uint32_t>(g1 - g0) * 4u);
            }
        }

        // ---- OMP: orthonormalise psi_m against the basis Q of the atoms
        // selected so far (classical Gram-Schmidt, applied twice), then the
        // residual update below uses the new basis vector q = w2 / ||w2||
        // and alpha = <r, q>: r - alpha q = y - Psi_S x_S for the least-
        // squares x_S, which the back substitution after the loop recovers.
        T step = c;            // coefficient of this step's update
        T qscale = T(1);       // OMP: 1 / ||w2||
        if constexpr (OMP) {
            const int k = t;
            const int GW = G * ncw, gw = cta * ncw + cw;
            const int chunk = (ldN / kV + G - 1) / G * kV;
            const int n0 = min(ldN, cta * chunk), n1 = min(ldN, n0 + chunk);
            bool ok = k < a.kmax;
            if (!ok) rank_stop = true;
            for (int pass = 0; pass < 2 && ok; ++pass) {
                const T* v = pass == 0 ? a.psi + static_cast<size_t>(m) * ldN : a.w;
                T* hp = pass == 0 ? a.h : a.h2;
                T* wo = pass == 0 ? a.w : a.w2;
                for (int j = gw; j < k; j += GW) {
                    const T d = dot1(a.Q + static_cast<size_t>(j) * ldN, v, ldN, lane);
                    if (lane == 0) hp[j] = d;
                }
                if (!cta_grid_sync(a, sh, G, t * NB + 1 + 2 * pass, ct, nct)) {
                    ok = false;
                    aborted = true;
                    break;
                }
                // w_n = v_n - sum_j h_j Q[j][n] over the CTA's slice: the
                // j-sum of each element in 4 fixed quarters (one FMA chain
                // each, consecutive threads on consecutive n: coalesced rows
                // of Q), combined as v_n + ((s0 + s1) + (s2 + s3))
                const int nel = n1 - n0;
                for (int task = ct; task < 4 * nel; task += nct) {
                    const int qt = task / nel, n = n0 + task % nel;
                    const int j0 = (k * qt) / 4, j1 = (k * (qt + 1)) / 4;
                    T acc = T(0);
#pragma unroll 8
                    for (int j = j0; j < j1; ++j) acc = fmaf(-hp[j], a.Q[static_cast<size_t>(j) * ldN + n], acc);
                    a.wpart[static_cast<size_t>(qt) * ldN + n] = acc;
                }
                named_bar_sync(1, nct);
                double nacc = 0.0;
                for (int n = n0 + ct; n < n1; n += nct) {
                    const T* wp = a.wpart + n;
                    wo[n] = v[n] + ((wp[0] + wp[ldN]) + (wp[2 * ldN] + wp[3 * ldN]));
                }
                if (pass == 1) {
                    named_bar_sync(1, nct);
                    if (ct < kSumChains)
                        for (int n = n0 + ct; n < n1; n += kSumChains)
                            nacc = fma(static_cast<double>(wo[n]), static_cast<double>(wo[n]), nacc);
                }
                if (pass == 1) {
                    nacc = warp_sum_f64(nacc);
                    if (lane == 0) sh->wsum[cw] = nacc;
                    named_bar_sync(1, nct);
                    if (ct == 0) {
                        // the chain warps' sums in warp order (the others hold zeros)
                        double sum = 0.0;
                        for (int q = 0; q < kSumChains / 32; ++q) sum += sh->wsum[q];
                        a.nrm[cta] = sum;
                    }
                }
                if (!cta_grid_sync(a, sh, G, t * NB + 2 + 2 * pass, ct, nct)) {
                    ok = false;
                    aborted = true;
                    break;
                }
            }
            if (aborted) break;
            if (ok) {
                // ||w2||^2 in one fixed order, the same value in every CTA:
                // lane l of warp 0 sums the CTA partials l, l + 32, ... in
                // turn, then the warp butterfly; lane 0 also takes sqrt and
                // its reciprocal once for the CTA.  Broadcast through the
                // last wsum slots, which no warp index reaches (at most 9
                // warps)
                if (cw == 0) {
                    double sum = 0.0;
                    for (int q = lane; q < G; q += 32) sum += a.nrm[q];
                    sum = warp_sum_f64(sum);
                    if (lane == 0) {
                        const double rt = sqrt(sum);
                        sh->wsum[kMaxWarps - 1] = sum;
                        sh->wsum[kMaxWarps - 3] = rt;
                        sh->wsum[kMaxWarps - 4] = 1.0 / rt;
                    }
                }
                named_bar_sync(1, nct);
                const double nw2 = sh->wsum[kMaxWarps - 1];
                // unit atoms: a component below 1e-4 is rounding, not a new direction
                if (!(nw2 > 1e-8)) rank_stop = true;
                else qscale = static_cast<T>(sh->wsum[kMaxWarps - 4]);
                if (!rank_stop) {
                    if (cw == 0) {
                        const T al = dot1_scaled(a.w2, qscale, r, ldN, lane);
                        if (lane == 0) sh->wsum[kMaxWarps - 2] = static_cast<double>(al);
                    }
                    named_bar_sync(1, nct);
                    step = static_cast<T>(sh->wsum[kMaxWarps - 2]);
                    if (cta == 0) {
                        // record the basis vector, R's column k and alpha_k
                        for (int n = ct; n < ldN; n += nct) a.Q[static_cast<size_t>(k) * ldN + n] = a.w2[n] * qscale;
                        const size_t ck = static_cast<size_t>(k) * (k + 1) / 2;
                        for (int j = ct; j < k; j += nct) a.Rc[ck + j] = a.h[j] + a.h2[j];
                        if (ct == 0) {
                            a.Rc[ck + k] = static_cast<T>(sh->wsum[kMaxWarps - 3]);
                            a.alpha[k] = step;
                            a.sel[k] = m;
                        }
                    }
                }
            }
            if (rank_stop) break;
        }

        // ---- Eq. 11: r <- r - c psi_m, and e = sum r^2 in FP64 (OMP:
        // r <- r - alpha q).  In the cluster shape psi_m is resident in its
        // owner CTA's shared memory and is read from there over DSMEM;
        // otherwise from global memory.
        const V* pm = reinterpret_cast<const V*>(OMP ? a.w2 : a.psi + static_cast<size_t>(m) * ldN);
        uint32_t pm_cluster = 0;
        if (CLUSTER) {
            // owner of atom m under the slice split above
            const int big = rem * (base + 1);
            const int own = m < big ? m / (base + 1) : rem + (m - big) / base;
            const int own_a0 = own * base + min(own, rem);
            pm_cluster = mapa_shared(smem_u32(data + static_cast<size_t>(m - own_a0) * ldN), static_cast<uint32_t>(own));
        }
        // the first kSumChains threads update r and run the energy chains
        // in the same pass (the other threads of 256-thread shapes idle here)
        acc = 0.0;
        if (ct < kSumChains) {
            for (int k = ct; k < nvr; k += kSumChains) {
                V pv;
                if (CLUSTER) dsmem_ld(pm_cluster + 16u * k, &pv);
                else if (OMP) pv = scale_vec(pm[k], qscale);
                else pv = __ldg(pm + k);
                const V v = sub_scaled(step, pv, rv[k]);
                rv[k] = v;
                acc = sq_acc(v, acc);
            }
        }
        acc = warp_sum_f64(acc);
        if (lane == 0) sh->wsum[cw] = acc;
        named_bar_sync(1, nct);
        double e_new = 0.0;
        for (int w = 0; w < kSumChains / 32; ++w) e_new += sh->wsum[w];

        // ---- Eq. 10 and bookkeeping (one thread of CTA 0)
        if (cta == 0 && ct == 0) {
            // fire-and-forget: same-address reductions from one thread apply
            // in program order, so x~_m accumulates exactly as x~_m += c would
            // (OMP: x~ comes from the back substitution after the loop)
            if (!OMP) red_add(a.x + m, c);
            if (t < a.tr_cap) {
                if (a.tr_atoms) a.tr_atoms[t] = m;
                if (a.tr_coefs) a.tr_coefs[t] = c;
                if (a.tr_energy) a.tr_energy[t] = e_new;
            }
            const double cc = static_cast<double>(step);
            // (e0 > 0 and rounded division is monotonic, so dividing the
            // maximum once gives the same bits as the maximum of quotients,
            // without an FP64 division on every iteration's critical path)
            audit = fmax(audit, fabs(e_new - (e - cc * cc)));
        }
        e = e_new;
        m_prev = m;
        c_prev = c;
        ++t;  // Eq. 12
    }

    if (STREAM && ct == 0) *reinterpret_cast<volatile int*>(&sh->done) = 1;
    if constexpr (OMP) {
        // R x_S = alpha by back substitution over R's packed columns, then
        // x~[sel_i] = x_i (CTA 0; every other CTA zeroed its x~ slice at the
        // start, before the first grid barrier)
        if (cta == 0 && !aborted) {
            for (int i = ct; i < t; i += nct) a.xs[i] = a.alpha[i];
            named_bar_sync(1, nct);
            for (int i = t - 1; i >= 0; --i) {
                const size_t ci = static_cast<size_t>(i) * (i + 1) / 2;
                const T xi = a.xs[i] / a.Rc[ci + i];
                for (int j = ct; j < i; j += nct) a.xs[j] = fmaf(-a.Rc[ci + j], xi, a.xs[j]);
                if (ct == 0) a.x[a.sel[i]] = xi;
                named_bar_sync(1, nct);
            }
        }
    }
    if (cta == 0 && a.tr_resid)
        for (int i = ct; i < a.N; i += nct) a.tr_resid[i] = r[i];
    if (cta == 0 && ct == 0) {
        PlainDevResult& res = a.ws->res;
        res.iters = t;
        res.e0 = e0;
        res.e = e;
        res.audit_max = e0 > 0.0 ? audit / e0 : 0.0;
        res.stop_reason = e0 == 0.0 ? MP_STOP_ZERO_Y
                          : rank_stop ? MP_STOP_RANK
                                      : (e <= thr2 ? MP_STOP_CONVERGED : MP_STOP_MAX_ITERS);
        res.status = !finite0 ? MP_ERR_NONFINITE : (aborted ? MP_ERR_TIMEOUT : MP_OK);
    }
    if (CLUSTER) cluster_sync_all();  // peers may still read this CTA's key slot
}
// ------------------------------------------------------------------ host side
static int round_up_i(int v, int m) { return (v + m - 1) / m * m; }

template <typename T, int MODE>
static cudaError_t prepare_kernel_attrs(int max_smem) {
    static int done_smem = -1;
    cudaError_t e = cudaSuccess;
    if (done_smem != max_smem) {
        e = cudaFuncSetAttribute(mp_plain_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e == cudaSuccess && MODE == 1)
            e = cudaFuncSetAttribute(mp_plain_kernel<T, MODE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) done_smem = max_smem;
    }
    return e;
}

template <typename T>
static int max_cluster_size(int smem, int threads, int max_smem) {
    static int cached[2] = {-1, -1};  // [smem key, result]
    if (cached[0] == smem) return cached[1];
    int best = 0;
    if (prepare_kernel_attrs<T, 1>(max_smem) == cudaSuccess) {
        for (int c : {16, 8}) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(c);
            lc.blockDim = dim3(threads);
            lc.dynamicSmemBytes = smem;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            lc.attrs = at;
            lc.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, mp_plain_kernel<T, 1>, &lc) == cudaSuccess && n > 0) {
                best = c;
                break;
            }
            cudaGetLastError();
        }
    }
    cached[0] = smem;
    cached[1] = best;
    return best;
}

// omp: the OMP decode (grid shapes only: its Gram-Schmidt phases need grid
// barriers), reported as mode 5 (grid-resident) or 6 (grid-streaming).
template <typename T>
static mp_status plain_configure_t(PlanImpl* p, PlainConfig* cfg, bool omp = false) {
    *cfg = PlainConfig();
    const long long atom_bytes = static_cast<long long>(p->ldN) * sizeof(T);
    const int r_bytes = round_up_i(p->ldN * static_cast<int>(sizeof(T)), 128);
    const int sh_bytes = round_up_i(static_cast<int>(sizeof(PlainShared<T>)), 128);
    cfg->off_sh = r_bytes;
    cfg->off_data = r_bytes + sh_bytes;
    const long long budget = static_cast<long long>(p->max_smem_optin) - cfg->off_data;
    if (budget < atom_bytes)
        return fail(MP_ERR_UNSUPPORTED, "plain decode: N=" + std::to_string(p->N) +
                                            " is too large for the shared-memory residual");
    const int M = p->M;
    int G = p->grid_ctas > 0 ? std::min(p->grid_ctas, p->sm_count) : p->sm_count;
    G = std::max(1, std::min(G, M));

    auto cluster_ok = [&](int* C_out) {
        int C = 1;
        while (C * 2 <= std::min(16, M)) C *= 2;
        const long long apc = (M + C - 1) / C;
        const long long smem = cfg->off_data + apc * atom_bytes;
        if (smem > p->max_smem_optin) return false;
        const int cmax = max_cluster_size<T>(static_cast<int>(smem), kResidentThreads, p->max_smem_optin);
        if (cmax == 0) return false;
        if (C > cmax) {
            C = cmax;
            if (cfg->off_data + static_cast<long long>((M + C - 1) / C) * atom_bytes > p->max_smem_optin)
                return false;
        }
        *C_out = C;
        return true;
    };
    auto gridres_ok = [&]() {
        const long long apc = (M + G - 1) / G;
        return cfg->off_data + apc * atom_bytes <= p->max_smem_optin;
    };

    if (sizeof(T) == 4 && p->gram_period > 0 && !omp) {
        // mode 4: r and the CTA's correlations on chip, atoms and G from HBM
        const long long apc = (M + G - 1) / G;
        if (cfg->off_data + apc * static_cast<long long>(sizeof(T)) > p->max_smem_optin)
            return fail(MP_ERR_UNSUPPORTED, "Gram decode: the correlations do not fit shared memory");
        cfg->mode = 4;
        cfg->ctas = G;
        cfg->threads = kResidentThreads;
        cfg->smem = static_cast<int>(cfg->off_data + apc * static_cast<long long>(sizeof(T)));
        return MP_OK;
    }
    int mode = p->forced_mode;
    int C = 0;
    if (omp && mode == 1) return fail(MP_ERR_UNSUPPORTED, "OMP decode: no one-cluster launch shape");
    if (mode == 0) {
        if (!omp && cluster_ok(&C)) mode = 1;
        else if (gridres_ok()) mode = 2;
        else mode = 3;
    } else if (mode == 1 && !cluster_ok(&C)) {
        return fail(MP_ERR_UNSUPPORTED, "plain decode: dictionary does not fit one cluster");
    } else if (mode == 2 && !gridres_ok()) {
        return fail(MP_ERR_UNSUPPORTED, "plain decode: dictionary does not fit the grid's shared memory");
    }
    cfg->mode = mode;
    if (mode == 1) {
        cfg->ctas = C;
        cfg->threads = kResidentThreads;
        cfg->smem = static_cast<int>(cfg->off_data + static_cast<long long>((M + C - 1) / C) * atom_bytes);
        return MP_OK;
    }
    if (mode == 2) {
        cfg->mode = omp ? 5 : 2;
        cfg->ctas = G;
        cfg->threads = kResidentThreads;
        cfg->smem = static_cast<int>(cfg->off_data + static_cast<long long>((M + G - 1) / G) * atom_bytes);
        return MP_OK;
    }
    // mode 3: atoms per stage A, ring depth D, consumer warps W
    // A: whole atoms per stage, at least stage_bytes when that still leaves
    // a ring of 4 stages (larger copies stream faster; 4 stages keep 4
    // consumer warps busy), else at most stage_bytes (and at least one atom)
    const long long apc = (M + G - 1) / G;
    long long A = std::max<long long>(1, (p->stage_bytes + atom_bytes - 1) / atom_bytes);
    if (budget / (A * atom_bytes) < 4) A = std::max<long long>(1, p->stage_bytes / atom_bytes);
    A = std::min(A, apc);
    long long stage_bytes = A * atom_bytes;
    // as deep a ring as fits; 4 consumer warps (kSumChains threads), each
    // owning the slots s with s % 4 == its index (D need not be a multiple
    // of 4; with D < 4 some warps own no slot)
    long long D = std::min<long long>(kMaxStages, budget / stage_bytes);
    const int W = kSumChains / 32;
    // FP64 is bound by the FP64 units, not by HBM: keep all 4 SM sub-
    // partitions' FP64 pipes fed.  For atoms of 8 KB or more, or when the
    // ring cannot give every warp two whole-atom slots (its next atom
    // loading while it computes one), 4 warps share every stage, one class
    // of segments each, an atom streams as pieces of whole 4-segment groups
    // of about stage_bytes, and two such groups take alternate atoms where
    // the ring holds an atom for each (a warp fed from shared memory cannot
    // keep its sub-partition's FP64 pipe busy alone); otherwise every warp
    // owns the same number of whole-atom slots.  FP32 keeps the deepest ring
    // of whole atoms.
    int groups = 1;
    if (sizeof(T) == 8 && !omp) {
        if (atom_bytes >= 8192 || budget < 2LL * W * atom_bytes) {
            const long long nseg = (p->ldN + 63) / 64;
            long long np = std::max<long long>(1, (atom_bytes + p->stage_bytes - 1) / p->stage_bytes);
            const long long spp = ((nseg + np - 1) / np + 3) / 4 * 4;
            np = (nseg + spp - 1) / spp;
            const long long pe = spp * 64;
            cfg->coop = 1;
            cfg->pieces = static_cast<int>(np);
            cfg->piece_elems = static_cast<int>(pe);
            A = 1;
            stage_bytes = pe * static_cast<long long>(sizeof(T));
            D = std::min<long long>(kMaxStages, budget / stage_bytes);
            // two groups of 4 warps (two per SM sub-partition) when the ring
            // holds a whole atom for each, the ring a multiple of 2 atoms
            if (D >= kCoopGroups * np) {
                groups = kCoopGroups;
                D -= D % (kCoopGroups * np);
            }
        } else if (D >= W) {
            D -= D % W;
        }
    }
    if (D < 2)
        return fail(MP_ERR_UNSUPPORTED, "plain decode: N=" + std::to_string(p->N) +
                                            " leaves no room for a two-stage ring");
    cfg->mode = omp ? 6 : 3;
    cfg->ctas = G;
    cfg->threads = 32 * (1 + W * groups);
    cfg->stage_atoms = static_cast<int>(A);
    cfg->stages = static_cast<int>(D);
    cfg->smem = static_cast<int>(cfg->off_data + D * stage_bytes);
    return MP_OK;
}

mp_status plain_configure(PlanImpl* p, PlainConfig* cfg) { return plain_configure_t<float>(p, cfg); }
mp_status plain_configure64(PlanImpl* p, PlainConfig* cfg) { return plain_configure_t<double>(p, cfg); }

template <typename T>
static mp_status plain_launch_t(PlanImpl* p, const T* psi, const T* y, T* x, const mp_stop* stop, int* tr_atoms,
                                T* tr_coefs, double* tr_energy, T* tr_resid, int tr_cap, PlainWorkspace* ws,
                                cudaStream_t st, bool omp = false) {
    PlainConfig cfg;
    mp_status s = plain_configure_t<T>(p, &cfg, omp);
    if (s != MP_OK) return s;
    PlainArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.psi = psi;
    a.y = y;
    a.x = x;
    a.N = p->N;
    a.ldN = p->ldN;
    a.M = p->M;
    a.T_max = stop->max_iters;
    a.eps2 = stop->eps * stop->eps;
    a.stage_atoms = cfg.stage_atoms;
    a.stages = cfg.stages;
    a.pieces = cfg.coop ? cfg.pieces : 1;
    a.piece_elems = cfg.coop ? cfg.piece_elems : 0;
    a.stage_elems = cfg.coop ? cfg.piece_elems : cfg.stage_atoms * p->ldN;
    a.prefetch = cfg.mode == 3 ? p->prefetch_stages : 0;
    a.evict_first = p->evict_first;
    if (cfg.mode == 3 || cfg.mode == 6) {
        const long long atom_bytes = static_cast<long long>(p->ldN) * sizeof(T);
        const long long keep = p->l2_keep_bytes / std::max<long long>(1, atom_bytes * cfg.ctas);
        a.l2_keep_atoms = static_cast<int>(std::min<long long>(keep, (p->M + cfg.ctas - 1) / cfg.ctas));
    }
    a.off_sh = cfg.off_sh;
    a.off_data = cfg.off_data;
    a.ws = ws;
    a.slots = static_cast<Key128*>(p->slots64);
    a.tr_atoms = tr_atoms;
    a.tr_coefs = tr_coefs;
    a.tr_energy = tr_energy;
    a.tr_resid = tr_resid;
    a.tr_cap = std::max(0, tr_cap);
    a.watchdog_ns = static_cast<unsigned long long>(p->watchdog_ns);
    a.skip_cta = cfg.mode == 1 ? -1 : p->skip_cta;
    a.coop = cfg.coop;
    if (cfg.mode == 4) {
        a.G = reinterpret_cast<const T*>(p->gram);
        a.ldG = p->ldG;
        a.gram_period = p->gram_period;
    }
    if (omp) {
        OmpWorkspace& o = p->omp;
        a.Q = reinterpret_cast<T*>(o.Q);
        a.Rc = reinterpret_cast<T*>(o.Rc);
        a.alpha = reinterpret_cast<T*>(o.alpha);
        a.sel = o.sel;
        a.h = reinterpret_cast<T*>(o.h);
        a.h2 = reinterpret_cast<T*>(o.h2);
        a.w = reinterpret_cast<T*>(o.w);
        a.w2 = reinterpret_cast<T*>(o.w2);
        a.wpart = reinterpret_cast<T*>(o.wpart);
        a.nrm = o.nrm;
        a.xs = reinterpret_cast<T*>(o.xs);
        a.kmax = std::min(stop->max_iters, p->N);
    }

    MP_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(PlainWorkspace), st));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.ctas);
    lc.blockDim = dim3(cfg.threads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    if (cfg.mode == 1) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cfg.ctas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
    } else {
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
    }
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e;
    switch (cfg.mode) {
        case 1:
            MP_CUDA_TRY((prepare_kernel_attrs<T, 1>(p->max_smem_optin)));
            e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 1>, a);
            break;
        case 2:
            MP_CUDA_TRY((prepare_kernel_attrs<T, 2>(p->max_smem_optin)));
            e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 2>, a);
            break;
        case 3:
            MP_CUDA_TRY((prepare_kernel_attrs<T, 3>(p->max_smem_optin)));
            e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 3>, a);
            break;
        default:
            if constexpr (sizeof(T) == 4) {
                if (cfg.mode == 4) {
                    MP_CUDA_TRY((prepare_kernel_attrs<T, 4>(p->max_smem_optin)));
                    e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 4>, a);
                } else if (cfg.mode == 5) {
                    MP_CUDA_TRY((prepare_kernel_attrs<T, 5>(p->max_smem_optin)));
                    e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 5>, a);
                } else {
                    MP_CUDA_TRY((prepare_kernel_attrs<T, 6>(p->max_smem_optin)));
                    e = cudaLaunchKernelEx(&lc, mp_plain_kernel<T, 6>, a);
                }
            } else {
                e = cudaErrorInvalidConfiguration;
            }
            break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "plain decode launch");
    p->launches++;
    return MP_OK;
}

mp_status plain_launch(PlanImpl* p, const float* y, float* x, const mp_stop* stop, const mp_trace* trace,
                       PlainWorkspace* ws, cudaStream_t st) {
    if (p->gram_period > 0) {
        const mp_status s = gram_prepare(p, st);
        if (s != MP_OK) return s;
    }
    if (!trace) return plain_launch_t<float>(p, p->psi32, y, x, stop, nullptr, nullptr, nullptr, nullptr, 0, ws, st);
    return plain_launch_t<float>(p, p->psi32, y, x, stop, trace->atoms, trace->coefs, trace->energies,
                                 trace->residual, trace->capacity, ws, st);
}

// OMP scratch for up to kmax selected atoms (grown on demand, kept by the plan).
static mp_status omp_prepare(PlanImpl* p, int kmax) {
    OmpWorkspace& o = p->omp;
    if (o.kmax >= kmax && o.G >= p->sm_count) return MP_OK;
    omp_free(&o);
    const size_t ld = static_cast<size_t>(p->ldN), k = static_cast<size_t>(std::max(1, kmax));
    const size_t G = static_cast<size_t>(std::max(1, p->sm_count));
    MP_CUDA_TRY(cudaMalloc(&o.Q, k * ld * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.Rc, k * (k + 1) / 2 * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.alpha, k * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.sel, k * sizeof(int)));
    MP_CUDA_TRY(cudaMalloc(&o.h, k * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.h2, k * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.w, ld * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.w2, ld * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.wpart, 4 * ld * sizeof(float)));
    MP_CUDA_TRY(cudaMalloc(&o.nrm, G * sizeof(double)));
    MP_CUDA_TRY(cudaMalloc(&o.xs, k * sizeof(float)));
    o.kmax = static_cast<int>(k);
    o.G = static_cast<int>(G);
    o.bytes = (k * ld + k * (k + 1) / 2 + 5 * k + 6 * ld) * sizeof(float) + G * sizeof(double);
    return MP_OK;
}

mp_status plain_launch_omp(PlanImpl* p, const float* y, float* x, const mp_stop* stop, const mp_trace* trace,
                           PlainWorkspace* ws, cudaStream_t st) {
    const mp_status s = omp_prepare(p, std::min(std::max(stop->max_iters, 1), p->N));
    if (s != MP_OK) return s;
    if (!trace)
        return plain_launch_t<float>(p, p->psi32, y, x, stop, nullptr, nullptr, nullptr, nullptr, 0, ws, st, true);
    return plain_launch_t<float>(p, p->psi32, y, x, stop, trace->atoms, trace->coefs, trace->energies,
                                 trace->residual, trace->capacity, ws, st, true);
}

mp_status plain_launch64(PlanImpl* p, const double* y, double* x, const mp_stop* stop, const mp_trace_f64* trace,
                         PlainWorkspace* ws, cudaStream_t st) {
    if (!p->psi64 || !p->slots64)
        return fail(MP_ERR_UNSUPPORTED, "the plan holds no FP64 dictionary (prec_mask bit MP_PREC_FP64)");
    if (!trace) return plain_launch_t<double>(p, p->psi64, y, x, stop, nullptr, nullptr, nullptr, nullptr, 0, ws, st);
    return plain_launch_t<double>(p, p->psi64, y, x, stop, trace->atoms, trace->coefs, trace->energies,
                                  trace->residual, trace->capacity, ws, st);
}

mp_status plain_result_to_host(const PlanImpl*, const PlainWorkspace* h, mp_result* out) {
    const PlainDevResult& r = h->res;
    std::memset(out, 0, sizeof(*out));
    out->iters = r.iters;
    out->stop_reason = r.stop_reason;
    mp_status s = static_cast<mp_status>(r.status);
    if (s == MP_OK && h->err != 0) s = static_cast<mp_status>(h->err);
    out->status = s;
    out->rel_residual = r.e0 > 0.0 ? std::sqrt(r.e / r.e0) : 0.0;
    out->energy_audit_max = r.audit_max;
    if (s == MP_ERR_TIMEOUT) set_error("a device-side wait exceeded the watchdog limit");
    if (s == MP_ERR_NONFINITE) set_error("y has a non-finite entry");
    return s;
}

static mp_status check_stop(const mp_stop* stop) {
    if (!stop) return fail(MP_ERR_INVALID, "stop is NULL");
    if (!(stop->eps >= 0.0) || !std::isfinite(stop->eps)) return fail(MP_ERR_INVALID, "eps must be finite and >= 0");
    if (stop->max_iters < 0) return fail(MP_ERR_INVALID, "max_iters must be >= 0");
    if (stop->reserved != 0) return fail(MP_ERR_INVALID, "stop.reserved must be 0");
    return MP_OK;
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

mp_status mp_recover(mp_plan_t plan, const float* y, float* x, const mp_stop* stop, const mp_trace* trace,
                     mp_result* host_out, void* stream) {
    clear_error();
    if (!plan || !y || !x) return fail(MP_ERR_INVALID, "mp_recover: NULL plan, y or x");
    mp_status s = check_stop(stop);
    if (s != MP_OK) return s;
    PlanImpl* p = &plan->impl;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = plain_launch(p, y, x, stop, trace, p->ws, st);
    if (s != MP_OK) return s;
    p->last_stream = st;
    p->have_pending = true;
    if (!host_out) return MP_OK;
    return mp_plan_last_result(plan, host_out);
}

mp_status mp_recover_omp(mp_plan_t plan, const float* y, float* x, const mp_stop* stop, const mp_trace* trace,
                         mp_result* host_out, void* stream) {
    clear_error();
    if (!plan || !y || !x) return fail(MP_ERR_INVALID, "mp_recover_omp: NULL plan, y or x");
    mp_status s = check_stop(stop);
    if (s != MP_OK) return s;
    PlanImpl* p = &plan->impl;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = plain_launch_omp(p, y, x, stop, trace, p->ws, st);
    if (s != MP_OK) return s;
    p->last_stream = st;
    p->have_pending = true;
    if (!host_out) return MP_OK;
    return mp_plan_last_result(plan, host_out);
}

mp_status mp_recover_f64(mp_plan_t plan, const double* y, double* x, const mp_stop* stop,
                         const mp_trace_f64* trace, mp_result* host_out, void* stream) {
    clear_error();
    if (!plan || !y || !x) return fail(MP_ERR_INVALID, "mp_recover_f64: NULL plan, y or x");
    mp_status s = check_stop(stop);
    if (s != MP_OK) return s;
    PlanImpl* p = &plan->impl;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = plain_launch64(p, y, x, stop, trace, p->ws, st);
    if (s != MP_OK) return s;
    p->last_stream = st;
    p->have_pending = true;
    if (!host_out) return MP_OK;
    return mp_plan_last_result(plan, host_out);
}

mp_status mp_plan_last_result(mp_plan_t plan, mp_result* out) {
    if (!plan || !out) return fail(MP_ERR_INVALID, "mp_plan_last_result: NULL argument");
    PlanImpl* p = &plan->impl;
    if (!p->have_pending) return fail(MP_ERR_INVALID, "mp_plan_last_result: no decode was issued");
    MP_CUDA_TRY(cudaMemcpyAsync(p->ws_host, p->ws, sizeof(PlainWorkspace), cudaMemcpyDeviceToHost, p->last_stream));
    MP_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    return plain_result_to_host(p, p->ws_host, out);
}

mp_status mp_recover_host(mp_plan_t plan, const float* y_host, float* x_host, const mp_stop* stop,
                          mp_result* out) {
    clear_error();
    if (!plan || !y_host || !x_host || !out) return fail(MP_ERR_INVALID, "mp_recover_host: NULL argument");
    mp_status s = check_stop(stop);
    if (s != MP_OK) return s;
    PlanImpl* p = &plan->impl;
    if (!p->own_stream) MP_CUDA_TRY(cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking));
    if (!p->y_stage) {
        MP_CUDA_TRY(cudaMalloc(&p->y_stage, sizeof(float) * p->N));
        MP_CUDA_TRY(cudaMalloc(&p->x_stage, sizeof(float) * p->M));
        MP_CUDA_TRY(cudaMallocHost(&p->h_y, sizeof(float) * p->N));
        MP_CUDA_TRY(cudaMallocHost(&p->h_x, sizeof(float) * p->M));
    }
    cudaStream_t st = p->own_stream;
    std::memcpy(p->h_y, y_host, sizeof(float) * p->N);
    MP_CUDA_TRY(cudaMemcpyAsync(p->y_stage, p->h_y, sizeof(float) * p->N, cudaMemcpyHostToDevice, st));
    s = plain_launch(p, p->y_stage, p->x_stage, stop, nullptr, p->ws, st);
    if (s != MP_OK) return s;
    p->last_stream = st;
    p->have_pending = true;
    MP_CUDA_TRY(cudaMemcpyAsync(p->h_x, p->x_stage, sizeof(float) * p->M, cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(p->ws_host, p->ws, sizeof(PlainWorkspace), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    std::memcpy(x_host, p->h_x, sizeof(float) * p->M);
    return plain_result_to_host(p, p->ws_host, out);
}

}  // extern "C"
