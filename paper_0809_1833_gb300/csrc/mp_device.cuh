// Device-side helpers shared by the Matching Pursuit kernels (sm_103a):
// mbarriers, 1-D bulk copies, cluster shared-memory access, ordered global
// atomics, the packed argmax key and bounded waits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MP_DEV __device__ __forceinline__

namespace mpgb {

// ---------------------------------------------------------------- timers
MP_DEV uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

MP_DEV uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
MP_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
MP_DEV void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
MP_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Arrive on an mbarrier of another CTA of the cluster (cluster address).
MP_DEV void mbar_arrive_remote(uint32_t bar_cl) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cl) : "memory");
}
MP_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
MP_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of `parity` to complete, giving up after `limit_ns`.
MP_DEV bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t deadline = globaltimer_ns() + limit_ns;
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() > deadline) return false;
    }
}

// ---------------------------------------------------------------- bulk copy
// 1-D bulk copy global -> shared, completion counted on `bar` (tx bytes).
// dst and src 16-byte aligned, bytes a multiple of 16.
MP_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Same with an L2 cache policy (createpolicy: evict-first for data read
// once per pass, evict-last for data kept resident across passes).
MP_DEV void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
        "[%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// Fire-and-forget prefetch of [src, src+bytes) into L2 (16-byte aligned,
// bytes a multiple of 16).
MP_DEV void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy operations (bulk copies) on the same shared memory.
MP_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// One 128-byte line toward L2 (fire and forget).
MP_DEV void prefetch_line_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
MP_DEV uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
MP_DEV uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// ---------------------------------------------------------------- barriers
MP_DEV void named_bar_sync(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
MP_DEV void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
MP_DEV uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
MP_DEV uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Address of the same shared variable in CTA `rank` of this cluster.
MP_DEV uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
MP_DEV float4 dsmem_ld_f32x4(uint32_t cluster_addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(cluster_addr)
                 : "memory");
    return v;
}
MP_DEV double2 dsmem_ld_f64x2(uint32_t cluster_addr) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(cluster_addr) : "memory");
    return v;
}
MP_DEV void red_add(float* p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
MP_DEV void red_add(double* p, double v) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
MP_DEV void dsmem_st_u64(uint32_t cluster_addr, uint64_t v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(cluster_addr), "l"(v) : "memory");
}
MP_DEV uint64_t dsmem_ld_u64(uint32_t cluster_addr) {
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(cluster_addr) : "memory");
    return v;
}
// ---------------------------------------------------------------- global atomics
MP_DEV void red_release_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
MP_DEV unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
MP_DEV unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
MP_DEV void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
MP_DEV int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// ---------------------------------------------------------------- argmax key
// Packs (|c|, index, sign(c)) into one integer whose unsigned order is the
// selection order of Sec. 3 / Sec. 4: larger |c| first, then the smaller
// index.  |c| >= 0, so its IEEE bits order like its value.  The sign rides
// in the lowest bit so the coefficient is recovered exactly.
MP_DEV unsigned long long pack_key(float c, int idx) {
    const uint32_t bits = __float_as_uint(c);
    const uint32_t mag = bits & 0x7fffffffu;
    const uint32_t lo = ((0x7fffffffu - static_cast<uint32_t>(idx)) << 1) | (bits >> 31);
    return (static_cast<unsigned long long>(mag) << 32) | lo;
}
MP_DEV int key_index(unsigned long long k) {
    return static_cast<int>(0x7fffffffu - (static_cast<uint32_t>(k) >> 1));
}
MP_DEV float key_coef(unsigned long long k) {
    const uint32_t mag = static_cast<uint32_t>(k >> 32);
    const uint32_t sgn = static_cast<uint32_t>(k) & 1u;
    return __uint_as_float(mag | (sgn << 31));
}
MP_DEV unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// The same order for FP64 correlations, with |c| kept to all 63 bits: the
// magnitude in the high word, (index, sign) packed as above in the low word,
// compared as one 128-bit unsigned number.
struct Key128 {
    unsigned long long hi, lo;
};
MP_DEV Key128 pack_key(double c, int idx) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(c));
    Key128 k;
    k.hi = bits & 0x7fffffffffffffffull;
    k.lo = (static_cast<unsigned long long>(0x7fffffffu - static_cast<uint32_t>(idx)) << 1) | (bits >> 63);
    return k;
}
MP_DEV int key_index(Key128 k) { return static_cast<int>(0x7fffffffu - static_cast<uint32_t>(k.lo >> 1)); }
MP_DEV double key_coef(Key128 k) {
    return __longlong_as_double(static_cast<long long>(k.hi | ((k.lo & 1ull) << 63)));
}
MP_DEV Key128 kmax(Key128 a, Key128 b) { return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b; }
MP_DEV unsigned long long kmax(unsigned long long a, unsigned long long b) { return umax64(a, b); }

// ---------------------------------------------------------------- reductions
// Butterfly sums: every lane ends with the same bits (each step adds the
// same two operands on both partner lanes).
MP_DEV float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
MP_DEV double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
MP_DEV unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
MP_DEV Key128 warp_max_key(Key128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Key128 w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = kmax(v, w);
    }
    return v;
}
MP_DEV unsigned long long warp_max_key(unsigned long long v) { return warp_max_u64(v); }

}  // namespace mpgb
