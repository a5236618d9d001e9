// Plans: the dictionary Psi (Sec. 2, Eq. 3) copied to the device in the
// layouts the decode kernels read, with the unit-norm precondition of Eq. 4
// checked (or enforced) on the device.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mp_batch.cuh"
#include "mp_device.cuh"
#include "mp_internal.h"

namespace mpgb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
mp_status fail(mp_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
mp_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? MP_ERR_NOMEM : MP_ERR_CUDA;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Per-atom statistics gathered by the preparation kernel.
struct AtomStats {
    double norm2;       // sum of squares of the input atom (FP64)
    float maxabs;       // max |entry| of the stored atom
    int nonfinite;      // any NaN / Inf entry
};

// One CTA per atom: read psi_m from the caller's layout (FP32 or FP64),
// reduce its squared norm in FP64, optionally scale it to unit norm, and
// write the padded FP32 row plus the requested FP64 and low-precision rows.
// FP32 input: the FP64 row is the stored FP32 row widened (exact).  FP64
// input: the FP64 row is the (scaled) input, the FP32 row its rounding.
template <typename TIn>
__global__ void __launch_bounds__(256) prep_atoms_kernel(
    const TIn* __restrict__ src, int layout, int N, int M, int normalize, float* __restrict__ psi32,
    int ldN, double* __restrict__ psi64, __nv_bfloat16* __restrict__ psi16, int ldK16,
    __nv_fp8_storage_t* __restrict__ psi8, int ldK8, float* __restrict__ scale8, AtomStats* __restrict__ stats) {
    constexpr bool kIn64 = sizeof(TIn) == 8;
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    __shared__ double s_d[8];
    __shared__ float s_f[8];
    __shared__ int s_i[8];
    auto at = [&](int n) -> TIn {
        return layout == MP_LAYOUT_ATOM_MAJOR ? src[static_cast<size_t>(m) * N + n]
                                              : src[static_cast<size_t>(n) * M + m];
    };
    // pass 1: squared norm, finiteness
    double acc = 0.0;
    int bad = 0;
    for (int n = tid; n < N; n += blockDim.x) {
        const TIn v = at(n);
        if (!isfinite(static_cast<double>(v))) bad = 1;
        acc = fma(static_cast<double>(v), static_cast<double>(v), acc);
    }
    acc = warp_sum_f64(acc);
    bad = __any_sync(0xffffffffu, bad);
    if ((tid & 31) == 0) {
        s_d[tid >> 5] = acc;
        s_i[tid >> 5] = bad;
    }
    __syncthreads();
    double norm2 = 0.0;
    int anybad = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        norm2 += s_d[w];
        anybad |= s_i[w];
    }
    const double scale = (normalize && norm2 > 0.0) ? 1.0 / sqrt(norm2) : 1.0;
    // pass 2: stored FP32 row (zero padded) and its max |entry|
    float mx = 0.f;
    float* row = psi32 + static_cast<size_t>(m) * ldN;
    double* row64 = psi64 ? psi64 + static_cast<size_t>(m) * ldN : nullptr;
    for (int n = tid; n < ldN; n += blockDim.x) {
        float v = 0.f;
        double v64 = 0.0;
        if (n < N) {
            if (kIn64) {
                v64 = normalize ? static_cast<double>(at(n)) * scale : static_cast<double>(at(n));
                v = static_cast<float>(v64);
            } else {
                v = normalize ? static_cast<float>(static_cast<double>(at(n)) * scale) : static_cast<float>(at(n));
                v64 = static_cast<double>(v);
            }
        }
        row[n] = v;
        if (row64) row64[n] = v64;
        mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((tid & 31) == 0) s_f[tid >> 5] = mx;
    __syncthreads();
    float amax = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmaxf(amax, s_f[w]);
    // BF16 copy (round to nearest even), zero padded to ldK16
    if (psi16) {
        __nv_bfloat16* r16 = psi16 + static_cast<size_t>(m) * ldK16;
        for (int n = tid; n < ldK16; n += blockDim.x)
            r16[n] = __float2bfloat16_rn(n < N ? row[n] : 0.f);
    }
    // FP8-E4M3 copy with per-atom scale max|psi_m| / 448 (448 = largest
    // finite E4M3 value), zero padded to ldK8
    if (psi8) {
        const float s = amax > 0.f ? amax / 448.f : 1.f;
        const float inv = amax > 0.f ? 448.f / amax : 1.f;
        __nv_fp8_storage_t* r8 = psi8 + static_cast<size_t>(m) * ldK8;
        for (int n = tid; n < ldK8; n += blockDim.x)
            r8[n] = __nv_cvt_float_to_fp8(n < N ? row[n] * inv : 0.f, __NV_SATFINITE, __NV_E4M3);
        if (tid == 0) scale8[m] = s;
    }
    if (tid == 0) {
        stats[m].norm2 = norm2;
        stats[m].maxabs = amax;
        stats[m].nonfinite = anybad;
    }
}

static void plan_free(PlanImpl* p) {
    if (!p) return;
    if (p->batch) batch_destroy(p->batch);
    cudaFree(p->psi32);
    cudaFree(p->psi16);
    cudaFree(p->psi8);
    cudaFree(p->scale8);
    cudaFree(p->psi64);
    cudaFree(p->slots64);
    cudaFree(p->gram);
    omp_free(&p->omp);
    cudaFree(p->ws);
    cudaFree(p->y_stage);
    cudaFree(p->x_stage);
    cudaFreeHost(p->ws_host);
    cudaFreeHost(p->h_y);
    cudaFreeHost(p->h_x);
    if (p->own_stream) cudaStreamDestroy(p->own_stream);
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

const char* mp_status_string(mp_status s) {
    switch (s) {
        case MP_OK: return "MP_OK";
        case MP_PENDING: return "MP_PENDING";
        case MP_ERR_INVALID: return "MP_ERR_INVALID";
        case MP_ERR_NOMEM: return "MP_ERR_NOMEM";
        case MP_ERR_BUSY: return "MP_ERR_BUSY";
        case MP_ERR_TIMEOUT: return "MP_ERR_TIMEOUT";
        case MP_ERR_NONFINITE: return "MP_ERR_NONFINITE";
        case MP_ERR_CUDA: return "MP_ERR_CUDA";
        case MP_ERR_UNSUPPORTED: return "MP_ERR_UNSUPPORTED";
        case MP_ERR_NOT_FOUND: return "MP_ERR_NOT_FOUND";
    }
    return "MP_UNKNOWN_STATUS";
}

const char* mp_last_error_message(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace mpgb {

template <typename TIn>
static mp_status plan_create_t(mp_plan_t* out, const mp_plan_desc* desc, const TIn* psi, void* stream) {
    clear_error();
    if (!out) return fail(MP_ERR_INVALID, "mp_plan_create: out is NULL");
    *out = nullptr;
    if (!desc || !psi) return fail(MP_ERR_INVALID, "mp_plan_create: desc or psi is NULL");
    if (desc->N < 1 || desc->M < 1)
        return fail(MP_ERR_INVALID, "mp_plan_create: N and M must be >= 1");
    if (desc->layout != MP_LAYOUT_ATOM_MAJOR && desc->layout != MP_LAYOUT_ROW_MAJOR)
        return fail(MP_ERR_INVALID, "mp_plan_create: unknown layout");
    if (desc->reserved != 0) return fail(MP_ERR_INVALID, "mp_plan_create: reserved must be 0");
    if (desc->prec_mask & ~15u) return fail(MP_ERR_INVALID, "mp_plan_create: unknown precision bit");
    if (sizeof(TIn) == 8 && !(desc->prec_mask & (1u << MP_PREC_FP64)))
        return fail(MP_ERR_INVALID, "mp_plan_create_f64: prec_mask must include MP_PREC_FP64");
    if (static_cast<long long>(desc->N) * desc->M > (1LL << 40))
        return fail(MP_ERR_INVALID, "mp_plan_create: dictionary too large");

    mp_plan_s* plan = new (std::nothrow) mp_plan_s();
    if (!plan) return fail(MP_ERR_NOMEM, "mp_plan_create: host allocation failed");
    PlanImpl* p = &plan->impl;
    auto bail = [&](mp_status s) {
        plan_free(p);
        delete plan;
        return s;
    };
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->N = desc->N;
    p->M = desc->M;
    p->ldN = round_up(p->N, 32);
    p->ldK16 = round_up(p->N, 64);
    p->ldK8 = round_up(p->N, 128);
    p->prec_mask = desc->prec_mask | 1u;
    cudaError_t e;
    if ((e = cudaGetDevice(&p->device)) != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    if ((e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(multiprocessor count)"));
    if ((e = cudaDeviceGetAttribute(&p->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(shared memory per block, opt-in)"));
    if ((e = cudaDeviceGetAttribute(&p->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(shared memory per multiprocessor)"));

    const size_t n32 = static_cast<size_t>(p->M) * p->ldN;
    if ((e = cudaMalloc(&p->psi32, n32 * sizeof(float))) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMalloc(psi32)"));
    p->device_bytes += n32 * sizeof(float);
    if (p->prec_mask & (1u << MP_PREC_BF16)) {
        const size_t b = static_cast<size_t>(p->M) * p->ldK16 * sizeof(__nv_bfloat16);
        if ((e = cudaMalloc(&p->psi16, b)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(psi16)"));
        p->device_bytes += b;
    }
    if (p->prec_mask & (1u << MP_PREC_FP8E4M3)) {
        const size_t b = static_cast<size_t>(p->M) * p->ldK8;
        if ((e = cudaMalloc(&p->psi8, b)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(psi8)"));
        if ((e = cudaMalloc(&p->scale8, p->M * sizeof(float))) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc(scale8)"));
        p->device_bytes += b + p->M * sizeof(float);
    }
    if (p->prec_mask & (1u << MP_PREC_FP64)) {
        const size_t b = n32 * sizeof(double);
        if ((e = cudaMalloc(&p->psi64, b)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(psi64)"));
        const size_t sb = 2 * static_cast<size_t>(std::max(1, p->sm_count)) * 16;
        if ((e = cudaMalloc(&p->slots64, sb)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(slots64)"));
        p->device_bytes += b + sb;
    }
    if ((e = cudaMalloc(&p->ws, sizeof(PlainWorkspace))) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMalloc(workspace)"));
    if ((e = cudaMallocHost(&p->ws_host, sizeof(PlainWorkspace))) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocHost(workspace)"));

    AtomStats* d_stats = nullptr;
    if ((e = cudaMallocAsync(&d_stats, p->M * sizeof(AtomStats), st)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocAsync(stats)"));
    prep_atoms_kernel<TIn><<<p->M, 256, 0, st>>>(
        psi, desc->layout, p->N, p->M, desc->normalize ? 1 : 0, p->psi32, p->ldN, p->psi64,
        static_cast<__nv_bfloat16*>(p->psi16), p->ldK16, static_cast<__nv_fp8_storage_t*>(p->psi8),
        p->ldK8, p->scale8, d_stats);
    p->launches++;
    std::vector<AtomStats> h(p->M);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_stats, p->M * sizeof(AtomStats), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d_stats, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "mp_plan_create: atom preparation"));
    for (int m = 0; m < p->M; ++m) {
        if (h[m].nonfinite)
            return bail(fail(MP_ERR_NONFINITE, "mp_plan_create: atom " + std::to_string(m) +
                                                   " has a non-finite entry"));
        const double nrm = std::sqrt(h[m].norm2);
        if (desc->normalize) {
            if (!(nrm > 0.0))
                return bail(fail(MP_ERR_INVALID,
                                 "mp_plan_create: atom " + std::to_string(m) + " is zero"));
        } else if (std::fabs(nrm - 1.0) > 1e-5) {
            return bail(fail(MP_ERR_INVALID, "mp_plan_create: atom " + std::to_string(m) +
                                                 " has norm " + std::to_string(nrm) +
                                                 " (unit norm required, Eq. 4)"));
        }
    }
    PlainConfig cfg;
    plain_configure(p, &cfg);   // validates that a plain launch shape exists (or not)
    *out = plan;
    return MP_OK;
}

}  // namespace mpgb

extern "C" {

mp_status mp_plan_create(mp_plan_t* out, const mp_plan_desc* desc, const float* psi, void* stream) {
    return plan_create_t<float>(out, desc, psi, stream);
}

mp_status mp_plan_create_f64(mp_plan_t* out, const mp_plan_desc* desc, const double* psi, void* stream) {
    return plan_create_t<double>(out, desc, psi, stream);
}

mp_status mp_plan_destroy(mp_plan_t plan) {
    clear_error();
    if (!plan) return MP_OK;
    cudaDeviceSynchronize();
    plan_free(&plan->impl);
    delete plan;
    return MP_OK;
}

mp_status mp_plan_set_option(mp_plan_t plan, int option, long long value) {
    clear_error();
    if (!plan) return fail(MP_ERR_INVALID, "mp_plan_set_option: plan is NULL");
    PlanImpl* p = &plan->impl;
    switch (option) {
        case MP_OPT_PLAIN_MODE:
            if (value < 0 || value > 3) return fail(MP_ERR_INVALID, "plain mode must be 0..3");
            p->forced_mode = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_WATCHDOG_NS:
            if (value < 1000) return fail(MP_ERR_INVALID, "watchdog must be >= 1000 ns");
            p->watchdog_ns = value;
            return MP_OK;
        case MP_OPT_DEBUG_SKIP_ARRIVE:
            p->skip_cta = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_GRID_CTAS:
            if (value < 0) return fail(MP_ERR_INVALID, "grid CTA count must be >= 0");
            p->grid_ctas = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_PLAIN_PREFETCH:
            if (value < 0 || value > 256) return fail(MP_ERR_INVALID, "prefetch distance must be 0..256");
            p->prefetch_stages = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_PLAIN_STAGE_BYTES:
            if (value < 16 || value > (1 << 20)) return fail(MP_ERR_INVALID, "stage bytes must be 16..1 MiB");
            p->stage_bytes = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_PLAIN_L2_KEEP_BYTES:
            if (value < 0) return fail(MP_ERR_INVALID, "L2 keep bytes must be >= 0");
            p->l2_keep_bytes = value;
            return MP_OK;
        case MP_OPT_PLAIN_EVICT_FIRST:
            p->evict_first = value ? 1 : 0;
            return MP_OK;
        case MP_OPT_PLAIN_GRAM:
            if (value < 0 || value > (1 << 20)) return fail(MP_ERR_INVALID, "Gram refresh period must be 0..2^20");
            p->gram_period = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_BATCH_AUTOTUNE:
            p->batch_autotune = value ? 1 : 0;
            return MP_OK;
        case MP_OPT_BATCH_TILE_N:
            // 128, 160, 192, 224 or 256 atoms per tile
            if (value != 0 && (value < 128 || value > 256 || value % 32))
                return fail(MP_ERR_INVALID, "batch tile must be 0 or 128..256 in steps of 32");
            p->batch_tile_n = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_BATCH_GRAM:
            if (value < 0 || value > (1 << 20) || value % 16)
                return fail(MP_ERR_INVALID, "batch Gram period must be 0 or a multiple of 16 up to 2^20");
            p->batch_gram = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_BATCH_GRAM_BELOW:
            if (value < 0 || value > (1 << 30))
                return fail(MP_ERR_INVALID, "batch Gram switch threshold must be 0..2^30 signals");
            p->batch_gram_below = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_BATCH_PAIR:
            if (value < 0 || value > 2) return fail(MP_ERR_INVALID, "batch pair option must be 0, 1 or 2");
            p->batch_pair = static_cast<int>(value);
            return MP_OK;
        case MP_OPT_BATCH_TILE_M:
            if (value != 0 && value != 128 && value != 256)
                return fail(MP_ERR_INVALID, "batch tile rows must be 0, 128 or 256");
            p->batch_tile_m = static_cast<int>(value);
            return MP_OK;
    }
    return fail(MP_ERR_INVALID, "unknown option " + std::to_string(option));
}

mp_status mp_plan_query(mp_plan_t plan, int what, long long* value) {
    clear_error();
    if (!plan || !value) return fail(MP_ERR_INVALID, "mp_plan_query: NULL argument");
    PlanImpl* p = &plan->impl;
    PlainConfig cfg;
    mp_status s = plain_configure(p, &cfg);
    switch (what) {
        case MP_Q_PLAIN_MODE: *value = s == MP_OK ? cfg.mode : 0; return MP_OK;
        case MP_Q_PLAIN_CTAS: *value = cfg.ctas; return MP_OK;
        case MP_Q_PLAIN_THREADS: *value = cfg.threads; return MP_OK;
        case MP_Q_PLAIN_SMEM: *value = cfg.smem; return MP_OK;
        case MP_Q_PLAIN_STAGE_ATOMS: *value = cfg.stage_atoms; return MP_OK;
        case MP_Q_PLAIN_STAGES: *value = cfg.stages; return MP_OK;
        case MP_Q_LD_FP32: *value = p->ldN; return MP_OK;
        case MP_Q_DEVICE_BYTES: *value = static_cast<long long>(p->device_bytes); return MP_OK;
        case MP_Q_KERNEL_LAUNCHES: *value = p->launches; return MP_OK;
        case MP_Q_BATCH_TILE_N: *value = p->batch ? p->batch->TN : 0; return MP_OK;
        case MP_Q_BATCH_TILE_M: *value = p->batch ? p->batch->TM : 0; return MP_OK;
        case MP_Q_BATCH_GRAM: *value = p->batch ? p->batch->gram_R : 0; return MP_OK;
        case MP_Q_BATCH_PAIR: *value = p->batch ? p->batch->pair : 0; return MP_OK;
        case MP_Q_BATCH_GRAM_BELOW: *value = p->batch ? p->batch->gram_below : 0; return MP_OK;
        case MP_Q_PLAN_N: *value = p->N; return MP_OK;
        case MP_Q_PLAN_M: *value = p->M; return MP_OK;
        case MP_Q_GRAM_BYTES:
            *value = p->gram ? static_cast<long long>(p->M) * p->ldG * 4 : 0;
            return MP_OK;
        case MP_Q_PLAIN64_MODE:
        case MP_Q_PLAIN64_STAGES:
        case MP_Q_PLAIN64_PIECES: {
            PlainConfig c64;
            const bool ok = p->psi64 && plain_configure64(p, &c64) == MP_OK;
            *value = !ok ? 0
                         : (what == MP_Q_PLAIN64_MODE     ? c64.mode
                            : what == MP_Q_PLAIN64_STAGES ? c64.stages
                                                          : (c64.coop ? c64.pieces : 0));
            clear_error();
            return MP_OK;
        }
    }
    return fail(MP_ERR_INVALID, "unknown query " + std::to_string(what));
}

}  // extern "C"
