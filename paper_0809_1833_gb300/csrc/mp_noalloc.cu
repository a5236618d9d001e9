// Allocation-free single-signal decode.
//
// Some callers cannot allocate GPU memory at all: code running where
// cudaMalloc is forbidden or unavailable (inside a pre-sized memory pool, a
// plugin that only receives buffers from its host application, or a real-time
// loop that must not touch the allocator).  mp_recover_noalloc serves them:
// it runs the same persistent FP32 kernel as mp_recover on a dictionary the
// caller already holds on the device, and keeps the kernel's scratch (the
// argmax key slots, the grid-barrier arrival counter, the error word and the
// result record) in the file-scope array below instead of in plan memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mpgb_noalloc.h"
#include "mp_internal.h"

namespace mpgb {

// Upper bound on the scratch this entry point may use.  The module holds the
// array on every GPU that loads the library, for the life of the process.
constexpr size_t kNoAllocScratchBytes = 256;
static_assert(sizeof(PlainWorkspace) <= kNoAllocScratchBytes, "plain workspace exceeds the static scratch");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, once per device, with that device current.  A
// cudaDeviceReset of that device invalidates the cached address (as it does
// every other device pointer the caller holds).
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static mp_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(MP_ERR_UNSUPPORTED, "mp_recover_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MP_OK;
}

}  // namespace mpgb

using namespace mpgb;

extern "C" {

mp_status mp_recover_noalloc(const float* psi, int N, int M, int ld, const float* y, float* x, const mp_stop* stop,
                             const mp_trace* trace, mp_result* host_out, void* stream) {
    clear_error();
    if (!psi || !y || !x || !stop || !host_out) return fail(MP_ERR_INVALID, "mp_recover_noalloc: NULL argument");
    if (N < 1 || M < 1) return fail(MP_ERR_INVALID, "mp_recover_noalloc: N and M must be >= 1");
    if (ld < N || ld % 4 != 0)
        return fail(MP_ERR_INVALID, "mp_recover_noalloc: ld must be >= N and a multiple of 4");
    if (reinterpret_cast<uintptr_t>(psi) % 16 != 0)
        return fail(MP_ERR_INVALID, "mp_recover_noalloc: psi must be 16-byte aligned");
    if (static_cast<long long>(M) * ld > (1LL << 40)) return fail(MP_ERR_INVALID, "mp_recover_noalloc: dictionary too large");
    if (!(stop->eps >= 0.0) || !std::isfinite(stop->eps) || stop->max_iters < 0 || stop->reserved != 0)
        return fail(MP_ERR_INVALID, "mp_recover_noalloc: bad stop parameters (eps must be finite and >= 0, T >= 0)");
    if (trace && trace->capacity < 0) return fail(MP_ERR_INVALID, "mp_recover_noalloc: trace capacity < 0");
    if (sizeof(PlainWorkspace) > kNoAllocScratchBytes)
        return fail(MP_ERR_UNSUPPORTED, "mp_recover_noalloc: scratch need exceeds the 256-byte static array");

    // A plan-shaped description of the caller's dictionary; nothing here
    // allocates (the struct lives on the stack and points at caller memory).
    PlanImpl p;
    cudaError_t e = cudaGetDevice(&p.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st) {
        // the kernel runs on the current device: a stream of another device
        // is a caller error, reported here rather than as a launch failure
        int sdev = -1;
        e = cudaStreamGetDevice(st, &sdev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetDevice");
        if (sdev != p.device)
            return fail(MP_ERR_INVALID, "mp_recover_noalloc: the stream belongs to device " + std::to_string(sdev) +
                                            ", the current device is " + std::to_string(p.device));
    }
    e = cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, p.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(multiprocessor count)");
    e = cudaDeviceGetAttribute(&p.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(shared memory per block, opt-in)");
    p.N = N;
    p.M = M;
    p.ldN = ld;
    p.psi32 = const_cast<float*>(psi);
    void* scratch = nullptr;
    mp_status s = scratch_address(p.device, &scratch);
    if (s != MP_OK) return s;
    PlainWorkspace* ws = static_cast<PlainWorkspace*>(scratch);
    // plain_launch clears the scratch on `st` before the kernel starts
    s = plain_launch(&p, y, x, stop, trace, ws, st);
    if (s != MP_OK) return s;
    PlainWorkspace h;
    std::memset(&h, 0, sizeof(h));
    MP_CUDA_TRY(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    return plain_result_to_host(&p, &h, host_out);
}

}  // extern "C"
