// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mpgb.h"

namespace mpgb {

// Thread-local error text behind mp_last_error_message().
void set_error(const std::string& msg);
void clear_error();
mp_status fail(mp_status s, const std::string& msg);
mp_status cuda_fail(cudaError_t e, const char* what);

#define MP_CUDA_TRY(expr)                                          \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ::mpgb::cuda_fail(_e, #expr); \
    } while (0)

// Device-side result of one plain decode, written by the kernel.
struct PlainDevResult {
    int iters;
    int stop_reason;
    int status;            // mp_status of the decode (set by the kernel)
    int pad;
    double e0;
    double e;
    double audit_max;
};

// Scratch of the plain kernel: the argmax key slots and the arrival
// counter of the grid barrier, an error word, and the result.
struct PlainWorkspace {
    unsigned long long keys[4];
    unsigned long long count;
    int err;
    int pad;
    PlainDevResult res;
};

// Launch shape of the plain kernel, derived from (N, M) and the device.
struct PlainConfig {
    int mode = 0;          // 1 cluster-resident, 2 grid-resident, 3 grid-stream, 4 Gram
    int ctas = 0;          // grid size (= cluster size in mode 1)
    int threads = 0;
    int smem = 0;          // dynamic shared memory bytes
    int stage_atoms = 0;   // mode 3
    int stages = 0;        // mode 3
    int off_data = 0;      // byte offsets inside dynamic smem
    int off_sh = 0;
    int coop = 0;          // FP64 streaming: 4 warps share every stage
    int pieces = 1;        // coop: stages per atom (pieces of whole 4-segment groups)
    int piece_elems = 0;   // coop: elements per piece (a multiple of 256), the stage stride
};

// OMP decode scratch (mp_plain.cu): basis, packed R, alpha = Q^T y,
// selected atoms, Gram-Schmidt vectors, per-CTA norm partials, solution.
struct OmpWorkspace {
    float* Q = nullptr;
    float* Rc = nullptr;
    float* alpha = nullptr;
    int* sel = nullptr;
    float* h = nullptr;
    float* h2 = nullptr;
    float* w = nullptr;
    float* w2 = nullptr;
    float* wpart = nullptr;
    double* nrm = nullptr;
    float* xs = nullptr;
    int kmax = 0;
    int G = 0;
    size_t bytes = 0;
};

inline void omp_free(OmpWorkspace* o) {
    cudaFree(o->Q);
    cudaFree(o->Rc);
    cudaFree(o->alpha);
    cudaFree(o->sel);
    cudaFree(o->h);
    cudaFree(o->h2);
    cudaFree(o->w);
    cudaFree(o->w2);
    cudaFree(o->wpart);
    cudaFree(o->nrm);
    cudaFree(o->xs);
    *o = OmpWorkspace();
}

struct BatchEngine;        // batched decode state (mp_batched.cu)

// Shape of the batched correlation GEMM's tiles: TM signal rows (128, or
// 256 = two 128-row MMAs sharing each atom stage) and TN atoms (128 or 256).
struct GemmShape {
    int tm = 128;
    int tn = 256;
    int pair = 0;   // 1: two-SM tiles of 256 rows (clusters of two CTAs), tn a multiple of 32 in [128, 256]
};

// Autotuned batched-GEMM shape for one (precision, batch-size bucket).
struct TuneEntry {
    int prec;
    int bucket;
    GemmShape shape;
    double us;             // measured GEMM time per launch
    int lo = 0;            // the smaller batch the shapes were also timed on (0: a quarter)
};

struct PlanImpl {
    int N = 0, M = 0;
    int ldN = 0;           // FP32 atom stride (floats), multiple of 32
    int ldK16 = 0;         // BF16 atom stride (elements), multiple of 64
    int ldK8 = 0;          // FP8 atom stride (bytes), multiple of 128
    unsigned prec_mask = 0;
    int device = 0;
    int sm_count = 0;
    int max_smem_optin = 0;
    int smem_per_sm = 0;            // shared memory of one SM (all its CTAs together)
    size_t device_bytes = 0;

    float* psi32 = nullptr;
    void* psi16 = nullptr;          // __nv_bfloat16
    void* psi8 = nullptr;           // __nv_fp8_e4m3
    float* scale8 = nullptr;        // per-atom FP8 scale
    double* psi64 = nullptr;        // FP64 atom-major copy, stride ldN
    void* slots64 = nullptr;        // FP64 grid exchange slots (2 x sm_count keys)
    float* gram = nullptr;          // Gram matrix Psi^T Psi (M x ldG), built on demand
    int ldG = 0;

    PlainWorkspace* ws = nullptr;   // device
    PlainWorkspace* ws_host = nullptr;  // pinned mirror
    cudaStream_t last_stream = nullptr;
    bool have_pending = false;

    // staging for mp_recover_host
    float* y_stage = nullptr;       // device N
    float* x_stage = nullptr;       // device M
    float* h_y = nullptr;           // pinned N
    float* h_x = nullptr;           // pinned M
    cudaStream_t own_stream = nullptr;

    // options
    int forced_mode = 0;
    long long watchdog_ns = 2000000000LL;
    int skip_cta = -1;
    int grid_ctas = 0;
    int batch_tile_n = 0;
    int batch_tile_m = 0;           // batched GEMM signal rows per tile (0 = auto)
    int batch_pair = 0;             // two-SM GEMM tiles: 0 = auto, 1 = off, 2 = on
    int batch_autotune = 1;         // time the GEMM shapes on first use of a batch size
    std::vector<TuneEntry> tuned;
    int prefetch_stages = 0;        // plain streaming: L2 prefetch distance (measured slower; off)
    int stage_bytes = 32768;        // plain streaming: target bytes per ring stage
    int evict_first = 1;            // plain streaming: L2 evict-first hint on the stream
    long long l2_keep_bytes = 0;    // plain streaming: dictionary bytes kept resident in L2
    int gram_period = 0;            // > 0: Gram-updated correlations, direct every R steps
    int batch_gram = 0;             // batched / served BF16: Gram mode period (0 = off)
    int batch_gram_below = 0;       // batched BF16 with batch_gram > 0: direct steps while more
                                    // signals than this are active, Gram steps after (0 = off)

    long long launches = 0;
    BatchEngine* batch = nullptr;
    OmpWorkspace omp;
};

// Plain-kernel helpers (mp_plain.cu).
mp_status plain_configure(PlanImpl* p, PlainConfig* cfg);
mp_status plain_launch(PlanImpl* p, const float* y, float* x, const mp_stop* stop,
                       const mp_trace* trace, PlainWorkspace* ws, cudaStream_t st);
mp_status plain_result_to_host(const PlanImpl* p, const PlainWorkspace* h, mp_result* out);
// Gram matrix of the plan's FP32 atoms (mp_gram.cu); builds it once.
mp_status gram_prepare(PlanImpl* p, cudaStream_t st);
// The FP64 decode (the same kernel instantiated for double).
mp_status plain_configure64(PlanImpl* p, PlainConfig* cfg);
mp_status plain_launch64(PlanImpl* p, const double* y, double* x, const mp_stop* stop,
                         const mp_trace_f64* trace, PlainWorkspace* ws, cudaStream_t st);

// Batched engine teardown (mp_batched.cu).
void batch_destroy(BatchEngine* b);
// GEMM shape (signals and atoms per tile) for a batch of B signals: the
// plan's options if set, else the autotuned choice (timed now on first use
// of the batch-size bucket, on rows R when given), else a fixed rule.
// lo_rows > 0: the fewest active rows a GEMM of this decode will see (the
// autotuner times each shape on the full batch and on that many rows; by
// default on a quarter of the batch).
mp_status batch_shape(PlanImpl* p, int prec, int B, const float* R, cudaStream_t st, GemmShape* shape,
                      int lo_rows = 0);

}  // namespace mpgb

struct mp_plan_s {
    mpgb::PlanImpl impl;
};
