// Definitions shared by the batched decode (mp_batched.cu), its correlation
// GEMM (mp_corr.cu) and the request server (mp_server.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mp_internal.h"

namespace mpgb {

constexpr int kBM = 128;            // signals per row block = TMEM lanes = UMMA M
constexpr int kRowBytes = 128;      // bytes of K per operand row per stage (one swizzle row)
constexpr int kMaxStages = 16;      // GEMM shared-memory pipeline depth, upper bound
constexpr int kSmemOptin = 232448;  // shared memory a CTA may opt into on sm_103a

constexpr int kTop = 8;             // low-precision candidates kept per signal and list
constexpr int kEpiGroups = 4;       // epilogue warp groups: each scans 1/4 of a tile's atoms
// shared memory besides the stages: alignment slack, barriers, and the
// epilogue's list exchange (3 groups x 8 keys x 128 rows x 4 bytes)
constexpr int kCorrFixedSmem = 2048 + (kEpiGroups - 1) * kTop * kBM * 4;

// Pipeline depth for a TM x TN tile: as many A+B stages as fit, at most 8.
constexpr int corr_stages(int TM, int TN) {
    return (kSmemOptin - kCorrFixedSmem) / (TM * kRowBytes + TN * kRowBytes) < kMaxStages
               ? (kSmemOptin - kCorrFixedSmem) / (TM * kRowBytes + TN * kRowBytes)
               : kMaxStages;
}
constexpr int kGemmThreads = 32 * (2 + 4 * kEpiGroups);   // warp 0 TMA, warp 1 MMA, then epilogue

// Arguments of the correlation GEMM.
struct CorrArgs {
    const int* n_act;       // active rows this step (rows 0..n_act-1 of the A operand)
    int TN;                 // atoms per tile (128 or 256; two-SM tiles: 128..256, step 32)
    int RM;                 // 128-row blocks per tile (1 or 2)
    int n_at;               // atom tiles
    int M;
    int nk;                 // K blocks of 128 bytes
    int fp8;
    int tmem_cols;
    int stages;             // pipeline depth, corr_stages(128 * RM, TN)
    const float* colscale;  // FP8 per-atom scale
    uint2* cand;            // [row][n_at][8] = (score bits, atom), each tile's list sorted
    unsigned long long watchdog_ns;
    int* err;
    float* dump;            // diagnostic: full correlation rows (row * M + m), or NULL
    const float* rscale;    // diagnostic FP8: per-row scale of the quantised residual
    int* zero_next;         // step: the other half's survivor count, set to 0 here (or NULL)
    int half_ok;            // tmBh holds TN/2-row boxes: a launch may take tiles of TN/2 atoms
    int* n_at_out;          // atom tiles (candidate lists per row) this launch used, or NULL
    int ks2_ok;             // tmA3 / tmB3 are set: 128-atom one-block tiles may stage two K slices
};

int corr_smem_bytes(int TM, int TN);
cudaError_t corr_prepare();
int corr_max_ctas();
// Launch: tmA's box is 128 signal rows (a partial row block is loaded
// whole), tmB's TN atom rows, tmBh's (when a.half_ok) TN/2 atom rows; with
// a.ks2_ok, tmA3 / tmB3 are the same operands as 3-D views (128-byte K
// slice, rows, slice index) with boxes of 128 rows x 2 slices, used by
// launches whose tile is one row block by 128 atoms.  max_rows bounds the
// active rows any step of this launch can see (it sizes the grid).
cudaError_t launch_corr_top8(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmBh,
                             const CUtensorMap& tmA3, const CUtensorMap& tmB3, const CorrArgs& a, int max_rows,
                             cudaStream_t st);
// The same GEMM on two-SM tiles (clusters of two CTAs, tcgen05 cta_group::2):
// 256 signal rows x a.TN atoms per cluster, a.TN a multiple of 32 in
// [128, 256], a.RM = 2, a.stages = corr_stages(128, a.TN / 2), a.half_ok = 0;
// tmBp's box is a.TN / 2 atom rows.
int pair_smem_bytes(int TN);
cudaError_t pair_prepare();
int pair_max_clusters(int TN, bool fp8);
cudaError_t launch_corr_pair(const CUtensorMap& tmA, const CUtensorMap& tmBp, const CorrArgs& a, int max_rows,
                             cudaStream_t st);

// ------------------------------------------------------------------ batch engine
// Per-signal state of a slot.
struct SlotState {
    double e0, e, thr2, audit;   // audit: max |e_t - (e_{t-1} - c^2)| (reported / e0)
    int t, T, status, stop_reason;
};

// Outputs the kernels write, read through one device pointer so a captured
// graph does not depend on the caller's buffers.
struct BatchIO {
    float* X;              // slot s row at X + s * ldx
    long long ldx;
    int* tr_atoms;         // slot s row at tr_atoms + s * tr_cap (optional)
    float* tr_coefs;
    double* tr_energy;
    int tr_cap;
    int pad;
};

// Device state of `cap` decode slots over one dictionary at one precision:
// FP32 residuals, the quantised GEMM operand (one row per active signal),
// the active-row table, candidates, slot states, and the step graph.
//
// The operand and the active-row table have two halves.  A step reads half p
// (rows 0..counters[p ? 3 : 0]-1) and every signal still running after it
// takes the next free row of half 1-p with one atomic, writing its slot id
// and quantised residual there; so the next step's rows are compact without
// a separate compaction pass.  Step graphs hold an even number of steps, so
// between graph launches (admission, the host's reads) the current half is 0.
// The order of rows within a half does not change any signal's result: every
// row's products, top-8 and update are its own.
struct BatchEngine {
    int cap = 0;            // slots (= GEMM rows available)
    int cap_pad = 0;        // rows of the GEMM operand (multiple of 128)
    int prec = -1;
    int TM = 128;           // signal rows per GEMM tile
    int TN = 0;
    int pair = 0;           // two-SM tiles (TM = 256 over a cluster of two CTAs)
    int n_at = 0;
    int ldq = 0;            // operand row: elements (BF16) or bytes (FP8)
    float* R32 = nullptr;
    void* Rq = nullptr;        // 2 x cap_pad operand rows (half 0, then half 1)
    SlotState* st = nullptr;
    int* act = nullptr;        // 2 x cap slot ids by row (half 0, then half 1)
    int* counters = nullptr;   // [0] rows of half 0, [1] rows just admitted, [2] finished count, [3] rows of half 1,
                               // [4] candidate lists per row of the last GEMM, [5] Gram mode: select CTAs done
    int* done = nullptr;
    int* holes = nullptr;
    int* surv = nullptr;
    uint2* cand = nullptr;
    double* eps2 = nullptr;
    int* T = nullptr;
    int* err = nullptr;
    BatchIO* io = nullptr;
    float* rscale = nullptr;
    int* fin_list = nullptr;   // slots that stopped since the last retire
    SlotState* h_st = nullptr;
    int* h_cnt = nullptr;
    double* h_eps2 = nullptr;
    int* h_T = nullptr;
    BatchIO* h_io = nullptr;
    int* h_err = nullptr;
    CUtensorMap tmA, tmA1, tmB, tmBh;   // operand half 0, half 1, atoms (TN-row and TN/2-row boxes)
    CUtensorMap tmBp;                   // two-SM tiles: atoms in TN/2-row boxes
    CUtensorMap tmA3, tmA1_3, tmB3;     // 3-D views (slice, rows, slice index): 128 rows x 2 K slices
    // Gram mode (gram_R > 0): each slot keeps its correlations Psi^T r in
    // FP32 (Cg, M of ldC floats), computed directly at admission and every
    // gram_R of its own steps, and updated from one row of G = Psi^T Psi in
    // every step; gtop carries the row's 8 largest |c| (keys as in the
    // candidate lists).  No GEMM runs in this mode.
    int gram_R = 0;
    float* Cg = nullptr;
    int ldC = 0;
    unsigned long long* gtop = nullptr;
    // Switched mode (gram_below > 0, with gram_R > 0): the decode runs direct
    // GEMM steps (`graph`) while more than gram_below signals are active,
    // then computes every active signal's correlations directly once and
    // runs Gram-updated steps (`graph_g`) to the end.  Admission computes no
    // correlation rows in this mode.
    int gram_below = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t graph_g = nullptr;
    // Gram steps without the refresh at the start of the replay: a batched
    // decode's signals all start together, so the host knows which replays
    // begin at a multiple of the period and runs this graph for the others
    cudaGraphExec_t graph_gn = nullptr;
    int graph_steps = 0;
    int graph_kernels = 0;          // kernels one replay of the graph launches
    int graph_g_kernels = 0;        // the same for graph_g
    int graph_gn_kernels = 0;       // the same for graph_gn
    bool graph_retire = false;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cnt_ready[2] = {nullptr, nullptr};   // active-count reads of alternate replays
    size_t bytes = 0;
};

// Bytes of device memory one slot costs (residual, operand row, candidates,
// state, an output row of M floats when the engine owns X).
size_t engine_slot_bytes(const PlanImpl* p, int prec, bool with_x, int gram_R = 0);
// gram_R: 0, or the Gram mode's refresh period (a multiple of 16; BF16 or
// FP32 plans; the plan's Gram matrix must exist); gram_below > 0 (with
// gram_R > 0): the switched mode
mp_status engine_alloc(BatchEngine* e, PlanImpl* p, int prec, int cap, const GemmShape& shape, int gram_R = 0,
                       int gram_below = 0);
void engine_free(BatchEngine* e);
// Admit n signals: rows Y (device, n x N), into slots `slots_dev` (device,
// NULL = 0..n-1), with per-signal eps^2 and T already in e->eps2 / e->T.
// Signals that need no iteration are reported in fin_list at once.
cudaError_t engine_admit(PlanImpl* p, BatchEngine* e, const float* Y, int n, const int* slots_dev, cudaStream_t st);
// Capture `steps` steps (and, if `retire`, a copy of the finished slots'
// results to host-mapped memory) as the engine's graph.
mp_status engine_build_graph(PlanImpl* p, BatchEngine* e, int steps, bool retire, float* out_x_dev,
                             SlotState* out_state_dev, int* out_list_dev, int* out_count_dev);

}  // namespace mpgb
