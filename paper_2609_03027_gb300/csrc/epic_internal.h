// Internal declarations shared by the host plan, the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/epic.h"

namespace epic {

// Occupied part of one channel's grid: every GCF tap of every element lies in
// rows [y0, y0+ny) and columns [x0, x0+nx).
struct Box {
    int x0, y0, nx, ny;
};

// Device tables of one plan (all channels concatenated).
struct DeviceTables {
    int4* box = nullptr;          // [C] (x0, y0, nx, ny)
    int* cell_off = nullptr;      // [C+1] offset of channel c's first cell in cell_ptr
    int* cell_ptr = nullptr;      // per channel nx*ny+1 offsets (absolute into contrib arrays)
    int* contrib_e = nullptr;     // element of each (cell, element) contribution
    float2* contrib_w = nullptr;  // conj(W) * (-1)^(x+y) of each contribution
    float2* twiddle = nullptr;    // [N/2] exp(+2 pi i m / N)
    int* first_xy = nullptr;      // [C][A] packed first tap (y << 16 | x)
    float2* w_taps = nullptr;     // [C][A][K][K] weights (conj, shift sign folded)
    float4* jones = nullptr;      // [C][A][2] polarisation mixing: (conj J^{a0}, conj J^{a1}) per output pol a
    uint16_t* dft_f16 = nullptr;  // DFT-as-GEMM operand tables (tensor path)
    size_t dft_bytes = 0;
};

// Tensor-core path state (k_dftgemm.cu).
struct TcState {
    uint16_t* a1 = nullptr;        // stage-1 DFT operands per (channel, 64-column kx pair), FP16
    uint16_t* a2 = nullptr;        // stage-2 DFT operands per (channel, 128-row ky block), FP16
    long long* a1_off = nullptr;   // element offsets into a1 / a2
    long long* a2_off = nullptr;
    int* status = nullptr;         // device flag: 1 = a bounded wait ran out
    int smem = 0;
    unsigned sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0;
    int n_g = 0, n_kb = 0, n_s = 0;
    int cg = 0, tc = 0;            // channels per group, time samples per chunk
    size_t stride = 0;             // bytes per grid tile in the chunk buffer
    unsigned b1_bytes = 0;         // bytes per shared-memory tile buffer
    int nb = 1;                    // tile buffers (2 = next tile prefetched)
    int grid_smem = 0;             // dynamic shared memory of the gridding kernel
    bool grid_csr_smem = false;    // gridding kernel stages the cell lists in shared memory
    int grid_frames = 1;           // frames gridded per pass by the gridding kernel
    bool grid_ps = false;          // persistent gridding kernel (cell lists staged per channel)
    bool grid_cplx = false;        // complex GCF weights (table GCF)
    int grid_blocks = 0;           // blocks of the persistent gridding kernel
    int grid_max_cells = 0;        // largest occupied box (cells)
    int grid_max_list = 0;         // (cell, element) entries per channel
    int grid_variant = 1;          // 1: persistent row-major gather, 2: balanced task lists, 3: pair lists
    long long* wcum = nullptr;     // [C + 1] prefix sums of k_dftgemm_ws3 item costs per frame (work split)
    int* item_order = nullptr;     // k_dftgemm_ws3 whole items: per channel group, the order items are dealt to blocks
    int* pl_ptr = nullptr;         // pair-list gridding: per channel entry offsets of the box's cell
    int* pl_off = nullptr;         //   pairs (row-major) and where each channel's start
    int* pl_e = nullptr;           //   entries: element
    float2* pl_w = nullptr;        //   entries: weights at x and x + 1
    int pl_max_ptr = 0;            //   most offsets / entries of one channel
    int pl_max_ent = 0;
    bool pl_stage = false;         //   the kernel stages a channel's lists in shared memory
    int4* gtask = nullptr;         // balanced gridding: per-channel task lists (device)
    int* gtask_off = nullptr;      // [C + 1]
    int gtask_max = 0;             // largest task list
    int* gell_e = nullptr;         // balanced gridding: interleaved entries, element
    void* gell_w = nullptr;        //   and the weights of its run of cells (one per cell)
    int* gell_off = nullptr;       // [C + 1]
    int gell_max = 0;              // largest entry list (with padding)
    bool fast = false;             // TMEM-resident stage-2 operand, double-buffered stage 1 / B2
    uint32_t* a2w = nullptr;       // stage-2 operand rows as packed FP16 pairs (fast variant)
    long long* a2w_off = nullptr;
    unsigned b2_bytes = 0;
    int d1_cols = 0;
    bool ws = false;               // warp-specialised 64-column-pair kernel
    int ws_variant = 0;            // 1: epilogue warps issue the MMAs; 2: a control warp does
    uint16_t* a1p = nullptr;       // stage-1 operands per (channel, 64-column kx pair)
    long long* a1p_off = nullptr;
    int n_gp = 0;                  // 64-column pairs per channel
    float* partial = nullptr;      // k_dftgemm_ws3: partial sums of items split between blocks
    int* counters = nullptr;       // k_dftgemm_ws3: per item, parts stored so far
    int split = -1;                // k_dftgemm_ws3 work split: -1 auto, 0 whole items, 1 equal shares
    int group = 0;                 // channels per launch: 0 groups of about two work items per SM,
    int cg_items = 0;              //   1 every channel (cg_items: the size group 0 gives)
    // Row parts of k_dftgemm_ws3: channel c's box rows are cut into H parts of nyh rows
    // (padded to H * nyh rows, the extra rows zero); each part is a grid tile of its own
    // (P * nyh rows) and a stage-1 / stage-2 step of its own, so tall boxes fit in TMEM.
    std::vector<int4> tbox_h;      // [C] (nyh, H, H * nyh, 0) on the host
    int4* tbox = nullptr;          // same, on the device (every tensor-path plan)
    bool parts = false;            // some channel has H > 1 (only k_dftgemm_ws3 takes it)
    int nbt = 2;                   // k_dftgemm_ws3: tile-part buffers in shared memory (2..4)
    size_t n_counters = 0;         // entries of `counters`
};

// Device memory one epic_image call writes besides its images: the grid / tile scratch, the
// tensor path's split bookkeeping (partial sums, per-item counters, which the last block of
// an item resets to zero) and the bounded-wait flag.  A plan owns one set; the streaming
// server gives each of its slots its own, so that calls of one plan overlap on the device.
struct CallScratch {
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    float* partial = nullptr;
    size_t partial_bytes = 0;
    int* counters = nullptr;
    size_t n_counters = 0;
    int* status = nullptr;
};

struct KernelEvent {
    const char* name;
    cudaEvent_t start, stop;
};

}  // namespace epic

struct epic_plan_s {
    // descriptor copy
    int A = 0, P = 0, C = 0, N = 0, K = 0, nprod = 0, path = 0, max_time = 0;
    int bits = 4;                         // input samples: 4 (4+4-bit bytes) or 8 (8+8-bit pairs)
    int sub = 0;                          // samples per image set (0 = the whole block)
    int logN = 0;
    int device = 0;
    std::vector<double> pos, freq, cell;
    epic_gcf_desc gcf{};
    std::vector<float> table;
    std::vector<float> jones;             // [C][A][2][2] complex pairs, empty = no polarisation mixing

    // host geometry (FP64 computed, stored as used by the kernels)
    std::vector<epic::Box> box;           // [C]
    std::vector<int> first_x, first_y;    // [C][A]
    std::vector<double> w_re, w_im;       // [C][A][K][K], conj(W) * (-1)^(jx+jy)
    int box_max_x = 0, box_max_y = 0;
    size_t n_contrib = 0;
    double tc_flops_per_sample = 0.0;     // pruned DFT-as-GEMM flops per time sample (tensor path)

    // device state
    epic::DeviceTables dt;
    size_t table_bytes = 0;
    void* scratch = nullptr;              // path-specific per-call scratch
    size_t scratch_bytes = 0;
    int time_chunk = 0;
    uint8_t* stage_volt = nullptr;        // host-API staging
    cudaStream_t copy_stream = nullptr;   // host-API copies overlapped with the tensor path's groups
    std::vector<cudaEvent_t> copy_ev;
    float* stage_out = nullptr;
    size_t stage_bytes = 0;
    int sm_count = 0;
    int smem_optin = 0;
    epic::TcState tc;                     // tensor-core path
    int fused_variant = 0;                // kernel variant chosen for fused paths
    bool auto_path = false;               // created with EPIC_PATH_AUTO: the tuner may change path
    int slab = 0;                         // output columns per work item (fused paths)
    int plain_fft = 0;                    // plain path FFT kernels: 0 register two-pass, 1 shared-memory Stockham

    size_t chunk_budget = 0;              // scratch budget of one time chunk (chunked paths)

    // errors / timing
    std::string last_error;
    cudaStream_t last_stream = nullptr;
    bool timing = false;
    std::vector<epic::KernelEvent> events;
    size_t n_events = 0;

    // CUDA-graph replay (EPIC_GRAPH)
    cudaStream_t cap_stream = nullptr;    // plan-owned stream the launches are recorded on
    bool capturing = false;
    cudaGraphExec_t gexec = nullptr;
    const void* g_volt = nullptr;         // arguments the graph was recorded for
    const float* g_out = nullptr;
    int g_T = -1;
    unsigned g_flags = 0;
    size_t g_events = 0;                  // timing events recorded in the graph
};

namespace epic {

// plan.cpp
epic_status build_geometry(epic_plan_s* p, std::string* err);
void build_csr(const epic_plan_s* p, std::vector<int>& cell_off, std::vector<int>& cell_ptr,
               std::vector<int>& contrib_e, std::vector<float2>& contrib_w);
void build_twiddles(int N, std::vector<float2>& tw);
void order_warp_entries(const std::vector<std::vector<int2>>& cells, int nmax, int2* out);

// api.cu helpers used by the kernels' launch code
// Let kernel `fn` take as much dynamic shared memory as the device allows (its
// static shared memory subtracted).  Kernels are shared by every plan, so this
// limit is never set to one plan's need: a plan created later must not shrink
// what the launches of an earlier plan ask for.
cudaError_t allow_max_smem(const void* fn, int optin);
void ev_begin(epic_plan_s* p, const char* name, cudaStream_t s);
void ev_end(epic_plan_s* p, cudaStream_t s);
epic_status cuda_fail(epic_plan_s* p, cudaError_t e, const char* what);
// Switch the plan to another path (frees the current path's tables and scratch, sets up the
// new one; on failure the plan is back on its previous path and the status is returned).
epic_status set_path(epic_plan_s* p, int path);
// one epic_image call after argument checks (flags without EPIC_GRAPH handling)
// Host-side hooks around each channel group of a tensor-path call: before(c0, ng) runs
// before the group's first launch is issued, after(c0, ng) after its last (the pipelined
// host-buffer call puts its per-group copies there).  Other paths ignore them.
struct GroupHooks {
    std::function<epic_status(int, int)> before, after;
};

epic_status image_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, unsigned flags,
                      const GroupHooks* hooks = nullptr);
// Grow c (zeroed on allocation) to what a call of p needs; allocates, so not on a hot path.
epic_status call_scratch_fit(epic_plan_s* p, CallScratch& c);
void call_scratch_free(CallScratch& c);
// image_run with c's memory in place of the plan's (same host thread as every other call of p)
epic_status image_run_with(epic_plan_s* p, CallScratch& c, const uint8_t* volt, int T, cudaStream_t s, float* out,
                           unsigned flags);

// k_plain.cu
epic_status plain_setup(epic_plan_s* p);
epic_status plain_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate);
epic_status plain_set_chunk(epic_plan_s* p, size_t budget);
epic_status plain_set_fft(epic_plan_s* p, int v);

// k_fused.cu
epic_status fused_setup(epic_plan_s* p);
epic_status fused_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate);
epic_status fused_set_slab(epic_plan_s* p, int SW);

// k_dftgemm.cu
epic_status dftgemm_setup(epic_plan_s* p);
epic_status dftgemm_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate,
                        const GroupHooks* hooks = nullptr);
epic_status dftgemm_grid_config(epic_plan_s* p, int F);
epic_status dftgemm_set_chunk(epic_plan_s* p, size_t budget);
epic_status dftgemm_set_kernel(epic_plan_s* p, int variant);
epic_status dftgemm_set_grid_kernel(epic_plan_s* p, int variant);
epic_status dftgemm_set_split(epic_plan_s* p, int mode);
epic_status dftgemm_set_group(epic_plan_s* p, int v);

}  // namespace epic
