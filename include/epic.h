/*
 * epic.h -- C ABI of the GB300 EPIC imaging library (libepic.so).
 *
 * EPIC (E-field Parallel Imaging "Correlator", paper Sec. 2) turns channelised,
 * calibrated element voltages into all-sky polarised intensity images without
 * forming pairwise correlations:
 *   Eq. 1  grid the voltages of every element onto a regular aperture grid with a
 *          gridding convolution function (GCF), then take a 2-D spatial Fourier
 *          transform (the paper implements it as an FFT);
 *   Eq. 2  form the pixelwise outer product of the polarisations and average it
 *          over the integration time.
 * One call of epic_image runs, on the GPU, for every time sample, channel and
 * polarisation of a voltage block: 4+4-bit unpack -> gridding -> 2-D transform
 * -> XX/YY/XY products -> accumulation (Sec. 2, Eq. 1-2; 4-bit input and the
 * power-of-two grid finer than lambda/2 follow the workload of Sec. 4).
 *
 * Conventions shared by every call:
 *   - Every function returns an epic_status; nothing throws across the ABI.
 *   - Voltages: uint8 [T][n_chan][n_ant][n_pol], one byte per complex sample,
 *     real part in the high nibble, imaginary in the low nibble, 4-bit two's
 *     complement (values -8..7).
 *   - Images: float32 [n_chan][n_prod][N][N], n_prod = 1 (XX) for one pol and
 *     4 (XX, YY, Re XY, Im XY; XY = E_X conj(E_Y), YX = conj(XY) not stored) for
 *     two.  Row index = m (y), column = l (x); index i holds direction cosine
 *     (i - N/2) * lambda_c / (N * Delta_c) (zero direction at N/2, "fftshifted").
 *   - The transform has the + sign of Eq. 1, no 1/N factor, and unit cell area
 *     (delta^2 r_j = 1).  The images are SUMS over the block's time samples; divide
 *     by T for the average of Eq. 2.
 *   - Grid geometry: cell spacing Delta_c (default lambda_c/2), origin at the array
 *     centroid placed at cell (N/2, N/2).  Odd K: anchor = nearest cell (ties up),
 *     taps anchor +- (K-1)/2; even K: taps floor(u)-K/2+1 .. floor(u)+K/2.  No tap
 *     may leave the grid (EPIC_ERR_GRID_OVERFLOW at plan creation).
 *   - Both polarisations share one GCF W; a per-element 2x2 polarisation-mixing
 *     kernel may multiply it (epic_plan_desc.jones, Eq. 1's W_e^{ap}).
 *   - Device pointers must come from cudaMalloc (or torch) on the device that is
 *     current when the plan is created; host pointers are plain host memory.
 *   - Calls are stream-ordered and asynchronous unless stated; CUDA errors of
 *     kernels surface as EPIC_ERR_CUDA from a later call or from epic_sync.
 *   - No CPU fallback: without a usable sm_103a GPU, plan creation fails.
 */
#ifndef EPIC_H
#define EPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EPIC_OK = 0,
    EPIC_ERR_INVALID_ARG = 1,   /* bad size, pointer, flag or descriptor field; nothing launched */
    EPIC_ERR_GRID_OVERFLOW = 2, /* a GCF tap falls outside the N x N grid (plan creation)        */
    EPIC_ERR_OOM = 3,           /* device or host allocation failed, or a server memory limit    */
    EPIC_ERR_BUSY = 4,          /* server: no free slot or memory now; retry later               */
    EPIC_ERR_TIMEOUT = 5,       /* a bounded wait ran out                                         */
    EPIC_ERR_CUDA = 6,          /* a CUDA call failed; epic_last_error() has the text             */
    EPIC_ERR_UNSUPPORTED = 7,   /* valid request this build cannot run (e.g. path/size combo)    */
    EPIC_ERR_NOT_FOUND = 8      /* unknown server ticket                                          */
} epic_status;

/* Which implementation of the hot path a plan uses. */
typedef enum {
    EPIC_PATH_PLAIN_FP32 = 0,   /* unfused FP32: grid kernel -> HBM -> row FFT -> HBM -> column FFT
                                   -> HBM -> square/accumulate kernel (the plain comparator)      */
    EPIC_PATH_FUSED_FP32 = 1,   /* one fused kernel per block: grid -> FP32 FFT -> products ->
                                   on-chip accumulation, images written once                      */
    EPIC_PATH_DFTGEMM_FP16 = 2, /* a gridding kernel writes FP16 grid tiles, then one tensor-core
                                   kernel runs the 2-D transform as two DFT-as-GEMM stages on the
                                   tcgen05 tensor cores (FP16 operands, FP32 accumulation), the
                                   products and the accumulation; per (channel group, time chunk) */
    EPIC_PATH_AUTO = 3          /* the DFT-as-GEMM path where the plan's occupied grid fits it,
                                   else the plain FP32 path; epic_plan_tune then times every path
                                   that takes the plan on the caller's block and keeps the
                                   fastest (tuning parameter "path")                              */
} epic_path;

typedef enum {
    EPIC_GCF_GAUSSIAN = 0,      /* W(d) = exp(-|d|^2 / (2 sigma_c^2)), d in cells, not renormalised */
    EPIC_GCF_TABLE = 1          /* complex W sampled on a (K*os+1)^2 table, nearest sample        */
} epic_gcf_kind;

/* Gridding convolution function (Eq. 1: W_e^{ap}(r_j - r_e), here one W for all
 * elements and both polarisations; the conjugate W* is what multiplies E). */
typedef struct {
    int kind;               /* epic_gcf_kind                                                      */
    int K;                  /* taps per side, 1..8 (2 = the paper's 2x2 kernel, Sec. 4)           */
    double sigma_cells;     /* GAUSSIAN: sigma in grid cells at f_ref_hz                          */
    double f_ref_hz;        /* GAUSSIAN: reference frequency of sigma                             */
    int freq_scaled;        /* GAUSSIAN: nonzero -> sigma_c = sigma_cells * f_c / f_ref_hz        */
    int oversample;         /* TABLE: samples per cell os >= 1                                    */
    const float* table;     /* TABLE: host, complex float pairs [(K*os+1)][(K*os+1)]; sample
                               (iy, ix) is W at offset (ix/os - K/2, iy/os - K/2) cells; copied   */
} epic_gcf_desc;

/* Everything epic_image needs besides the voltages (Eq. 1: element positions r_e,
 * grid r_j, kernel W; Eq. 2: polarisations).  All host arrays are copied. */
typedef struct {
    int n_ant;              /* elements A >= 1                                                    */
    const double* pos_m;    /* host [n_ant][2] x, y in metres                                     */
    int n_pol;              /* 1 or 2                                                             */
    int n_chan;             /* channels C >= 1, C x n_pol <= 65535                                */
    const double* freq_hz;  /* host [n_chan] centre frequency of each channel, > 0                */
    const double* cell_m;   /* host [n_chan] grid spacing Delta_c, or NULL for lambda_c / 2       */
    int grid_n;             /* N: power of two, 8..512                                            */
    epic_gcf_desc gcf;
    int path;               /* epic_path                                                          */
    int max_time;           /* largest T of one call (sizes scratch and host staging), >= 1       */
    int input_bits;         /* 4 (or 0): one 4+4-bit byte per complex sample, real in the high
                               nibble; 8: two bytes per sample, real then imaginary, two's
                               complement (paper Sec. 4)                                          */
    int sub_int;            /* 0: one image set per call (Eq. 2's average over the whole block);
                               S > 0: one image set per S samples (sub-integrations, Sec. 4) --
                               T of every call a multiple of S, 1 <= S <= max_time; the tensor
                               path needs its control-warp kernel for it (UNSUPPORTED otherwise) */
    const float* jones;     /* NULL: no polarisation mixing (W_e^{ap} = delta_ap W).  Otherwise host
                               [n_chan][n_ant][2][2] complex float pairs J_{c,e}^{ap} (output pol a,
                               input pol p), copied: the per-element kernel of Eq. 1 is
                               W_e^{ap}(r) = J_{c,e}^{ap} W(r), a direction-independent 2x2
                               leakage/gain matrix per element and channel times the shared GCF,
                               so output pol a grids sum_p conj(J^{ap}) E^p.  Needs n_pol == 2;
                               every value finite (INVALID_ARG otherwise)                          */
} epic_plan_desc;

typedef struct epic_plan_s* epic_plan_t;

/* What a plan resolved to (for logging and roofline bookkeeping). */
typedef struct {
    int path;               /* the epic_path actually used (never EPIC_PATH_AUTO)                 */
    int n_prod;             /* 1 or 4                                                             */
    int box_max_x;          /* largest occupied-grid width over channels (cells)                  */
    int box_max_y;          /* largest occupied-grid height over channels (cells)                 */
    int time_chunk;         /* time samples per internal pass                                     */
    size_t device_bytes;    /* device memory owned by the plan                                    */
    size_t scratch_bytes;   /* part of device_bytes used as per-call scratch                      */
    int n_kernels;          /* kernels in one epic_image call for T = max_time                    */
    double gemm_flops_per_sample; /* DFT-as-GEMM path: flops of the pruned two-stage transform per
                                     time sample over all channels and pols (8 per complex MAC over
                                     the occupied box); 0 for the FFT paths                        */
    int input_bits;         /* 4 or 8                                                             */
    int sub_int;            /* samples per image set, 0 = the whole block                         */
    int pol_mix;            /* 1 when the plan has a polarisation-mixing kernel (jones)           */
    int tc_kernel;          /* DFT-as-GEMM path: transform kernel of a call -- 3 the warp-
                               specialised control-warpgroup kernel, 1 / 2 its older warp-
                               specialised forms, 4 / 5 the 32-column-slab fallbacks; 0 for the
                               FFT paths                                                          */
    int row_parts;          /* DFT-as-GEMM path: most row parts of a channel's occupied grid (tall
                               grids are transformed in parts of rows whose stage-2 sums add up);
                               1 when every channel is one part; 0 for the FFT paths              */
} epic_plan_info;

/* flags of epic_image / epic_image_host */
#define EPIC_RESET       0u /* out = images of this block                                         */
#define EPIC_ACCUMULATE  1u /* out += images of this block (continue an integration / resume)     */
#define EPIC_TIME_KERNELS 2u /* record CUDA events around each kernel (see epic_kernel_times)     */
#define EPIC_GRAPH       4u /* replay the call's kernel sequence as one CUDA graph (see epic_image) */

/* Build a plan: geometry and GCF taps in FP64 on the host (Eq. 1 bracket), the
 * inverse cell -> (element, weight) lists, transform tables, device uploads.
 * Returns EPIC_ERR_INVALID_ARG for a bad descriptor, EPIC_ERR_GRID_OVERFLOW if a
 * footprint leaves the grid, EPIC_ERR_UNSUPPORTED for a path this build cannot
 * run at these sizes, EPIC_ERR_CUDA / EPIC_ERR_OOM on device failure.  On error
 * *out is NULL and nothing is leaked.  The plan owns all its device memory. */
epic_status epic_plan_create(const epic_plan_desc* desc, epic_plan_t* out);

/* Free a plan and its device memory (synchronises the plan's last stream). NULL is OK. */
epic_status epic_plan_destroy(epic_plan_t plan);

/* Image one voltage block (Eq. 1-2) on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  volt: device uint8[T][C][A][P] (uint8[T][C][A][P][2] for 8+8-bit
 * input); out: device float32 [C][n_prod][N][N] ([T/S][C][n_prod][N][N] with
 * sub-integrations of S samples), written (EPIC_RESET) or added to (EPIC_ACCUMULATE).
 * 0 <= T <= max_time; T = 0 with EPIC_RESET zeroes out.  Asynchronous: returns
 * after launching.  The plan's scratch is reused by every call, so calls on one
 * plan must not overlap on different streams.
 * EPIC_GRAPH: the plan records the call's launches (for these volt, out, T and
 * flags) on a stream of its own into a CUDA graph and launches that graph on
 * `stream`; later calls with the same arguments only launch the graph again
 * (one launch per call instead of one per kernel), a call with other arguments
 * records again and updates the graph in place.  Same images as without the flag. */
epic_status epic_image(epic_plan_t plan, const uint8_t* volt, int T, void* stream, float* out,
                       unsigned flags);

/* Same as epic_image with HOST buffers: copies volt_host (T*C*A*P bytes) to the
 * plan's device staging buffer, images it, copies the images to out_host
 * (C*n_prod*N*N floats; with EPIC_ACCUMULATE its old content is uploaded first)
 * and synchronises the stream before returning.  Pinned host memory is fastest.
 * On the tensor path with several channel groups (and no sub-integrations or
 * EPIC_ACCUMULATE) the copies overlap the computation: each group's voltages (its
 * channel range of every sample) go up on a copy stream the plan owns, the group's
 * kernels wait only for them, and its images come back while the next group
 * computes; the images are the same.  EPIC_GRAPH is then ignored.
 * Returns EPIC_ERR_TIMEOUT when a bounded device-side wait ran out during this call
 * (or during an earlier call of the plan not yet reported by epic_sync). */
epic_status epic_image_host(epic_plan_t plan, const uint8_t* volt_host, int T, void* stream,
                            float* out_host, unsigned flags);

/* Wait for the plan's last stream and report any asynchronous CUDA error, or
 * EPIC_ERR_TIMEOUT when a bounded device-side wait of one of the plan's kernels
 * ran out since the last report (the images of that call are incomplete; the
 * plan stays usable).  The flag is read and cleared here and by epic_image_host. */
epic_status epic_sync(epic_plan_t plan);

/* Failure-detection self-test: on `stream`, one block that holds tensor memory
 * waits budget_cycles (1..4e9 SM clock cycles) on a barrier nothing signals, then
 * raises the plan's bounded-wait flag, frees its tensor memory and returns -- the
 * path the tensor-core kernels take when a wait runs out.  A following epic_sync
 * (or epic_image_host) returns EPIC_ERR_TIMEOUT.  Nothing traps or faults.  The
 * paper has no counterpart: it checks this implementation's own error handling. */
epic_status epic_selftest_bounded_wait(epic_plan_t plan, long long budget_cycles, void* stream);

/* Kernel durations (ms) of the last call made with EPIC_TIME_KERNELS, in launch
 * order, with static kernel names.  Synchronises on the recorded events.
 * *n_out = number of kernels (<= max entries are written). */
epic_status epic_kernel_times(epic_plan_t plan, const char** names, float* ms, int max, int* n_out);

epic_status epic_plan_get_info(epic_plan_t plan, epic_plan_info* info);

/* Autotuner: times epic_image on the caller's block (device volt, T samples, out
 * as in epic_image; out is overwritten) for the candidate values of each of the
 * plan's tuning parameters in turn, keeping the fastest value of each, and leaves
 * the plan configured with them.  Parameters by path:
 *   AUTO plans    path         0 plain FP32, 1 fused FP32, 2 DFT-as-GEMM (timed first; the chosen
 *                              path's own parameters follow)
 *   PLAIN_FP32    fft          FFT kernels: 0 register-resident two-pass transforms (one
 *                              shared-memory exchange), 1 radix-4/2 Stockham in shared memory
 *                 chunk_mb     grid-buffer budget of one time chunk (MiB)
 *   FUSED_FP32    slab         image columns per work item
 *   DFTGEMM_FP16  group        channels per launch: 0 groups of about two work items per SM,
 *                              1 every channel in one launch (fewer launches, larger tile buffer)
 *                 mma_kernel   1: epilogue warps issue the tensor-core work, 2: a
 *                              control warp does, 3: a control warpgroup with its own
 *                              register budget does (when the occupied box allows each);
 *                 split        work of the control-warp kernel: -1 automatic (equal shares unless
 *                              the items divide evenly), 0 whole work items per SM, 1 equal
 *                              (item, time sample) shares per SM;
 *                 grid_kernel  gridding kernel: 1 row-major cell walk, 2 cells in lists sorted
 *                              by length (Gaussian GCF, when its tiles fit in shared memory);
 *                 grid_frames  frames per pass of the gridding kernel;
 *                 chunk_mb     tile-buffer budget of one (channel group, time chunk), 96 MiB to
 *                              24 GiB (the block's samples at most)
 * Images after tuning equal those before up to FP32 rounding order.  reps calls
 * are timed per candidate (1..100) after one untimed call.  May reallocate the
 * plan's scratch (EPIC_ERR_OOM if that fails; the plan then keeps working with
 * its previous values).  Synchronous.  The paper has no counterpart: this picks
 * the implementation's tiling for the GPU it runs on. */
typedef struct {
    int n_timed;            /* candidate configurations timed                                      */
    float default_ms;       /* one call with the configuration the plan had before                 */
    float best_ms;          /* one call with the chosen configuration                              */
    int n_params;           /* entries of names / values                                           */
    const char* names[8];   /* static parameter names                                              */
    int values[8];          /* chosen values                                                       */
} epic_tune_report;
epic_status epic_plan_tune(epic_plan_t plan, const uint8_t* volt, int T, void* stream, float* out, int reps,
                           epic_tune_report* report);

/* Set / read one tuning parameter by the names above (e.g. to apply values an
 * earlier epic_plan_tune reported).  EPIC_ERR_NOT_FOUND: no such parameter on
 * this plan's path; EPIC_ERR_UNSUPPORTED: the value is not possible for this
 * plan (the plan is unchanged); EPIC_ERR_OOM when a larger scratch cannot be
 * allocated.  Images change at most by FP32 rounding order.  Not during a call
 * in flight on another stream.  The paper has no counterpart. */
epic_status epic_plan_set_param(epic_plan_t plan, const char* name, int value);
epic_status epic_plan_get_param(epic_plan_t plan, const char* name, int* value);

/* Static text of a status code, and the detail of the last error on a plan
 * (or of the last failed epic_plan_create when plan is NULL).  Never NULL. */
const char* epic_status_str(epic_status s);
const char* epic_last_error(epic_plan_t plan);

/* Library and device facts: SM count and opt-in shared memory of the current
 * device; returns EPIC_ERR_CUDA without a usable device. */
epic_status epic_device_query(int* sm_count, int* smem_optin_bytes, int* cc_major, int* cc_minor);

/* Same result as epic_image, but the call allocates no device memory and uses no
 * plan scratch: its grid scratch is a fixed 32 MiB array in the library's device
 * image (held by every GPU that loads the library until the process exits).  For
 * callers that may not call cudaMalloc while imaging -- e.g. code running inside
 * a framework that owns the device memory through its own pool, or real-time
 * loops where an allocation could stall the device.  The paper has no
 * counterpart; it runs the plain FP32 pipeline (grid, row FFT, column FFT,
 * products) in time chunks that fit the array, with any plan.
 * - EPIC_ERR_UNSUPPORTED (with the sizes in epic_last_error) when one time sample
 *   of the plan needs more than 32 MiB of grids (n_chan x n_pol x N^2 x 8 bytes),
 *   and for plans with 8+8-bit input, sub-integrations or polarisation mixing.
 * - The first call on a device looks up the array's device address and sets the
 *   kernels' shared-memory limits there; make that first call before any stream
 *   capture.
 * - All calls share the array (it keeps the last call's contents; each call writes
 *   every byte it reads first): calls that overlap on the GPU race on it.
 * flags: EPIC_RESET or EPIC_ACCUMULATE.  Stream-ordered, asynchronous. */
epic_status epic_image_static_scratch(epic_plan_t plan, const uint8_t* volt, int T, void* cuda_stream, float* out,
                                      unsigned flags);

/* ---------------------------------------------------------------------------
 * Streaming server (continuous batching).  Voltage blocks from several stations
 * (one plan per station type) are admitted as they arrive and imaged
 * concurrently: each block waits until one of max_slots CUDA streams is free,
 * a range of the server's device pool (max_device_bytes, allocated once at
 * creation) holds it, and no earlier block with the same output images is still
 * queued or running -- blocks that write one set of images run in submission
 * order, all others (those of one plan included) overlap on the device.  Each
 * slot has its own call memory (a plan's grid / tile scratch and bookkeeping),
 * allocated the first time the slot runs a plan that needs more: up to max_slots
 * times the largest plan scratch (epic_plan_info.scratch_bytes) besides the pool.
 * Images go to caller-owned device accumulators (use EPIC_ACCUMULATE to continue
 * an integration across blocks).  Latency of a block = wall time from submission
 * to completion of its kernels.  A block whose bounded device wait ran out
 * completes with EPIC_ERR_TIMEOUT.  A plan given to a server must not be used by
 * other epic_image calls until its blocks are done.  The server's streams do not
 * wait for work the caller queued on other streams: the accumulators must be
 * complete (e.g. the caller's stream synchronised) when a block is submitted.
 * ------------------------------------------------------------------------- */
typedef struct epic_server_s* epic_server_t;

/* max_slots in 1..64; max_device_bytes >= 256.  EPIC_ERR_OOM if the pool cannot
 * be allocated. */
epic_status epic_server_create(size_t max_device_bytes, int max_slots, epic_server_t* out);

/* Queue one block: volt_host = host uint8[T][C][A][P] of `plan` (must stay valid and
 * unchanged until the ticket completes), out_dev = device images of the plan's
 * shape, flags EPIC_RESET or EPIC_ACCUMULATE.  Returns at once with a ticket;
 * EPIC_ERR_BUSY when the admission queue (4 x max_slots blocks) is full,
 * EPIC_ERR_OOM when the block can never fit the pool. */
epic_status epic_server_submit(epic_server_t server, epic_plan_t plan, const uint8_t* volt_host, int T,
                               float* out_dev, unsigned flags, uint64_t* ticket);

/* Non-blocking: *done = 1 once the block's images are complete (then returns the
 * block's status and its latency in ms). */
epic_status epic_server_poll(epic_server_t server, uint64_t ticket, int* done, double* latency_ms);

/* Block up to timeout_ms for a ticket, then release it and return the block's
 * status (EPIC_ERR_TIMEOUT if not done in time; EPIC_ERR_NOT_FOUND for an unknown or
 * already released ticket -- when several threads wait on one ticket, one of them
 * collects it and the others get EPIC_ERR_NOT_FOUND). */
epic_status epic_server_wait(epic_server_t server, uint64_t ticket, int timeout_ms, double* latency_ms);

/* Completed blocks so far, p50 / p99 of their latencies (ms; -1 when none), blocks
 * on the device now. */
epic_status epic_server_stats(epic_server_t server, int* completed, double* p50_ms, double* p99_ms, int* in_flight);

/* Stop admitting, finish blocks already on the device, free everything. NULL is OK. */
epic_status epic_server_destroy(epic_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* EPIC_H */
