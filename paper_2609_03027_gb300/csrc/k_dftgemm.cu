// Tensor-core path: the 2-D transform of Eq. 1 as two DFT-as-GEMM stages on the
// sm_103a tcgen05 tensor cores (FP16 operands, FP32 accumulation in TMEM),
// fused with the polarisation products and the time accumulation of Eq. 2.
//
// Per (channel c, time t) the gridded voltages G_p[y][x] occupy a box of nyp x
// nxp cells (padded).  With F[j][k] = exp(+2 pi i j k / N) and the fftshift sign
// folded into the gridding weights:
//   stage 1 (along x):  H_p[y][kx]  = sum_x G_p[y][x] F[x][kx]
//   stage 2 (along y):  E_p[ky][kx] = sum_y F[y][ky] H_p[y][kx]
// as real GEMMs on [re | im] blocks:
//   stage 1: D1[(q, kx)][(p, y)] = A1[(q, kx)][(q', x)] . B1[(p, y)][(q', x)]
//            A1 rows (re, kx) = [ Fr | -Fi ], rows (im, kx) = [ Fi | Fr ]   (128 = 2 x 64 kx)
//            B1 row (p, y)   = [ Gr_p[y][:] | Gi_p[y][:] ]                  (the grid tile)
//   stage 2: D2_p[ky][n]     = A2[ky][(q', y)] . B2_p[n][(q', y)]
//            A2 row ky       = [ Fr[:][ky] | Fi[:][ky] ]
//            B2_p row kx     = [ Hr[:][kx] | -Hi[:][kx] ],  row 32+kx = [ Hi | Hr ]
//   so that D2_p[ky][kx] = Re E_p, D2_p[ky][32+kx] = Im E_p.
// A work item is (channel, block of 128 ky, slab of kx: 32 in the fallback kernels,
// a pair of 32 in the warp-specialised ones); the XX, YY, Re/Im XY sums of its pixels
// stay in registers over every frame of a chunk.
//
// Two kernels per (channel group, time chunk), stream-ordered; the grid tiles of a
// chunk go through HBM between them (gigabytes per chunk, far more than L2; the
// autotuner's chunk budget reaches 24 GiB, a whole block per channel group):
//   k_dftgemm_grid_*  gather-grid every (t, c) frame of the chunk into FP16 tiles
//                     already in the 128-byte swizzled UMMA K-major layout (tall
//                     boxes: one such operand per row part)
//   k_dftgemm_ws3     (or an older variant) stage 1 -> TMEM -> FP16 shared B2 ->
//                     stage 2 -> TMEM -> products -> register accumulation; images
//                     written (or added) once per chunk
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "epic_internal.h"
#include "kcommon.cuh"
#include "tc_ptx.cuh"

namespace epic {

namespace {

constexpr int kThreads = 256;
constexpr size_t kScratchBudget = 3072ull << 20;  // grid tiles of one (channel group, time chunk)
constexpr long long kWaitBudget = 4000000000LL;  // clock cycles before a wait gives up (~2 s)
constexpr int kGridFramesPerBlock = 8;            // frames gridded per block (cell lists read once)

// ------------------------------------------------------------------ host helpers
// IEEE binary16 bits of v, round to nearest even (written from the format definition).
uint16_t f16_bits(double v)
{
    const uint16_t sign = std::signbit(v) ? 0x8000 : 0;
    const double a = fabs(v);
    if (std::isnan(v)) return 0x7e00;
    if (a >= 65520.0) return sign | 0x7c00;
    if (a < ldexp(1.0, -14)) {  // subnormal range: multiples of 2^-24
        const double k = nearbyint(a * ldexp(1.0, 24));
        return sign | (uint16_t)k;  // k == 1024 is the smallest normal, encoded the same way
    }
    int e;
    const double m = frexp(a, &e);  // a = m 2^e, m in [0.5, 1)
    const int ex = e - 1;           // a = (2m) 2^ex
    double mant = nearbyint((2.0 * m - 1.0) * 1024.0);
    int E = ex + 15;
    if (mant >= 1024.0) {
        mant = 0.0;
        E += 1;
    }
    if (E >= 31) return sign | 0x7c00;
    return sign | (uint16_t)(E << 10) | (uint16_t)mant;
}

// element offset (in halves) of (row r, column k) in an R-row operand stored in the
// 128-byte swizzled K-major layout: 64-wide K panels of R rows x 128 bytes, the
// 16-byte chunk c of row r at chunk position c ^ (r & 7).
inline size_t sw_off(int r, int k, int R)
{
    return (size_t)(k >> 6) * ((size_t)R * 64) + (size_t)r * 64 + ((((k >> 3) & 7) ^ (r & 7)) << 3) + (k & 7);
}

__host__ __device__ inline int pad64(int k) { return (k + 63) & ~63; }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Row parts of a box of `rows` rows (a multiple of 8 for two pols, 16 for one) for
// k_dftgemm_ws3 with D1 slots of D TMEM columns: the fewest parts H whose equal height
// nyh (rounded up to that multiple) gives P * nyh <= D.  Returns (nyh, H, H * nyh, 0),
// or H = 0 when no height fits.
inline int4 row_parts(int rows, int P, int D)
{
    const int q = P == 2 ? 8 : 16;
    for (int H = 1; H <= rows / q; ++H) {
        const int nyh = ((rows + H - 1) / H + q - 1) / q * q;
        if (P * nyh <= D) return make_int4(nyh, H, H * nyh, 0);
    }
    return make_int4(0, 0, 0, 0);
}

inline int __float_as_int_host(float f)
{
    int i;
    std::memcpy(&i, &f, sizeof i);
    return i;
}

// ------------------------------------------------------------------ device
struct MmaArgs {
    const uint8_t* tiles;
    unsigned long long tile_stride;
    int c0, n_ch, nt, n_kb, n_s, n_g, N, P, nprod;
    const int4* box;
    const uint16_t* a1;
    const uint16_t* a2;
    const long long* a1_off;
    const long long* a2_off;
    float* out;
    int accumulate;
    int* status;
    unsigned sA1, sA2, sB1, sB2;
    unsigned b1_bytes;  // bytes per tile buffer in shared memory
    // fast variant only
    const uint32_t* a2w;        // stage-2 DFT operand rows as packed FP16 pairs, per (channel, ky block)
    const long long* a2w_off;   // word offsets into a2w
    unsigned b2_bytes;          // bytes per B2 buffer
    int d1_cols;                // TMEM columns per D1 slot
    // warp-specialised variant only
    const uint16_t* a1p;        // stage-1 operands per (channel, 64-column kx pair)
    const long long* a1p_off;
    float* partial;             // k_dftgemm_ws3: 2 slots per block of 4 x 128 x 64 partial sums
    int* counters;              // k_dftgemm_ws3: per item, blocks that stored a part (reset by the last)
    int sub;                    // k_dftgemm_ws3<2>: samples per image set
    int iv0;                    // k_dftgemm_ws3<2>: image set of the chunk's first sample
    int C;                      // channels of the plan (image sets are [C][nprod][N][N])
    const int4* tbox;           // k_dftgemm_ws3: per channel row parts (nyh, H, H nyh, 0)
    int nbt;                    // k_dftgemm_ws3: tile-part buffers in shared memory (2..4)
    const long long* wcum;      // k_dftgemm_ws3<1>: [C + 1] prefix sums of the channels' item costs per frame
    const int* item_order;      // k_dftgemm_ws3<0>: per channel group (from c0 ipc), items in the order dealt to blocks
};

__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// byte offset of 16-byte chunk c (8 halves of K) of row r in an R-row operand in the
// 128-byte swizzled K-major layout
__device__ __forceinline__ size_t sw_chunk(int r, int c, int R)
{
    return (size_t)(c >> 3) * ((size_t)R * 128) + (size_t)r * 128 + (((c & 7) ^ (r & 7)) << 4);
}

// 16 consecutive image pixels of one product: written, or added to what is there.
__device__ __forceinline__ void store_pixels16(float* op, int nk, int accumulate, const float (&v)[16])
{
    if (nk == 16) {
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            float4 w = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            if (accumulate) {
                const float4 u = *reinterpret_cast<const float4*>(op + i);
                w.x += u.x;
                w.y += u.y;
                w.z += u.z;
                w.w += u.w;
            }
            *reinterpret_cast<float4*>(op + i) = w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i < nk) op[i] = (accumulate ? op[i] : 0.f) + v[i];
    }
}

// store_pixels16 for the sub-integration flush of k_dftgemm_ws3<2>: the same stores, the tail
// of a tile cut by an 8-column grid in a rolled loop.  Indexing the sums at run time there
// makes the compiler keep them in memory rather than spill the frame loop around an unrolled
// flush inside it: measured 10.1 against 17-20 ms for the LWA block with an image set every 4
// samples.  (The other schedules store once per work item and keep the unrolled form: for them
// sums in memory cost 2x.)
__device__ __forceinline__ void store_pixels16_flush(float* op, int nk, int accumulate, const float (&v)[16])
{
    if (nk == 16) {
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            float4 w = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            if (accumulate) {
                const float4 u = *reinterpret_cast<const float4*>(op + i);
                w.x += u.x;
                w.y += u.y;
                w.z += u.z;
                w.w += u.w;
            }
            *reinterpret_cast<float4*>(op + i) = w;
        }
    } else {
        for (int i = 0; i < nk; ++i) op[i] = (accumulate ? op[i] : 0.f) + v[i];
    }
}

// First unit of block b of G when a launch's units -- ipc items of each of n_ch channels from
// c0 in channel order, nt frames per item, item-major -- are cut into G ranges of equal cost,
// a unit costing its channel's weight (wcum: prefix sums of the weights over the plan's
// channels).  Without weights, G ranges of equal numbers of units.  Non-decreasing in b,
// 0 at b = 0 and every unit at b = G.
__device__ __forceinline__ long long split_start(const long long* wcum, int c0, int n_ch, int ipc, int nt, int b, int G)
{
    const long long per = (long long)ipc * nt;  // units of one channel
    if (!wcum) return (long long)n_ch * per * b / G;
    const long long base = wcum[c0];
    const long long s = per * (wcum[c0 + n_ch] - base) * b / G;  // cost position of the block's start
    int lo = 0, hi = n_ch;                                        // last channel whose units start at or before s
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (per * (wcum[c0 + mid] - base) <= s) lo = mid;
        else hi = mid;
    }
    const long long w = wcum[c0 + lo + 1] - wcum[c0 + lo];
    const long long u = min(per, (s - per * (wcum[c0 + lo] - base)) / w);
    return (long long)lo * per + u;
}

// Unpack and gather-grid frames of one chunk into FP16 UMMA tiles.  A block
// handles `fpc` consecutive frames of one channel, F frames per pass; a thread
// owns two horizontally adjacent cells, walks their (element, weight) lists once
// per pass and applies every entry to the F frames (F independent accumulators),
// then writes the cells as FP16 pairs: consecutive threads cover consecutive
// cell pairs of a row, so a warp fills whole 128-byte rows of the swizzled tile.
// With CSR_SMEM the channel's cell lists sit in shared memory as (element, real
// weight) pairs (Gaussian GCF), otherwise they are read through L1.
template <bool CSR_SMEM, int F>
__global__ void __launch_bounds__(kThreads) k_dftgemm_grid(const uint8_t* __restrict__ volt, int t0, int c0,
                                                           int n_ch, int nt, int fpc, int C, int A, int P,
                                                           int bits, const int4* __restrict__ box,
                                                           const int* __restrict__ cell_off,
                                                           const int* __restrict__ cell_ptr,
                                                           const int* __restrict__ ce,
                                                           const float2* __restrict__ cw,
                                                           const float4* __restrict__ jones,
                                                           const int4* __restrict__ tbox,
                                                           uint8_t* __restrict__ tiles,
                                                           unsigned long long tile_stride)
{
    extern __shared__ __align__(128) uint8_t gsm[];
    float4* sv = reinterpret_cast<float4*>(gsm);  // [F][A]: (re X, im X, re Y, im Y)
    const int cl = blockIdx.y, c = c0 + cl;
    const float4* jm = jones ? jones + (size_t)c * A * 2 : nullptr;  // polarisation mixing
    const int4 b = box[c];
    const int nxp = b.z, nyp = b.w, ncell = nxp * nyp;
    const int4 tp = tbox[c];  // row parts: rows nyp .. H nyh - 1 are written as zeros
    const int nyh = tp.x, N1h = P * nyh;
    const uint32_t part_bytes = (uint32_t)N1h * pad64(2 * nxp) * 2;
    const int* gptr = cell_ptr + cell_off[c];
    const int* ptr = gptr;
    int2* con = nullptr;
    if (CSR_SMEM) {
        int* sptr = reinterpret_cast<int*>(gsm + sizeof(float4) * (size_t)F * A);
        con = reinterpret_cast<int2*>(sptr + ((ncell + 2) & ~1));
        const int base = gptr[0];
        const int ncon = gptr[ncell] - base;
        for (int i = threadIdx.x; i <= ncell; i += blockDim.x) sptr[i] = gptr[i] - base;
        for (int i = threadIdx.x; i < ncon; i += blockDim.x)
            con[i] = make_int2(ce[base + i], __float_as_int(cw[base + i].x));
        ptr = sptr;
    }
    const int f0 = blockIdx.x * fpc, f1 = min(nt, f0 + fpc);
    const int half = nxp >> 1;
    const int tasks = tp.z * half;
    for (int tb = f0; tb < f1; tb += F) {
        const int nf = min(F, f1 - tb);
        __syncthreads();
        for (int i = threadIdx.x; i < nf * A; i += blockDim.x) {
            const int f = i / A, e = i - f * A;
            const uint8_t* fr = volt + ((size_t)(t0 + tb + f) * C + c) * (size_t)A * P * (bits / 4);
            sv[f * A + e] = load_quad(fr, e, P, bits, jm);
        }
        __syncthreads();
        for (int task = threadIdx.x; task < tasks; task += blockDim.x) {
            const int y = task / half, x = 2 * (task - y * half);
            float4 g[2][F];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int f = 0; f < F; ++f) g[j][f] = make_float4(0.f, 0.f, 0.f, 0.f);
                const int r = y * nxp + x + j;
                const int q1 = y < nyp ? ptr[r + 1] : 0;
                for (int q = y < nyp ? ptr[r] : 0; q < q1; ++q) {
                    int e;
                    float2 w;
                    if (CSR_SMEM) {
                        const int2 cr = con[q];
                        e = cr.x;
                        w = make_float2(__int_as_float(cr.y), 0.f);
                    } else {
                        e = ce[q];
                        w = cw[q];
                    }
#pragma unroll
                    for (int f = 0; f < F; ++f) {
                        const float4 v = sv[f * A + e];
                        if (CSR_SMEM) {
                            g[j][f].x = fmaf(w.x, v.x, g[j][f].x);
                            g[j][f].y = fmaf(w.x, v.y, g[j][f].y);
                            g[j][f].z = fmaf(w.x, v.z, g[j][f].z);
                            g[j][f].w = fmaf(w.x, v.w, g[j][f].w);
                        } else {
                            const float2 gx = cfma(w, make_float2(v.x, v.y), make_float2(g[j][f].x, g[j][f].y));
                            const float2 gy = cfma(w, make_float2(v.z, v.w), make_float2(g[j][f].z, g[j][f].w));
                            g[j][f] = make_float4(gx.x, gx.y, gy.x, gy.y);
                        }
                    }
                }
            }
            // cells (y, x) and (y, x+1): K index x (re) and nxp + x (im), in row part y / nyh at
            // rows p*nyh + y % nyh
            const int kc_re = x >> 3, kc_im = (nxp + x) >> 3, within = (x & 7) * 2;
            const int hpart = y / nyh, R0 = y - hpart * nyh;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (f >= nf) break;
                uint8_t* tile = tiles + ((size_t)(tb + f) * n_ch + cl) * tile_stride + (size_t)hpart * part_bytes;
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_re, N1h) + within) = pack_h2(g[0][f].x, g[1][f].x);
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_im, N1h) + within) = pack_h2(g[0][f].y, g[1][f].y);
                if (P == 2) {
                    const int R1 = nyh + R0;
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_re, N1h) + within) = pack_h2(g[0][f].z, g[1][f].z);
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_im, N1h) + within) = pack_h2(g[0][f].w, g[1][f].w);
                }
            }
        }
    }
}

// Persistent gridding kernel: block b owns the contiguous range [w0, w1) of the
// chunk's (channel, frame) pairs in channel-major order, so every block grids the
// same number of frames (+-1) and stages the cell lists of at most a few channels.
// Frames go in passes of up to F frames of one channel; the raw voltage bytes of
// the next pass are fetched by the TMA engine (one bulk copy per frame) while the
// current pass is gridded.  Each thread owns two horizontally adjacent cells per
// task, walks their (element, weight) lists once per pass and applies every entry
// to the pass's frames, then writes FP16 pairs into the swizzled UMMA tiles as the
// gather kernel above does.  CPLX selects complex weights (table GCF).
struct GridArgs {
    const uint8_t* volt;
    int t0, c0, n_ch, nt, C, A, P;
    const int4* box;
    const int* cell_off;
    const int* cell_ptr;
    const int* ce;
    const float2* cw;
    uint8_t* tiles;
    unsigned long long tile_stride;
    int* status;
    int max_cells;  // largest nx * ny over the channels
    int max_list;   // largest number of (cell, element) entries of a channel
    int bulk;       // 1: voltage frames copied by the TMA engine (frame bytes % 16 == 0, 16-byte aligned base)
    int bits;       // 4: 4+4-bit bytes, 8: 8+8-bit sample pairs
    const float4* jones;  // [C][A][2] polarisation-mixing rows (conj J), or nullptr
    const int4* tbox;     // [C] row parts of the tiles: (nyh, H, H nyh, 0)
};

__host__ __device__ inline size_t grid_ps_smem(int F, int A, int frame_bytes, int max_cells, int max_list, bool cplx)
{
    const size_t ap = (size_t)((frame_bytes + 15) & ~15);
    size_t b = 2ull * F * ap + 16ull * F * A + 4ull * ((max_cells + 2) & ~1);
    b += cplx ? 4ull * ((max_list + 1) & ~1) + 8ull * max_list : 8ull * max_list;
    return b;
}

template <bool CPLX, int F>
__global__ void __launch_bounds__(kThreads) k_dftgemm_grid_ps(GridArgs a)
{
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ uint64_t bar_raw[2];
    const int tid = threadIdx.x;
    const int A = a.A, P = a.P, AP = A * P * (a.bits / 4);  // bytes of one frame
    const int APr = (AP + 15) & ~15;
    uint8_t* raw = gsm;                                                  // [2][F][APr]
    float4* sv = reinterpret_cast<float4*>(gsm + 2 * F * APr);           // [F][A]
    int* sptr = reinterpret_cast<int*>(sv + F * A);                      // [ncell + 1], relative
    int2* con = reinterpret_cast<int2*>(sptr + ((a.max_cells + 2) & ~1));  // real: (e, w)
    int* cone = reinterpret_cast<int*>(con);                             // complex: e ...
    float2* conw = reinterpret_cast<float2*>(cone + ((a.max_list + 1) & ~1));  // ... and w

    // (channel, frame) pairs [w0, w1) of this block
    const long long w0 = split_start(nullptr, a.c0, a.n_ch, 1, a.nt, blockIdx.x, gridDim.x);
    const long long w1 = split_start(nullptr, a.c0, a.n_ch, 1, a.nt, blockIdx.x + 1, gridDim.x);
    if (tid == 0) {
        tc::mbar_init(&bar_raw[0], 1);
        tc::mbar_init(&bar_raw[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (w0 >= w1) return;

    auto pass_len = [&](long long w) {
        const int f = (int)(w % a.nt);
        return (int)min((long long)min(F, a.nt - f), w1 - w);
    };
    auto fetch = [&](long long w, int b) {  // thread 0: raw bytes of the pass starting at w -> buffer b
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        tc::mbar_expect_tx(&bar_raw[b], (uint32_t)(nf * AP));
        for (int i = 0; i < nf; ++i)
            tc::bulk_g2s(raw + (size_t)(b * F + i) * APr,
                         a.volt + ((size_t)(a.t0 + f + i) * a.C + a.c0 + cl) * (size_t)AP, (uint32_t)AP, &bar_raw[b]);
    };

    uint32_t ph = 0;          // parity bit per raw buffer
    uint32_t pending = 0;     // bit b: a bulk copy into raw buffer b is in flight (thread 0)
    int staged = -1, buf = 0;
    bool ok = true;
    if (a.bulk && tid == 0) {
        fetch(w0, 0);
        pending = 1u;
    }
    for (long long w = w0; w < w1;) {
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        const long long wn = w + nf;
        const int c = a.c0 + cl;
        const int4 b = a.box[c];
        const int nxp = b.z, nyp = b.w, ncell = nxp * nyp;
        const int4 tp = a.tbox[c];  // row parts: rows nyp .. H nyh - 1 are written as zeros
        const int nyh = tp.x, N1h = P * nyh;
        const uint32_t part_bytes = (uint32_t)N1h * pad64(2 * nxp) * 2;
        const float4* jm = a.jones ? a.jones + (size_t)c * A * 2 : nullptr;  // polarisation mixing
        if (a.bulk && tid == 0 && wn < w1) {  // the other buffer was consumed by the previous pass
            fetch(wn, buf ^ 1);
            pending |= 1u << (buf ^ 1);
        }
        if (cl != staged) {  // cell lists of channel c -> shared memory
            const int* gptr = a.cell_ptr + a.cell_off[c];
            const int base = gptr[0];
            const int ncon = gptr[ncell] - base;
            for (int i = tid; i <= ncell; i += blockDim.x) sptr[i] = gptr[i] - base;
            for (int i = tid; i < ncon; i += blockDim.x) {
                if (CPLX) {
                    cone[i] = a.ce[base + i];
                    conw[i] = a.cw[base + i];
                } else {
                    con[i] = make_int2(a.ce[base + i], __float_as_int(a.cw[base + i].x));
                }
            }
            staged = cl;
        }
        // unpack the pass's voltages: (re X, im X, re Y, im Y) per element and frame
        if (a.bulk) {
            const bool got = tc::mbar_wait(&bar_raw[buf], (ph >> buf) & 1u, kWaitBudget);
            if (got) {
                ph ^= 1u << buf;
                pending &= ~(1u << buf);
            }
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            for (int i = tid; i < nf * A; i += blockDim.x) {
                const int fi = i / A, e = i - fi * A;
                const uint8_t* fr = raw + (size_t)(buf * F + fi) * APr;
                sv[fi * A + e] = load_quad(fr, e, P, a.bits, jm);
            }
        } else {
            for (int i = tid; i < nf * A; i += blockDim.x) {
                const int fi = i / A, e = i - fi * A;
                const uint8_t* fr = a.volt + ((size_t)(a.t0 + f + fi) * a.C + c) * (size_t)AP;
                sv[fi * A + e] = load_quad(fr, e, P, a.bits, jm);
            }
        }
        __syncthreads();
        const int half = nxp >> 1;
        const int tasks = tp.z * half;
        for (int task = tid; task < tasks; task += blockDim.x) {
            const int y = task / half, x = 2 * (task - y * half);
            float4 g[2][F];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int fi = 0; fi < F; ++fi) g[j][fi] = make_float4(0.f, 0.f, 0.f, 0.f);
                const int r = y * nxp + x + j;
                const int q1 = y < nyp ? sptr[r + 1] : 0;
                for (int q = y < nyp ? sptr[r] : 0; q < q1; ++q) {
                    int e;
                    float2 wv;
                    if (CPLX) {
                        e = cone[q];
                        wv = conw[q];
                    } else {
                        const int2 cr = con[q];
                        e = cr.x;
                        wv = make_float2(__int_as_float(cr.y), 0.f);
                    }
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) {
                        if (fi < nf) {
                            const float4 v = sv[fi * A + e];
                            if (!CPLX) {
                                g[j][fi].x = fmaf(wv.x, v.x, g[j][fi].x);
                                g[j][fi].y = fmaf(wv.x, v.y, g[j][fi].y);
                                g[j][fi].z = fmaf(wv.x, v.z, g[j][fi].z);
                                g[j][fi].w = fmaf(wv.x, v.w, g[j][fi].w);
                            } else {
                                const float2 gx = cfma(wv, make_float2(v.x, v.y), make_float2(g[j][fi].x, g[j][fi].y));
                                const float2 gy = cfma(wv, make_float2(v.z, v.w), make_float2(g[j][fi].z, g[j][fi].w));
                                g[j][fi] = make_float4(gx.x, gx.y, gy.x, gy.y);
                            }
                        }
                    }
                }
            }
            const int kc_re = x >> 3, kc_im = (nxp + x) >> 3, within = (x & 7) * 2;
            const int hpart = y / nyh, R0 = y - hpart * nyh;
#pragma unroll
            for (int fi = 0; fi < F; ++fi) {
                if (fi >= nf) break;
                uint8_t* tile =
                    a.tiles + ((size_t)(f + fi) * a.n_ch + cl) * a.tile_stride + (size_t)hpart * part_bytes;
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_re, N1h) + within) = pack_h2(g[0][fi].x, g[1][fi].x);
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_im, N1h) + within) = pack_h2(g[0][fi].y, g[1][fi].y);
                if (P == 2) {
                    const int R1 = nyh + R0;
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_re, N1h) + within) =
                        pack_h2(g[0][fi].z, g[1][fi].z);
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_im, N1h) + within) =
                        pack_h2(g[0][fi].w, g[1][fi].w);
                }
            }
        }
        __syncthreads();  // sv and the cell lists are reused by the next pass
        w = wn;
        buf ^= 1;
    }
    if (!ok && tid == 0) {
        // leave no bulk copy in flight into this block's shared memory
        for (int b2 = 0; b2 < 2; ++b2)
            if ((pending >> b2) & 1u) tc::mbar_wait(&bar_raw[b2], (ph >> b2) & 1u, kWaitBudget);
        atomicExch(a.status, 1);
    }
}

// Balanced gridding kernel (real GCF weights).  A task is a run of kTaskCells
// horizontally adjacent cells (x a multiple of kTaskCells) of a channel's box: its
// list holds every element whose footprint covers any of them, with one weight per
// cell (zero where the footprint ends), so each voltage read serves all the cells and
// their FP16 results in a tile row leave as one 2 x kTaskCells-byte word.  Tasks are taken from a per-channel list
// sorted by entry count, so the 32 lanes of a warp walk lists of nearly equal length
// (a row-major walk keeps about 40% of the lanes busy), and the F frames of a pass are
// assembled in shared-memory tiles that the TMA engine then stores with one bulk copy
// per frame.  Tile buffers are double buffered across passes; cells no task touches
// stay zero from the channel's first pass.  The entries of the 32 tasks a warp handles
// together are interleaved (entry k of lane l at 32 k + l: elements as one 128-byte row,
// weights as one 32 x 4 x kTaskCells-byte row per step).  With H the unpacked voltages are held
// as FP16 pairs, the F frames of an element side by side (F x 8 bytes: X, Y of frame
// 0, ...), so one 16-byte load per entry serves two frames; 4- and 8-bit samples are
// exact in FP16, so the sums are bitwise those of the FP32 form (which polarisation
// mixing uses).
constexpr int kTaskCells = 2;                             // cells per gridding task (2 or 4; 4 measured no faster)
using TaskW = std::conditional<kTaskCells == 4, float4, float2>::type;  // one weight per cell
__host__ __device__ __forceinline__ void task_w_get(const float2& w, float* q) { q[0] = w.x; q[1] = w.y; }
__host__ __device__ __forceinline__ void task_w_get(const float4& w, float* q)
{
    q[0] = w.x;
    q[1] = w.y;
    q[2] = w.z;
    q[3] = w.w;
}
__host__ __device__ __forceinline__ void task_w_set(float2& w, const float* q) { w = make_float2(q[0], q[1]); }
__host__ __device__ __forceinline__ void task_w_set(float4& w, const float* q) { w = make_float4(q[0], q[1], q[2], q[3]); }
__device__ __forceinline__ void store_words(uint8_t* dst, const uint32_t (&w)[1]) { *reinterpret_cast<uint32_t*>(dst) = w[0]; }
__device__ __forceinline__ void store_words(uint8_t* dst, const uint32_t (&w)[2])
{
    *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
}
constexpr int kGridBalThreads = 512;                      // gridding threads
constexpr int kGridBalBlock = kGridBalThreads + 32;        // + one warp that issues the bulk copies

struct GridBalArgs {
    GridArgs g;
    const int4* tasks;      // per channel: (cell run | group's longest list << 24, group's first
                            //  entry, tile byte offsets of the run's re X and im X words, or -1
                            //  for a padding task); warp w takes groups w, w + 16, ... of 32 tasks
    const int* task_off;    // [C + 1]
    const int* ell_e;       // per channel: element of each entry, 32 lanes interleaved per group
    const TaskW* ell_w;     // per channel: weights at x, x + 1, ... of each entry
    const int* ell_off;     // [C + 1]
    int max_tasks;          // largest task count of a channel
    int max_ell;            // largest entry count of a channel (with padding)
    unsigned tile_max;      // shared-memory bytes per tile (largest channel)
};

__host__ __device__ inline size_t grid_bal_smem(int F, int A, int frame_bytes, int max_tasks, int max_list,
                                               unsigned tile_max)
{
    const size_t ap = (size_t)((frame_bytes + 15) & ~15);
    size_t b = 2ull * F * ap + 16ull * F * A;  // raw voltages, unpacked voltages
    b = (b + 127) & ~(size_t)127;
    b += 2ull * F * tile_max;                  // tile buffers
    b += 16ull * max_tasks + (4ull + sizeof(TaskW)) * max_list;  // task list, entries (weights, elements)
    return b;
}

__host__ __device__ __forceinline__ uint32_t tile_half_off(int R, int k, int N1)
{
    return (uint32_t)((k >> 6) * (N1 * 128) + R * 128 + ((((k >> 3) & 7) ^ (R & 7)) << 4) + ((k & 7) << 1));
}

// Byte offset of the FP16 at (pol-X row y, K index k) of a grid tile cut into row parts of
// nyh rows: part h = y / nyh is an operand of its own (P nyh rows: pol X rows 0..nyh-1, pol
// Y rows nyh..2 nyh-1, so a pol-Y value sits nyh * 128 bytes after its pol-X value),
// part_bytes apart.  One part (nyh = box rows) is the plain layout.
__host__ __device__ __forceinline__ uint32_t tile_part_off(int y, int k, int nyh, int P, uint32_t part_bytes)
{
    const int h = y / nyh;
    return (uint32_t)h * part_bytes + tile_half_off(y - h * nyh, k, P * nyh);
}

template <int F, bool H>
__global__ void __launch_bounds__(kGridBalBlock, 1) k_dftgemm_grid_bal(GridBalArgs ba)
{
    const GridArgs& a = ba.g;
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ uint64_t bar_raw[2];
    const int tid = threadIdx.x;
    // Threads 0..kGridBalThreads-1 grid; the first thread of the last warp issues every bulk
    // copy (raw frames of the next pass, tile stores of the previous one) while the others
    // work, so that no gridding thread waits for the copy engine to accept a copy.
    const bool tma = tid == kGridBalThreads;
    const int nthr = kGridBalThreads;
    const int A = a.A, P = a.P, AP = A * P * (a.bits / 4);  // bytes of one frame
    const int APr = (AP + 15) & ~15;
    uint8_t* raw = gsm;                                                // [2][F][APr]
    float4* sv = reinterpret_cast<float4*>(gsm + 2 * F * APr);         // [F][A] (FP32) or [A][F] (H)
    uint2* svh = reinterpret_cast<uint2*>(sv);
    const size_t tiles_at = ((size_t)2 * F * APr + 16ull * F * A + 127) & ~(size_t)127;
    uint8_t* stile = gsm + tiles_at;                                   // [2][F][tile_max]
    int4* stask = reinterpret_cast<int4*>(stile + 2ull * F * ba.tile_max);
    TaskW* sell_w = reinterpret_cast<TaskW*>(stask + ba.max_tasks);
    int* sell_e = reinterpret_cast<int*>(sell_w + ba.max_ell);

    const long long W = (long long)a.n_ch * a.nt;
    const long long w0 = W * blockIdx.x / gridDim.x, w1 = W * (blockIdx.x + 1) / gridDim.x;
    if (tma) {
        tc::mbar_init(&bar_raw[0], 1);
        tc::mbar_init(&bar_raw[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < F * A; i += blockDim.x) sv[i] = make_float4(0.f, 0.f, 0.f, 0.f);  // short passes read all F
    __syncthreads();
    if (w0 >= w1) return;

    auto pass_len = [&](long long w) {
        const int f = (int)(w % a.nt);
        return (int)min((long long)min(F, a.nt - f), w1 - w);
    };
    auto fetch = [&](long long w, int b) {  // copy thread: raw bytes of the pass starting at w -> buffer b
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        tc::mbar_expect_tx(&bar_raw[b], (uint32_t)(nf * AP));
        for (int i = 0; i < nf; ++i)
            tc::bulk_g2s(raw + (size_t)(b * F + i) * APr,
                         a.volt + ((size_t)(a.t0 + f + i) * a.C + a.c0 + cl) * (size_t)AP, (uint32_t)AP, &bar_raw[b]);
    };

    uint32_t ph = 0, pending = 0;
    int staged = -1, buf = 0, tb = 0, ntask = 0;
    bool ok = true;
    if (a.bulk && tma) {
        fetch(w0, 0);
        pending = 1u;
    }
    // tile stores of the last finished pass, issued by the copy thread one pass later
    int d_nf = 0, d_f = 0, d_cl = 0, d_tb = 0;
    uint32_t d_bytes = 0;
    auto store_deferred = [&]() {
        if (d_nf == 0) return;
        for (int fi = 0; fi < d_nf; ++fi)
            tc::bulk_s2g(a.tiles + ((size_t)(d_f + fi) * a.n_ch + d_cl) * a.tile_stride,
                         stile + ((size_t)d_tb * F + fi) * ba.tile_max, d_bytes);
        tc::bulk_commit();
        d_nf = 0;
    };
    int4 b = make_int4(0, 0, 0, 0);  // box of the staged channel (read once per channel, not per pass)
    int4 tp = make_int4(0, 0, 0, 0);  // and its row parts
    for (long long w = w0; w < w1;) {
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        const long long wn = w + nf;
        const int c = a.c0 + cl;
        if (cl != staged) b = a.box[c];
        if (cl != staged) tp = a.tbox[c];
        const int nxp = b.z, nyh = tp.x;
        const float4* jm = a.jones ? a.jones + (size_t)c * A * 2 : nullptr;  // polarisation mixing
        const uint32_t tile_bytes = (uint32_t)(P * tp.z) * pad64(2 * nxp) * 2;  // every part
        if (cl != staged) {  // new channel: zeroed tile buffers, its task list and entries
            if (tma) {
                store_deferred();
                tc::bulk_wait_read<0>();
            }
            __syncthreads();
            const int nz = (int)((2ull * F * ba.tile_max) >> 4);
            for (int i = tid; i < nz; i += blockDim.x) reinterpret_cast<uint4*>(stile)[i] = make_uint4(0, 0, 0, 0);
            ntask = ba.task_off[c + 1] - ba.task_off[c];
            const int t0 = ba.task_off[c];
            for (int i = tid; i < ntask; i += blockDim.x) stask[i] = ba.tasks[t0 + i];
            const int e0 = ba.ell_off[c], nell = ba.ell_off[c + 1] - e0;
            for (int i = tid; i < nell; i += blockDim.x) {
                sell_w[i] = ba.ell_w[e0 + i];
                sell_e[i] = ba.ell_e[e0 + i];
            }
            staged = cl;
        }
        if (a.bulk) {
            const bool got = tc::mbar_wait(&bar_raw[buf], (ph >> buf) & 1u, kWaitBudget);
            if (got) {
                ph ^= 1u << buf;
                pending &= ~(1u << buf);
            }
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            for (int i = tid; i < nf * A && tid < nthr; i += nthr) {
                const int fi = i / A, e = i - fi * A;
                const uint8_t* fr = raw + (size_t)(buf * F + fi) * APr;
                const float4 q = load_quad(fr, e, P, a.bits, jm);
                if (H) svh[e * F + fi] = make_uint2(pack_h2(q.x, q.y), pack_h2(q.z, q.w));
                else sv[fi * A + e] = q;
            }
        } else {
            for (int i = tid; i < nf * A && tid < nthr; i += nthr) {
                const int fi = i / A, e = i - fi * A;
                const uint8_t* fr = a.volt + ((size_t)(a.t0 + f + fi) * a.C + c) * (size_t)AP;
                const float4 q = load_quad(fr, e, P, a.bits, jm);
                if (H) svh[e * F + fi] = make_uint2(pack_h2(q.x, q.y), pack_h2(q.z, q.w));
                else sv[fi * A + e] = q;
            }
        }
        if (tma) {  // the previous pass's tiles go out; those of the pass before last have been read
            store_deferred();
            tc::bulk_wait_read<1>();
        }
        __syncthreads();
        if (a.bulk && tma && wn < w1) {  // raw frames of the next pass, while the others grid
            fetch(wn, buf ^ 1);
            pending |= 1u << (buf ^ 1);
        }
        uint8_t* tset = stile + (size_t)tb * F * ba.tile_max;
        for (int s = tid; s < ntask && tid < nthr; s += nthr) {
            const int4 tk = stask[s];
            const int n = (int)((unsigned)tk.x >> 24);
            float4 g[kTaskCells][F];  // cells x, x + 1, ...
#pragma unroll
            for (int q = 0; q < kTaskCells; ++q)
#pragma unroll
                for (int fi = 0; fi < F; ++fi) g[q][fi] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int* le = sell_e + tk.y + (s & 31);
            const TaskW* lw = sell_w + tk.y + (s & 31);
            auto apply = [&](TaskW w, const float4 (&v)[F]) {
                float wq[kTaskCells];
                task_w_get(w, wq);
#pragma unroll
                for (int q = 0; q < kTaskCells; ++q)
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) {
                        g[q][fi].x = fmaf(wq[q], v[fi].x, g[q][fi].x);
                        g[q][fi].y = fmaf(wq[q], v[fi].y, g[q][fi].y);
                        g[q][fi].z = fmaf(wq[q], v[fi].z, g[q][fi].z);
                        g[q][fi].w = fmaf(wq[q], v[fi].w, g[q][fi].w);
                    }
            };
            auto load = [&](int el, float4 (&v)[F]) {  // frames past nf read stale but valid entries
                if constexpr (H) {
                    uint2 h[F];
                    if constexpr (F == 1) {
                        h[0] = svh[el];
                    } else {
                        const uint4* q = reinterpret_cast<const uint4*>(svh + el * F);
#pragma unroll
                        for (int j = 0; j < F / 2; ++j) {
                            const uint4 u = q[j];
                            h[2 * j] = make_uint2(u.x, u.y);
                            h[2 * j + 1] = make_uint2(u.z, u.w);
                        }
                    }
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) {
                        const float2 x = __half22float2(*reinterpret_cast<const __half2*>(&h[fi].x));
                        const float2 y = __half22float2(*reinterpret_cast<const __half2*>(&h[fi].y));
                        v[fi] = make_float4(x.x, x.y, y.x, y.y);
                    }
                } else {
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) v[fi] = sv[fi * A + el];
                }
            };
            int k = 0;
            for (; k + 1 < n; k += 2) {  // two entries in flight, applied in list order
                const int e0 = le[32 * k], e1 = le[32 * (k + 1)];
                const TaskW w0 = lw[32 * k], w1 = lw[32 * (k + 1)];
                float4 v0[F], v1[F];
                load(e0, v0);
                load(e1, v1);
                apply(w0, v0);
                apply(w1, v1);
            }
            if (k < n) {
                const int e0 = le[32 * k];
                const TaskW w0 = lw[32 * k];
                float4 v0[F];
                load(e0, v0);
                apply(w0, v0);
            }
            // pol-Y rows sit nyh rows below the pol-X rows of their part within every 64-column
            // panel, with the same swizzle phase (nyh is a multiple of 8)
            const uint32_t o_rx = (uint32_t)tk.z, o_ix = (uint32_t)tk.w;
            const uint32_t o_ry = o_rx + (uint32_t)nyh * 128, o_iy = o_ix + (uint32_t)nyh * 128;
#pragma unroll
            for (int fi = 0; fi < F; ++fi) {
                if (fi >= nf || tk.z < 0) break;  // tk.z < 0: padding task
                uint8_t* t = tset + (size_t)fi * ba.tile_max;
                uint32_t rx[kTaskCells / 2], ix[kTaskCells / 2], ry[kTaskCells / 2], iy[kTaskCells / 2];
#pragma unroll
                for (int q = 0; q < kTaskCells / 2; ++q) {
                    rx[q] = pack_h2(g[2 * q][fi].x, g[2 * q + 1][fi].x);
                    ix[q] = pack_h2(g[2 * q][fi].y, g[2 * q + 1][fi].y);
                    ry[q] = pack_h2(g[2 * q][fi].z, g[2 * q + 1][fi].z);
                    iy[q] = pack_h2(g[2 * q][fi].w, g[2 * q + 1][fi].w);
                }
                store_words(t + o_rx, rx);
                store_words(t + o_ix, ix);
                if (P == 2) {
                    store_words(t + o_ry, ry);
                    store_words(t + o_iy, iy);
                }
            }
        }
        tc::fence_proxy_async();  // tile writes -> visible to the bulk copies
        __syncthreads();
        if (tma) {  // stored at the next pass (or after the loop)
            d_nf = nf;
            d_f = f;
            d_cl = cl;
            d_tb = tb;
            d_bytes = tile_bytes;
        }
        w = wn;
        buf ^= 1;
        tb ^= 1;
    }
    if (tma) {
        if (ok) store_deferred();
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // tile stores complete
        if (!ok) {
            for (int b2 = 0; b2 < 2; ++b2)
                if ((pending >> b2) & 1u) tc::mbar_wait(&bar_raw[b2], (ph >> b2) & 1u, kWaitBudget);
            atomicExch(a.status, 1);
        }
    }
}

// Row-major pair-list gridding kernel (real GCF weights): persistent like
// k_dftgemm_grid_ps, but a task's list is that of a run of two horizontally adjacent
// cells (every element reaching either cell, one weight per cell), so each voltage
// read serves both cells, and the lists are read through L1 instead of being staged in
// shared memory -- only the pass's voltages are, so boxes of any size fit.  Every cell
// pair of the box (row parts padded, no entries for those rows) is a task, so each
// pass writes every tile byte but the K padding (zero from the buffer's first use).
// Threads take consecutive cell pairs of a row: a warp's stores fill whole 128-byte
// rows of the swizzled tile.  With H the unpacked voltages are FP16 pairs, the F frames
// of an element side by side (exact for 4- and 8-bit samples), so one 16-byte load
// serves two frames.
constexpr int kGridPlThreads = 512;

struct GridPlArgs {
    GridArgs g;
    const int* pl_ptr;    // per channel: entry offsets of the box's cell pairs, row-major, + 1
    const int* pl_off;    // [C] start of channel c's offsets in pl_ptr
    const int* pl_e;      // entries: element
    const float2* pl_w;   // entries: weights at cells x and x + 1
    int max_ptr;          // S: most offsets of a channel (box pairs + 1)
    int max_ent;          // S: most entries of a channel
};

// Shared memory of k_dftgemm_grid_pl: raw frames, unpacked voltages and, with S, one
// channel's offsets (relative) and entries.
__host__ __device__ inline size_t grid_pl_smem(int F, int A, int frame_bytes, bool H, bool S = false, int max_ptr = 0,
                                              int max_ent = 0)
{
    const size_t ap = (size_t)((frame_bytes + 15) & ~15);
    size_t b = 2ull * F * ap + (H ? 8ull : 16ull) * F * A;
    if (S) b += 4ull * ((max_ptr + 1) & ~1) + 4ull * ((max_ent + 1) & ~1) + 8ull * max_ent;
    return b;
}

// S: the lists of the channel a pass grids are staged in shared memory (when they fit) instead
// of being read through L1.
template <int F, bool H, bool S>
__global__ void __launch_bounds__(kGridPlThreads) k_dftgemm_grid_pl(GridPlArgs pa)
{
    const GridArgs& a = pa.g;
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ uint64_t bar_raw[2];
    const int tid = threadIdx.x;
    const int A = a.A, P = a.P, AP = A * P * (a.bits / 4);  // bytes of one frame
    const int APr = (AP + 15) & ~15;
    uint8_t* raw = gsm;                                          // [2][F][APr]
    float4* sv = reinterpret_cast<float4*>(gsm + 2 * F * APr);   // [F][A] (FP32) or [A][F] (H)
    uint2* svh = reinterpret_cast<uint2*>(sv);
    int* sptr = reinterpret_cast<int*>(gsm + 2 * F * APr + (H ? 8 : 16) * F * A);  // S: offsets, then
    int* sent = sptr + ((pa.max_ptr + 1) & ~1);                                    // elements and
    float2* swt = reinterpret_cast<float2*>(sent + ((pa.max_ent + 1) & ~1));       // weights

    // (channel, frame) pairs [w0, w1) of this block
    const long long w0 = split_start(nullptr, a.c0, a.n_ch, 1, a.nt, blockIdx.x, gridDim.x);
    const long long w1 = split_start(nullptr, a.c0, a.n_ch, 1, a.nt, blockIdx.x + 1, gridDim.x);
    if (tid == 0) {
        tc::mbar_init(&bar_raw[0], 1);
        tc::mbar_init(&bar_raw[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < F * A; i += blockDim.x) {  // short passes read all F frames: start them at zero
        if (H) svh[i] = make_uint2(0u, 0u);  // 8 bytes per (element, frame): the buffer holds F A of them
        else sv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (w0 >= w1) return;

    auto pass_len = [&](long long w) {
        const int f = (int)(w % a.nt);
        return (int)min((long long)min(F, a.nt - f), w1 - w);
    };
    auto fetch = [&](long long w, int b) {  // thread 0: raw bytes of the pass starting at w -> buffer b
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        tc::mbar_expect_tx(&bar_raw[b], (uint32_t)(nf * AP));
        for (int i = 0; i < nf; ++i)
            tc::bulk_g2s(raw + (size_t)(b * F + i) * APr,
                         a.volt + ((size_t)(a.t0 + f + i) * a.C + a.c0 + cl) * (size_t)AP, (uint32_t)AP, &bar_raw[b]);
    };

    uint32_t ph = 0, pending = 0;
    int buf = 0, staged = -1;
    bool ok = true;
    if (a.bulk && tid == 0) {
        fetch(w0, 0);
        pending = 1u;
    }
    for (long long w = w0; w < w1;) {
        const int cl = (int)(w / a.nt), f = (int)(w % a.nt), nf = pass_len(w);
        const long long wn = w + nf;
        const int c = a.c0 + cl;
        const int4 b = a.box[c];
        const int nxp = b.z, nyp = b.w;
        const int4 tp = a.tbox[c];
        const int nyh = tp.x, N1h = P * nyh;
        const uint32_t part_bytes = (uint32_t)N1h * pad64(2 * nxp) * 2;
        if (S && cl != staged) {  // the channel's offsets (relative to its first entry) and entries
            const int* gp = pa.pl_ptr + pa.pl_off[c];
            const int np = nyp * (nxp >> 1) + 1, e0 = __ldg(gp), ne = __ldg(gp + np - 1) - e0;
            for (int i = tid; i < np; i += blockDim.x) sptr[i] = __ldg(gp + i) - e0;
            for (int i = tid; i < ne; i += blockDim.x) {
                sent[i] = __ldg(pa.pl_e + e0 + i);
                swt[i] = __ldg(pa.pl_w + e0 + i);
            }
            staged = cl;  // read by the task loop after the barrier below
        }
        const float4* jm = a.jones ? a.jones + (size_t)c * A * 2 : nullptr;  // polarisation mixing
        if (a.bulk && tid == 0 && wn < w1) {  // the other buffer was consumed by the previous pass
            fetch(wn, buf ^ 1);
            pending |= 1u << (buf ^ 1);
        }
        if (a.bulk) {
            const bool got = tc::mbar_wait(&bar_raw[buf], (ph >> buf) & 1u, kWaitBudget);
            if (got) {
                ph ^= 1u << buf;
                pending &= ~(1u << buf);
            }
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
        }
        for (int i = tid; i < nf * A; i += blockDim.x) {
            const int fi = i / A, e = i - fi * A;
            const uint8_t* fr = a.bulk ? raw + (size_t)(buf * F + fi) * APr
                                       : a.volt + ((size_t)(a.t0 + f + fi) * a.C + c) * (size_t)AP;
            const float4 q = load_quad(fr, e, P, a.bits, jm);
            if (H) svh[e * F + fi] = make_uint2(pack_h2(q.x, q.y), pack_h2(q.z, q.w));
            else sv[fi * A + e] = q;
        }
        __syncthreads();
        const int half = nxp >> 1;
        const int tasks = tp.z * half;
        const int* ptr_c = S ? sptr : pa.pl_ptr + pa.pl_off[c];
        const int* ent_e = S ? sent : pa.pl_e;
        const float2* ent_w = S ? swt : pa.pl_w;
        for (int task = tid; task < tasks; task += blockDim.x) {
            const int y = task / half, x = 2 * (task - y * half);
            float4 g[2][F];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int fi = 0; fi < F; ++fi) g[j][fi] = make_float4(0.f, 0.f, 0.f, 0.f);
            auto load = [&](int e, float4 (&v)[F]) {  // the pass's F frames of element e
                if constexpr (H) {
                    uint2 hv[F];
                    if constexpr (F == 1) {
                        hv[0] = svh[e];
                    } else {
                        const uint4* q = reinterpret_cast<const uint4*>(svh + e * F);
#pragma unroll
                        for (int jj = 0; jj < F / 2; ++jj) {
                            const uint4 u = q[jj];
                            hv[2 * jj] = make_uint2(u.x, u.y);
                            hv[2 * jj + 1] = make_uint2(u.z, u.w);
                        }
                    }
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) {
                        const float2 xx = __half22float2(*reinterpret_cast<const __half2*>(&hv[fi].x));
                        const float2 yy = __half22float2(*reinterpret_cast<const __half2*>(&hv[fi].y));
                        v[fi] = make_float4(xx.x, xx.y, yy.x, yy.y);
                    }
                } else {
#pragma unroll
                    for (int fi = 0; fi < F; ++fi) v[fi] = sv[fi * A + e];
                }
            };
            auto apply = [&](float2 wv, const float4 (&v)[F]) {  // packed FP32 FMAs, rounded as fmaf
                const float2 w0 = make_float2(wv.x, wv.x), w1 = make_float2(wv.y, wv.y);
#pragma unroll
                for (int fi = 0; fi < F; ++fi) {
                    const float2 vx = make_float2(v[fi].x, v[fi].y), vy = make_float2(v[fi].z, v[fi].w);
                    const float2 a0 = tc::fma2(w0, vx, make_float2(g[0][fi].x, g[0][fi].y));
                    const float2 b0 = tc::fma2(w0, vy, make_float2(g[0][fi].z, g[0][fi].w));
                    const float2 a1 = tc::fma2(w1, vx, make_float2(g[1][fi].x, g[1][fi].y));
                    const float2 b1 = tc::fma2(w1, vy, make_float2(g[1][fi].z, g[1][fi].w));
                    g[0][fi] = make_float4(a0.x, a0.y, b0.x, b0.y);
                    g[1][fi] = make_float4(a1.x, a1.y, b1.x, b1.y);
                }
            };
            const int k1 = y < nyp ? ptr_c[task + 1] : 0;
            int k = y < nyp ? ptr_c[task] : 0;
            for (; k + 1 < k1; k += 2) {  // two list entries in flight, applied in list order
                const int e0 = ent_e[k], e1 = ent_e[k + 1];
                const float2 w0 = ent_w[k], w1 = ent_w[k + 1];
                float4 v0[F], v1[F];
                load(e0, v0);
                load(e1, v1);
                apply(w0, v0);
                apply(w1, v1);
            }
            if (k < k1) {
                float4 v0[F];
                load(ent_e[k], v0);
                apply(ent_w[k], v0);
            }
            const int kc_re = x >> 3, kc_im = (nxp + x) >> 3, within = (x & 7) * 2;
            const int hpart = y / nyh, R0 = y - hpart * nyh;
#pragma unroll
            for (int fi = 0; fi < F; ++fi) {
                if (fi >= nf) break;
                uint8_t* tile =
                    a.tiles + ((size_t)(f + fi) * a.n_ch + cl) * a.tile_stride + (size_t)hpart * part_bytes;
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_re, N1h) + within) = pack_h2(g[0][fi].x, g[1][fi].x);
                *reinterpret_cast<uint32_t*>(tile + sw_chunk(R0, kc_im, N1h) + within) = pack_h2(g[0][fi].y, g[1][fi].y);
                if (P == 2) {
                    const int R1 = nyh + R0;
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_re, N1h) + within) =
                        pack_h2(g[0][fi].z, g[1][fi].z);
                    *reinterpret_cast<uint32_t*>(tile + sw_chunk(R1, kc_im, N1h) + within) =
                        pack_h2(g[0][fi].w, g[1][fi].w);
                }
            }
        }
        __syncthreads();  // the voltages are reused by the next pass
        w = wn;
        buf ^= 1;
    }
    if (!ok && tid == 0) {
        // leave no bulk copy in flight into this block's shared memory
        for (int b2 = 0; b2 < 2; ++b2)
            if ((pending >> b2) & 1u) tc::mbar_wait(&bar_raw[b2], (ph >> b2) & 1u, kWaitBudget);
        atomicExch(a.status, 1);
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ bool wait_flag_uniform(uint64_t* bar, uint32_t parity, const volatile int* err)
{
    const bool ok = tc::mbar_wait(bar, parity, kWaitBudget);
    return __syncthreads_and(ok && *err == 0) != 0;
}

// Epilogue 2: products of the stage-2 result in TMEM columns col0.. (pol X at
// col0, pol Y at col0 + 64; re at +0, im at +32) added to the accumulators.
__device__ __forceinline__ void epilogue2(uint32_t taddr, int P, float (&axx)[16], float (&ayy)[16], float (&arx)[16],
                                          float (&aix)[16])
{
    uint32_t xr[16], xi[16];
    tc::tmem_ld16(taddr, xr);
    tc::tmem_ld16(taddr + 32, xi);
    if (P == 2) {
        uint32_t yr[16], yi[16];
        tc::tmem_ld16(taddr + 64, yr);
        tc::tmem_ld16(taddr + 96, yi);
        tc::tmem_wait_ld(xr);
        tc::tmem_wait_ld(xi);
        tc::tmem_wait_ld(yr);
        tc::tmem_wait_ld(yi);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float Xr = __uint_as_float(xr[i]), Xi = __uint_as_float(xi[i]);
            const float Yr = __uint_as_float(yr[i]), Yi = __uint_as_float(yi[i]);
            axx[i] = fmaf(Xr, Xr, fmaf(Xi, Xi, axx[i]));
            ayy[i] = fmaf(Yr, Yr, fmaf(Yi, Yi, ayy[i]));
            arx[i] = fmaf(Xr, Yr, fmaf(Xi, Yi, arx[i]));
            aix[i] = fmaf(Xi, Yr, fmaf(-Xr, Yi, aix[i]));
        }
    } else {
        tc::tmem_wait_ld(xr);
        tc::tmem_wait_ld(xi);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float Xr = __uint_as_float(xr[i]), Xi = __uint_as_float(xi[i]);
            axx[i] = fmaf(Xr, Xr, fmaf(Xi, Xi, axx[i]));
        }
    }
}

// Epilogue 1 of one pol: the stage-1 result of this warp's lane quarter (lanes =
// the slab's 32 kx; quarter 0 holds Hr, quarter 1 Hi) for the pol's nyp columns,
// converted to FP16 and written as the stage-2 operand B2_p:
//   row kx      = [ Hr[0..nyp) | -Hi[0..nyp) ],  row 32+kx = [ Hi | Hr ].
// TMEM loads are issued 32 columns at a time before one wait.
__device__ __forceinline__ void epilogue1(uint32_t taddr, int nyp, bool imw, int lane, uint8_t* b2, int p, int R2)
{
    const int n0 = 64 * p + lane, n1 = 64 * p + 32 + lane;
    for (int y0 = 0; y0 < nyp; y0 += 32) {
        const int ng = min(4, (nyp - y0) >> 3);  // groups of 8 columns in this batch
        uint32_t r[32];
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (g < ng) tmem_ld8(taddr + y0 + 8 * g, r + 8 * g);
        tc::tmem_wait_ld(r);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            if (g >= ng) break;
            uint4 pos, neg;
            pos.x = pack_h2(__uint_as_float(r[8 * g + 0]), __uint_as_float(r[8 * g + 1]));
            pos.y = pack_h2(__uint_as_float(r[8 * g + 2]), __uint_as_float(r[8 * g + 3]));
            pos.z = pack_h2(__uint_as_float(r[8 * g + 4]), __uint_as_float(r[8 * g + 5]));
            pos.w = pack_h2(__uint_as_float(r[8 * g + 6]), __uint_as_float(r[8 * g + 7]));
            neg.x = pos.x ^ 0x80008000u;  // FP16 negation = sign-bit flip
            neg.y = pos.y ^ 0x80008000u;
            neg.z = pos.z ^ 0x80008000u;
            neg.w = pos.w ^ 0x80008000u;
            const int kc_lo = (y0 >> 3) + g, kc_hi = (nyp >> 3) + kc_lo;
            if (!imw) {  // Hr: B2[kx][y] and B2[32+kx][nyp+y]
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_lo, R2)) = pos;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_hi, R2)) = pos;
            } else {     // Hi: B2[kx][nyp+y] = -Hi, B2[32+kx][y] = Hi
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_hi, R2)) = neg;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_lo, R2)) = pos;
            }
        }
    }
}

// MMA chains over KS K steps accumulating into one TMEM tile.  Descriptors are
// derived from a base by adding, in 16-byte units, (k / 4) * panel + (k % 4) * 2
// (a 64-wide K panel of the swizzled layout, then 32 bytes per K step inside it);
// the loops are unrolled at compile time so that issuing costs no more than the
// tensor core's own time per MMA.
template <int KS>
__device__ __forceinline__ void chain_ss(uint32_t d, uint64_t da, uint64_t db, uint32_t pa16, uint32_t pb16,
                                         uint32_t id)
{
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16(d, da + (uint64_t)((k >> 2) * pa16 + (k & 3) * 2), db + (uint64_t)((k >> 2) * pb16 + (k & 3) * 2),
                    id, k > 0);
}

template <int KS>
__device__ __forceinline__ void chain_ts(uint32_t d, uint32_t at, uint64_t db, uint32_t pb16, uint32_t id, bool acc)
{
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16_ta(d, at + 8 * k, db + (uint64_t)((k >> 2) * pb16 + (k & 3) * 2), id, acc || k > 0);
}

#define EPIC_KS_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// A and B in shared memory (both 128-byte swizzled, K-major)
__device__ __forceinline__ void issue_ss(int ks, uint32_t d, uint32_t sa, uint32_t sb, uint32_t a_panel_bytes,
                                         uint32_t b_panel_bytes, uint32_t id)
{
    const uint64_t da = tc::smem_desc_sw128(sa), db = tc::smem_desc_sw128(sb);
    const uint32_t pa = a_panel_bytes >> 4, pb = b_panel_bytes >> 4;
    switch (ks) {
#define EPIC_SS(n) \
    case n: chain_ss<n>(d, da, db, pa, pb, id); break;
        EPIC_KS_CASES(EPIC_SS)
#undef EPIC_SS
        default:
            for (int k = 0; k < ks; ++k)
                tc::mma_f16(d, da + (uint64_t)((k >> 2) * pa + (k & 3) * 2), db + (uint64_t)((k >> 2) * pb + (k & 3) * 2),
                            id, k > 0);
    }
}

// A in TMEM (K halves packed in pairs: 8 columns per K step), B in shared memory; with
// acc the chain adds to what D holds (a later row part of the same stage-2 sum)
__device__ __forceinline__ void issue_ts(int ks, uint32_t d, uint32_t at, uint32_t sb, uint32_t b_panel_bytes,
                                         uint32_t id, bool acc = false)
{
    const uint64_t db = tc::smem_desc_sw128(sb);
    const uint32_t pb = b_panel_bytes >> 4;
    switch (ks) {
#define EPIC_TS(n) \
    case n: chain_ts<n>(d, at, db, pb, id, acc); break;
        EPIC_KS_CASES(EPIC_TS)
#undef EPIC_TS
        default:
            for (int k = 0; k < ks; ++k)
                tc::mma_f16_ta(d, at + 8 * k, db + (uint64_t)((k >> 2) * pb + (k & 3) * 2), id, acc || k > 0);
    }
}

// Stage 1 + stage 2 + products + accumulation for the work items of one chunk.
// Warps 0-7 do the epilogues; lane 0 of warp 3 (which has no epilogue-1 work)
// also drives the TMA engine and the tensor core.  The frame loop is
// software-pipelined:
//   all wait until S2(t-1) and S1(t) are complete
//   control: refill the tile buffer S1(t) released with tile t+NB
//   warps 0,1 (pol X) and 4,5 (pol Y): epilogue 1 (t): D1 -> FP16 B2     | barrier
//   control: issue S2(t) into D2[t&1], then S1(t+1) into D1, commit
//   warps 0-7: epilogue 2 (t-1) from D2[(t-1)&1] while the tensor core runs
// TMEM: D1 in columns [0, 256), D2[b] in [256 + 128 b, 384 + 128 b).
// A1 rows 0..31 = re, 32..63 = im of the item's own 32 kx (rows 64..127 zero),
// so epilogue 1 reads lane quarters 0 (Hr) and 1 (Hi).
constexpr int kMmaThreads = 256;

template <int NB>
__global__ void __launch_bounds__(kMmaThreads, 1) k_dftgemm_mma(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_mma, bar_a, bar_tile[2];
    __shared__ uint32_t tmem_sh;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctl = tid == 3 * 32;  // the control thread (warp 3, lane 0)
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (ctl) {
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_init(&bar_a, 1);
        tc::mbar_init(&bar_tile[0], 1);
        tc::mbar_init(&bar_tile[1], 1);
        err_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    // swizzled operands need 1024-byte aligned bases (the swizzle uses address bits 4-9)
    uint8_t* sbase = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    uint8_t* sA1 = sbase + a.sA1;
    uint8_t* sA2 = sbase + a.sA2;
    uint8_t* sB2 = sbase + a.sB2;
    uint32_t ph_mma = 0, ph_a = 0;
    uint32_t ph_tile = 0;  // bit b = parity of tile buffer b (control thread only)
    bool ok = true;
    const int items = a.n_ch * a.n_kb * a.n_s;
    const int q4 = warp & 3, hc = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    const bool epi1 = q4 < 2 && (warp >> 2) < a.P;  // warps 0, 1 (pol 0) and 4, 5 (pol 1)

    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int s = item % a.n_s, kb = (item / a.n_s) % a.n_kb, cl = item / (a.n_s * a.n_kb);
        const int c = a.c0 + cl;
        const int4 bx = a.box[c];
        const int nxp = bx.z, nyp = bx.w;
        const int K1 = 2 * nxp, K2 = 2 * nyp, N1 = a.P * nyp;
        const int K1s = pad64(K1), K2s = pad64(K2);
        const uint32_t a1_bytes = 256u * K1s, a2_bytes = 256u * K2s;
        const uint32_t tile_bytes = (uint32_t)N1 * K1s * 2;
        const uint8_t* tiles_c = a.tiles + (size_t)cl * a.tile_stride;
        const size_t frame_step = (size_t)a.n_ch * a.tile_stride;
        const uint32_t id1 = tc::idesc_f16_f32(128, N1), id2 = tc::idesc_f16_f32(128, 64 * a.P);
        const int nt = a.nt;

        auto issue_s1 = [&](int b) {
            issue_ss(K1 / 16, tmem, tc::smem_u32(sA1), tc::smem_u32(sbase + a.sB1 + (size_t)b * a.b1_bytes), 128 * 128,
                     N1 * 128, id1);
        };
        auto issue_s2 = [&](int d) {  // both pols in one MMA: B2 rows 0..63 pol X, 64..127 pol Y
            issue_ss(K2 / 16, tmem + 256 + 128 * d, tc::smem_u32(sA2), tc::smem_u32(sB2), 128 * 128, 64 * a.P * 128,
                     id2);
        };
        auto load_tile = [&](int t, int b) {
            tc::mbar_expect_tx(&bar_tile[b], tile_bytes);
            tc::bulk_g2s(sbase + a.sB1 + (size_t)b * a.b1_bytes, tiles_c + (size_t)t * frame_step, tile_bytes,
                         &bar_tile[b]);
        };
        auto wait_tile = [&](int b) -> bool {
            const bool r = tc::mbar_wait(&bar_tile[b], (ph_tile >> b) & 1u, kWaitBudget);
            ph_tile ^= 1u << b;
            if (!r) err_sh = 1;
            return r;
        };

        if (ctl) {
            tc::mbar_expect_tx(&bar_a, a1_bytes + a2_bytes);
            tc::bulk_g2s(sA1, a.a1 + a.a1_off[(size_t)c * a.n_s + s], a1_bytes, &bar_a);
            tc::bulk_g2s(sA2, a.a2 + a.a2_off[(size_t)c * a.n_kb + kb], a2_bytes, &bar_a);
            for (int j = 0; j < NB && j < nt; ++j) load_tile(j, j);
        }
        ok = wait_flag_uniform(&bar_a, ph_a, &err_sh);
        ph_a ^= 1;
        if (!ok) break;
        if (ctl) {
            if (wait_tile(0)) {
                tc::fence_after_sync();
                issue_s1(0);
            }
            tc::mma_commit(&bar_mma);
        }

        float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;

        for (int t = 0; ok && t < nt; ++t) {
            ok = wait_flag_uniform(&bar_mma, ph_mma, &err_sh);  // S2(t-1) and S1(t) complete
            ph_mma ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
            if (ctl && t + NB < nt) load_tile(t + NB, t % NB);  // S1(t) has released that buffer
            if (epi1) {
                const int p = warp >> 2;
                epilogue1(tmem + ((uint32_t)(32 * q4) << 16) + p * nyp, nyp, q4 == 1, lane, sB2, p, 64 * a.P);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (ctl) {
                issue_s2(t & 1);
                if (t + 1 < nt && wait_tile((t + 1) % NB)) {
                    tc::fence_after_sync();
                    issue_s1((t + 1) % NB);
                }
                tc::mma_commit(&bar_mma);
            }
            __syncwarp();
            if (t >= 1)
                epilogue2(tmem + lane_base + 256 + 128 * ((t - 1) & 1) + 16 * hc, a.P, axx, ayy, arx, aix);
            tc::fence_before_sync();
        }
        if (ok && nt > 0) {
            ok = wait_flag_uniform(&bar_mma, ph_mma, &err_sh);  // S2(nt-1)
            ph_mma ^= 1;
            if (ok) {
                tc::fence_after_sync();
                epilogue2(tmem + lane_base + 256 + 128 * ((nt - 1) & 1) + 16 * hc, a.P, axx, ayy, arx, aix);
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
        if (!ok) break;
        // ---- images: written (first chunk, reset) or added
        const int ky = 128 * kb + 32 * q4 + lane;
        const int kx0 = 32 * s + 16 * hc;
        if (ky < a.N && kx0 < a.N) {
            const size_t NN = (size_t)a.N * a.N;
            float* o = a.out + (size_t)c * a.nprod * NN + (size_t)ky * a.N + kx0;
            const int nk = min(16, a.N - kx0);
            store_pixels16(o, nk, a.accumulate, axx);
            if (a.nprod == 4) {
                store_pixels16(o + NN, nk, a.accumulate, ayy);
                store_pixels16(o + 2 * NN, nk, a.accumulate, arx);
                store_pixels16(o + 3 * NN, nk, a.accumulate, aix);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if ((!ok || err_sh) && tid == 0) atomicExch(a.status, 1);
}

// Fast variant for occupied boxes small enough that two stage-1 results, the
// stage-2 DFT operand and two stage-2 results all fit in TMEM (2 N1 + K2/2 <= 256
// columns) and three grid tiles plus two B2 buffers fit in shared memory.
//   TMEM: D1[b] at b*d1_cols, A2 (FP16 pairs) at 2*d1_cols, D2[b] at 256 + 128 b.
//   The stage-2 A operand (the constant ky DFT rows) is read from TMEM, so stage 2
//   streams only B2 from shared memory.
// Schedule (tensor order S1(0) S1(1) S2(0) S1(2) S2(1) S1(3) ...):
//   iteration t: wait S1(t) -> control refills tile t+3 -> epilogue 1 (t): D1[t&1] ->
//   B2[t&1] | barrier | control issues S2(t) -> D2[t&1] (commit s2[t&1]) and
//   S1(t+2) -> D1[t&1] (commit s1[t&1]) | epilogue 2 (t-1) after S2(t-1).
// While the warps convert frame t the tensor core runs S1(t+1) and S2(t-1).
template <int dummy>
__global__ void __launch_bounds__(kMmaThreads, 1) k_dftgemm_mma_fast(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_a, bar_s1[2], bar_s2[2], bar_tile[3];
    __shared__ uint32_t tmem_sh;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctl = tid == 3 * 32;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (ctl) {
        tc::mbar_init(&bar_a, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&bar_s1[i], 1);
            tc::mbar_init(&bar_s2[i], 1);
        }
        for (int i = 0; i < 3; ++i) tc::mbar_init(&bar_tile[i], 1);
        err_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    uint8_t* sbase = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    uint8_t* sA1 = sbase + a.sA1;
    uint32_t ph_a = 0, ph_s1 = 0, ph_s2 = 0;  // bit b: parity of slot b
    uint32_t ph_tile = 0;                     // control thread: bit b parity of tile buffer b
    bool ok = true;
    const int items = a.n_ch * a.n_kb * a.n_s;
    const int q4 = warp & 3, hc = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    const bool epi1 = q4 < 2 && (warp >> 2) < a.P;
    const uint32_t a2col = 2u * a.d1_cols;

    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int s = item % a.n_s, kb = (item / a.n_s) % a.n_kb, cl = item / (a.n_s * a.n_kb);
        const int c = a.c0 + cl;
        const int4 bx = a.box[c];
        const int nxp = bx.z, nyp = bx.w;
        const int K1 = 2 * nxp, K2 = 2 * nyp, N1 = a.P * nyp;
        const int K1s = pad64(K1);
        const uint32_t a1_bytes = 256u * K1s;
        const uint32_t tile_bytes = (uint32_t)N1 * K1s * 2;
        const uint8_t* tiles_c = a.tiles + (size_t)cl * a.tile_stride;
        const size_t frame_step = (size_t)a.n_ch * a.tile_stride;
        const uint32_t id1 = tc::idesc_f16_f32(128, N1), id2 = tc::idesc_f16_f32(128, 64 * a.P);
        const int nt = a.nt;
        const int R2 = 64 * a.P;

        auto issue_s1 = [&](int b, int slot) {
            issue_ss(K1 / 16, tmem + slot * a.d1_cols, tc::smem_u32(sA1),
                     tc::smem_u32(sbase + a.sB1 + (size_t)b * a.b1_bytes), 128 * 128, N1 * 128, id1);
        };
        auto issue_s2 = [&](int slot) {
            issue_ts(K2 / 16, tmem + 256 + 128 * slot, tmem + a2col,
                     tc::smem_u32(sbase + a.sB2 + (size_t)slot * a.b2_bytes), R2 * 128, id2);
        };
        auto load_tile = [&](int t) {
            const int b = t % 3;
            tc::mbar_expect_tx(&bar_tile[b], tile_bytes);
            tc::bulk_g2s(sbase + a.sB1 + (size_t)b * a.b1_bytes, tiles_c + (size_t)t * frame_step, tile_bytes,
                         &bar_tile[b]);
        };
        auto wait_tile = [&](int t) -> bool {
            const int b = t % 3;
            const bool r = tc::mbar_wait(&bar_tile[b], (ph_tile >> b) & 1u, kWaitBudget);
            ph_tile ^= 1u << b;
            if (!r) err_sh = 1;
            return r;
        };
        auto wait_slot = [&](uint64_t* bars, uint32_t& ph, int slot) -> bool {
            const bool r = tc::mbar_wait(&bars[slot], (ph >> slot) & 1u, kWaitBudget);
            ph ^= 1u << slot;
            if (!r) err_sh = 1;
            return r;
        };

        if (ctl) {
            tc::mbar_expect_tx(&bar_a, a1_bytes);
            tc::bulk_g2s(sA1, a.a1 + a.a1_off[(size_t)c * a.n_s + s], a1_bytes, &bar_a);
            for (int j = 0; j < 3 && j < nt; ++j) load_tile(j);
        }
        __syncwarp();
        // stage-2 DFT operand -> TMEM (warps 0-3: lane = ky row)
        if (warp < 4) {
            const uint32_t* src = a.a2w + a.a2w_off[(size_t)c * a.n_kb + kb] + (size_t)(32 * warp + lane) * (K2 / 2);
            for (int j = 0; j < K2 / 2; j += 8) {
                uint32_t r[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = src[j + i];
                tc::tmem_st8(tmem + lane_base + a2col + j, r);
            }
            tc::tmem_wait_st();
        }
        tc::fence_before_sync();
        ok = wait_flag_uniform(&bar_a, (ph_a & 1u), &err_sh);
        ph_a ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
        if (ctl) {
            for (int j = 0; j < 2 && j < nt; ++j) {
                if (wait_tile(j)) {
                    tc::fence_after_sync();
                    issue_s1(j % 3, j);
                }
                tc::mma_commit(&bar_s1[j]);
            }
        }

        float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;

        for (int t = 0; ok && t < nt; ++t) {
            const int sl = t & 1;
            bool w = wait_slot(bar_s1, ph_s1, sl);           // S1(t) (and S2(t-2)) complete
            ok = __syncthreads_and(w && err_sh == 0) != 0;
            if (!ok) break;
            tc::fence_after_sync();
            if (ctl && t + 3 < nt) load_tile(t + 3);          // S1(t) released tile buffer t % 3
            if (epi1) {
                const int p = warp >> 2;
                epilogue1(tmem + ((uint32_t)(32 * q4) << 16) + sl * a.d1_cols + p * nyp, nyp, q4 == 1, lane,
                          sbase + a.sB2 + (size_t)sl * a.b2_bytes, p, R2);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (ctl) {
                issue_s2(sl);
                tc::mma_commit(&bar_s2[sl]);
                if (t + 2 < nt) {
                    if (wait_tile(t + 2)) {
                        tc::fence_after_sync();
                        issue_s1((t + 2) % 3, sl);
                    }
                    tc::mma_commit(&bar_s1[sl]);
                }
            }
            __syncwarp();
            if (t >= 1) {
                const bool w2 = wait_slot(bar_s2, ph_s2, (t - 1) & 1);
                __syncwarp();
                if (w2) {
                    tc::fence_after_sync();
                    epilogue2(tmem + lane_base + 256 + 128 * ((t - 1) & 1) + 16 * hc, a.P, axx, ayy, arx, aix);
                }
            }
            tc::fence_before_sync();
        }
        if (ok && nt > 0) {
            const bool w = wait_slot(bar_s2, ph_s2, (nt - 1) & 1);
            __syncwarp();
            if (w) {
                tc::fence_after_sync();
                epilogue2(tmem + lane_base + 256 + 128 * ((nt - 1) & 1) + 16 * hc, a.P, axx, ayy, arx, aix);
            }
            tc::fence_before_sync();
            ok = __syncthreads_and(w && err_sh == 0) != 0;
            tc::fence_after_sync();
        }
        if (!ok) break;
        const int ky = 128 * kb + 32 * q4 + lane;
        const int kx0 = 32 * s + 16 * hc;
        if (ky < a.N && kx0 < a.N) {
            const size_t NN = (size_t)a.N * a.N;
            float* o = a.out + (size_t)c * a.nprod * NN + (size_t)ky * a.N + kx0;
            const int nk = min(16, a.N - kx0);
            store_pixels16(o, nk, a.accumulate, axx);
            if (a.nprod == 4) {
                store_pixels16(o + NN, nk, a.accumulate, ayy);
                store_pixels16(o + 2 * NN, nk, a.accumulate, arx);
                store_pixels16(o + 3 * NN, nk, a.accumulate, aix);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if ((!ok || err_sh) && tid == 0) atomicExch(a.status, 1);
}

// ---------------------------------------------------------------------------------
// Warp-specialised variant: a work item is (channel, 128-row ky block, 64-column kx
// pair), so stage 1 uses all 128 rows (re and im of 64 kx) and stage 2 runs as two
// N = 64 P halves (kx 0..31 and 32..63 of the pair).  16 warps do the epilogues;
// three lanes issue the tensor core work and the tile copies; all hand-offs go
// through mbarriers, never a block-wide barrier inside the frame loop:
//   d1_full[s]  commit after S1 into D1[s]          (waited by every warp)
//   b2_full[s]  16 warp arrivals after epilogue 1   (waited by the three issuers)
//   d2_full[h]  commit after S2 of half h           (waited by every warp)
//   d2_empty[h] 8 warp arrivals after epilogue 2 h  (waited by the issuer of h)
//   tile[b]     TMA completion of grid tile buffer b
// Per frame t every warp: wait S1(t) -> (issuer B: copy tile t+2) -> epilogue 1 (t)
// into B2[t&1] -> arrive b2_full -> wait S2(t-1) -> epilogue 2 (t-1) -> arrive
// d2_empty; issuers then queue S2a(t), S2b(t) (after b2_full(t) and d2_empty(t-1))
// and S1(t+2) (after b2_full(t) frees D1[t&1] and tile t+2 has landed).
// TMEM: D1[0..1] at 0 and d1_cols, A2 at 2 d1_cols, D2 half h at 256 + 128 h.
constexpr int kWsThreads = 512;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Epilogue 1 of one warp: the stage-1 result in this warp's lane quarter (lanes =
// 32 kx of half h; part 0 = Hr, part 1 = Hi), columns [c0, c1) of pol p, written to
// the B2 rows of half h / pol p (row kx = [Hr | -Hi], row 32+kx = [Hi | Hr]).
__device__ __forceinline__ void ws_epilogue1(uint32_t taddr, int nyp, int yc0, int yc1, bool imw, int lane,
                                             uint8_t* b2, int row0, int R2)
{
    const int n0 = row0 + lane, n1 = row0 + 32 + lane;
    for (int yb = yc0; yb < yc1; yb += 2) {
        const int ng = min(2, yc1 - yb);
        uint32_t r[16];
#pragma unroll
        for (int g = 0; g < 2; ++g)
            if (g < ng) tmem_ld8(taddr + 8 * (yb + g), r + 8 * g);
        tc::tmem_wait_ld(r);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (g >= ng) break;
            uint4 pos, neg;
            pos.x = pack_h2(__uint_as_float(r[8 * g + 0]), __uint_as_float(r[8 * g + 1]));
            pos.y = pack_h2(__uint_as_float(r[8 * g + 2]), __uint_as_float(r[8 * g + 3]));
            pos.z = pack_h2(__uint_as_float(r[8 * g + 4]), __uint_as_float(r[8 * g + 5]));
            pos.w = pack_h2(__uint_as_float(r[8 * g + 6]), __uint_as_float(r[8 * g + 7]));
            neg.x = pos.x ^ 0x80008000u;
            neg.y = pos.y ^ 0x80008000u;
            neg.z = pos.z ^ 0x80008000u;
            neg.w = pos.w ^ 0x80008000u;
            const int kc_lo = yb + g, kc_hi = (nyp >> 3) + kc_lo;
            if (!imw) {
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_lo, R2)) = pos;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_hi, R2)) = pos;
            } else {
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_hi, R2)) = neg;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_lo, R2)) = pos;
            }
        }
    }
}

// Epilogue 2 of one warp: 16 kx x (X, Y) of its 32 ky rows, 4 kx per TMEM batch.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// c0 += a0 b0, c1 += a1 b1 as one paired FP32 fused multiply-add (fma.rn.f32x2, sm_100
// family): each lane rounds exactly as fmaf does, in half the issue slots.
__device__ __forceinline__ void fma2x2(float& c0, float& c1, float a0, float a1, float b0, float b1)
{
    const float2 r = tc::fma2(make_float2(a0, a1), make_float2(b0, b1), make_float2(c0, c1));
    c0 = r.x;
    c1 = r.y;
}

// Products of W pixels (TMEM loads of X re / im and Y re / im, W even) added to the
// accumulators o .. o+W-1, two pixels per paired FMA; same roundings as fmaf.
template <int W, int NA>
__device__ __forceinline__ void products(const uint32_t* xr, const uint32_t* xi, const uint32_t* yr,
                                         const uint32_t* yi, int P, int o, float (&axx)[NA], float (&ayy)[NA],
                                         float (&arx)[NA], float (&aix)[NA])
{
#pragma unroll
    for (int i = 0; i < W; i += 2) {
        const float Xr0 = __uint_as_float(xr[i]), Xi0 = __uint_as_float(xi[i]);
        const float Xr1 = __uint_as_float(xr[i + 1]), Xi1 = __uint_as_float(xi[i + 1]);
        fma2x2(axx[o + i], axx[o + i + 1], Xi0, Xi1, Xi0, Xi1);
        fma2x2(axx[o + i], axx[o + i + 1], Xr0, Xr1, Xr0, Xr1);
        if (P == 2) {
            const float Yr0 = __uint_as_float(yr[i]), Yi0 = __uint_as_float(yi[i]);
            const float Yr1 = __uint_as_float(yr[i + 1]), Yi1 = __uint_as_float(yi[i + 1]);
            fma2x2(ayy[o + i], ayy[o + i + 1], Yi0, Yi1, Yi0, Yi1);
            fma2x2(ayy[o + i], ayy[o + i + 1], Yr0, Yr1, Yr0, Yr1);
            fma2x2(arx[o + i], arx[o + i + 1], Xi0, Xi1, Yi0, Yi1);
            fma2x2(arx[o + i], arx[o + i + 1], Xr0, Xr1, Yr0, Yr1);
            fma2x2(aix[o + i], aix[o + i + 1], -Xr0, -Xr1, Yi0, Yi1);
            fma2x2(aix[o + i], aix[o + i + 1], Xi0, Xi1, Yr0, Yr1);
        }
    }
}

__device__ __forceinline__ void ws_epilogue2(uint32_t taddr, int P, float (&axx)[16], float (&ayy)[16],
                                             float (&arx)[16], float (&aix)[16])
{
#pragma unroll
    for (int hb = 0; hb < 4; ++hb) {
        uint32_t xr[4], xi[4], yr[4], yi[4];
        tmem_ld4(taddr + 4 * hb, xr);
        tmem_ld4(taddr + 32 + 4 * hb, xi);
        if (P == 2) {
            tmem_ld4(taddr + 64 + 4 * hb, yr);
            tmem_ld4(taddr + 96 + 4 * hb, yi);
        }
        tc::tmem_wait_ld(xr);
        tc::tmem_wait_ld(xi);
        if (P == 2) {
            tc::tmem_wait_ld(yr);
            tc::tmem_wait_ld(yi);
        }
        products<4>(xr, xi, yr, yi, P, 4 * hb, axx, ayy, arx, aix);
    }
}

template <int dummy>
__global__ void __launch_bounds__(kWsThreads, 1) k_dftgemm_ws(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_a, d1_full[2], b2_full[2], d2_full[2], d2_empty[2], tile_full[2];
    __shared__ uint32_t tmem_sh;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool isB = tid == 5 * 32;    // stage 1 + tile copies (sub-partition 1)
    const bool isA = tid == 2 * 32;    // stage 2, kx half 0 (sub-partition 2)
    const bool isC = tid == 15 * 32;   // stage 2, kx half 1 (sub-partition 3)
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_a, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&d1_full[i], 1);
            tc::mbar_init(&b2_full[i], 16);
            tc::mbar_init(&d2_full[i], 1);
            tc::mbar_init(&d2_empty[i], 8);
            tc::mbar_init(&tile_full[i], 1);
        }
        err_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    uint8_t* sbase = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    uint8_t* sA1 = sbase + a.sA1;
    // parities (bit s per slot); every thread waits each phase it tracks exactly once
    uint32_t ph_d1 = 0, ph_d2 = 0, ph_b2 = 0, ph_e2 = 0, ph_tile = 0, ph_a = 0;
    bool ok = true;
    const int P = a.P;
    const int q4 = warp & 3, j4 = warp >> 2;       // lane quarter, column group
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    const int R2 = 2 * 64 * P;                      // B2 rows: half h at 64 P h, pol p at 64 p
    const uint32_t a2col = 2u * a.d1_cols;
    const int items = a.n_ch * a.n_kb * a.n_g;
    // epilogue-2 part of this warp: quarter q4 (ky), kx group j4 -> half h2, 16 kx at 16 (j4 & 1)
    const int h2 = j4 >> 1;

    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int g = item % a.n_g, kb = (item / a.n_g) % a.n_kb, cl = item / (a.n_g * a.n_kb);
        const int c = a.c0 + cl;
        const int4 bx = a.box[c];
        const int nxp = bx.z, nyp = bx.w;
        const int K1 = 2 * nxp, K2 = 2 * nyp, N1 = P * nyp;
        const int K1s = pad64(K1);
        const uint32_t a1_bytes = 256u * K1s;
        const uint32_t tile_bytes = (uint32_t)N1 * K1s * 2;
        const uint8_t* tiles_c = a.tiles + (size_t)cl * a.tile_stride;
        const size_t frame_step = (size_t)a.n_ch * a.tile_stride;
        const uint32_t id1 = tc::idesc_f16_f32(128, N1), id2 = tc::idesc_f16_f32(128, 64 * P);
        const int nt = a.nt;

        auto wait_bit = [&](uint64_t* bar, uint32_t& ph, int slot) -> bool {
            const bool r = tc::mbar_wait(bar, (ph >> slot) & 1u, kWaitBudget);
            ph ^= 1u << slot;
            if (!r) err_sh = 1;
            return r;
        };
        auto load_tile = [&](int t) {
            const int b = t & 1;
            tc::mbar_expect_tx(&tile_full[b], tile_bytes);
            tc::bulk_g2s(sbase + a.sB1 + (size_t)b * a.b1_bytes, tiles_c + (size_t)t * frame_step, tile_bytes,
                         &tile_full[b]);
        };
        auto issue_s1 = [&](int t) {  // issuer B: tile t (buffer t&1) -> D1[t&1]
            issue_ss(K1 / 16, tmem + (t & 1) * a.d1_cols, tc::smem_u32(sA1),
                     tc::smem_u32(sbase + a.sB1 + (size_t)(t & 1) * a.b1_bytes), 128 * 128, N1 * 128, id1);
            tc::mma_commit(&d1_full[t & 1]);
        };
        auto issue_s2 = [&](int t, int h) {  // issuers A / C: B2[t&1] half h -> D2 half h
            const uint32_t b2 = tc::smem_u32(sbase + a.sB2 + (size_t)(t & 1) * a.b2_bytes) + (uint32_t)(64 * P * h) * 128;
            issue_ts(K2 / 16, tmem + 256 + 128 * h, tmem + a2col, b2, R2 * 128, id2);
            tc::mma_commit(&d2_full[h]);
        };

        // ---- item prologue
        if (isB) {
            tc::mbar_expect_tx(&bar_a, a1_bytes);
            tc::bulk_g2s(sA1, a.a1p + a.a1p_off[(size_t)c * a.n_g + g], a1_bytes, &bar_a);
            for (int j = 0; j < 2 && j < nt; ++j) load_tile(j);
        }
        __syncwarp();
        if (warp < 4) {  // stage-2 DFT operand -> TMEM (lane = ky row)
            const uint32_t* src = a.a2w + a.a2w_off[(size_t)c * a.n_kb + kb] + (size_t)(32 * warp + lane) * (K2 / 2);
            for (int jj = 0; jj < K2 / 2; jj += 8) {
                uint32_t r[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = src[jj + i];
                tc::tmem_st8(tmem + lane_base + a2col + jj, r);
            }
            tc::tmem_wait_st();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (isB) {
            if (wait_bit(&bar_a, ph_a, 0)) {
                for (int j = 0; j < 2 && j < nt; ++j)
                    if (wait_bit(&tile_full[j], ph_tile, j)) {
                        tc::fence_after_sync();
                        issue_s1(j);
                    }
            }
        }
        __syncwarp();

        float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;

        for (int t = 0; t < nt; ++t) {
            const int sl = t & 1;
            // (1) S1(t) complete
            bool w = wait_bit(&d1_full[sl], ph_d1, sl);
            __syncwarp();
            tc::fence_after_sync();
            // (2) issuer B: the tile buffer of S1(t) is free -> copy tile t+2
            if (isB && t + 2 < nt) load_tile(t + 2);
            __syncwarp();
            // (3) epilogue 1 (t): quarter q4 (half q4&1, part q4>>1); columns of pol / y-range by j4
            if (w) {
                const int hh = q4 & 1;
                const bool imw = (q4 >> 1) != 0;
                const int nyc = nyp >> 3;
                int p, yc0, yc1;
                if (P == 2) {
                    p = j4 >> 1;
                    const int mid = (nyc + 1) >> 1;
                    yc0 = (j4 & 1) ? mid : 0;
                    yc1 = (j4 & 1) ? nyc : mid;
                } else {
                    p = 0;
                    yc0 = (nyc * j4) >> 2;
                    yc1 = (nyc * (j4 + 1)) >> 2;
                }
                ws_epilogue1(tmem + lane_base + sl * a.d1_cols + p * nyp, nyp, yc0, yc1, imw, lane,
                             sbase + a.sB2 + (size_t)sl * a.b2_bytes, 64 * P * hh + 64 * p, R2);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&b2_full[sl]);
            // (4) epilogue 2 (t-1) after S2(t-1) of both halves
            if (t >= 1) {
                const bool wa = wait_bit(&d2_full[0], ph_d2, 0);
                const bool wb = wait_bit(&d2_full[1], ph_d2, 1);
                __syncwarp();
                tc::fence_after_sync();
                if (wa && wb)
                    ws_epilogue2(tmem + lane_base + 256 + 128 * h2 + 16 * (j4 & 1), P, axx, ayy, arx, aix);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&d2_empty[h2]);
            }
            // (5) issuers
            if (isA || isC) {
                const int h = isA ? 0 : 1;
                bool r = wait_bit(&b2_full[sl], ph_b2, sl);
                if (t >= 1) r = wait_bit(&d2_empty[h], ph_e2, h) && r;
                if (r) {
                    tc::fence_after_sync();
                    issue_s2(t, h);
                } else {
                    tc::mma_commit(&d2_full[h]);
                }
            }
            if (isB && t + 2 < nt) {
                bool r = wait_bit(&b2_full[sl], ph_b2, sl);  // every warp has read D1[sl]
                r = wait_bit(&tile_full[sl], ph_tile, sl) && r;
                if (r) {
                    tc::fence_after_sync();
                    issue_s1(t + 2);
                } else {
                    tc::mma_commit(&d1_full[sl]);
                }
            } else if (isB) {
                wait_bit(&b2_full[sl], ph_b2, sl);  // keep the phase count in step
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, err_sh != 0)) break;
        }
        // final epilogue 2 (nt-1)
        if (nt > 0 && !err_sh) {
            const bool wa = wait_bit(&d2_full[0], ph_d2, 0);
            const bool wb = wait_bit(&d2_full[1], ph_d2, 1);
            __syncwarp();
            tc::fence_after_sync();
            if (wa && wb)
                ws_epilogue2(tmem + lane_base + 256 + 128 * h2 + 16 * (j4 & 1), P, axx, ayy, arx, aix);
        }
        tc::fence_before_sync();
        ok = __syncthreads_and(err_sh == 0) != 0;
        tc::fence_after_sync();
        if (!ok) break;
        // ---- images: row ky = 128 kb + 32 q4 + lane, 16 kx from 64 g + 32 h2 + 16 (j4 & 1)
        const int ky = 128 * kb + 32 * q4 + lane;
        const int kx0 = 64 * g + 32 * h2 + 16 * (j4 & 1);
        if (ky < a.N && kx0 < a.N) {
            const size_t NN = (size_t)a.N * a.N;
            float* o = a.out + (size_t)c * a.nprod * NN + (size_t)ky * a.N + kx0;
            const int nk = min(16, a.N - kx0);
            store_pixels16(o, nk, a.accumulate, axx);
            if (a.nprod == 4) {
                store_pixels16(o + NN, nk, a.accumulate, ayy);
                store_pixels16(o + 2 * NN, nk, a.accumulate, arx);
                store_pixels16(o + 3 * NN, nk, a.accumulate, aix);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if ((!ok || err_sh) && tid == 0) atomicExch(a.status, 1);
}

// ---------------------------------------------------------------------------------
// Second warp-specialised kernel: the work item and operands of k_dftgemm_ws, but
// no thread waits to issue tensor-core work.  The warp that completes a step issues
// the next one: after every warp has finished epilogue 1 (t) and epilogue 2 (t-1)
// -- counted on a shared-memory counter -- the last one to arrive issues stage 2
// of frame t as one MMA chain with N = 128 P (both kx halves, both pols) and
// stage 1 of frame t+2, so the MMA issue never delays a warp the others wait for.
// Per frame t, every warp:
//   wait d1_full(t) -> (warp 0: copy tile t+2 into the buffer S1(t) has read)
//   -> epilogue 1 (t): D1[t&1] -> FP16 B2[t&1], up to three TMEM loads per wait
//   -> wait d2_full(t-1) -> epilogue 2 (t-1), four kx per TMEM load
//   -> arrive; the 16th arrival issues S2(t) -> d2_full and S1(t+2) -> d1_full[t&1]
// TMEM: D1[0..1] at 0 and d1_cols, A2 at 2 d1_cols, D2 at 256 (N = 128 P columns).
// Barrier parities follow from the frame index; every thread flips them alike.
constexpr int kWs2Threads = 512;

// Epilogue 1: D1 columns (chunks [yc0, yc1) of 8 y) of this warp's lane quarter ->
// B2 rows of half / pol `row0`, up to G TMEM loads per wait.
template <int G>
__device__ __forceinline__ void ws2_epilogue1(uint32_t taddr, int nyp, int yc0, int yc1, bool imw, int lane,
                                              uint8_t* b2, int row0, int R2)
{
    const int n0 = row0 + lane, n1 = row0 + 32 + lane;
    for (int yb = yc0; yb < yc1; yb += G) {
        const int ng = min(G, yc1 - yb);
        uint32_t r[8 * G];
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < ng) tmem_ld8(taddr + 8 * (yb + g), r + 8 * g);
        tc::tmem_wait_ld(r);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= ng) break;
            uint4 pos, neg;
            pos.x = pack_h2(__uint_as_float(r[8 * g + 0]), __uint_as_float(r[8 * g + 1]));
            pos.y = pack_h2(__uint_as_float(r[8 * g + 2]), __uint_as_float(r[8 * g + 3]));
            pos.z = pack_h2(__uint_as_float(r[8 * g + 4]), __uint_as_float(r[8 * g + 5]));
            pos.w = pack_h2(__uint_as_float(r[8 * g + 6]), __uint_as_float(r[8 * g + 7]));
            neg.x = pos.x ^ 0x80008000u;
            neg.y = pos.y ^ 0x80008000u;
            neg.z = pos.z ^ 0x80008000u;
            neg.w = pos.w ^ 0x80008000u;
            const int kc_lo = yb + g, kc_hi = (nyp >> 3) + kc_lo;
            if (!imw) {
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_lo, R2)) = pos;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_hi, R2)) = pos;
            } else {
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n0, kc_hi, R2)) = neg;
                *reinterpret_cast<uint4*>(b2 + sw_chunk(n1, kc_lo, R2)) = pos;
            }
        }
    }
}

template <int dummy>
__global__ void __launch_bounds__(kWs2Threads, 1) k_dftgemm_ws2(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_a, d1_full[2], d2_full, tile_full[2];
    __shared__ uint32_t tmem_sh;
    __shared__ unsigned arrivals;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_a, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&d1_full[i], 1);
            tc::mbar_init(&tile_full[i], 1);
        }
        tc::mbar_init(&d2_full, 1);
        arrivals = 0;
        err_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    uint8_t* sbase = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    uint8_t* sA1 = sbase + a.sA1;
    uint32_t ph_d1 = 0, ph_tile = 0, ph_a = 0, ph_d2 = 0;
    bool ok = true;
    const int P = a.P;
    const int q4 = warp & 3, j4 = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    const int R2 = 2 * 64 * P;
    const uint32_t a2col = 2u * a.d1_cols;
    const int items = a.n_ch * a.n_kb * a.n_g;
    const int h2 = j4 >> 1;  // epilogue 2: kx half of this warp, 16 kx at 16 (j4 & 1)

    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int g = item % a.n_g, kb = (item / a.n_g) % a.n_kb, cl = item / (a.n_g * a.n_kb);
        const int c = a.c0 + cl;
        const int4 bx = a.box[c];
        const int nxp = bx.z, nyp = bx.w;
        const int K1 = 2 * nxp, K2 = 2 * nyp, N1 = P * nyp;
        const int nt = a.nt;
        const uint32_t tile_bytes = (uint32_t)N1 * pad64(K1) * 2;
        const uint8_t* tiles_c = a.tiles + (size_t)cl * a.tile_stride;
        const size_t frame_step = (size_t)a.n_ch * a.tile_stride;
        const uint32_t id1 = tc::idesc_f16_f32(128, N1), id2 = tc::idesc_f16_f32(128, 128 * P);

        // ---- item prologue: A1 and the first two tiles by the TMA engine, A2 -> TMEM
        if (tid == 0) {
            const uint32_t a1_bytes = 256u * pad64(K1);
            tc::mbar_expect_tx(&bar_a, a1_bytes);
            tc::bulk_g2s(sA1, a.a1p + a.a1p_off[(size_t)c * a.n_g + g], a1_bytes, &bar_a);
            for (int j = 0; j < 2 && j < nt; ++j) {
                tc::mbar_expect_tx(&tile_full[j], tile_bytes);
                tc::bulk_g2s(sbase + a.sB1 + (size_t)j * a.b1_bytes, tiles_c + (size_t)j * frame_step, tile_bytes,
                             &tile_full[j]);
            }
        }
        if (warp < 4) {  // stage-2 DFT operand -> TMEM (lane = ky row)
            const uint32_t* src = a.a2w + a.a2w_off[(size_t)c * a.n_kb + kb] + (size_t)(32 * warp + lane) * (K2 / 2);
            for (int jj = 0; jj < K2 / 2; jj += 8) {
                uint32_t r[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = src[jj + i];
                tc::tmem_st8(tmem + lane_base + a2col + jj, r);
            }
            tc::tmem_wait_st();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        auto issue_s1 = [&](int t) {
            issue_ss(K1 / 16, tmem + (t & 1) * a.d1_cols, tc::smem_u32(sA1),
                     tc::smem_u32(sbase + a.sB1 + (size_t)(t & 1) * a.b1_bytes), 128 * 128, N1 * 128, id1);
            tc::mma_commit(&d1_full[t & 1]);
        };
        if (tid == 0) {
            bool good = tc::mbar_wait(&bar_a, ph_a & 1u, kWaitBudget);
            for (int j = 0; j < 2 && j < nt && good; ++j) {
                good = tc::mbar_wait(&tile_full[j], (ph_tile >> j) & 1u, kWaitBudget);
                if (good) {
                    tc::fence_after_sync();
                    issue_s1(j);
                }
            }
            if (!good) err_sh = 1;
        }
        ph_a ^= 1u;
        for (int j = 0; j < 2 && j < nt; ++j) ph_tile ^= 1u << j;
        __syncwarp();

        float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;
        // epilogue-1 part of this warp: lane quarter q4 = (part q4 >> 1, half q4 & 1);
        // columns: pol j4 >> 1 and half of the y chunks (P = 2), or a quarter of them (P = 1)
        const int hh = q4 & 1;
        const bool imw = (q4 >> 1) != 0;
        const int nyc = nyp >> 3;
        int p1, yc0, yc1;
        if (P == 2) {
            p1 = j4 >> 1;
            const int mid = (nyc + 1) >> 1;
            yc0 = (j4 & 1) ? mid : 0;
            yc1 = (j4 & 1) ? nyc : mid;
        } else {
            p1 = 0;
            yc0 = (nyc * j4) >> 2;
            yc1 = (nyc * (j4 + 1)) >> 2;
        }
        const uint32_t e2addr = tmem + lane_base + 256 + 64 * P * h2 + 16 * (j4 & 1);
        for (int t = 0; t < nt; ++t) {
            const int sl = t & 1;
            // epilogue 1 (t)
            const bool w = tc::mbar_wait(&d1_full[sl], (ph_d1 >> sl) & 1u, kWaitBudget);
            ph_d1 ^= 1u << sl;
            if (!w) err_sh = 1;
            __syncwarp();
            tc::fence_after_sync();
            if (tid == 0 && w && t + 2 < nt) {  // S1(t) has read tile buffer sl: copy tile t+2 into it
                tc::mbar_expect_tx(&tile_full[sl], tile_bytes);
                tc::bulk_g2s(sbase + a.sB1 + (size_t)sl * a.b1_bytes, tiles_c + (size_t)(t + 2) * frame_step,
                             tile_bytes, &tile_full[sl]);
            }
            if (w)
                ws2_epilogue1<3>(tmem + lane_base + sl * a.d1_cols + p1 * nyp, nyp, yc0, yc1, imw, lane,
                              sbase + a.sB2 + (size_t)sl * a.b2_bytes, 64 * P * hh + 64 * p1, R2);
            tc::fence_proxy_async();
            // epilogue 2 (t-1)
            if (t >= 1) {
                const bool w2 = tc::mbar_wait(&d2_full, ph_d2 & 1u, kWaitBudget);
                ph_d2 ^= 1u;
                if (!w2) err_sh = 1;
                __syncwarp();
                tc::fence_after_sync();
                if (w2) ws_epilogue2(e2addr, P, axx, ayy, arx, aix);
            }
            // arrival: the 16th warp issues S2(t) and S1(t+2)
            tc::fence_before_sync();
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) {
                __threadfence_block();
                last = (atomicAdd(&arrivals, 1u) & 15u) == 15u;
                if (last) __threadfence_block();
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last && lane == 0 && !err_sh) {
                tc::fence_after_sync();
                issue_ts(K2 / 16, tmem + 256, tmem + a2col, tc::smem_u32(sbase + a.sB2 + (size_t)sl * a.b2_bytes),
                         R2 * 128, id2);
                tc::mma_commit(&d2_full);
                if (t + 2 < nt) {
                    if (tc::mbar_wait(&tile_full[sl], (ph_tile >> sl) & 1u, kWaitBudget)) {
                        tc::fence_after_sync();
                        issue_s1(t + 2);
                    } else {
                        err_sh = 1;
                    }
                }
            }
            if (t + 2 < nt) ph_tile ^= 1u << sl;
            __syncwarp();
            if (__any_sync(0xffffffffu, err_sh != 0)) break;
        }
        // epilogue 2 (nt-1)
        if (nt > 0 && !err_sh) {
            const bool w2 = tc::mbar_wait(&d2_full, ph_d2 & 1u, kWaitBudget);
            ph_d2 ^= 1u;
            if (!w2) err_sh = 1;
            __syncwarp();
            tc::fence_after_sync();
            if (w2) ws_epilogue2(e2addr, P, axx, ayy, arx, aix);
        }
        tc::fence_before_sync();
        ok = __syncthreads_and(err_sh == 0) != 0;
        tc::fence_after_sync();
        if (!ok) break;
        // images: row ky = 128 kb + 32 q4 + lane, 16 kx from 64 g + 32 h2 + 16 (j4 & 1)
        const int ky = 128 * kb + 32 * q4 + lane;
        const int kx0 = 64 * g + 32 * h2 + 16 * (j4 & 1);
        if (ky < a.N && kx0 < a.N) {
            const size_t NN = (size_t)a.N * a.N;
            float* o = a.out + (size_t)c * a.nprod * NN + (size_t)ky * a.N + kx0;
            const int nk = min(16, a.N - kx0);
            store_pixels16(o, nk, a.accumulate, axx);
            if (a.nprod == 4) {
                store_pixels16(o + NN, nk, a.accumulate, ayy);
                store_pixels16(o + 2 * NN, nk, a.accumulate, arx);
                store_pixels16(o + 3 * NN, nk, a.accumulate, aix);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if ((!ok || err_sh) && tid == 0) atomicExch(a.status, 1);
}

// ---------------------------------------------------------------------------------
// Third warp-specialised kernel: 16 epilogue warps and a control warpgroup in
// separate register budgets (setmaxnreg), so that the threads issuing the MMAs and
// tile copies -- blocking while the tensor pipe is busy -- hold up no epilogue warp.
// Work item, operands and TMEM layout as k_dftgemm_ws2, except that a channel's box rows
// may come in H row parts (tall boxes): stage 2 sums over the box rows, so part h of frame t
// is a step of its own -- its tile part through stage 1 (D1 of P nyh columns), epilogue 1 and
// a stage-2 chain over its K range that adds to D2 (h > 0) -- and D2 holds the frame once
// its last part is in.  Sub-frame u = t H + h; NB (2..4) tile-part buffers:
//   copy thread (warp 18, lane 0), per sub-frame u:
//     wait d1_full(u) -> copy tile part u+NB into the buffer S1(u) read (frames ahead -> L2)
//   stage-1 issuer (warp 17, lane 0), per sub-frame u:
//     wait b2_full(u) and tile part u+2 -> S1(u+2) -> d1_full[u&1]
//   stage-2 issuer (warp 16, lane 0), per sub-frame u:
//     wait b2_full(u) [and, at h = 0, d2_empty(t-1)] -> S2(u) -> b2_free[u&1] (H > 1),
//     and at h = H-1 -> d2_full
//   epilogue warps 0-15, per sub-frame u:
//     wait d1_full(u) [and b2_free(u-2)] -> epilogue 1 (u) -> arrive b2_full[u&1];
//     at h = 0: wait d2_full(t-1) -> epilogue 2 (t-1) -> arrive d2_empty
// Epilogue 2 of frame t-1 runs after epilogue 1 of part 0 of frame t, before the later parts,
// so the stage-2 chain of part 0 (which waits for it) never waits on a later epilogue 1.
// Items are separated by two block-wide named barriers (operands loaded; item done).
constexpr int kWs3Threads = 640;
// Grid tiles requested into L2 this many frames before the shared-memory copy that
// needs them: with two tile buffers a tile is copied only one frame ahead of its
// stage-1 MMAs, which is less than the HBM latency; from L2 it arrives in time.
constexpr int kTilePrefetch = 8;
constexpr int kWs3MaxBlocks = 256;  // blocks per launch (one per SM) the split bookkeeping holds
constexpr int kWs3MaxTileBufs = 4;  // tile-part buffers of k_dftgemm_ws3 (short row parts need more in flight)

__device__ __forceinline__ void bar_all(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kWs3Threads) : "memory");
}

// A split work item (k_dftgemm_ws3, equal shares) after this block stored its part
// to its slot: the block that stores the item's last part -- counted on the item's
// counter -- adds all parts in block order and writes (or adds) the images.  Kept
// out of line so that the frame loop's register allocation does not carry it.
__device__ __noinline__ void ws3_split_finish(const MmaArgs& a, int item, int c, int ky, int kx0, size_t px,
                                              long long U, int tid, int* split_slot, int* split_n)
{
    __threadfence();
    asm volatile("bar.sync 3, 512;" ::: "memory");
    if (tid == 0) {
        const long long s0 = (long long)item * a.nt, s1 = s0 + a.nt - 1;
        const int G = gridDim.x, ipc = a.n_kb * a.n_g;
        auto start = [&](int b) { return split_start(a.wcum, a.c0, a.n_ch, ipc, a.nt, b, G); };
        auto owner = [&](long long f) {  // the block whose range [start(b), start(b + 1)) holds f
            int lo = 0, hi = G;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (start(mid) <= f) lo = mid;
                else hi = mid;
            }
            return lo;
        };
        (void)U;
        int n = 0;
        const int b1 = owner(s1);
        for (int b = owner(s0); b <= b1; ++b) {
            const long long bw0 = start(b);
            if (bw0 == start(b + 1)) continue;  // no frames: no part
            split_slot[n++] = 2 * b + (s0 <= bw0 ? 0 : 1);
        }
        const bool last = atomicAdd(&a.counters[item], 1) == n - 1;
        if (last) a.counters[item] = 0;  // ready for the next launch
        *split_n = last ? n : 0;
    }
    asm volatile("bar.sync 3, 512;" ::: "memory");
    const int n = *split_n;
    if (n > 0 && ky < a.N && kx0 < a.N) {
        __threadfence();
        const size_t NN = (size_t)a.N * a.N;
        const int nk = min(16, a.N - kx0);
        for (int pr = 0; pr < a.nprod; ++pr) {  // one product at a time: 16 live sums
            float sum[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) sum[i] = 0.f;
            for (int k = 0; k < n; ++k) {
                const float* q = a.partial + ((size_t)split_slot[k] * 4 + pr) * 8192 + px;
#pragma unroll
                for (int i = 0; i < 16; i += 4) {
                    const float4 u = __ldcg(reinterpret_cast<const float4*>(q + i));
                    sum[i] += u.x;
                    sum[i + 1] += u.y;
                    sum[i + 2] += u.z;
                    sum[i + 3] += u.w;
                }
            }
            store_pixels16(a.out + ((size_t)c * a.nprod + pr) * NN + (size_t)ky * a.N + kx0, nk, a.accumulate, sum);
        }
    }
}

// MODE 0: whole items, 1: equal shares (split items), 2: whole items, sub-integrations.
// PARTS: some channel of the plan has more than one row part (else every H is 1 at compile time).
template <int MODE, bool PARTS>
__global__ void __launch_bounds__(kWs3Threads, 1) k_dftgemm_ws3(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_a, d1_full[2], b2_full[2], b2_free[2], d2_full, d2_empty, tile_full[kWs3MaxTileBufs],
        tile_free[kWs3MaxTileBufs], drain[2];
    __shared__ uint32_t tmem_sh;
    __shared__ int err_sh;
    __shared__ int split_slot[kWs3MaxBlocks];  // partial slots of a split item, in block order
    __shared__ int split_n;                    // > 0: this block completes the item; sum split_n slots
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_a, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&d1_full[i], 1);
            tc::mbar_init(&b2_full[i], 16);
            tc::mbar_init(&b2_free[i], 1);
            tc::mbar_init(&drain[i], 1);
        }
        for (int i = 0; i < kWs3MaxTileBufs; ++i) {
            tc::mbar_init(&tile_full[i], 1);
            tc::mbar_init(&tile_free[i], 1);
        }
        tc::mbar_init(&d2_full, 1);
        tc::mbar_init(&d2_empty, 16);
        err_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    uint8_t* sbase = smem + ((1024u - (tc::smem_u32(smem) & 1023u)) & 1023u);
    uint8_t* sA1 = sbase + a.sA1;
    const int P = a.P;
    const int R2 = 2 * 64 * P;
    const uint32_t a2col = 2u * a.d1_cols;
    const int items = a.n_ch * a.n_kb * a.n_g;
    // this block's share of the launch.  split: the (item, frame) pairs [wb0, wb1) in
    // item-major order (equal shares; items cut at share boundaries are summed by the
    // block that stores their last part); else whole items blockIdx.x, + gridDim.x, ...
    const long long U = (long long)items * a.nt;
    const int ipc = a.n_kb * a.n_g;  // items per channel
    const long long wb0 = split_start(a.wcum, a.c0, a.n_ch, ipc, a.nt, blockIdx.x, gridDim.x);
    const long long wb1 = split_start(a.wcum, a.c0, a.n_ch, ipc, a.nt, blockIdx.x + 1, gridDim.x);

    if (warp >= 16) {
        // ------------------------------------------------------------ control warpgroup
        // 4 control warps x 32 lanes x 32 registers + 16 epilogue warps x 32 lanes x 112 =
        // 61,440: exactly the 640 threads x 96 registers the block is launched with
        asm volatile("setmaxnreg.dec.sync.aligned.u32 32;" ::: "memory");
        uint32_t ph_d1 = 0, ph_b2 = 0, ph_tile = 0, ph_free = 0, ph_a = 0, ph_e2 = 0;
        uint32_t pend = 0;  // copy thread: bulk copies in flight (bit j tile buffer j, bit 7 A1)
        uint32_t cph = 0;   // copy thread: parity of the phase the next copy into buffer j (bit j)
                            // or of A1 (bit 7) completes
        const bool iss1 = warp == 17 && lane == 0;  // stage 1: S1 chains
        const bool iss2 = warp == 16 && lane == 0;  // stage 2 chains
        const bool cpy = warp == 18 && lane == 0;   // A1 and tile-part copies, L2 prefetches
        const int NB = a.nbt;                       // tile-part buffers in shared memory (2..4)
        long long w = wb0;
        for (int it = 0;; ++it) {
            int item, fs, nt;  // work item, its first frame and the frames of this segment
            if (MODE == 1) {
                if (w >= wb1) break;
                item = (int)(w / a.nt);
                fs = (int)(w % a.nt);
                nt = (int)min((long long)(a.nt - fs), wb1 - w);
                w += nt;
            } else {
                item = blockIdx.x + it * gridDim.x;
                if (item >= items) break;
                if (a.item_order) item = a.item_order[(size_t)a.c0 * ipc + item];
                fs = 0;
                nt = a.nt;
            }
            const int g = item % a.n_g, cl = item / (a.n_g * a.n_kb);
            const int c = a.c0 + cl;
            const int4 bx = a.box[c];
            const int4 tp = a.tbox[c];
            const int nxp = bx.z, nyh = tp.x, H = PARTS ? tp.y : 1;
            const int K1 = 2 * nxp, K2h = 2 * nyh, N1 = P * nyh;
            const int NU = nt * H;  // sub-frames u = t H + h: frame t, row part h
            const uint32_t part_bytes = (uint32_t)N1 * pad64(K1) * 2;
            auto buf = [&](int b) { return sbase + a.sB1 + (size_t)b * a.b1_bytes; };
            auto wait_bit = [&](uint64_t* bar, uint32_t& ph, int slot) -> bool {
                const bool r = tc::mbar_wait(bar, (ph >> slot) & 1u, kWaitBudget);
                if (r) ph ^= 1u << slot;
                return r;
            };
            // copy thread: A1 and the first NB tile parts now, then part u+NB once S1(u) has read
            // its buffer (after the barrier: S1 is issued only past it)
            const size_t frame_step = (size_t)a.n_ch * a.tile_stride;
            const uint8_t* tiles_c = a.tiles + (size_t)cl * a.tile_stride + (size_t)fs * frame_step;
            const uint8_t* nxt = tiles_c;  // next part to copy, advanced without division
            int nxt_h = 0;
            auto copy_next = [&](int b) {
                tc::mbar_expect_tx(&tile_full[b], part_bytes);
                tc::bulk_g2s(buf(b), nxt, part_bytes, &tile_full[b]);
                pend |= 1u << b;
                cph ^= 1u << b;
                if (++nxt_h == H) {
                    nxt_h = 0;
                    nxt += frame_step - (size_t)(H - 1) * part_bytes;
                } else {
                    nxt += part_bytes;
                }
            };
            if (cpy) {
                const uint32_t a1_bytes = 256u * pad64(K1);
                tc::mbar_expect_tx(&bar_a, a1_bytes);
                tc::bulk_g2s(sA1, a.a1p + a.a1p_off[(size_t)c * a.n_g + g], a1_bytes, &bar_a);
                pend |= 0x80u;
                cph ^= 0x80u;
                for (int j = 0; j < NB && j < NU; ++j) copy_next(j);
                for (int j = 1; j <= kTilePrefetch && j < nt; ++j)  // later frames: HBM -> L2 ahead of use
                    tc::bulk_prefetch_l2(tiles_c + (size_t)j * frame_step, part_bytes * H);
            }
            bar_all(1);  // A2 is in TMEM
            if (iss1) {  // per sub-frame u: E1(u) has read D1[u&1] and tile part u+2 is in -> S1(u+2)
                const uint32_t id1 = tc::idesc_f16_f32(128, N1);
                auto issue_s1 = [&](int slot, int b) {
                    issue_ss(K1 / 16, tmem + slot * a.d1_cols, tc::smem_u32(sA1), tc::smem_u32(buf(b)), 128 * 128,
                             N1 * 128, id1);
                    tc::mma_commit(&d1_full[slot]);
                    tc::mma_commit(&tile_free[b]);  // the copy thread's signal that buffer b was read
                };
                bool good = wait_bit(&bar_a, ph_a, 0);
                for (int j = 0; j < 2 && j < NU && good; ++j) {
                    good = wait_bit(&tile_full[j], ph_tile, j);
                    if (good) {
                        tc::fence_after_sync();
                        issue_s1(j, j);
                    }
                }
                int bu2 = 2 % NB;  // buffer of sub-frame u + 2
                for (int u = 0; u < NU - 2 && good; ++u) {
                    const int sl = u & 1;
                    good = wait_bit(&b2_full[sl], ph_b2, sl);  // E1(u) has read D1[sl]
                    if (good) good = wait_bit(&tile_full[bu2], ph_tile, bu2);
                    if (good) {
                        tc::fence_after_sync();
                        issue_s1(sl, bu2);
                    }
                    if (++bu2 == NB) bu2 = 0;
                }
                for (int u = max(0, NU - 2); u < NU && good; ++u)  // the last two E1s, so parities stay paired
                    good = wait_bit(&b2_full[u & 1], ph_b2, u & 1);
                if (!good) err_sh = 1;
            } else if (iss2) {  // per sub-frame u: E1(u) wrote B2[u&1] (and E2(t-1) read D2) -> S2(u)
                const uint32_t id2 = tc::idesc_f16_f32(128, 128 * P);
                bool good = true;
                for (int t = 0; t < nt && good; ++t)
                    for (int h = 0; h < H && good; ++h) {
                        const int sl = (t * H + h) & 1;
                        good = wait_bit(&b2_full[sl], ph_b2, sl);
                        if (good && h == 0 && t >= 1) good = wait_bit(&d2_empty, ph_e2, 0);
                        if (!good) break;
                        tc::fence_after_sync();
                        issue_ts(K2h / 16, tmem + 256, tmem + a2col + h * nyh,
                                 tc::smem_u32(sbase + a.sB2 + (size_t)sl * a.b2_bytes), R2 * 128, id2, h > 0);
                        if (H > 1) tc::mma_commit(&b2_free[sl]);  // S2(u) has read B2[sl]
                        if (h == H - 1) tc::mma_commit(&d2_full);
                    }
                if (!good) err_sh = 1;
            } else if (cpy) {
                bool good = true;
                int bu = 0, hu = 0, tu = 0;  // buffer, row part and frame of u
                for (int u = 0; u < NU && good; ++u) {
                    // S1(u) done: buffer bu is free.  Its own barrier, not d1_full[u & 1]: with
                    // more than two buffers S1(u + 2) needs no refill from this thread, so
                    // d1_full[u & 1] could complete twice before this wait and its parity alias;
                    // tile_free[bu] cannot complete again before this thread refills bu
                    good = wait_bit(&tile_free[bu], ph_free, bu);
                    if (good) pend &= ~((1u << bu) | 0x80u);  // its copy (and A1) had landed: S1(u) read them
                    if (good && u + NB < NU) copy_next(bu);
                    if (good && hu == 0 && tu + 1 + kTilePrefetch < nt)
                        tc::bulk_prefetch_l2(tiles_c + (size_t)(tu + 1 + kTilePrefetch) * frame_step, part_bytes * H);
                    if (++bu == NB) bu = 0;
                    if (++hu == H) {
                        hu = 0;
                        ++tu;
                    }
                }
                if (!good) err_sh = 1;
            }
            __syncwarp();
            bar_all(2);  // item done
            if (err_sh) break;
        }
        if (err_sh && (iss1 || iss2)) {  // a wait ran out: let this thread's MMAs finish (bounded)
            tc::mma_commit(&drain[iss2 ? 1 : 0]);
            tc::mbar_wait(&drain[iss2 ? 1 : 0], 0, kWaitBudget);
        }
        if (err_sh && cpy) {  // and the bulk copies in flight, before the block releases its memory
            for (int j = 0; j < kWs3MaxTileBufs; ++j)  // a pending copy completes the phase before cph's
                if ((pend >> j) & 1u) tc::mbar_wait(&tile_full[j], ((cph >> j) & 1u) ^ 1u, kWaitBudget);
            if (pend & 0x80u) tc::mbar_wait(&bar_a, ((cph >> 7) & 1u) ^ 1u, kWaitBudget);
        }
    } else {
        // ------------------------------------------------------------ epilogue warps
        asm volatile("setmaxnreg.inc.sync.aligned.u32 112;" ::: "memory");
        uint32_t ph_d1 = 0, ph_d2 = 0, ph_bf = 0;
        const int q4 = warp & 3, j4 = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        const int h2 = j4 >> 1;
        long long w = wb0;
        for (int it = 0;; ++it) {
            int item, fs, nt;  // work item, its first frame and the frames of this segment
            if (MODE == 1) {
                if (w >= wb1) break;
                item = (int)(w / a.nt);
                fs = (int)(w % a.nt);
                nt = (int)min((long long)(a.nt - fs), wb1 - w);
                w += nt;
            } else {
                item = blockIdx.x + it * gridDim.x;
                if (item >= items) break;
                if (a.item_order) item = a.item_order[(size_t)a.c0 * ipc + item];
                fs = 0;
                nt = a.nt;
            }
            const bool first_seg = it == 0;
            const int g = item % a.n_g, kb = (item / a.n_g) % a.n_kb, cl = item / (a.n_g * a.n_kb);
            const int c = a.c0 + cl;
            const int4 tp = a.tbox[c];
            const int nyh = tp.x, H = PARTS ? tp.y : 1, nyt = tp.z;
            if (warp < 4) {  // stage-2 DFT operand (every row part) -> TMEM (lane = ky row)
                // rows of nyt words (a multiple of 8) from a 32-byte aligned table: 32 words per
                // round of 16-byte loads, so an item waits for nyt / 32 load latencies, not nyt / 8
                const uint4* src = reinterpret_cast<const uint4*>(a.a2w + a.a2w_off[(size_t)c * a.n_kb + kb] +
                                                                  (size_t)(32 * warp + lane) * nyt);
                for (int jj = 0; jj < nyt; jj += 32) {
                    uint4 q[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        q[i] = jj + 4 * i < nyt ? __ldg(src + (jj >> 2) + i) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (jj + 8 * g >= nyt) break;
                        const uint32_t r[8] = {q[2 * g].x,     q[2 * g].y,     q[2 * g].z,     q[2 * g].w,
                                               q[2 * g + 1].x, q[2 * g + 1].y, q[2 * g + 1].z, q[2 * g + 1].w};
                        tc::tmem_st8(tmem + lane_base + a2col + jj + 8 * g, r);
                    }
                }
                tc::tmem_wait_st();
            }
            tc::fence_before_sync();
            bar_all(1);
            tc::fence_after_sync();
            float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;
            const int hh = q4 & 1;
            const bool imw = (q4 >> 1) != 0;
            const int nyc = nyh >> 3;
            int p1, yc0, yc1;
            if (P == 2) {
                p1 = j4 >> 1;
                const int mid = (nyc + 1) >> 1;
                yc0 = (j4 & 1) ? mid : 0;
                yc1 = (j4 & 1) ? nyc : mid;
            } else {
                p1 = 0;
                yc0 = (nyc * j4) >> 2;
                yc1 = (nyc * (j4 + 1)) >> 2;
            }
            const uint32_t e2addr = tmem + lane_base + 256 + 64 * P * h2 + 16 * (j4 & 1);
            // sub-integrations: after frame f (chunk-local) ends an interval, write (or add)
            // the sums to image set iv0 + f / sub and restart them
            auto flush_interval = [&](int f) {
                const int ky = 128 * kb + 32 * q4 + lane;
                const int kx0 = 64 * g + 32 * h2 + 16 * (j4 & 1);
                if (ky < a.N && kx0 < a.N) {
                    const size_t NN = (size_t)a.N * a.N;
                    float* o = a.out + ((size_t)(a.iv0 + f / a.sub) * a.C + c) * a.nprod * NN + (size_t)ky * a.N + kx0;
                    const int nk = min(16, a.N - kx0);
                    store_pixels16_flush(o, nk, a.accumulate, axx);
                    if (a.nprod == 4) {
                        store_pixels16_flush(o + NN, nk, a.accumulate, ayy);
                        store_pixels16_flush(o + 2 * NN, nk, a.accumulate, arx);
                        store_pixels16_flush(o + 3 * NN, nk, a.accumulate, aix);
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;
            };
            const int NU = nt * H;
            bool live = true;
            for (int u = 0, t = 0, h = 0; u < NU && live; ++u) {
                const int sl = u & 1;
                bool w = tc::mbar_wait(&d1_full[sl], (ph_d1 >> sl) & 1u, kWaitBudget);
                ph_d1 ^= 1u << sl;
                if (w && H > 1 && u >= 2) {  // S2(u-2) has read B2[sl]
                    w = tc::mbar_wait(&b2_free[sl], (ph_bf >> sl) & 1u, kWaitBudget);
                    ph_bf ^= 1u << sl;
                }
                __syncwarp();
                tc::fence_after_sync();
                if (w)
                    // one TMEM load per round without row parts (fewer spills), two with them (a
                    // short part's stores cannot hide a second round's load latency)
                    ws2_epilogue1<PARTS ? 2 : 1>(tmem + lane_base + sl * a.d1_cols + p1 * nyh, nyh, yc0, yc1, imw, lane,
                                  sbase + a.sB2 + (size_t)sl * a.b2_bytes, 64 * P * hh + 64 * p1, R2);
                tc::fence_proxy_async();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&b2_full[sl]);
                bool w2 = true;
                if (h == 0 && t >= 1) {
                    w2 = tc::mbar_wait(&d2_full, ph_d2 & 1u, kWaitBudget);
                    ph_d2 ^= 1u;
                    __syncwarp();
                    tc::fence_after_sync();
                    if (w2) ws_epilogue2(e2addr, P, axx, ayy, arx, aix);
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&d2_empty);
                    if (MODE == 2 && w2 && t % a.sub == 0) flush_interval(t - 1);  // frame t-1 ends one
                }
                if (!w || !w2) err_sh = 1;
                live = !__any_sync(0xffffffffu, err_sh != 0);
                if (++h == H) {
                    h = 0;
                    ++t;
                }
            }
            if (nt > 0 && live) {
                bool w2 = tc::mbar_wait(&d2_full, ph_d2 & 1u, kWaitBudget);
                ph_d2 ^= 1u;
                // the last two stage-2 steps' B2 releases, waited on by no later epilogue 1
                for (int u = max(0, NU - 2); w2 && H > 1 && u < NU; ++u) {
                    w2 = tc::mbar_wait(&b2_free[u & 1], (ph_bf >> (u & 1)) & 1u, kWaitBudget);
                    ph_bf ^= 1u << (u & 1);
                }
                if (!w2) err_sh = 1;
                __syncwarp();
                tc::fence_after_sync();
                if (w2) ws_epilogue2(e2addr, P, axx, ayy, arx, aix);
                if (MODE == 2 && w2) flush_interval(nt - 1);
            }
            tc::fence_before_sync();
            bar_all(2);
            tc::fence_after_sync();
            if (err_sh) break;
            // images: row ky = 128 kb + 32 q4 + lane, 16 kx from 64 g + 32 h2 + 16 (j4 & 1); a
            // segment that is only part of its item goes to this block's partial slot
            const int ky = 128 * kb + 32 * q4 + lane;
            const int kx0 = 64 * g + 32 * h2 + 16 * (j4 & 1);
            if (MODE == 1 && (fs != 0 || nt != a.nt)) {
                const size_t px = (size_t)(32 * q4 + lane) * 64 + 32 * h2 + 16 * (j4 & 1);
                float* o = a.partial + (2 * (size_t)blockIdx.x + (first_seg ? 0 : 1)) * 4 * 8192 + px;
                store_pixels16(o, 16, 0, axx);
                if (a.nprod == 4) {
                    store_pixels16(o + 8192, 16, 0, ayy);
                    store_pixels16(o + 2 * 8192, 16, 0, arx);
                    store_pixels16(o + 3 * 8192, 16, 0, aix);
                }
                ws3_split_finish(a, item, c, ky, kx0, px, U, tid, split_slot, &split_n);
            } else if (MODE != 2 && ky < a.N && kx0 < a.N) {
                const size_t NN = (size_t)a.N * a.N;
                float* o = a.out + (size_t)c * a.nprod * NN + (size_t)ky * a.N + kx0;
                const int nk = min(16, a.N - kx0);
                store_pixels16(o, nk, a.accumulate, axx);
                if (a.nprod == 4) {
                    store_pixels16(o + NN, nk, a.accumulate, ayy);
                    store_pixels16(o + 2 * NN, nk, a.accumulate, arx);
                    store_pixels16(o + 3 * NN, nk, a.accumulate, aix);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
    if (err_sh && tid == 0) atomicExch(a.status, 1);
}





}  // namespace

// Time samples per chunk so that the grid tiles of one (channel group, time
// chunk) take at most `budget` bytes, and the tile buffer for them.
epic_status dftgemm_set_kernel(epic_plan_s* p, int variant)
{
    if (variant < 1 || variant > 3 || !p->tc.ws || ((p->sub > 0 || p->tc.parts) && variant != 3) ||
        (variant == 3 && p->sm_count > kWs3MaxBlocks))
        return EPIC_ERR_UNSUPPORTED;
    p->tc.ws_variant = variant;
    return EPIC_OK;
}

static epic_status upload_item_order(epic_plan_s* p);

// Channels per launch of the warp-specialised kernels: 0 = groups of about two work items
// per SM (whole items per block balance), 1 = every channel in one group (the fewest
// launches; with equal (item, frame) shares the item count need not divide evenly).  The
// tile buffer is resized for the group at the current chunk budget.
epic_status dftgemm_set_group(epic_plan_s* p, int v)
{
    if (!p->tc.ws || v < 0 || v > 1) return EPIC_ERR_UNSUPPORTED;
    const int cg_old = p->tc.cg, group_old = p->tc.group;
    p->tc.group = v;
    p->tc.cg = v == 1 ? p->C : p->tc.cg_items;
    epic_status st = dftgemm_set_chunk(p, p->chunk_budget);
    if (st != EPIC_OK) {
        p->tc.group = group_old;
        p->tc.cg = cg_old;
        dftgemm_set_chunk(p, p->chunk_budget);
    }
    const epic_status so = upload_item_order(p);  // the groups changed
    return st != EPIC_OK ? st : so;
}

// Work split of k_dftgemm_ws3: -1 = automatic (equal shares unless the launch's items are
// a whole number per SM), 0 = whole items per block, 1 = equal (item, frame) shares.
epic_status dftgemm_set_split(epic_plan_s* p, int mode)
{
    if (!p->tc.ws || mode < -1 || mode > 1 || (p->sub > 0 && mode == 1)) return EPIC_ERR_UNSUPPORTED;
    p->tc.split = mode;
    return EPIC_OK;
}

// Order in which k_dftgemm_ws3 deals a channel group's whole work items to its blocks (block b
// takes the items at positions b, b + G, b + 2 G, ... of the group's list, G blocks): items
// sorted by modelled cost per frame (the work-split weight of their channel) and dealt in
// snake order -- round k forward when k is even, backward when odd -- so that a block's
// items add up to about the same cost (costliest with cheapest); a last partial round is
// dealt forward, to the first blocks, as the kernel expects.
static epic_status upload_item_order(epic_plan_s* p)
{
    cudaFree(p->tc.item_order);
    p->tc.item_order = nullptr;
    if (!p->tc.ws) return EPIC_OK;
    const int C = p->C, ipc = p->tc.n_kb * p->tc.n_gp;
    std::vector<int> ord((size_t)C * ipc);
    for (int c0 = 0; c0 < C; c0 += p->tc.cg) {
        const int ng = std::min(p->tc.cg, C - c0), L = ng * ipc, G = std::min(L, p->sm_count);
        auto w = [&](int i) {
            const int4 r = p->tc.tbox_h[c0 + i / ipc];
            return 1000LL + 1200LL * r.y + 10LL * r.z;
        };
        std::vector<int> idx(L);
        for (int i = 0; i < L; ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int u, int v) { return w(u) > w(v); });
        for (int r = 0; r < L; ++r) {
            const int k = r / G, j = r % G;
            const bool partial = (k + 1) * G > L;
            const int b = (k & 1) && !partial ? G - 1 - j : j;
            ord[(size_t)c0 * ipc + (size_t)k * G + b] = idx[r];
        }
    }
    cudaError_t e = cudaMalloc(&p->tc.item_order, ord.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.item_order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(p, e, "work-item order upload");
    return EPIC_OK;
}

epic_status dftgemm_set_chunk(epic_plan_s* p, size_t budget)
{
    const size_t per_t = (size_t)p->tc.cg * p->tc.stride;
    int tcn = (int)std::max<size_t>(1, std::min<size_t>((size_t)p->max_time, budget / per_t));
    if (p->sub > 0) tcn = std::max(p->sub, tcn - tcn % p->sub);  // whole sub-integrations per chunk
    const size_t bytes = per_t * tcn;
    p->chunk_budget = budget;
    p->tc.tc = tcn;
    p->time_chunk = tcn;
    if (p->scratch && bytes == p->scratch_bytes) return EPIC_OK;
    cudaFree(p->scratch);
    p->scratch = nullptr;
    p->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&p->scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMalloc(tensor path tile buffer)");
    // zero once: tile bytes no gridding kernel writes (K padding past 2 nx) then hold zeros or
    // FP16 values of other tiles, never stale non-finite bits, and meet zero DFT operands
    e = cudaMemset(p->scratch, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemset(tensor path tile buffer)");
    p->scratch_bytes = bytes;
    return EPIC_OK;
}

static epic_status grid_bal_config(epic_plan_s* p, int F);

// Frames per pass and grid size of the pair-list gridding kernel (UNSUPPORTED when F
// frames of voltages do not fit in shared memory).
static epic_status grid_pl_config(epic_plan_s* p, int F)
{
    if (!p->tc.pl_ptr || (F != 1 && F != 2 && F != 4 && F != 8)) return EPIC_ERR_UNSUPPORTED;
    const bool H = p->jones.empty();  // FP16-pair voltages unless polarisation mixing
    const int fb = p->A * p->P * (p->bits / 4);
    // the lists in shared memory when they fit beside the voltages
    const bool S =
        grid_pl_smem(F, p->A, fb, H, true, p->tc.pl_max_ptr, p->tc.pl_max_ent) + 2048 <= (size_t)p->smem_optin;
    const size_t bytes = grid_pl_smem(F, p->A, fb, H, S, p->tc.pl_max_ptr, p->tc.pl_max_ent);
#define EPIC_PL_FN(FF)                                                                                   \
    (H ? (S ? (const void*)k_dftgemm_grid_pl<FF, true, true> : (const void*)k_dftgemm_grid_pl<FF, true, false>) \
       : (S ? (const void*)k_dftgemm_grid_pl<FF, false, true> : (const void*)k_dftgemm_grid_pl<FF, false, false>))
    const void* fn = F == 8 ? EPIC_PL_FN(8) : F == 4 ? EPIC_PL_FN(4) : F == 2 ? EPIC_PL_FN(2) : EPIC_PL_FN(1);
#undef EPIC_PL_FN
    p->tc.pl_stage = S;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncGetAttributes(k_dftgemm_grid_pl)");
    if (bytes + fa.sharedSizeBytes > (size_t)p->smem_optin) return EPIC_ERR_UNSUPPORTED;
    e = allow_max_smem(fn, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_grid_pl)");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kGridPlThreads, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_dftgemm_grid_pl)");
    if (occ < 1) return EPIC_ERR_UNSUPPORTED;
    p->tc.grid_frames = F;
    p->tc.grid_smem = (int)bytes;
    p->tc.grid_blocks = p->sm_count * occ;
    return EPIC_OK;
}

// Frames per pass of the persistent gridding kernel and its grid size (the blocks
// that fit on the GPU at once).  UNSUPPORTED when F frames do not fit in shared memory.
epic_status dftgemm_grid_config(epic_plan_s* p, int F)
{
    if (p->tc.grid_variant == 2) return grid_bal_config(p, F);
    if (p->tc.grid_variant == 3) return grid_pl_config(p, F);
    if (F != 1 && F != 2 && F != 4 && F != 8) return EPIC_ERR_UNSUPPORTED;
    const size_t bytes =
        grid_ps_smem(F, p->A, p->A * p->P * (p->bits / 4), p->tc.grid_max_cells, p->tc.grid_max_list, p->tc.grid_cplx);
    const void* fn = nullptr;
    if (p->tc.grid_cplx) {
        fn = F == 8 ? (const void*)k_dftgemm_grid_ps<true, 8> : F == 4 ? (const void*)k_dftgemm_grid_ps<true, 4>
           : F == 2 ? (const void*)k_dftgemm_grid_ps<true, 2> : (const void*)k_dftgemm_grid_ps<true, 1>;
    } else {
        fn = F == 8 ? (const void*)k_dftgemm_grid_ps<false, 8> : F == 4 ? (const void*)k_dftgemm_grid_ps<false, 4>
           : F == 2 ? (const void*)k_dftgemm_grid_ps<false, 2> : (const void*)k_dftgemm_grid_ps<false, 1>;
    }
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncGetAttributes(k_dftgemm_grid_ps)");
    if (bytes + fa.sharedSizeBytes > (size_t)p->smem_optin) return EPIC_ERR_UNSUPPORTED;
    e = allow_max_smem(fn, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_grid_ps)");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_dftgemm_grid_ps)");
    if (occ < 1) return EPIC_ERR_UNSUPPORTED;
    p->tc.grid_frames = F;
    p->tc.grid_smem = (int)bytes;
    p->tc.grid_blocks = p->sm_count * occ;
    return EPIC_OK;
}

// Frames per pass and grid size of the balanced gridding kernel (UNSUPPORTED when
// F tile buffers, the task list and the entries do not fit in shared memory).
static epic_status grid_bal_config(epic_plan_s* p, int F)
{
    if (!p->tc.gtask || (F != 1 && F != 2 && F != 4)) return EPIC_ERR_UNSUPPORTED;
    const size_t bytes =
        grid_bal_smem(F, p->A, p->A * p->P * (p->bits / 4), p->tc.gtask_max, p->tc.gell_max, (unsigned)p->tc.stride);
    // FP16-pair voltages (H) unless polarisation mixing makes them non-integer
    const bool H = p->jones.empty();
    const void* fn = H ? (F == 4 ? (const void*)k_dftgemm_grid_bal<4, true>
                             : F == 2 ? (const void*)k_dftgemm_grid_bal<2, true> : (const void*)k_dftgemm_grid_bal<1, true>)
                       : (F == 4 ? (const void*)k_dftgemm_grid_bal<4, false>
                             : F == 2 ? (const void*)k_dftgemm_grid_bal<2, false> : (const void*)k_dftgemm_grid_bal<1, false>);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncGetAttributes(k_dftgemm_grid_bal)");
    if (bytes + fa.sharedSizeBytes > (size_t)p->smem_optin) return EPIC_ERR_UNSUPPORTED;
    e = allow_max_smem(fn, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_grid_bal)");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kGridBalBlock, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(k_dftgemm_grid_bal)");
    if (occ < 1) return EPIC_ERR_UNSUPPORTED;
    p->tc.grid_frames = F;
    p->tc.grid_smem = (int)bytes;
    p->tc.grid_blocks = p->sm_count * occ;
    return EPIC_OK;
}

// Gridding kernel variant: 1 = persistent row-major gather, 2 = balanced task lists,
// 3 = row-major pair lists.  Keeps the frames per pass if the variant allows them, else
// the largest it allows.
epic_status dftgemm_set_grid_kernel(epic_plan_s* p, int variant)
{
    if (variant < 1 || variant > 3) return EPIC_ERR_UNSUPPORTED;
    if (variant == 2 && !p->tc.gtask) return EPIC_ERR_UNSUPPORTED;
    if (variant == 3 && !p->tc.pl_ptr) return EPIC_ERR_UNSUPPORTED;
    if (variant == 1 && !p->tc.grid_ps) return EPIC_ERR_UNSUPPORTED;
    const int old_variant = p->tc.grid_variant, old_f = p->tc.grid_frames;
    p->tc.grid_variant = variant;
    epic_status st = EPIC_ERR_UNSUPPORTED;
    for (int F = old_f; F >= 1 && st == EPIC_ERR_UNSUPPORTED; F >>= 1) st = dftgemm_grid_config(p, F);
    if (st != EPIC_OK) {
        p->tc.grid_variant = old_variant;
        dftgemm_grid_config(p, old_f);
    }
    return st;
}

epic_status dftgemm_setup(epic_plan_s* p)
{
    const int N = p->N, C = p->C, P = p->P;
    const int n_kb = (N + 127) / 128, n_s = (N + 31) / 32;
    // shared-memory budget from the largest box; two tile buffers when they fit
    const int K1max = pad64(2 * p->box_max_x), K2max = pad64(2 * p->box_max_y), N1max = P * p->box_max_y;
    if (N1max > 256) {
        p->last_error = "tensor path: occupied grid too tall (pols x rows > 256)";
        return EPIC_ERR_UNSUPPORTED;
    }
    const size_t b1 = align_up(2ull * N1max * K1max, 1024);
    auto layout = [&](int nb, size_t* sA1, size_t* sA2, size_t* sB1, size_t* sB2) {
        size_t off = 0;
        *sA1 = off;
        off = align_up(off + 256ull * K1max, 1024);
        *sA2 = off;
        off = align_up(off + 256ull * K2max, 1024);
        *sB1 = off;
        off += nb * b1;
        *sB2 = off;
        off = align_up(off + 2ull * 64 * P * K2max, 1024);
        return off;
    };
    size_t sA1, sA2, sB1, sB2;
    const size_t limit = (size_t)p->smem_optin - 2048;
    // warp-specialised variant (64-column pairs): A1 + NB tile parts + 2 B2 buffers in shared
    // memory; 2 D1 slots + A2 + D2 in TMEM.  Each channel's box rows go in H_c parts of nyh_c
    // rows (row_parts), chosen for the largest D1 slot width D that fits both memories.
    p->tc.tbox_h.assign(C, make_int4(0, 0, 0, 0));
    p->tc.parts = false;
    p->tc.ws = false;
    for (int D = 256; D >= 16 && !p->tc.ws; D -= 16) {
        int dmax = 0, a2max = 0, nyh_max = 0;
        bool ok = true, split = false;
        std::vector<int4> tb(C);
        for (int c = 0; c < C && ok; ++c) {
            const int4 r = row_parts(p->box[c].ny, P, D);
            if (r.y == 0) ok = false;
            tb[c] = r;
            dmax = std::max(dmax, P * r.x);
            a2max = std::max(a2max, r.z);
            nyh_max = std::max(nyh_max, r.x);
            split = split || r.y > 1;
        }
        if (!ok || 2 * dmax + a2max > 256) continue;
        const size_t b1p = align_up(2ull * dmax * K1max, 1024);
        const size_t b2w = align_up(2ull * 2 * 64 * P * pad64(2 * nyh_max), 1024);
        // as many tile-part buffers (2..4) as fit: row parts are short steps, so more copies
        // must be in flight to cover their latency
        int nbt = 4;
        auto need_for = [&](int nb) { return align_up(256ull * K1max, 1024) + nb * b1p + 2 * b2w; };
        while (nbt > 2 && need_for(nbt) > limit) --nbt;
        const size_t need_ws = need_for(nbt);
        if (need_ws > limit) continue;
        p->tc.ws = true;
        p->tc.parts = split;
        p->tc.tbox_h = tb;
        p->tc.nbt = nbt;
        p->tc.sA1 = 0;
        p->tc.sB1 = (unsigned)align_up(256ull * K1max, 1024);
        p->tc.sB2 = (unsigned)(p->tc.sB1 + nbt * b1p);
        p->tc.b1_bytes = (unsigned)b1p;
        p->tc.b2_bytes = (unsigned)b2w;
        p->tc.d1_cols = dmax;
        p->tc.smem = (int)(need_ws + 1024);
    }
    if (!p->tc.ws)  // one part per channel for the other kernels' tile layout
        for (int c = 0; c < C; ++c) p->tc.tbox_h[c] = make_int4(p->box[c].ny, 1, p->box[c].ny, 0);
    // fast variant: 2 D1 slots + A2 (FP16 pairs) in TMEM columns [0, 256); 3 tiles + 2 B2 in shared memory
    {
        const int tm = 2 * N1max + p->box_max_y;  // 2 N1 + K2/2 columns
        const size_t b2 = align_up(2ull * 64 * P * K2max, 1024);
        const size_t need_fast = align_up(256ull * K1max, 1024) + 3 * b1 + 2 * b2;
        p->tc.fast = !p->tc.ws && tm <= 256 && need_fast <= limit;
        if (p->tc.fast) {
            p->tc.sA1 = 0;
            p->tc.sB1 = (unsigned)align_up(256ull * K1max, 1024);
            p->tc.sB2 = (unsigned)(p->tc.sB1 + 3 * b1);
            p->tc.b1_bytes = (unsigned)b1;
            p->tc.b2_bytes = (unsigned)b2;
            p->tc.d1_cols = N1max;
            p->tc.smem = (int)std::max<size_t>(need_fast + 1024, 120 * 1024);
        }
    }
    int nb = 2;
    size_t need = layout(2, &sA1, &sA2, &sB1, &sB2);
    if (need > limit) {
        nb = 1;
        need = layout(1, &sA1, &sA2, &sB1, &sB2);
    }
    if (need > limit) {
        p->last_error = "tensor path: occupied grid too large for shared memory";
        return EPIC_ERR_UNSUPPORTED;
    }
    // +1 KB to align the operand base at run time; at least 120 KB so that one CTA
    // per SM owns all 512 TMEM columns
    const size_t smem = std::max<size_t>(need + 1024, 120 * 1024);
    if (!p->tc.fast && !p->tc.ws) {
        p->tc.smem = (int)smem;
        p->tc.sA1 = (unsigned)sA1;
        p->tc.sA2 = (unsigned)sA2;
        p->tc.sB1 = (unsigned)sB1;
        p->tc.sB2 = (unsigned)sB2;
        p->tc.b1_bytes = (unsigned)b1;
    }
    p->tc.nb = nb;
    p->tc.n_g = n_s;
    p->tc.n_kb = n_kb;
    p->tc.n_s = n_s;

    // DFT operand tables in the K-major core-matrix layout (FP64 -> FP16).
    // A1 per (channel, 32-column slab s): rows 0..31 re, 32..63 im of kx = 32 s + j.
    std::vector<long long> a1_off((size_t)C * n_s), a2_off((size_t)C * n_kb);
    size_t n1 = 0, n2 = 0;
    for (int c = 0; c < C; ++c) {
        for (int sl = 0; sl < n_s; ++sl) {
            a1_off[(size_t)c * n_s + sl] = (long long)n1;
            n1 += 128ull * pad64(2 * p->box[c].nx);
        }
        for (int kb = 0; kb < n_kb; ++kb) {
            a2_off[(size_t)c * n_kb + kb] = (long long)n2;
            n2 += 128ull * pad64(2 * p->box[c].ny);
        }
    }
    std::vector<uint16_t> a1(n1, 0), a2(n2, 0);
    const double kPi = 3.14159265358979323846;
    auto F = [&](long long j, long long k, double* re, double* im) {
        const double ang = 2.0 * kPi * (double)((j * k) % N) / (double)N;
        *re = cos(ang);
        *im = sin(ang);
    };
    for (int c = 0; c < C; ++c) {
        const Box b = p->box[c];
        const int K1 = 2 * b.nx, K2 = 2 * b.ny;
        for (int sl = 0; sl < n_s; ++sl) {
            uint16_t* t = &a1[a1_off[(size_t)c * n_s + sl]];
            for (int r = 0; r < 64; ++r) {
                const int q = r / 32, kx = 32 * sl + r % 32;
                if (kx >= N) continue;
                for (int k = 0; k < K1; ++k) {
                    const int x = b.x0 + (k % b.nx);
                    double fr, fi;
                    F(x, kx, &fr, &fi);
                    double v;
                    if (q == 0) v = k < b.nx ? fr : -fi;
                    else v = k < b.nx ? fi : fr;
                    t[sw_off(r, k, 128)] = f16_bits(v);
                }
            }
        }
        for (int kb = 0; kb < n_kb; ++kb) {
            uint16_t* t = &a2[a2_off[(size_t)c * n_kb + kb]];
            for (int r = 0; r < 128; ++r) {
                const int ky = 128 * kb + r;
                if (ky >= N) continue;
                for (int k = 0; k < K2; ++k) {
                    const int y = b.y0 + (k % b.ny);
                    double fr, fi;
                    F(y, ky, &fr, &fi);
                    t[sw_off(r, k, 128)] = f16_bits(k < b.ny ? fr : fi);
                }
            }
        }
    }
    // A1 per (channel, 64-column pair g): rows 0..63 re, 64..127 im of kx = 64 g + j
    const int n_gp = (N + 63) / 64;
    std::vector<long long> a1p_off((size_t)C * n_gp);
    size_t n1p = 0;
    for (int c = 0; c < C; ++c)
        for (int g = 0; g < n_gp; ++g) {
            a1p_off[(size_t)c * n_gp + g] = (long long)n1p;
            n1p += 128ull * pad64(2 * p->box[c].nx);
        }
    std::vector<uint16_t> a1p(n1p, 0);
    for (int c = 0; c < C; ++c) {
        const Box b = p->box[c];
        const int K1 = 2 * b.nx;
        for (int g = 0; g < n_gp; ++g) {
            uint16_t* t = &a1p[a1p_off[(size_t)c * n_gp + g]];
            for (int r = 0; r < 128; ++r) {
                const int q = r / 64, kx = 64 * g + r % 64;
                if (kx >= N) continue;
                for (int k = 0; k < K1; ++k) {
                    const int x = b.x0 + (k % b.nx);
                    double fr, fi;
                    F(x, kx, &fr, &fi);
                    const double v = q == 0 ? (k < b.nx ? fr : -fi) : (k < b.nx ? fi : fr);
                    t[sw_off(r, k, 128)] = f16_bits(v);
                }
            }
        }
    }
    p->tc.n_gp = n_gp;
    // row-major stage-2 operand as packed FP16 pairs (lower K in the low half) for TMEM, per
    // row part: part h of a row holds words [h nyh, (h + 1) nyh), K = (re | im) of its nyh box
    // rows; rows past the box (part padding) are zero
    std::vector<long long> a2w_off((size_t)C * n_kb);
    size_t nw = 0;
    for (int c = 0; c < C; ++c)
        for (int kb = 0; kb < n_kb; ++kb) {
            a2w_off[(size_t)c * n_kb + kb] = (long long)nw;
            nw += 128ull * p->tc.tbox_h[c].z;  // H nyh words per row
        }
    std::vector<uint32_t> a2w(nw, 0);
    for (int c = 0; c < C; ++c) {
        const Box b = p->box[c];
        const int nyh = p->tc.tbox_h[c].x, H = p->tc.tbox_h[c].y, nyt = p->tc.tbox_h[c].z;
        for (int kb = 0; kb < n_kb; ++kb) {
            uint32_t* t = &a2w[a2w_off[(size_t)c * n_kb + kb]];
            for (int r = 0; r < 128; ++r) {
                const int ky = 128 * kb + r;
                if (ky >= N) continue;
                for (int h = 0; h < H; ++h)
                    for (int j = 0; j < nyh; ++j) {
                        uint16_t hv[2];
                        for (int u = 0; u < 2; ++u) {
                            const int k = 2 * j + u;                           // K index within the part
                            const int yb = h * nyh + (k < nyh ? k : k - nyh);  // box row
                            double fr = 0.0, fi = 0.0;
                            if (yb < b.ny) F(b.y0 + yb, ky, &fr, &fi);
                            hv[u] = f16_bits(k < nyh ? fr : fi);
                        }
                        t[(size_t)r * nyt + h * nyh + j] = (uint32_t)hv[0] | ((uint32_t)hv[1] << 16);
                    }
            }
        }
    }
    cudaError_t e = cudaMalloc(&p->tc.a1, n1 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a1p, n1p * 2);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a1p, a1p.data(), n1p * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a1p_off, a1p_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a1p_off, a1p_off.data(), a1p_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2w, nw * 4);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a2w, a2w.data(), nw * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2w_off, a2w_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a2w_off, a2w_off.data(), a2w_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a1, a1.data(), n1 * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2, n2 * 2);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a2, a2.data(), n2 * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a1_off, a1_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a1_off, a1_off.data(), a1_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2_off, a2_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a2_off, a2_off.data(), a2_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.tbox, (size_t)C * sizeof(int4));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.tbox, p->tc.tbox_h.data(), (size_t)C * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !p->tc.status) e = cudaMalloc(&p->tc.status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->tc.status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(p, e, "tensor path table upload");
    p->dt.dft_bytes = (n1 + n2 + n1p) * 2 + nw * 4 +
                      (a1_off.size() + a2_off.size() + a1p_off.size() + a2w_off.size()) * sizeof(long long);

    // Work split weights of k_dftgemm_ws3's equal shares, per frame of a channel's work item:
    // a fixed epilogue 2, an epilogue 1 per row part and stage-2 work in proportion to the rows
    // (about 1000 + 1200 H + 10 H nyh SM cycles, from clock64 timelines of the kernel).
    {
        std::vector<long long> wc(C + 1, 0);
        for (int c = 0; c < C; ++c) {
            const int4 r = p->tc.tbox_h[c];
            wc[c + 1] = wc[c] + 1000 + 1200LL * r.y + 10LL * r.z;
        }
        cudaError_t ew = cudaMalloc(&p->tc.wcum, (C + 1) * sizeof(long long));
        if (ew == cudaSuccess) ew = cudaMemcpy(p->tc.wcum, wc.data(), (C + 1) * sizeof(long long), cudaMemcpyHostToDevice);
        if (ew != cudaSuccess) return cuda_fail(p, ew, "work-split weights upload");
    }

    // algorithmic work of the pruned DFT-as-GEMM per time sample (all channels, pols):
    // complex MACs  nyp*nxp*N (rows along x) + N*nyp*N (columns along y), 8 flops each
    double fl = 0.0;
    for (int c = 0; c < C; ++c) fl += 8.0 * P * ((double)p->box[c].ny * p->box[c].nx * N + (double)N * p->box[c].ny * N);
    p->tc_flops_per_sample = fl;

    // chunking: channel groups big enough to fill the GPU, time chunks whose tiles fit the budget
    size_t stride = 0;
    for (int c = 0; c < C; ++c)
        stride = std::max(stride, (size_t)P * p->tc.tbox_h[c].z * pad64(2 * p->box[c].nx) * 2);
    stride = align_up(stride, 128);
    const int per_ch = n_kb * (p->tc.ws ? n_gp : n_s);
    p->tc.cg_items = std::min(C, std::max(1, (2 * p->sm_count + per_ch - 1) / per_ch));
    p->tc.cg = p->tc.group == 1 && p->tc.ws ? C : p->tc.cg_items;
    p->tc.stride = stride;
    epic_status cst = dftgemm_set_chunk(p, kScratchBudget);
    if (cst != EPIC_OK) return cst;
    cst = upload_item_order(p);
    if (cst != EPIC_OK) return cst;

    // gridding kernel: the persistent one when the cell lists of the largest channel fit in
    // shared memory next to F frames of voltages, else the gather kernel reading them through L1
    int max_cells = 0;
    for (int c = 0; c < C; ++c) max_cells = std::max(max_cells, p->box[c].nx * p->box[c].ny);
    const int max_list = p->A * p->K * p->K;
    const bool cplx = p->gcf.kind != EPIC_GCF_GAUSSIAN;
    p->tc.grid_max_cells = max_cells;
    p->tc.grid_max_list = max_list;
    p->tc.grid_cplx = cplx;
    e = cudaSuccess;
    p->tc.grid_ps = false;
    p->tc.grid_variant = 1;
    for (int gf = 4; gf >= 1 && !p->tc.grid_ps; gf >>= 1) {
        const epic_status gst = dftgemm_grid_config(p, gf);
        if (gst == EPIC_OK) p->tc.grid_ps = true;
        else if (gst != EPIC_ERR_UNSUPPORTED) return gst;
    }
    if (!cplx) {  // per-channel task lists of non-empty cell pairs, longest list first
        std::vector<int> coff, cptr, ce;
        std::vector<float2> cw;
        build_csr(p, coff, cptr, ce, cw);
        // A task is the run of kTaskCells cells (x, x + 1, ...), x a multiple of kTaskCells,
        // of one row of a channel's box; its entries are the elements that reach any of them
        // (the union of the cells' element-ordered lists) with one weight per cell.  Runs of
        // a channel are sorted by entry count (equal counts in Morton order, so that a warp's
        // runs are near one another and share elements); groups of 32 consecutive runs (the
        // lanes of one warp) store their entries interleaved, entry k of lane l at 32 k + l,
        // padded with zero weights to the group's longest list, in the order
        // order_warp_entries picks.
        std::vector<int4> tasks;
        std::vector<int> ell_e;
        std::vector<TaskW> ell_w;
        std::vector<int> toff(C + 1, 0), eoff(C + 1, 0);
        std::vector<TaskW> pw;  // weights of the channel's run lists
        std::vector<int2> ord;
        std::vector<int> pl_ptr, pl_off(C), pl_e;  // the same lists row-major (pair-list kernel)
        std::vector<TaskW> pl_w;
        bool fits = true;
        int tmax = 0, emax = 0;
        for (int c = 0; c < C && fits; ++c) {
            toff[c] = (int)tasks.size();
            eoff[c] = (int)ell_e.size();
            const int* ptr = &cptr[coff[c]];
            const Box bx = p->box[c];
            const int hp = bx.nx / kTaskCells;  // runs per row (nx is a multiple of 8)
            std::vector<std::vector<int2>> plist((size_t)hp * bx.ny);  // (element, 1 + index into pw)
            pw.clear();
            for (int y = 0; y < bx.ny; ++y)
                for (int j = 0; j < hp; ++j) {
                    const int r0 = y * bx.nx + kTaskCells * j;
                    int at[kTaskCells];
                    for (int q = 0; q < kTaskCells; ++q) at[q] = ptr[r0 + q];
                    std::vector<int2>& L = plist[(size_t)y * hp + j];
                    for (;;) {  // merge of the cells' element-ordered lists
                        int el = INT32_MAX;
                        for (int q = 0; q < kTaskCells; ++q)
                            if (at[q] < ptr[r0 + q + 1]) el = std::min(el, ce[at[q]]);
                        if (el == INT32_MAX) break;
                        float wq[4] = {0.f, 0.f, 0.f, 0.f};
                        for (int q = 0; q < kTaskCells; ++q)
                            if (at[q] < ptr[r0 + q + 1] && ce[at[q]] == el) wq[q] = cw[at[q]++].x;
                        TaskW w;
                        task_w_set(w, wq);
                        pw.push_back(w);
                        L.push_back(make_int2(el, (int)pw.size()));
                    }
                }
            pl_off[c] = (int)pl_ptr.size();
            for (const std::vector<int2>& L : plist) {
                pl_ptr.push_back((int)pl_e.size());
                for (const int2& en : L) {
                    pl_e.push_back(en.x);
                    pl_w.push_back(pw[en.y - 1]);
                }
            }
            pl_ptr.push_back((int)pl_e.size());
            std::vector<int> idx;
            for (int q = 0; q < hp * bx.ny; ++q)
                if (!plist[q].empty()) idx.push_back(q);
            auto morton = [hp](int q) {
                const unsigned x = (unsigned)(kTaskCells * (q % hp)), y = (unsigned)(q / hp);
                unsigned m = 0;
                for (int bit = 0; bit < 12; ++bit) m |= ((x >> bit) & 1u) << (2 * bit) | ((y >> bit) & 1u) << (2 * bit + 1);
                return m;
            };
            std::stable_sort(idx.begin(), idx.end(), [&](int u, int v) {
                const size_t nu = plist[u].size(), nv = plist[v].size();
                return nu != nv ? nu > nv : morton(u) < morton(v);
            });
            const int nyh = p->tc.tbox_h[c].x;
            const uint32_t part_bytes = (uint32_t)(p->P * nyh) * pad64(2 * bx.nx) * 2;
            std::vector<std::vector<int4>> gtasks;  // the 32 tasks of each group (padding tasks: no store)
            std::vector<int> gcost;
            for (size_t g0 = 0; g0 < idx.size(); g0 += 32) {
                const int members = (int)std::min<size_t>(32, idx.size() - g0);
                const int nmax = (int)plist[idx[g0]].size();
                const int base = (int)ell_e.size() - eoff[c];
                if (nmax > 255) fits = false;
                std::vector<std::vector<int2>> lists(members);
                for (int l = 0; l < members; ++l) lists[l] = plist[idx[g0 + l]];
                ord.assign(32ull * nmax, make_int2(0, 0));
                order_warp_entries(lists, nmax, ord.data());
                for (const int2& en : ord) {
                    ell_e.push_back(en.x);
                    ell_w.push_back(en.y > 0 ? pw[en.y - 1] : TaskW{});
                }
                std::vector<int4> gt(32, make_int4(nmax << 24, base, -1, -1));
                for (int l = 0; l < members; ++l) {
                    const int q = idx[g0 + l];
                    if (q >= (1 << 24)) fits = false;
                    const int y = q / hp, x = kTaskCells * (q % hp);
                    gt[l] = make_int4(q | (nmax << 24), base, (int)tile_part_off(y, x, nyh, p->P, part_bytes),
                                      (int)tile_part_off(y, bx.nx + x, nyh, p->P, part_bytes));
                }
                gtasks.push_back(gt);
                gcost.push_back(nmax + 1);  // list steps + the tile stores
            }
            // Warp w of the kernel takes groups w, w + W, w + 2 W, ... of the task list (W
            // gridding warps) and a pass ends when its slowest warp does, so the groups are
            // dealt out longest first to the least-loaded warp and laid out in that order;
            // positions a warp does not use hold groups of padding tasks (no entries, no store).
            const int W = kGridBalThreads / 32;
            std::vector<std::vector<int>> wl(W);
            std::vector<long long> load(W, 0);
            for (int g = 0; g < (int)gtasks.size(); ++g) {  // groups are in decreasing cost order
                int w = 0;
                for (int v = 1; v < W; ++v)
                    if (load[v] < load[w]) w = v;
                wl[w].push_back(g);
                load[w] += gcost[g];
            }
            size_t rounds = 0;
            for (const auto& l : wl) rounds = std::max(rounds, l.size());
            const std::vector<int4> pad(32, make_int4(0, 0, -1, -1));
            for (size_t j = 0; j < rounds; ++j)
                for (int w = 0; w < W; ++w) {
                    const std::vector<int4>& gt = j < wl[w].size() ? gtasks[wl[w][j]] : pad;
                    tasks.insert(tasks.end(), gt.begin(), gt.end());
                }
            tmax = std::max(tmax, (int)(tasks.size() - toff[c]));
            emax = std::max(emax, (int)ell_e.size() - eoff[c]);
        }
        toff[C] = (int)tasks.size();
        eoff[C] = (int)ell_e.size();
        for (int c = 0; c < C; ++c) {  // largest offsets / entries of a channel (staged lists)
            const int np = p->box[c].ny * (p->box[c].nx / kTaskCells) + 1;
            p->tc.pl_max_ptr = std::max(p->tc.pl_max_ptr, np);
            p->tc.pl_max_ent = std::max(p->tc.pl_max_ent, pl_ptr[pl_off[c] + np - 1] - pl_ptr[pl_off[c]]);
        }
        if (kTaskCells == 2 && !pl_e.empty() && pl_e.size() < (1u << 31)) {  // pair lists for k_dftgemm_grid_pl
            e = cudaMalloc(&p->tc.pl_ptr, pl_ptr.size() * sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemcpy(p->tc.pl_ptr, pl_ptr.data(), pl_ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.pl_off, pl_off.size() * sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemcpy(p->tc.pl_off, pl_off.data(), pl_off.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.pl_e, pl_e.size() * sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemcpy(p->tc.pl_e, pl_e.data(), pl_e.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.pl_w, pl_w.size() * sizeof(float2));
            if (e == cudaSuccess)
                e = cudaMemcpy(p->tc.pl_w, pl_w.data(), pl_w.size() * sizeof(float2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(p, e, "pair-list upload");
            p->dt.dft_bytes += (pl_ptr.size() + pl_off.size() + pl_e.size()) * sizeof(int) + pl_w.size() * sizeof(float2);
        }
        if (fits && !tasks.empty()) {
            e = cudaMalloc(&p->tc.gtask, tasks.size() * sizeof(int4));
            if (e == cudaSuccess) e = cudaMemcpy(p->tc.gtask, tasks.data(), tasks.size() * sizeof(int4),
                                                 cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.gtask_off, toff.size() * sizeof(int));
            if (e == cudaSuccess) e = cudaMemcpy(p->tc.gtask_off, toff.data(), toff.size() * sizeof(int),
                                                 cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.gell_e, ell_e.size() * sizeof(int));
            if (e == cudaSuccess) e = cudaMemcpy(p->tc.gell_e, ell_e.data(), ell_e.size() * sizeof(int),
                                                 cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.gell_w, ell_w.size() * sizeof(TaskW));
            if (e == cudaSuccess) e = cudaMemcpy(p->tc.gell_w, ell_w.data(), ell_w.size() * sizeof(TaskW),
                                                 cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&p->tc.gell_off, eoff.size() * sizeof(int));
            if (e == cudaSuccess) e = cudaMemcpy(p->tc.gell_off, eoff.data(), eoff.size() * sizeof(int),
                                                 cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(p, e, "gridding task lists upload");
            p->tc.gtask_max = tmax;
            p->tc.gell_max = emax;
            const int keep_f = p->tc.grid_frames;
            p->tc.grid_variant = 2;
            epic_status bst = EPIC_ERR_UNSUPPORTED;
            for (int gf = 2; gf >= 1 && bst == EPIC_ERR_UNSUPPORTED; gf >>= 1) bst = grid_bal_config(p, gf);
            if (bst != EPIC_OK) {  // the balanced kernel does not fit: the pair-list one, else row-major
                if (bst != EPIC_ERR_UNSUPPORTED) return bst;
                p->tc.grid_variant = 1;
                cudaFree(p->tc.gtask);
                cudaFree(p->tc.gtask_off);
                cudaFree(p->tc.gell_e);
                cudaFree(p->tc.gell_w);
                cudaFree(p->tc.gell_off);
                p->tc.gtask = nullptr;
                p->tc.gtask_off = nullptr;
                p->tc.gell_e = nullptr;
                p->tc.gell_w = nullptr;
                p->tc.gell_off = nullptr;
                p->tc.gtask_max = 0;
                if (p->tc.grid_ps) {
                    const epic_status kst = dftgemm_grid_config(p, keep_f);
                    if (kst != EPIC_OK) return kst;
                }
                if (p->tc.pl_ptr) {
                    p->tc.grid_variant = 3;
                    epic_status pst = EPIC_ERR_UNSUPPORTED;
                    for (int gf = 4; gf >= 1 && pst == EPIC_ERR_UNSUPPORTED; gf >>= 1) pst = grid_pl_config(p, gf);
                    if (pst != EPIC_OK) {
                        if (pst != EPIC_ERR_UNSUPPORTED) return pst;
                        p->tc.grid_variant = 1;
                        if (p->tc.grid_ps) {
                            const epic_status kst = dftgemm_grid_config(p, keep_f);
                            if (kst != EPIC_OK) return kst;
                        }
                    }
                }
            } else {
                p->dt.dft_bytes += tasks.size() * sizeof(int4) + ell_e.size() * (sizeof(int) + sizeof(TaskW)) +
                                   (toff.size() + eoff.size()) * sizeof(int);
            }
        }
    }
    const size_t max_list_l = (size_t)max_list;
    const size_t csr_bytes = sizeof(int) * (size_t)((max_cells + 2) & ~1) + sizeof(int2) * max_list_l;
    const size_t gl = (size_t)p->smem_optin;
    int gf = 4;
    while (gf > 1 && sizeof(float4) * (size_t)gf * p->A > gl / 2) gf >>= 1;
    size_t sv_bytes = sizeof(float4) * (size_t)gf * p->A;
    p->tc.grid_csr_smem = !cplx && sv_bytes + csr_bytes <= gl;
    if (!p->tc.grid_csr_smem) {
        while (gf > 1 && sizeof(float4) * (size_t)gf * p->A > gl) gf >>= 1;
        sv_bytes = sizeof(float4) * (size_t)gf * p->A;
    }
    if (!p->tc.grid_ps && p->tc.grid_variant == 1) {  // only the gather kernel is left: its frames and memory
        p->tc.grid_frames = gf;
        p->tc.grid_smem = (int)(sv_bytes + (p->tc.grid_csr_smem ? csr_bytes : 0));
        if (p->tc.grid_smem > p->smem_optin) {
            p->last_error = "tensor path: frame of A*P voltages does not fit in shared memory";
            return EPIC_ERR_UNSUPPORTED;
        }
    }
#define EPIC_GRID_ATTR(CS, FF)                                                                                      \
    if (e == cudaSuccess)                                                                                           \
        e = allow_max_smem((const void*)k_dftgemm_grid<CS, FF>, p->smem_optin);
    e = cudaSuccess;
    EPIC_GRID_ATTR(true, 4)
    EPIC_GRID_ATTR(true, 2)
    EPIC_GRID_ATTR(true, 1)
    EPIC_GRID_ATTR(false, 4)
    EPIC_GRID_ATTR(false, 2)
    EPIC_GRID_ATTR(false, 1)
#undef EPIC_GRID_ATTR
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_grid)");
    e = allow_max_smem((const void*)k_dftgemm_ws<0>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws2<0>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<0, false>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<1, false>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<2, false>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<0, true>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<1, true>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_ws3<2, true>, p->smem_optin);
    p->tc.ws_variant = p->tc.ws ? 3 : 0;
    if (p->tc.ws && p->sm_count > kWs3MaxBlocks) p->tc.ws_variant = 1;
    if (p->tc.parts && p->tc.ws_variant != 3) {
        p->last_error = "tensor path: an occupied grid this tall needs the control-warp kernel";
        return EPIC_ERR_UNSUPPORTED;
    }
    if (p->sub > 0 && p->tc.ws_variant != 3) {
        p->last_error = "tensor path: sub-integrations need a control-warp kernel (occupied grid too large)";
        return EPIC_ERR_UNSUPPORTED;
    }
    if (p->tc.ws && e == cudaSuccess) {
        const size_t n_items = (size_t)C * n_kb * n_gp;  // the largest channel group
        e = cudaMalloc(&p->tc.partial, (size_t)p->sm_count * 2 * 4 * 8192 * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&p->tc.counters, n_items * sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->tc.counters, 0, n_items * sizeof(int));
        if (e == cudaSuccess) p->tc.n_counters = n_items;
        if (e == cudaSuccess)
            p->dt.dft_bytes += (size_t)p->sm_count * 2 * 4 * 8192 * sizeof(float) + n_items * sizeof(int);
    }
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_mma_fast<0>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_mma<1>, p->smem_optin);
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_dftgemm_mma<2>, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_mma)");
    return EPIC_OK;
}

epic_status dftgemm_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate,
                        const GroupHooks* hooks)
{
    const int C = p->C, P = p->P, A = p->A;
    MmaArgs a{};
    a.tiles = (const uint8_t*)p->scratch;
    a.tile_stride = p->tc.stride;
    a.n_kb = p->tc.n_kb;
    a.n_s = p->tc.n_s;
    a.n_g = p->tc.n_g;
    a.N = p->N;
    a.P = P;
    a.nprod = p->nprod;
    a.box = p->dt.box;
    a.a1 = p->tc.a1;
    a.a2 = p->tc.a2;
    a.a1_off = p->tc.a1_off;
    a.a2_off = p->tc.a2_off;
    a.out = out;
    a.status = p->tc.status;
    a.sA1 = p->tc.sA1;
    a.sA2 = p->tc.sA2;
    a.sB1 = p->tc.sB1;
    a.sB2 = p->tc.sB2;
    a.b1_bytes = p->tc.b1_bytes;
    a.a2w = p->tc.a2w;
    a.a2w_off = p->tc.a2w_off;
    a.b2_bytes = p->tc.b2_bytes;
    a.d1_cols = p->tc.d1_cols;
    a.a1p = p->tc.a1p;
    a.a1p_off = p->tc.a1p_off;
    a.tbox = p->tc.tbox;
    a.nbt = p->tc.nbt;
    a.wcum = p->tc.wcum;
    a.item_order = p->tc.item_order;
    const int fpc = kGridFramesPerBlock;
    const int F = p->tc.grid_frames;
    for (int c0 = 0; c0 < C; c0 += p->tc.cg) {
        const int ng = std::min(p->tc.cg, C - c0);
        if (hooks && hooks->before) {
            const epic_status hs = hooks->before(c0, ng);
            if (hs != EPIC_OK) return hs;
        }
        for (int t0 = 0; t0 < T; t0 += p->tc.tc) {
            const int nt = std::min(p->tc.tc, T - t0);
            const dim3 gg((nt + fpc - 1) / fpc, ng);
            if (p->tc.grid_ps || p->tc.grid_variant >= 2) {
                // the launch's shared memory must be the chosen kernel's layout for F frames
                const int fb = A * P * (p->bits / 4);
                const size_t need = p->tc.grid_variant == 3 ? grid_pl_smem(F, A, fb, p->jones.empty(), p->tc.pl_stage,
                                                                             p->tc.pl_max_ptr, p->tc.pl_max_ent)
                                  : p->tc.grid_variant == 2
                                      ? grid_bal_smem(F, A, fb, p->tc.gtask_max, p->tc.gell_max, (unsigned)p->tc.stride)
                                      : grid_ps_smem(F, A, fb, p->tc.grid_max_cells, p->tc.grid_max_list, p->tc.grid_cplx);
                if (need != (size_t)p->tc.grid_smem) {
                    p->last_error = "tensor path: gridding kernel configuration out of step (internal)";
                    return EPIC_ERR_CUDA;
                }
                GridArgs g{};
                g.volt = volt;
                g.t0 = t0;
                g.c0 = c0;
                g.n_ch = ng;
                g.nt = nt;
                g.C = C;
                g.A = A;
                g.P = P;
                g.box = p->dt.box;
                g.cell_off = p->dt.cell_off;
                g.cell_ptr = p->dt.cell_ptr;
                g.ce = p->dt.contrib_e;
                g.cw = p->dt.contrib_w;
                g.tiles = (uint8_t*)p->scratch;
                g.tile_stride = p->tc.stride;
                g.status = p->tc.status;
                g.max_cells = p->tc.grid_max_cells;
                g.max_list = p->tc.grid_max_list;
                g.bits = p->bits;
                g.jones = p->dt.jones;
                g.tbox = p->tc.tbox;
                g.bulk = ((A * P * (p->bits / 4)) % 16 == 0 && ((uintptr_t)volt & 15) == 0) ? 1 : 0;
                const int gb = (int)std::min<long long>(p->tc.grid_blocks, (long long)ng * nt);
                ev_begin(p, "k_dftgemm_grid", s);
                if (p->tc.grid_variant == 3) {
                    GridPlArgs pa{};
                    pa.g = g;
                    pa.pl_ptr = p->tc.pl_ptr;
                    pa.pl_off = p->tc.pl_off;
                    pa.pl_e = p->tc.pl_e;
                    pa.pl_w = reinterpret_cast<const float2*>(p->tc.pl_w);
                    pa.max_ptr = p->tc.pl_max_ptr;
                    pa.max_ent = p->tc.pl_max_ent;
                    const size_t sm = p->tc.grid_smem;
#define EPIC_PL_LAUNCH(FF, HH, SS) k_dftgemm_grid_pl<FF, HH, SS><<<gb, kGridPlThreads, sm, s>>>(pa)
#define EPIC_PL_F(HH, SS)                       \
    if (F == 8) EPIC_PL_LAUNCH(8, HH, SS);      \
    else if (F == 4) EPIC_PL_LAUNCH(4, HH, SS); \
    else if (F == 2) EPIC_PL_LAUNCH(2, HH, SS); \
    else EPIC_PL_LAUNCH(1, HH, SS);
                    if (p->jones.empty()) {
                        if (p->tc.pl_stage) { EPIC_PL_F(true, true) } else { EPIC_PL_F(true, false) }
                    } else {
                        if (p->tc.pl_stage) { EPIC_PL_F(false, true) } else { EPIC_PL_F(false, false) }
                    }
#undef EPIC_PL_F
#undef EPIC_PL_LAUNCH
                } else if (p->tc.grid_variant == 2) {
                    GridBalArgs ba{};
                    ba.g = g;
                    ba.tasks = p->tc.gtask;
                    ba.task_off = p->tc.gtask_off;
                    ba.ell_e = p->tc.gell_e;
                    ba.ell_w = reinterpret_cast<const TaskW*>(p->tc.gell_w);
                    ba.ell_off = p->tc.gell_off;
                    ba.max_tasks = p->tc.gtask_max;
                    ba.max_ell = p->tc.gell_max;
                    ba.tile_max = (unsigned)p->tc.stride;
                    const size_t sm = p->tc.grid_smem;
                    if (p->jones.empty()) {  // FP16-pair voltages (exact for unmixed samples)
                        if (F == 4) k_dftgemm_grid_bal<4, true><<<gb, kGridBalBlock, sm, s>>>(ba);
                        else if (F == 2) k_dftgemm_grid_bal<2, true><<<gb, kGridBalBlock, sm, s>>>(ba);
                        else k_dftgemm_grid_bal<1, true><<<gb, kGridBalBlock, sm, s>>>(ba);
                    } else {
                        if (F == 4) k_dftgemm_grid_bal<4, false><<<gb, kGridBalBlock, sm, s>>>(ba);
                        else if (F == 2) k_dftgemm_grid_bal<2, false><<<gb, kGridBalBlock, sm, s>>>(ba);
                        else k_dftgemm_grid_bal<1, false><<<gb, kGridBalBlock, sm, s>>>(ba);
                    }
                } else {
#define EPIC_GRID_PS_LAUNCH(CX, FF) k_dftgemm_grid_ps<CX, FF><<<gb, kThreads, p->tc.grid_smem, s>>>(g)
                if (p->tc.grid_cplx) {
                    if (F == 8) EPIC_GRID_PS_LAUNCH(true, 8);
                    else if (F == 4) EPIC_GRID_PS_LAUNCH(true, 4);
                    else if (F == 2) EPIC_GRID_PS_LAUNCH(true, 2);
                    else EPIC_GRID_PS_LAUNCH(true, 1);
                } else {
                    if (F == 8) EPIC_GRID_PS_LAUNCH(false, 8);
                    else if (F == 4) EPIC_GRID_PS_LAUNCH(false, 4);
                    else if (F == 2) EPIC_GRID_PS_LAUNCH(false, 2);
                    else EPIC_GRID_PS_LAUNCH(false, 1);
                }
                }
#undef EPIC_GRID_PS_LAUNCH
                ev_end(p, s);
            } else {
            ev_begin(p, "k_dftgemm_grid", s);
#define EPIC_GRID_LAUNCH(CS, FF)                                                                                    \
    k_dftgemm_grid<CS, FF><<<gg, kThreads, p->tc.grid_smem, s>>>(volt, t0, c0, ng, nt, fpc, C, A, P, p->bits,         \
                                                              p->dt.box,                                               \
                                                              p->dt.cell_off, p->dt.cell_ptr, p->dt.contrib_e,         \
                                                              p->dt.contrib_w, p->dt.jones, p->tc.tbox,                \
                                                              (uint8_t*)p->scratch,                                    \
                                                              p->tc.stride)
            if (p->tc.grid_csr_smem) {
                if (F == 4) EPIC_GRID_LAUNCH(true, 4);
                else if (F == 2) EPIC_GRID_LAUNCH(true, 2);
                else EPIC_GRID_LAUNCH(true, 1);
            } else {
                if (F == 4) EPIC_GRID_LAUNCH(false, 4);
                else if (F == 2) EPIC_GRID_LAUNCH(false, 2);
                else EPIC_GRID_LAUNCH(false, 1);
            }
#undef EPIC_GRID_LAUNCH
            ev_end(p, s);
            }
            a.c0 = c0;
            a.n_ch = ng;
            a.nt = nt;
            a.accumulate = (accumulate || (t0 > 0 && p->sub == 0)) ? 1 : 0;
            a.sub = p->sub;
            a.iv0 = p->sub > 0 ? t0 / p->sub : 0;
            a.C = C;
            const int items = ng * a.n_kb * (p->tc.ws ? p->tc.n_gp : a.n_s);
            const int grid = std::min(items, p->sm_count);
            ev_begin(p, p->tc.ws ? (p->tc.ws_variant == 3 ? "k_dftgemm_ws3" : p->tc.ws_variant == 2 ? "k_dftgemm_ws2" : "k_dftgemm_ws")
                                 : p->tc.fast ? "k_dftgemm_mma_fast" : "k_dftgemm_mma", s);
            if (p->tc.ws) {
                a.n_g = p->tc.n_gp;
                if (p->tc.ws_variant == 3) {
                    a.partial = p->tc.partial;
                    a.counters = p->tc.counters;
                    if (p->sub > 0)
                        p->tc.parts ? k_dftgemm_ws3<2, true><<<grid, kWs3Threads, p->tc.smem, s>>>(a)
                                    : k_dftgemm_ws3<2, false><<<grid, kWs3Threads, p->tc.smem, s>>>(a);
                    else if (p->tc.split == 1 || (p->tc.split < 0 && items % p->sm_count != 0))
                        p->tc.parts ? k_dftgemm_ws3<1, true><<<p->sm_count, kWs3Threads, p->tc.smem, s>>>(a)
                                    : k_dftgemm_ws3<1, false><<<p->sm_count, kWs3Threads, p->tc.smem, s>>>(a);
                    else
                        p->tc.parts ? k_dftgemm_ws3<0, true><<<grid, kWs3Threads, p->tc.smem, s>>>(a)
                                    : k_dftgemm_ws3<0, false><<<grid, kWs3Threads, p->tc.smem, s>>>(a);
                }
                else if (p->tc.ws_variant == 2) k_dftgemm_ws2<0><<<grid, kWs2Threads, p->tc.smem, s>>>(a);
                else k_dftgemm_ws<0><<<grid, kWsThreads, p->tc.smem, s>>>(a);
            } else if (p->tc.fast) k_dftgemm_mma_fast<0><<<grid, kMmaThreads, p->tc.smem, s>>>(a);
            else if (p->tc.nb == 2) k_dftgemm_mma<2><<<grid, kMmaThreads, p->tc.smem, s>>>(a);
            else k_dftgemm_mma<1><<<grid, kMmaThreads, p->tc.smem, s>>>(a);
            ev_end(p, s);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(p, e, "tensor path launch");
        }
        if (hooks && hooks->after) {
            const epic_status hs = hooks->after(c0, ng);
            if (hs != EPIC_OK) return hs;
        }
    }
    return EPIC_OK;
}

}  // namespace epic
