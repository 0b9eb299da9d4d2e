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
// Work item = (channel, block of 128 ky, slab of 32 kx); the XX, YY, Re/Im XY
// sums of its 128 x 32 pixels stay in registers over every frame of a chunk.
//
// Two kernels per (channel group, time chunk), stream-ordered, with the grid
// tiles staying in L2 between them:
//   k_dftgemm_grid  gather-grid every (t, c) frame of the chunk into an FP16
//                   tile already in the UMMA K-major core-matrix layout
//   k_dftgemm_mma   stage 1 -> TMEM -> FP16 shared B2 -> stage 2 -> TMEM ->
//                   products -> register accumulation; images written (or
//                   added) once per chunk
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <cstring>

#include "epic_internal.h"
#include "kcommon.cuh"
#include "tc_ptx.cuh"

namespace epic {

namespace {

constexpr int kThreads = 256;
constexpr size_t kScratchBudget = 96ull << 20;  // grid tiles of one (channel group, time chunk)
constexpr long long kWaitBudget = 4000000000LL;  // clock cycles before a wait gives up (~2 s)

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

// element offset (in halves) of (row r, column k) in a [R][Kd] K-major core-matrix tile
inline size_t core_off(int r, int k, int Kd) { return ((size_t)(r >> 3) * (Kd >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

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
};

__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ bool wait_uniform(uint64_t* bar, uint32_t parity)
{
    const bool ok = tc::mbar_wait(bar, parity, kWaitBudget);
    return __syncthreads_and(ok) != 0;
}

// Eight grid cells (x8*8 .. x8*8+7) of tile row R as two 16-byte core-matrix rows:
// real parts at K chunk x8, imaginary parts at K chunk nxp/8 + x8.
__device__ __forceinline__ void store_tile_row(uint8_t* tile, int R, int K1, int nxp, int x8, const float2 (&g)[8])
{
    uint8_t* row = tile + ((size_t)(R >> 3) * (K1 >> 3)) * 128 + (R & 7) * 16;
    uint4 re, im;
    re.x = pack_h2(g[0].x, g[1].x);
    re.y = pack_h2(g[2].x, g[3].x);
    re.z = pack_h2(g[4].x, g[5].x);
    re.w = pack_h2(g[6].x, g[7].x);
    im.x = pack_h2(g[0].y, g[1].y);
    im.y = pack_h2(g[2].y, g[3].y);
    im.z = pack_h2(g[4].y, g[5].y);
    im.w = pack_h2(g[6].y, g[7].y);
    *reinterpret_cast<uint4*>(row + (size_t)x8 * 128) = re;
    *reinterpret_cast<uint4*>(row + (size_t)((nxp >> 3) + x8) * 128) = im;
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

// Unpack and gather-grid the frames of one chunk into FP16 UMMA tiles.
__global__ void __launch_bounds__(kThreads) k_dftgemm_grid(const uint8_t* __restrict__ volt, int t0, int c0,
                                                           int n_ch, int C, int A, int P,
                                                           const int4* __restrict__ box,
                                                           const int* __restrict__ cell_off,
                                                           const int* __restrict__ cell_ptr,
                                                           const int* __restrict__ ce,
                                                           const float2* __restrict__ cw, uint8_t* __restrict__ tiles,
                                                           unsigned long long tile_stride)
{
    extern __shared__ float2 sv[];  // [A][P]
    const int tl = blockIdx.x, cl = blockIdx.y, c = c0 + cl;
    const uint8_t* fr = volt + ((size_t)(t0 + tl) * C + c) * (size_t)A * P;
    for (int i = threadIdx.x; i < A * P; i += blockDim.x) sv[i] = unpack44(fr[i]);
    __syncthreads();
    const int4 b = box[c];
    const int nxp = b.z, nyp = b.w, K1 = 2 * nxp;
    const int* ptr = cell_ptr + cell_off[c];
    uint8_t* tile = tiles + ((size_t)tl * n_ch + cl) * tile_stride;
    const int tasks = nyp * (nxp >> 3);
    for (int task = threadIdx.x; task < tasks; task += blockDim.x) {
        const int y = task % nyp, x8 = task / nyp;
        const int r0 = y * nxp + x8 * 8;
        float2 gx[8], gy[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            gx[i] = make_float2(0.f, 0.f);
            gy[i] = make_float2(0.f, 0.f);
            const int q1 = ptr[r0 + i + 1];
            for (int q = ptr[r0 + i]; q < q1; ++q) {
                const int e = ce[q];
                const float2 w = cw[q];
                gx[i] = cfma(w, sv[e * P], gx[i]);
                if (P == 2) gy[i] = cfma(w, sv[e * P + 1], gy[i]);
            }
        }
        store_tile_row(tile, 0 * nyp + y, K1, nxp, x8, gx);
        if (P == 2) store_tile_row(tile, 1 * nyp + y, K1, nxp, x8, gy);
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

// Stage 1 + stage 2 + products + accumulation for the work items of one chunk.
__global__ void __launch_bounds__(kThreads, 1) k_dftgemm_mma(MmaArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_mma, bar_tma;
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_sh, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_init(&bar_tma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_sh;
    uint8_t* sA1 = smem + a.sA1;
    uint8_t* sA2 = smem + a.sA2;
    uint8_t* sB1 = smem + a.sB1;
    uint8_t* sB2 = smem + a.sB2;
    uint32_t ph_mma = 0, ph_tma = 0;
    bool ok = true;
    const int items = a.n_ch * a.n_kb * a.n_s;
    const int q4 = warp & 3, hc = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;

    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int s = item % a.n_s, kb = (item / a.n_s) % a.n_kb, cl = item / (a.n_s * a.n_kb);
        const int c = a.c0 + cl;
        const int4 bx = a.box[c];
        const int nxp = bx.z, nyp = bx.w;
        const int K1 = 2 * nxp, K2 = 2 * nyp, N1 = a.P * nyp;
        const int g = s >> 1, h = s & 1;
        const uint32_t a1_bytes = 256u * K1, a2_bytes = 256u * K2;
        const uint32_t tile_bytes = (uint32_t)N1 * K1 * 2;
        if (tid == 0) {
            tc::mbar_expect_tx(&bar_tma, a1_bytes + a2_bytes);
            tc::bulk_g2s(sA1, a.a1 + a.a1_off[(size_t)c * a.n_g + g], a1_bytes, &bar_tma);
            tc::bulk_g2s(sA2, a.a2 + a.a2_off[(size_t)c * a.n_kb + kb], a2_bytes, &bar_tma);
        }
        ok = wait_uniform(&bar_tma, ph_tma);
        ph_tma ^= 1;

        float axx[16], ayy[16], arx[16], aix[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;

        const uint32_t sbo1 = (uint32_t)(K1 / 8) * 128, sbo2 = (uint32_t)(K2 / 8) * 128;
        for (int t = 0; ok && t < a.nt; ++t) {
            // ---- grid tile of (t, c) -> shared memory
            if (tid == 0) {
                tc::mbar_expect_tx(&bar_tma, tile_bytes);
                tc::bulk_g2s(sB1, a.tiles + ((size_t)t * a.n_ch + cl) * a.tile_stride, tile_bytes, &bar_tma);
            }
            ok = wait_uniform(&bar_tma, ph_tma);
            ph_tma ^= 1;
            if (!ok) break;
            // ---- stage 1: D1 = A1 . B1^T  (M = 128, N = N1, K = K1)
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t ia = tc::smem_u32(sA1), ib = tc::smem_u32(sB1);
                const uint32_t id1 = tc::idesc_f16_f32(128, N1);
                for (int k = 0; k < K1 / 16; ++k)
                    tc::mma_f16(tmem, tc::smem_desc(ia + k * 256, 128, sbo1), tc::smem_desc(ib + k * 256, 128, sbo1),
                                id1, k > 0);
                tc::mma_commit(&bar_mma);
            }
            ok = wait_uniform(&bar_mma, ph_mma);
            ph_mma ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
            // ---- epilogue 1: H of this slab (lanes 32h.. re, 64+32h.. im) -> FP16 B2_p
            if (warp == h || warp == 2 + h) {
                const bool imw = warp >= 2;
                for (int p = 0; p < a.P; ++p) {
                    uint8_t* b2 = sB2 + (size_t)p * 64 * K2 * 2;
                    for (int yc = 0; yc < nyp / 8; ++yc) {
                        uint32_t r[8];
                        tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + p * nyp + yc * 8, r);
                        tc::tmem_wait_ld(r);
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
                        uint4 pos, neg;
                        pos.x = pack_h2(v[0], v[1]);
                        pos.y = pack_h2(v[2], v[3]);
                        pos.z = pack_h2(v[4], v[5]);
                        pos.w = pack_h2(v[6], v[7]);
                        neg.x = pack_h2(-v[0], -v[1]);
                        neg.y = pack_h2(-v[2], -v[3]);
                        neg.z = pack_h2(-v[4], -v[5]);
                        neg.w = pack_h2(-v[6], -v[7]);
                        const int n0 = lane, n1 = 32 + lane;
                        uint8_t* row0 = b2 + ((size_t)(n0 >> 3) * (K2 >> 3)) * 128 + (n0 & 7) * 16;
                        uint8_t* row1 = b2 + ((size_t)(n1 >> 3) * (K2 >> 3)) * 128 + (n1 & 7) * 16;
                        const int kc_lo = yc, kc_hi = (nyp >> 3) + yc;
                        if (!imw) {  // Hr: B2[kx][y] and B2[32+kx][nyp+y]
                            *reinterpret_cast<uint4*>(row0 + (size_t)kc_lo * 128) = pos;
                            *reinterpret_cast<uint4*>(row1 + (size_t)kc_hi * 128) = pos;
                        } else {     // Hi: B2[kx][nyp+y] = -Hi, B2[32+kx][y] = Hi
                            *reinterpret_cast<uint4*>(row0 + (size_t)kc_hi * 128) = neg;
                            *reinterpret_cast<uint4*>(row1 + (size_t)kc_lo * 128) = pos;
                        }
                    }
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            // ---- stage 2: D2_p = A2 . B2_p^T  (M = 128, N = 64, K = K2), TMEM columns 256 + 64 p
            if (tid == 0) {
                const uint32_t ia = tc::smem_u32(sA2);
                const uint32_t id2 = tc::idesc_f16_f32(128, 64);
                for (int p = 0; p < a.P; ++p) {
                    const uint32_t ib = tc::smem_u32(sB2) + (uint32_t)p * 64 * K2 * 2;
                    for (int k = 0; k < K2 / 16; ++k)
                        tc::mma_f16(tmem + 256 + 64 * p, tc::smem_desc(ia + k * 256, 128, sbo2),
                                    tc::smem_desc(ib + k * 256, 128, sbo2), id2, k > 0);
                }
                tc::mma_commit(&bar_mma);
            }
            ok = wait_uniform(&bar_mma, ph_mma);
            ph_mma ^= 1;
            if (!ok) break;
            tc::fence_after_sync();
            // ---- epilogue 2: products and accumulation (row ky = 32 q4 + lane, 16 kx per thread)
            {
                uint32_t xr[16], xi[16];
                tc::tmem_ld16(tmem + lane_base + 256 + 16 * hc, xr);
                tc::tmem_ld16(tmem + lane_base + 256 + 32 + 16 * hc, xi);
                if (a.P == 2) {
                    uint32_t yr[16], yi[16];
                    tc::tmem_ld16(tmem + lane_base + 256 + 64 + 16 * hc, yr);
                    tc::tmem_ld16(tmem + lane_base + 256 + 96 + 16 * hc, yi);
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
    if (!ok && tid == 0) atomicExch(a.status, 1);
}

}  // namespace

epic_status dftgemm_setup(epic_plan_s* p)
{
    const int N = p->N, C = p->C, P = p->P;
    const int n_g = (N + 63) / 64, n_kb = (N + 127) / 128, n_s = (N + 31) / 32;
    // shared-memory budget from the largest box
    const int K1max = 2 * p->box_max_x, K2max = 2 * p->box_max_y, N1max = P * p->box_max_y;
    if (N1max > 256) {
        p->last_error = "tensor path: occupied grid too tall (pols x rows > 256)";
        return EPIC_ERR_UNSUPPORTED;
    }
    size_t off = 0;
    const size_t sA1 = off;
    off = align_up(off + 256ull * K1max, 1024);
    const size_t sA2 = off;
    off = align_up(off + 256ull * K2max, 1024);
    const size_t sB1 = off;
    off = align_up(off + 2ull * N1max * K1max, 1024);
    const size_t sB2 = off;
    off = align_up(off + 2ull * P * 64 * K2max, 1024);
    size_t smem = std::max<size_t>(off, 120 * 1024);  // one CTA per SM (it owns all 512 TMEM columns)
    if ((int)smem > p->smem_optin - 1024) {
        p->last_error = "tensor path: occupied grid too large for shared memory";
        return EPIC_ERR_UNSUPPORTED;
    }
    p->tc.smem = (int)smem;
    p->tc.sA1 = (unsigned)sA1;
    p->tc.sA2 = (unsigned)sA2;
    p->tc.sB1 = (unsigned)sB1;
    p->tc.sB2 = (unsigned)sB2;
    p->tc.n_g = n_g;
    p->tc.n_kb = n_kb;
    p->tc.n_s = n_s;

    // DFT operand tables in the K-major core-matrix layout (FP64 -> FP16)
    std::vector<long long> a1_off((size_t)C * n_g), a2_off((size_t)C * n_kb);
    size_t n1 = 0, n2 = 0;
    for (int c = 0; c < C; ++c) {
        for (int g = 0; g < n_g; ++g) {
            a1_off[(size_t)c * n_g + g] = (long long)n1;
            n1 += 128ull * 2 * p->box[c].nx;
        }
        for (int kb = 0; kb < n_kb; ++kb) {
            a2_off[(size_t)c * n_kb + kb] = (long long)n2;
            n2 += 128ull * 2 * p->box[c].ny;
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
        for (int g = 0; g < n_g; ++g) {
            uint16_t* t = &a1[a1_off[(size_t)c * n_g + g]];
            for (int r = 0; r < 128; ++r) {
                const int q = r / 64, kx = 64 * g + r % 64;
                if (kx >= N) continue;
                for (int k = 0; k < K1; ++k) {
                    const int x = b.x0 + (k % b.nx);
                    double fr, fi;
                    F(x, kx, &fr, &fi);
                    double v;
                    if (q == 0) v = k < b.nx ? fr : -fi;
                    else v = k < b.nx ? fi : fr;
                    t[core_off(r, k, K1)] = f16_bits(v);
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
                    t[core_off(r, k, K2)] = f16_bits(k < b.ny ? fr : fi);
                }
            }
        }
    }
    cudaError_t e = cudaMalloc(&p->tc.a1, n1 * 2);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a1, a1.data(), n1 * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2, n2 * 2);
    if (e == cudaSuccess) e = cudaMemcpy(p->tc.a2, a2.data(), n2 * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a1_off, a1_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a1_off, a1_off.data(), a1_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.a2_off, a2_off.size() * sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tc.a2_off, a2_off.data(), a2_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc.status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->tc.status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(p, e, "tensor path table upload");
    p->dt.dft_bytes = (n1 + n2) * 2 + (a1_off.size() + a2_off.size()) * sizeof(long long);

    // chunking: channel groups big enough to fill the GPU, time chunks whose tiles fit the budget
    size_t stride = 0;
    for (int c = 0; c < C; ++c) stride = std::max(stride, (size_t)P * p->box[c].ny * 2 * p->box[c].nx * 2);
    stride = align_up(stride, 128);
    const int per_ch = n_kb * n_s;
    int cg = std::min(C, std::max(1, (2 * p->sm_count + per_ch - 1) / per_ch));
    int tcn = (int)std::max<size_t>(1, kScratchBudget / ((size_t)cg * stride));
    tcn = std::min(tcn, p->max_time);
    p->tc.cg = cg;
    p->tc.tc = tcn;
    p->tc.stride = stride;
    p->time_chunk = tcn;
    p->scratch_bytes = (size_t)cg * tcn * stride;
    e = cudaMalloc(&p->scratch, p->scratch_bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMalloc(tensor path tile buffer)");

    const size_t sg = sizeof(float2) * (size_t)p->A * P;
    if (sg > 48 * 1024) {
        if ((int)sg > p->smem_optin) {
            p->last_error = "tensor path: frame of A*P voltages does not fit in shared memory";
            return EPIC_ERR_UNSUPPORTED;
        }
        e = cudaFuncSetAttribute(k_dftgemm_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sg);
        if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_grid)");
    }
    e = cudaFuncSetAttribute(k_dftgemm_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, p->tc.smem);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_dftgemm_mma)");
    return EPIC_OK;
}

epic_status dftgemm_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate)
{
    const int C = p->C, P = p->P, A = p->A;
    const size_t sg = sizeof(float2) * (size_t)A * P;
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
    for (int c0 = 0; c0 < C; c0 += p->tc.cg) {
        const int ng = std::min(p->tc.cg, C - c0);
        for (int t0 = 0; t0 < T; t0 += p->tc.tc) {
            const int nt = std::min(p->tc.tc, T - t0);
            ev_begin(p, "k_dftgemm_grid", s);
            k_dftgemm_grid<<<dim3(nt, ng), kThreads, sg, s>>>(volt, t0, c0, ng, C, A, P, p->dt.box, p->dt.cell_off,
                                                            p->dt.cell_ptr, p->dt.contrib_e, p->dt.contrib_w,
                                                            (uint8_t*)p->scratch, p->tc.stride);
            ev_end(p, s);
            a.c0 = c0;
            a.n_ch = ng;
            a.nt = nt;
            a.accumulate = (accumulate || t0 > 0) ? 1 : 0;
            const int items = ng * a.n_kb * a.n_s;
            ev_begin(p, "k_dftgemm_mma", s);
            k_dftgemm_mma<<<std::min(items, p->sm_count), kThreads, p->tc.smem, s>>>(a);
            ev_end(p, s);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(p, e, "tensor path launch");
        }
    }
    return EPIC_OK;
}

}  // namespace epic
