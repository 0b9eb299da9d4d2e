// Fused FP32 path: one kernel per call runs, for every (channel, time sample,
// pol), unpack -> gridding -> 2-D transform -> polarisation products -> accumulation
// (paper Sec. 2, Eq. 1-2), with the images of a work item accumulated in
// registers over the whole block and written once.
//
// Work item = (channel c, slab of SW image columns kx).  Per frame:
//   for each chunk of 16 occupied grid rows: gather-grid the chunk (both pols)
//   into shared memory, then transform the rows only at the slab's SW columns, as
//   direct sums over the box's occupied columns (the other columns of a row are
//   zero; a full row FFT would compute N - SW outputs this item does not use);
//   FFT the slab's columns of both pols as one batch (radix-4/2 Stockham, + sign;
//   only the occupied rows are non-zero);
//   XX, YY, Re/Im XY of the slab's SW x N pixels are added to registers.
// The fftshift is folded into the gridding weights, so transform index k is image
// index k.  No atomics: reruns are bitwise identical.
#include <algorithm>

#include "epic_internal.h"
#include "kcommon.cuh"

namespace epic {

namespace {

constexpr int kFMaxThreads = 1024;  // threads per block: min(1024, SW x N), one pixel column per SW
constexpr int kRowChunk = 16;

struct FusedArgs {
    const uint8_t* volt;
    int T, C, A, P, N, logN, SW, n_s, nprod;
    const int4* box;
    const int* cell_off;
    const int* cell_ptr;
    const int* ce;
    const float2* cw;
    const float2* twiddle;
    float* out;
    int accumulate;
    int box_x, box_y;  // largest occupied box (for shared-memory carving)
    int bits;          // 4: 4+4-bit bytes, 8: 8+8-bit sample pairs
    int sub;           // samples per output image set (0 = the whole block)
    const float4* jones;  // [C][A][2] polarisation-mixing rows (conj J), or nullptr
};

// Shared memory carve-up (float2 units):
//   tw    [N/2]                      twiddles of the column FFT, exp(+2 pi i m / N)
//   twf   [N]                        exp(+2 pi i m / N) for all m (row sums)
//   vs    [A][P]                     unpacked voltages of the frame
//   gbuf  [P][16][box_x + 1]         gridded row chunk (odd row stride: column reads of many
//                                    rows hit different banks)
//   hbuf  [P][box_y][SW + 1]         row transforms at the slab's columns
//   fa,fb [P SW][N+1]                column FFT ping-pong buffers (both pols in one batch)
__host__ __device__ inline size_t fused_smem_elems(int N, int A, int P, int SW, int bx, int by)
{
    return (size_t)N / 2 + (size_t)N + (size_t)A * P + (size_t)P * kRowChunk * (bx + 1) +
           (size_t)P * by * (SW + 1) + 2ull * P * SW * (N + 1);
}

template <int NPT>  // accumulated pixels per thread (per product)
__global__ void __launch_bounds__(kFMaxThreads, 1) k_fused_fp32(FusedArgs a)
{
    extern __shared__ __align__(16) float2 fsm[];
    const int N = a.N, P = a.P, A = a.A, SW = a.SW;
    const int ldc = N + 1;  // padded column stride of the FFT buffers
    float2* tw = fsm;
    float2* twf = tw + N / 2;
    float2* vs = twf + N;
    float2* gbuf = vs + A * P;
    float2* hbuf = gbuf + P * kRowChunk * (a.box_x + 1);
    float2* fa = hbuf + P * a.box_y * (SW + 1);
    float2* fb = fa + (size_t)P * SW * ldc;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const float2 w = a.twiddle[i];
        tw[i] = w;
        twf[i] = w;
        twf[i + N / 2] = make_float2(-w.x, -w.y);  // exp(+2 pi i (m + N/2) / N) = -exp(+2 pi i m / N)
    }

    const int items = a.C * a.n_s;
    const int kxl = threadIdx.x % SW;              // slab-local column of this thread
    const int ky0 = threadIdx.x / SW, kys = blockDim.x / SW;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int s = item % a.n_s, c = item / a.n_s;
        const int4 b = a.box[c];
        const int x0 = b.x, y0 = b.y, nxp = b.z, nyp = b.w;
        const int gs = nxp + 1, hs = SW + 1;  // padded row strides of gbuf and hbuf
        const int* ptr = a.cell_ptr + a.cell_off[c];
        float axx[NPT], ayy[NPT], arx[NPT], aix[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;
        // write (or add) this thread's pixels to image set iv, then restart the sums
        auto store_images = [&](int iv) {
            const int kx = s * SW + kxl;
            if (kx < N) {
                const size_t NN = (size_t)N * N;
#pragma unroll
                for (int j = 0; j < NPT; ++j) {
                    const int ky = ky0 + j * kys;
                    if (ky >= N) continue;
                    float* o = a.out + ((size_t)iv * a.C + c) * a.nprod * NN + (size_t)ky * N + kx;
                    o[0] = (a.accumulate ? o[0] : 0.f) + axx[j];
                    if (a.nprod == 4) {
                        o[NN] = (a.accumulate ? o[NN] : 0.f) + ayy[j];
                        o[2 * NN] = (a.accumulate ? o[2 * NN] : 0.f) + arx[j];
                        o[3 * NN] = (a.accumulate ? o[3 * NN] : 0.f) + aix[j];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NPT; ++i) axx[i] = ayy[i] = arx[i] = aix[i] = 0.f;
        };

        for (int t = 0; t < a.T; ++t) {
            __syncthreads();
            const uint8_t* fr = a.volt + ((size_t)t * a.C + c) * (size_t)A * P * (a.bits / 4);
            stage_frame(vs, fr, A, P, a.bits, a.jones ? a.jones + (size_t)c * A * 2 : nullptr);
            __syncthreads();
            // ---- rows, 16 at a time: grid them, then sum each row at the slab's columns
            for (int r0 = 0; r0 < nyp; r0 += kRowChunk) {
                const int nr = min(kRowChunk, nyp - r0);
                for (int cell = threadIdx.x; cell < nr * nxp; cell += blockDim.x) {
                    const int r = cell / nxp, x = cell - r * nxp;
                    const int q0 = ptr[(r0 + r) * nxp + x], q1 = ptr[(r0 + r) * nxp + x + 1];
                    float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
                    for (int q = q0; q < q1; ++q) {
                        const int e = a.ce[q];
                        const float2 w = a.cw[q];
                        g0 = cfma(w, vs[e * P], g0);
                        if (P == 2) g1 = cfma(w, vs[e * P + 1], g1);
                    }
                    gbuf[r * gs + x] = g0;
                    if (P == 2) gbuf[kRowChunk * gs + r * gs + x] = g1;
                }
                __syncthreads();
                // H_p[y][kx] = sum_x G_p[y][x] exp(+2 pi i (x0 + x) kx / N), kx in the slab;
                // the lanes of a warp take different (pol, row) pairs of one kx, so each step
                // reads one twiddle for the whole warp
                const int prs = P * nr;
                for (int o = threadIdx.x; o < prs * SW; o += blockDim.x) {
                    const int k = o / prs, pr = o - k * prs, p = pr / nr, r = pr - p * nr;
                    const int kx = s * SW + k;
                    const float2* gr = gbuf + (p * kRowChunk + r) * gs;
                    int m = (x0 * kx) & (N - 1);
                    float2 h = make_float2(0.f, 0.f);
                    for (int x = 0; x < nxp; ++x) {
                        h = cfma(twf[m], gr[x], h);
                        m = (m + kx) & (N - 1);
                    }
                    hbuf[(p * a.box_y + r0 + r) * hs + k] = h;
                }
                __syncthreads();
            }
            // ---- columns: one batch of P x SW FFTs along y (rows outside the box are zero)
            for (int i = threadIdx.x; i < P * SW * N; i += blockDim.x) {
                const int pk = i / N, y = i - pk * N;  // pk = p * SW + k
                const int p = pk / SW, k = pk - p * SW;
                const int yr = y - y0;
                fa[pk * ldc + y] = (yr >= 0 && yr < nyp) ? hbuf[(p * a.box_y + yr) * hs + k] : make_float2(0.f, 0.f);
            }
            const float2* res = fft_stockham(fa, fb, a.logN, P * SW, 1, ldc, tw);
            // ---- products of this thread's pixels (kx = kxl, ky = ky0 + j kys)
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                const int ky = ky0 + j * kys;
                if (ky < N) {
                    const float2 X = res[kxl * ldc + ky];
                    axx[j] = fmaf(X.x, X.x, fmaf(X.y, X.y, axx[j]));
                    if (P == 2) {
                        const float2 Y = res[(SW + kxl) * ldc + ky];
                        ayy[j] = fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, ayy[j]));
                        arx[j] = fmaf(X.x, Y.x, fmaf(X.y, Y.y, arx[j]));
                        aix[j] = fmaf(X.y, Y.x, fmaf(-X.x, Y.y, aix[j]));
                    }
                }
            }
            if (a.sub > 0 && (t + 1) % a.sub == 0) store_images(t / a.sub);  // a sub-integration ends
        }
        // ---- images (the whole block)
        if (a.sub == 0) store_images(0);
    }
}

// threads per block and pixels per thread for a grid size: SW columns x N rows
int threads_for(int N, int SW) { return std::min(kFMaxThreads, SW * N); }
int npt_for(int N, int SW) { return SW * N / threads_for(N, SW); }

}  // namespace

// Image columns per work item (slab width SW); its pixels per thread pick the
// kernel variant.  UNSUPPORTED when SW is not a power of two in 8..min(N, 32)
// or the shared memory does not hold it.
epic_status fused_set_slab(epic_plan_s* p, int SW)
{
    const int N = p->N;
    if (SW < 8 || SW > std::min(32, N) || (SW & (SW - 1)) != 0) return EPIC_ERR_UNSUPPORTED;
    const int npt = npt_for(N, SW);
    if (npt > 16) return EPIC_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(float2) * fused_smem_elems(N, p->A, p->P, SW, p->box_max_x, p->box_max_y);
    if ((int)bytes > p->smem_optin) return EPIC_ERR_UNSUPPORTED;
    p->slab = SW;
    p->fused_variant = npt;
    return EPIC_OK;
}

epic_status fused_setup(epic_plan_s* p)
{
    const int N = p->N;
    // at most 4 pixels per thread; a narrower slab when the FFT buffers do not fit beside the voltages
    int SW = N >= 512 ? 8 : N >= 256 ? 16 : std::min(32, N);
    while (SW > 8 && sizeof(float2) * fused_smem_elems(N, p->A, p->P, SW, p->box_max_x, p->box_max_y) >
                         (size_t)p->smem_optin)
        SW >>= 1;
    const size_t bytes =
        sizeof(float2) * fused_smem_elems(N, p->A, p->P, SW, p->box_max_x, p->box_max_y);
    if ((int)bytes > p->smem_optin) {
        p->last_error = "fused FP32 path: occupied grid or element count too large for shared memory";
        return EPIC_ERR_UNSUPPORTED;
    }
    p->slab = SW;
    p->fused_variant = npt_for(N, SW);
    p->time_chunk = p->max_time;
    cudaError_t e = cudaSuccess;
#define EPIC_FUSED_ATTR(n)                                                                                      \
    if (e == cudaSuccess) e = allow_max_smem((const void*)k_fused_fp32<n>, p->smem_optin);
    EPIC_FUSED_ATTR(1)
    EPIC_FUSED_ATTR(2)
    EPIC_FUSED_ATTR(4)
    EPIC_FUSED_ATTR(8)
    EPIC_FUSED_ATTR(16)
#undef EPIC_FUSED_ATTR
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_fused_fp32)");
    return EPIC_OK;
}

epic_status fused_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate)
{
    FusedArgs a{};
    a.volt = volt;
    a.T = T;
    a.C = p->C;
    a.A = p->A;
    a.P = p->P;
    a.N = p->N;
    a.logN = p->logN;
    a.SW = p->slab;
    a.n_s = (p->N + p->slab - 1) / p->slab;
    a.nprod = p->nprod;
    a.box = p->dt.box;
    a.cell_off = p->dt.cell_off;
    a.cell_ptr = p->dt.cell_ptr;
    a.ce = p->dt.contrib_e;
    a.cw = p->dt.contrib_w;
    a.twiddle = p->dt.twiddle;
    a.out = out;
    a.accumulate = accumulate ? 1 : 0;
    a.box_x = p->box_max_x;
    a.box_y = p->box_max_y;
    a.bits = p->bits;
    a.sub = p->sub;
    a.jones = p->dt.jones;
    const size_t bytes = sizeof(float2) * fused_smem_elems(a.N, a.A, a.P, a.SW, a.box_x, a.box_y);
    const int items = a.C * a.n_s;
    const int grid = std::min(items, p->sm_count);
    const int nth = threads_for(a.N, a.SW);
    ev_begin(p, "k_fused_fp32", s);
    switch (p->fused_variant) {
        case 1: k_fused_fp32<1><<<grid, nth, bytes, s>>>(a); break;
        case 2: k_fused_fp32<2><<<grid, nth, bytes, s>>>(a); break;
        case 4: k_fused_fp32<4><<<grid, nth, bytes, s>>>(a); break;
        case 8: k_fused_fp32<8><<<grid, nth, bytes, s>>>(a); break;
        default: k_fused_fp32<16><<<grid, nth, bytes, s>>>(a); break;
    }
    ev_end(p, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "fused FP32 launch");
    return EPIC_OK;
}

}  // namespace epic
