// Plain, unfused FP32 path of the EPIC hot loop (paper Sec. 2, Eq. 1-2): the
// comparator for the fused paths.  Per chunk of time samples, four kernels with
// HBM round trips between them:
//   k_plain_grid     unpack the voltages (and mix polarisations, when the plan
//                    has a mixing kernel) and gather-grid every (t, c, p)
//                    frame onto a full N x N complex grid (Eq. 1 bracket)
//   k_plain_fft_rows radix-4/2 Stockham FFT along x of every grid row (Eq. 1 sum)
//   k_plain_fft_cols the same along y, on 16-column tiles
//   k_plain_sqacc    XX, YY, XY products summed over the chunk's frames and
//                    added to the images (Eq. 2)
#include <algorithm>

#include "epic_internal.h"
#include "kcommon.cuh"

namespace epic {

namespace {

constexpr int kThreads = 256;
constexpr int kColTile = 16;
constexpr size_t kGridBudget = 512ull << 20;  // bytes of the chunk grid buffer

__global__ void __launch_bounds__(kThreads) k_plain_grid(const uint8_t* __restrict__ volt, int t0, int C, int A,
                                                         int P, int N, int bits, const int4* __restrict__ box,
                                                         const int* __restrict__ cell_off,
                                                         const int* __restrict__ cell_ptr,
                                                         const int* __restrict__ ce, const float2* __restrict__ cw,
                                                         const float4* __restrict__ jones, float2* __restrict__ grid)
{
    extern __shared__ float2 sv[];  // [A][P] unpacked (and pol-mixed) voltages of this frame
    const int tl = blockIdx.x, c = blockIdx.y;
    const uint8_t* fr = volt + ((size_t)(t0 + tl) * C + c) * (size_t)A * P * (bits / 4);
    stage_frame(sv, fr, A, P, bits, jones ? jones + (size_t)c * A * 2 : nullptr);
    __syncthreads();
    const int4 b = box[c];
    const int* ptr = cell_ptr + cell_off[c];
    const size_t NN = (size_t)N * N;
    float2* g = grid + ((size_t)tl * C + c) * P * NN;
    for (int cell = threadIdx.x; cell < N * N; cell += blockDim.x) {
        const int y = cell / N, x = cell - y * N;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        const int rx = x - b.x, ry = y - b.y;
        if (rx >= 0 && rx < b.z && ry >= 0 && ry < b.w) {
            const int r = ry * b.z + rx;
            const int q1 = ptr[r + 1];
            for (int q = ptr[r]; q < q1; ++q) {
                const int e = ce[q];
                const float2 w = cw[q];
                a0 = cfma(w, sv[e * P], a0);
                if (P == 2) a1 = cfma(w, sv[e * P + 1], a1);
            }
        }
        g[cell] = a0;
        if (P == 2) g[NN + cell] = a1;
    }
}

// Same as k_plain_grid for frames whose A*P voltages do not fit in shared memory
// (very large arrays): each contribution reads and unpacks its voltage byte
// through the read-only data cache.
__global__ void __launch_bounds__(kThreads) k_plain_grid_g(const uint8_t* __restrict__ volt, int t0, int C, int A,
                                                           int P, int N, int bits, const int4* __restrict__ box,
                                                           const int* __restrict__ cell_off,
                                                           const int* __restrict__ cell_ptr,
                                                           const int* __restrict__ ce, const float2* __restrict__ cw,
                                                           const float4* __restrict__ jones, float2* __restrict__ grid)
{
    const int tl = blockIdx.x, c = blockIdx.y;
    const uint8_t* fr = volt + ((size_t)(t0 + tl) * C + c) * (size_t)A * P * (bits / 4);
    const float4* jm = jones ? jones + (size_t)c * A * 2 : nullptr;
    const int4 b = box[c];
    const int* ptr = cell_ptr + cell_off[c];
    const size_t NN = (size_t)N * N;
    float2* g = grid + ((size_t)tl * C + c) * P * NN;
    for (int cell = threadIdx.x; cell < N * N; cell += blockDim.x) {
        const int y = cell / N, x = cell - y * N;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        const int rx = x - b.x, ry = y - b.y;
        if (rx >= 0 && rx < b.z && ry >= 0 && ry < b.w) {
            const int r = ry * b.z + rx;
            const int q1 = ptr[r + 1];
            for (int q = ptr[r]; q < q1; ++q) {
                const int e = ce[q];
                const float2 w = cw[q];
                if (jm) {
                    const float4 v = load_pair(fr, e, bits, jm);
                    a0 = cfma(w, make_float2(v.x, v.y), a0);
                    a1 = cfma(w, make_float2(v.z, v.w), a1);
                } else {
                    a0 = cfma(w, load_sample(fr, (size_t)e * P, bits), a0);
                    if (P == 2) a1 = cfma(w, load_sample(fr, (size_t)e * P + 1, bits), a1);
                }
            }
        }
        g[cell] = a0;
        if (P == 2) g[NN + cell] = a1;
    }
}

__global__ void __launch_bounds__(kThreads) k_plain_fft_rows(float2* __restrict__ grid, size_t n_rows, int logN,
                                                             int rows_per_cta, const float2* __restrict__ twg)
{
    extern __shared__ float2 sm[];
    const int N = 1 << logN;
    float2* tw = sm;                       // [N/2]
    float2* a = sm + N / 2;                // [rows][N]
    float2* b = a + (size_t)rows_per_cta * N;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) tw[i] = twg[i];
    const size_t r0 = (size_t)blockIdx.x * rows_per_cta;
    const int nr = (int)min((size_t)rows_per_cta, n_rows - r0);
    const float2* src = grid + r0 * N;
    for (int i = threadIdx.x; i < nr * N; i += blockDim.x) a[i] = src[i];
    __syncthreads();
    float2* res = fft_stockham(a, b, logN, nr, 1, N, tw);
    float2* dst = grid + r0 * N;
    for (int i = threadIdx.x; i < nr * N; i += blockDim.x) dst[i] = res[i];
}

__global__ void __launch_bounds__(kThreads) k_plain_fft_cols(float2* __restrict__ grid, int logN, int tile,
                                                             const float2* __restrict__ twg)
{
    extern __shared__ float2 sm[];
    const int N = 1 << logN;
    const int ld = N + 1;                  // padded column stride in shared memory
    float2* tw = sm;
    float2* a = sm + N / 2;                // [tile][N + 1]
    float2* b = a + (size_t)tile * ld;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) tw[i] = twg[i];
    const size_t frame = blockIdx.y;
    const int x0 = blockIdx.x * tile;
    float2* g = grid + frame * (size_t)N * N;
    for (int i = threadIdx.x; i < N * tile; i += blockDim.x) {
        const int row = i / tile, col = i - row * tile;
        a[col * ld + row] = g[(size_t)row * N + x0 + col];
    }
    __syncthreads();
    float2* res = fft_stockham(a, b, logN, tile, 1, ld, tw);
    for (int i = threadIdx.x; i < N * tile; i += blockDim.x) {
        const int row = i / tile, col = i - row * tile;
        g[(size_t)row * N + x0 + col] = res[col * ld + row];
    }
}

// Products summed over the chunk's frames (sub = 0), or over each interval of sub
// frames (sub-integrations, paper Sec. 4): interval k of the chunk goes to image
// set out_iv0 + k.
__global__ void __launch_bounds__(kThreads) k_plain_sqacc(const float2* __restrict__ grid, int nt, int C, int P, int N,
                                                          float* __restrict__ out, int accumulate, int sub, int out_iv0)
{
    const size_t NN = (size_t)N * N;
    const size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (pix >= NN) return;
    const int nprod = P == 2 ? 4 : 1;
    const int span = sub > 0 ? sub : nt;
    for (int iv = 0; iv * span < nt; ++iv) {
    float xx = 0.f, yy = 0.f, rxy = 0.f, ixy = 0.f;
    for (int tl = iv * span; tl < (iv + 1) * span; ++tl) {
        const float2* g = grid + ((size_t)tl * C + c) * P * NN;
        const float2 X = g[pix];
        xx = fmaf(X.x, X.x, fmaf(X.y, X.y, xx));
        if (P == 2) {
            const float2 Y = g[NN + pix];
            yy = fmaf(Y.x, Y.x, fmaf(Y.y, Y.y, yy));
            rxy = fmaf(X.x, Y.x, fmaf(X.y, Y.y, rxy));
            ixy = fmaf(X.y, Y.x, fmaf(-X.x, Y.y, ixy));
        }
    }
    float* o = out + ((size_t)(out_iv0 + iv) * C + c) * nprod * NN + pix;
    if (accumulate) {
        o[0] += xx;
        if (P == 2) { o[NN] += yy; o[2 * NN] += rxy; o[3 * NN] += ixy; }
    } else {
        o[0] = xx;
        if (P == 2) { o[NN] = yy; o[2 * NN] = rxy; o[3 * NN] = ixy; }
    }
    }
}

int rows_per_cta_for(int N) { return std::max(1, 2048 / N); }

size_t rows_smem(int N) { return sizeof(float2) * ((size_t)N / 2 + 2ull * rows_per_cta_for(N) * N); }

int col_tile_for(int N) { return std::min(kColTile, N); }

size_t cols_smem(int N) { return sizeof(float2) * ((size_t)N / 2 + 2ull * col_tile_for(N) * (N + 1)); }

}  // namespace

// Time samples per chunk so that the chunk's grids take at most `budget` bytes
// (at least one sample), and the grid buffer for them.
epic_status plain_set_chunk(epic_plan_s* p, size_t budget)
{
    const size_t per_t = (size_t)p->C * p->P * p->N * p->N * sizeof(float2);
    // at most 65,535 (sample, channel, pol) columns: the second grid dimension of the column FFT
    const size_t max_t = 65535 / ((size_t)p->C * p->P);
    int tcn = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)p->max_time, max_t), budget / per_t));
    if (p->sub > 0) tcn = std::max(p->sub, tcn - tcn % p->sub);  // whole sub-integrations per chunk
    if ((size_t)tcn > max_t) {
        p->last_error = "plain path: sub_int x n_chan x n_pol exceeds 65,535";
        return EPIC_ERR_UNSUPPORTED;
    }
    const size_t bytes = per_t * tcn;
    p->chunk_budget = budget;
    if (p->scratch && bytes == p->scratch_bytes) {
        p->time_chunk = tcn;
        return EPIC_OK;
    }
    cudaFree(p->scratch);
    p->scratch = nullptr;
    p->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&p->scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMalloc(plain grid buffer)");
    p->scratch_bytes = bytes;
    p->time_chunk = tcn;
    return EPIC_OK;
}

epic_status plain_setup(epic_plan_s* p)
{
    epic_status st = plain_set_chunk(p, kGridBudget);
    if (st != EPIC_OK) return st;
    cudaError_t e = cudaSuccess;
    const size_t sg = sizeof(float2) * (size_t)p->A * p->P;
    if (sg > 48 * 1024 && (int)sg <= p->smem_optin) {  // larger frames use k_plain_grid_g
        e = allow_max_smem((const void*)k_plain_grid, p->smem_optin);
        if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_grid)");
    }
    e = allow_max_smem((const void*)k_plain_fft_rows, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_fft_rows)");
    e = allow_max_smem((const void*)k_plain_fft_cols, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_fft_cols)");
    return EPIC_OK;
}

epic_status plain_run(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, bool accumulate)
{
    const int C = p->C, P = p->P, N = p->N, A = p->A;
    float2* grid = (float2*)p->scratch;
    const size_t sg = sizeof(float2) * (size_t)A * P;
    const int bits = p->bits;
    for (int t0 = 0; t0 < T; t0 += p->time_chunk) {
        const int nt = std::min(p->time_chunk, T - t0);
        ev_begin(p, "k_plain_grid", s);
        if ((int)sg <= p->smem_optin)
            k_plain_grid<<<dim3(nt, C), kThreads, sg, s>>>(volt, t0, C, A, P, N, bits, p->dt.box, p->dt.cell_off,
                                                           p->dt.cell_ptr, p->dt.contrib_e, p->dt.contrib_w, p->dt.jones, grid);
        else
            k_plain_grid_g<<<dim3(nt, C), kThreads, 0, s>>>(volt, t0, C, A, P, N, bits, p->dt.box, p->dt.cell_off,
                                                            p->dt.cell_ptr, p->dt.contrib_e, p->dt.contrib_w, p->dt.jones, grid);
        ev_end(p, s);
        const size_t n_rows = (size_t)nt * C * P * N;
        const int rpc = rows_per_cta_for(N);
        ev_begin(p, "k_plain_fft_rows", s);
        k_plain_fft_rows<<<(unsigned)((n_rows + rpc - 1) / rpc), kThreads, rows_smem(N), s>>>(grid, n_rows, p->logN,
                                                                                           rpc, p->dt.twiddle);
        ev_end(p, s);
        ev_begin(p, "k_plain_fft_cols", s);
        k_plain_fft_cols<<<dim3(N / col_tile_for(N), (unsigned)((size_t)nt * C * P)), kThreads, cols_smem(N), s>>>(
            grid, p->logN, col_tile_for(N), p->dt.twiddle);
        ev_end(p, s);
        ev_begin(p, "k_plain_sqacc", s);
        k_plain_sqacc<<<dim3((unsigned)(((size_t)N * N + kThreads - 1) / kThreads), C), kThreads, 0, s>>>(
            grid, nt, C, P, N, out, (accumulate || (t0 > 0 && p->sub == 0)) ? 1 : 0, p->sub,
            p->sub > 0 ? t0 / p->sub : 0);
        ev_end(p, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(p, e, "plain path launch");
    }
    return EPIC_OK;
}

}  // namespace epic
