// Plain, unfused FP32 path of the EPIC hot loop (paper Sec. 2, Eq. 1-2): the
// comparator for the fused paths.  Per chunk of time samples, four kernels with
// HBM round trips between them:
//   k_plain_grid     unpack the voltages (and mix polarisations, when the plan
//                    has a mixing kernel) and gather-grid every (t, c, p)
//                    frame onto a full N x N complex grid (Eq. 1 bracket)
//   k_plain_fft_rows FFT along x of every grid row (Eq. 1 sum)
//   k_plain_fft_cols the same along y, on tiles of adjacent columns
// Two forms of the FFT kernels: register-resident two-pass transforms (the
// default, one shared-memory exchange per transform) and radix-4/2 Stockham
// transforms in shared memory (a pass over shared memory per radix-4 stage).
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

// ---- register-resident two-pass FFT ------------------------------------------
// A length-N transform X[k] = sum_n x[n] w^(nk), w = exp(+2 pi i / N) (Eq. 1: + sign,
// unnormalised), is split with N = N1 N2, n = n1 + N1 n2 and k = k2 + N2 k1 into
//   Y[n1][k2] = w^(n1 k2) sum_n2 x[n1 + N1 n2] w_N2^(n2 k2)       (pass 1)
//   X[k2 + N2 k1] = sum_n1 Y[n1][k2] w_N1^(n1 k1)                 (pass 2)
// (the Cooley-Tukey "four-step" factorisation).  Each thread holds whole N2- or
// N1-point transforms in registers; Y goes once through shared memory between
// the passes.  N1 is N2 or 2 N2, so both are at most 32 for N <= 512.

// exp(+2 pi i m / 32), m < 16: the twiddles inside the register transforms.
__constant__ float2 c_w32[16] = {
    {1.0f, 0.0f},                    {0.980785251f, 0.195090324f}, {0.923879504f, 0.382683426f},
    {0.831469595f, 0.555570245f},    {0.707106769f, 0.707106769f}, {0.555570245f, 0.831469595f},
    {0.382683426f, 0.923879504f},    {0.195090324f, 0.980785251f}, {0.0f, 1.0f},
    {-0.195090324f, 0.980785251f},   {-0.382683426f, 0.923879504f}, {-0.555570245f, 0.831469595f},
    {-0.707106769f, 0.707106769f},   {-0.831469595f, 0.555570245f}, {-0.923879504f, 0.382683426f},
    {-0.980785251f, 0.195090324f}};

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// k with its low `bits` bits reversed
__host__ __device__ constexpr int bit_reverse(int k, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1) << (bits - 1 - i);
    return r;
}

// d * exp(+2 pi i m / 32); m is a compile-time constant once the callers are unrolled
__device__ __forceinline__ float2 w32_mul(float2 d, int m)
{
    if (m == 0) return d;
    if (m == 8) return make_float2(-d.y, d.x);
    return cmul(d, c_w32[m]);
}

// In-place R-point transform (+ sign, unnormalised) of v by radix-2 decimation in
// frequency: afterwards v[bit_reverse(k, log2 R)] = sum_n v_in[n] exp(+2 pi i n k / R).
// A span-h stage maps (a, b) = (v[i], v[i + h]) to (a + b, (a - b) w_2h^j), j = i mod h.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R])
{
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const float2 x = v[b + j], y = v[b + j + h];
                v[b + j] = make_float2(x.x + y.x, x.y + y.y);
                v[b + j + h] = w32_mul(make_float2(x.x - y.x, x.y - y.y), j * (32 / (2 * h)));
            }
        }
    }
}

// tw[k2 N1 + n1] = w^(n1 k2) from the plan's table twg[m] = exp(+2 pi i m / N), m < N/2
template <int N1, int N2>
__device__ __forceinline__ void load_step_twiddles(float2* tw, const float2* __restrict__ twg)
{
    constexpr int N = N1 * N2;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int m = (i / N1) * (i % N1);  // < N
        const float2 t = twg[m < N / 2 ? m : m - N / 2];
        tw[i] = m < N / 2 ? t : make_float2(-t.x, -t.y);
    }
}

constexpr int kRegThreads = 256;

// Rows of N = N1 N2 points, 256 / N2 rows per block, N2 threads per row.  Thread j
// of a row takes n1 = j (and j + N2) in pass 1 and k2 = j in pass 2.  Y of a row is
// stored [k2][n1] with stride N1 + 1, which no pass-1 store or pass-2 load of a warp
// meets twice in one bank.
template <int N1, int N2>
__global__ void __launch_bounds__(kRegThreads) k_plain_fft_rows(float2* __restrict__ grid, size_t n_rows,
                                                                const float2* __restrict__ twg)
{
    constexpr int N = N1 * N2, RPC = kRegThreads / N2, S = N2 * (N1 + 1), T = N1 / N2;
    constexpr int L1 = ilog2(N1), L2 = ilog2(N2);
    extern __shared__ float2 sm[];
    float2* tw = sm;      // [N2][N1]
    float2* y = sm + N;   // [RPC][N2][N1 + 1]
    load_step_twiddles<N1, N2>(tw, twg);
    const int rl = threadIdx.x / N2, j = threadIdx.x % N2;
    const size_t r = (size_t)blockIdx.x * RPC + rl;
    const bool live = r < n_rows;
    float2* row = grid + (live ? r : 0) * N;
    float2 u[T][N2];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[t][n2] = live ? row[j + N2 * t + N1 * n2] : make_float2(0.f, 0.f);
    __syncthreads();  // twiddles
    float2* yr = y + rl * S;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        dft_reg<N2>(u[t]);
        const int n1 = j + N2 * t;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2)
            yr[k2 * (N1 + 1) + n1] = cmul(u[t][bit_reverse(k2, L2)], tw[k2 * N1 + n1]);
    }
    __syncthreads();
    float2 z[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) z[n1] = yr[j * (N1 + 1) + n1];
    dft_reg<N1>(z);
    if (live) {
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) row[j + N2 * k1] = z[bit_reverse(k1, L1)];
    }
}

// Columns of one N x N frame (blockIdx.y), TX adjacent columns per block, N2 threads
// per column; a warp's lanes take adjacent columns, so every global access of a warp
// is one contiguous run and Y ([n1][k2][column]) is read and written without bank
// conflicts.
template <int N1, int N2, int TX>
__global__ void __launch_bounds__(TX * N2) k_plain_fft_cols(float2* __restrict__ grid, const float2* __restrict__ twg)
{
    constexpr int N = N1 * N2, T = N1 / N2;
    constexpr int L1 = ilog2(N1), L2 = ilog2(N2);
    extern __shared__ float2 sm[];
    float2* tw = sm;      // [N2][N1]
    float2* y = sm + N;   // [N1][N2][TX]
    load_step_twiddles<N1, N2>(tw, twg);
    const int xl = threadIdx.x % TX, j = threadIdx.x / TX;
    float2* g = grid + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * TX + xl;
    float2 u[T][N2];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[t][n2] = g[(size_t)(j + N2 * t + N1 * n2) * N];
    __syncthreads();  // twiddles
#pragma unroll
    for (int t = 0; t < T; ++t) {
        dft_reg<N2>(u[t]);
        const int n1 = j + N2 * t;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2)
            y[(n1 * N2 + k2) * TX + xl] = cmul(u[t][bit_reverse(k2, L2)], tw[k2 * N1 + n1]);
    }
    __syncthreads();
    float2 z[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) z[n1] = y[(n1 * N2 + j) * TX + xl];
    dft_reg<N1>(z);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) g[(size_t)(j + N2 * k1) * N] = z[bit_reverse(k1, L1)];
}

// launch shapes of the register FFT kernels of one N
struct RegFft {
    void (*rows)(float2*, size_t, const float2*);
    void (*cols)(float2*, const float2*);
    int rows_per_cta, col_tile, col_threads;
    size_t rows_smem, cols_smem;
};

template <int N1, int N2>
RegFft reg_fft()
{
    constexpr int N = N1 * N2, TX = (N2 <= 8 ? 32 : 16) < N ? (N2 <= 8 ? 32 : 16) : N;
    return {k_plain_fft_rows<N1, N2>, k_plain_fft_cols<N1, N2, TX>, kRegThreads / N2, TX, TX * N2,
            sizeof(float2) * ((size_t)N + (size_t)(kRegThreads / N2) * N2 * (N1 + 1)),
            sizeof(float2) * ((size_t)N + (size_t)N * TX)};
}

// N = 2^logN, 8 <= N <= 512
RegFft reg_fft_for(int logN)
{
    switch (logN) {
        case 3: return reg_fft<4, 2>();
        case 4: return reg_fft<4, 4>();
        case 5: return reg_fft<8, 4>();
        case 6: return reg_fft<8, 8>();
        case 7: return reg_fft<16, 8>();
        case 8: return reg_fft<16, 16>();
        default: return reg_fft<32, 16>();
    }
}

// Zeros of the N x N planes (P of them, NN apart) outside the occupied box b =
// (x0, y0, width, height): pairs of cells wholly outside take one 16-byte store.
__device__ __forceinline__ void zero_outside_box(float2* g, int N, int P, int4 b)
{
    const size_t NN = (size_t)N * N;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < N * N / 2; i += blockDim.x) {
        const int cell = 2 * i, y = cell / N, x = cell - y * N;
        const bool row_in = y >= b.y && y < b.y + b.w;
        const bool in0 = row_in && x >= b.x && x < b.x + b.z;
        const bool in1 = row_in && x + 1 >= b.x && x + 1 < b.x + b.z;
        if (!in0 && !in1) {
            for (int p = 0; p < P; ++p) *reinterpret_cast<float4*>(g + p * NN + cell) = z4;
        } else if (in0 != in1) {
            const int zc = in0 ? cell + 1 : cell;
            for (int p = 0; p < P; ++p) g[p * NN + zc] = make_float2(0.f, 0.f);
        }
    }
}

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
    // the occupied box (its padding clipped to the grid), one cell per thread and step
    for (int i = threadIdx.x; i < b.z * b.w; i += blockDim.x) {
        const int ry = i / b.z, rx = i - ry * b.z;
        if (b.y + ry >= N || b.x + rx >= N) continue;  // box padding beyond the grid (empty lists)
        const size_t cell = (size_t)(b.y + ry) * N + b.x + rx;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        const int q1 = ptr[i + 1];
        for (int q = ptr[i]; q < q1; ++q) {
            const int e = ce[q];
            const float2 w = cw[q];
            a0 = cfma(w, sv[e * P], a0);
            if (P == 2) a1 = cfma(w, sv[e * P + 1], a1);
        }
        g[cell] = a0;
        if (P == 2) g[NN + cell] = a1;
    }
    zero_outside_box(g, N, P, b);
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
    for (int i = threadIdx.x; i < b.z * b.w; i += blockDim.x) {
        const int ry = i / b.z, rx = i - ry * b.z;
        if (b.y + ry >= N || b.x + rx >= N) continue;  // box padding beyond the grid (empty lists)
        const size_t cell = (size_t)(b.y + ry) * N + b.x + rx;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        const int q1 = ptr[i + 1];
        for (int q = ptr[i]; q < q1; ++q) {
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
        g[cell] = a0;
        if (P == 2) g[NN + cell] = a1;
    }
    zero_outside_box(g, N, P, b);
}

__global__ void __launch_bounds__(kThreads) k_plain_fft_rows_smem(float2* __restrict__ grid, size_t n_rows, int logN,
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

__global__ void __launch_bounds__(kThreads) k_plain_fft_cols_smem(float2* __restrict__ grid, int logN, int tile,
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
#pragma unroll 4
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

// FFT kernels of the plain path: 0 register two-pass, 1 shared-memory Stockham
epic_status plain_set_fft(epic_plan_s* p, int v)
{
    if (v != 0 && v != 1) {
        p->last_error = "plain path: FFT form must be 0 or 1";
        return EPIC_ERR_INVALID_ARG;
    }
    p->plain_fft = v;
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
    e = allow_max_smem((const void*)k_plain_fft_rows_smem, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_fft_rows_smem)");
    e = allow_max_smem((const void*)k_plain_fft_cols_smem, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_fft_cols_smem)");
    const RegFft rf = reg_fft_for(p->logN);
    if (rf.rows_smem > (size_t)p->smem_optin || rf.cols_smem > (size_t)p->smem_optin) {
        p->last_error = "plain path: FFT shared memory exceeds the device limit";
        return EPIC_ERR_UNSUPPORTED;
    }
    e = allow_max_smem((const void*)rf.rows, p->smem_optin);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute(k_plain_fft_rows)");
    e = allow_max_smem((const void*)rf.cols, p->smem_optin);
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
        if (p->plain_fft == 0) {
            const RegFft rf = reg_fft_for(p->logN);
            ev_begin(p, "k_plain_fft_rows", s);
            rf.rows<<<(unsigned)((n_rows + rf.rows_per_cta - 1) / rf.rows_per_cta), kRegThreads, rf.rows_smem, s>>>(
                grid, n_rows, p->dt.twiddle);
            ev_end(p, s);
            ev_begin(p, "k_plain_fft_cols", s);
            rf.cols<<<dim3(N / rf.col_tile, (unsigned)((size_t)nt * C * P)), rf.col_threads, rf.cols_smem, s>>>(
                grid, p->dt.twiddle);
            ev_end(p, s);
        } else {
            const int rpc = rows_per_cta_for(N);
            ev_begin(p, "k_plain_fft_rows_smem", s);
            k_plain_fft_rows_smem<<<(unsigned)((n_rows + rpc - 1) / rpc), kThreads, rows_smem(N), s>>>(
                grid, n_rows, p->logN, rpc, p->dt.twiddle);
            ev_end(p, s);
            ev_begin(p, "k_plain_fft_cols_smem", s);
            k_plain_fft_cols_smem<<<dim3(N / col_tile_for(N), (unsigned)((size_t)nt * C * P)), kThreads,
                                    cols_smem(N), s>>>(grid, p->logN, col_tile_for(N), p->dt.twiddle);
            ev_end(p, s);
        }
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
