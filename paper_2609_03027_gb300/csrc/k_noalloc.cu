// Imaging without any device allocation by the call: the plain FP32 pipeline
// (gather-grid -> row FFT -> column FFT -> products/accumulation) with its grid
// scratch taken from a fixed array that lives in this library's device memory
// image instead of from cudaMalloc.
//
// Who needs it: callers that may not allocate device memory while imaging --
// for example code running inside another framework that owns all device memory
// through its own pool (a second allocator would fragment or exceed it), or a
// real-time loop where a cudaMalloc (which can synchronise the device and take
// milliseconds) is not allowed.  They create plans once at start-up, pass input
// and output buffers they already own, and use this entry point per block.
//
// The scratch array is shared by every call in the process: calls whose work
// overlaps on the GPU (different streams, threads or plans at the same time) race
// on it.  Every scratch byte a call reads is first written by that same call, so
// nothing has to start at zero.  Its device address is looked up once per device
// by the first call made on that device (see epic.h).
#include <algorithm>
#include <mutex>

#include "epic_internal.h"
#include "kcommon.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB of FP32 complex grids per pass
constexpr int kMaxDevices = 64;
constexpr int kNaThreads = 256;
constexpr int kNaColTile = 16;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};
int g_smem_optin[kMaxDevices] = {0};

__global__ void k_na_grid(const uint8_t*, int, int, int, int, int, const int4*, const int*, const int*, const int*,
                          const float2*, float2*);
__global__ void k_na_fft_rows(float2*, size_t, int, int, const float2*);
__global__ void k_na_fft_cols(float2*, int, int, const float2*);

// One-time set-up on the current device: the device address of the scratch array
// (host code may not use the array's name as an address) and the kernels'
// shared-memory limits.  Allocates nothing.
cudaError_t device_setup(int dev, void** ptr, int* smem_optin)
{
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_na_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_na_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_na_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        g_smem_optin[dev] = optin;
        g_addr[dev] = p;
    }
    *ptr = g_addr[dev];
    *smem_optin = g_smem_optin[dev];
    return cudaSuccess;
}

__global__ void __launch_bounds__(kNaThreads) k_na_grid(const uint8_t* __restrict__ volt, int t0, int C, int A, int P,
                                                        int N, const int4* __restrict__ box,
                                                        const int* __restrict__ cell_off,
                                                        const int* __restrict__ cell_ptr,
                                                        const int* __restrict__ ce, const float2* __restrict__ cw,
                                                        float2* __restrict__ grid)
{
    extern __shared__ float2 sv[];  // [A][P]
    const int tl = blockIdx.x, c = blockIdx.y;
    const uint8_t* fr = volt + ((size_t)(t0 + tl) * C + c) * (size_t)A * P;
    for (int i = threadIdx.x; i < A * P; i += blockDim.x) sv[i] = epic::unpack44(fr[i]);
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
            for (int q = ptr[r]; q < ptr[r + 1]; ++q) {
                a0 = epic::cfma(cw[q], sv[ce[q] * P], a0);
                if (P == 2) a1 = epic::cfma(cw[q], sv[ce[q] * P + 1], a1);
            }
        }
        g[cell] = a0;  // every cell written: no scratch state carries over between calls
        if (P == 2) g[NN + cell] = a1;
    }
}

__global__ void __launch_bounds__(kNaThreads) k_na_fft_rows(float2* __restrict__ grid, size_t n_rows, int logN,
                                                            int rows_per_cta, const float2* __restrict__ twg)
{
    extern __shared__ float2 sm[];
    const int N = 1 << logN;
    float2* tw = sm;
    float2* a = sm + N / 2;
    float2* b = a + (size_t)rows_per_cta * N;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) tw[i] = twg[i];
    const size_t r0 = (size_t)blockIdx.x * rows_per_cta;
    const int nr = (int)min((size_t)rows_per_cta, n_rows - r0);
    for (int i = threadIdx.x; i < nr * N; i += blockDim.x) a[i] = grid[r0 * N + i];
    float2* res = epic::fft_stockham(a, b, logN, nr, 1, N, tw);
    for (int i = threadIdx.x; i < nr * N; i += blockDim.x) grid[r0 * N + i] = res[i];
}

__global__ void __launch_bounds__(kNaThreads) k_na_fft_cols(float2* __restrict__ grid, int logN, int tile,
                                                            const float2* __restrict__ twg)
{
    extern __shared__ float2 sm[];
    const int N = 1 << logN, ld = N + 1;
    float2* tw = sm;
    float2* a = sm + N / 2;
    float2* b = a + (size_t)tile * ld;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) tw[i] = twg[i];
    float2* g = grid + (size_t)blockIdx.y * N * N;
    const int x0 = blockIdx.x * tile;
    for (int i = threadIdx.x; i < N * tile; i += blockDim.x) {
        const int row = i / tile, col = i - row * tile;
        a[col * ld + row] = g[(size_t)row * N + x0 + col];
    }
    float2* res = epic::fft_stockham(a, b, logN, tile, 1, ld, tw);
    for (int i = threadIdx.x; i < N * tile; i += blockDim.x) {
        const int row = i / tile, col = i - row * tile;
        g[(size_t)row * N + x0 + col] = res[col * ld + row];
    }
}

__global__ void __launch_bounds__(kNaThreads) k_na_sqacc(const float2* __restrict__ grid, int nt, int C, int P, int N,
                                                         float* __restrict__ out, int accumulate)
{
    const size_t NN = (size_t)N * N;
    const size_t pix = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (pix >= NN) return;
    float xx = 0.f, yy = 0.f, rxy = 0.f, ixy = 0.f;
    for (int tl = 0; tl < nt; ++tl) {
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
    const int nprod = P == 2 ? 4 : 1;
    float* o = out + (size_t)c * nprod * NN + pix;
    o[0] = (accumulate ? o[0] : 0.f) + xx;
    if (P == 2) {
        o[NN] = (accumulate ? o[NN] : 0.f) + yy;
        o[2 * NN] = (accumulate ? o[2 * NN] : 0.f) + rxy;
        o[3 * NN] = (accumulate ? o[3 * NN] : 0.f) + ixy;
    }
}

}  // namespace

extern "C" epic_status epic_image_static_scratch(epic_plan_t p, const uint8_t* volt, int T, void* stream, float* out,
                                                 unsigned flags)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    if (T < 0 || T > p->max_time || !out || (T > 0 && !volt) || (flags & ~EPIC_ACCUMULATE)) {
        p->last_error = "static-scratch imaging: bad T, pointer or flags";
        return EPIC_ERR_INVALID_ARG;
    }
    const int C = p->C, P = p->P, N = p->N, A = p->A;
    const size_t per_t = (size_t)C * P * N * N * sizeof(float2);
    if (p->bits != 4 || p->sub != 0 || !p->jones.empty()) {
        p->last_error = "static-scratch imaging: 4+4-bit input, whole-block images, no polarisation mixing only";
        return EPIC_ERR_UNSUPPORTED;
    }
    if (per_t > kStaticScratchBytes) {
        p->last_error = "static-scratch imaging: one time sample needs " + std::to_string(per_t >> 20) +
                        " MiB of grid scratch (channels x pols x N^2 x 8 bytes); the static scratch holds " +
                        std::to_string(kStaticScratchBytes >> 20) + " MiB";
        return EPIC_ERR_UNSUPPORTED;
    }
    const size_t sg = sizeof(float2) * (size_t)A * P;
    const int rpc = std::max(1, 2048 / N);
    const int tile = std::min(kNaColTile, N);
    const size_t rows_smem = sizeof(float2) * ((size_t)N / 2 + 2ull * rpc * N);
    const size_t cols_smem = sizeof(float2) * ((size_t)N / 2 + 2ull * tile * (N + 1));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        p->last_error = "static-scratch imaging: no usable current device";
        return EPIC_ERR_CUDA;
    }
    void* scratch = nullptr;
    int optin = 0;
    e = device_setup(dev, &scratch, &optin);
    if (e != cudaSuccess) {
        p->last_error = std::string("static-scratch imaging: device set-up (cudaGetSymbolAddress) failed: ") +
                        cudaGetErrorString(e);
        return EPIC_ERR_CUDA;
    }
    if ((int)sg > optin || (int)rows_smem > optin || (int)cols_smem > optin) {
        p->last_error = "static-scratch imaging: element count or grid size needs more shared memory than the device has";
        return EPIC_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool acc = (flags & EPIC_ACCUMULATE) != 0;
    if (T == 0) {
        if (!acc) {
            e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)C * p->nprod * N * N, s);
            if (e != cudaSuccess) {
                p->last_error = std::string("static-scratch imaging: ") + cudaGetErrorString(e);
                return EPIC_ERR_CUDA;
            }
        }
        return EPIC_OK;
    }
    float2* grid = static_cast<float2*>(scratch);
    // time samples per chunk: what fits the array, and at most 65,535 (sample, channel, pol)
    // columns of the column-FFT launch's second grid dimension
    if ((size_t)C * P > 65535) {
        p->last_error = "static-scratch imaging: more than 65,535 channel-polarisations";
        return EPIC_ERR_UNSUPPORTED;
    }
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(kStaticScratchBytes / per_t, 65535 / ((size_t)C * P)));
    for (int t0 = 0; t0 < T; t0 += chunk) {
        const int nt = std::min(chunk, T - t0);
        k_na_grid<<<dim3(nt, C), kNaThreads, sg, s>>>(volt, t0, C, A, P, N, p->dt.box, p->dt.cell_off, p->dt.cell_ptr,
                                                      p->dt.contrib_e, p->dt.contrib_w, grid);
        const size_t n_rows = (size_t)nt * C * P * N;
        k_na_fft_rows<<<(unsigned)((n_rows + rpc - 1) / rpc), kNaThreads, rows_smem, s>>>(grid, n_rows, p->logN, rpc,
                                                                                           p->dt.twiddle);
        k_na_fft_cols<<<dim3(N / tile, (unsigned)((size_t)nt * C * P)), kNaThreads, cols_smem, s>>>(grid, p->logN, tile,
                                                                                                  p->dt.twiddle);
        k_na_sqacc<<<dim3((unsigned)(((size_t)N * N + kNaThreads - 1) / kNaThreads), C), kNaThreads, 0, s>>>(
            grid, nt, C, P, N, out, (acc || t0 > 0) ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            p->last_error = std::string("static-scratch imaging launch: ") + cudaGetErrorString(e);
            return EPIC_ERR_CUDA;
        }
    }
    return EPIC_OK;
}
