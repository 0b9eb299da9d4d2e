// Small device helpers shared by the EPIC kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace epic {

// One packed voltage byte -> complex float: real = high nibble, imaginary = low
// nibble, both 4-bit two's complement (sign-extended by arithmetic shifts).
__device__ __forceinline__ float2 unpack44(uint32_t b)
{
    const int re = ((int)(b << 24)) >> 28;
    const int im = ((int)(b << 28)) >> 28;
    return make_float2((float)re, (float)im);
}

// Complex sample idx (= element * P + pol) of one frame: a 4+4-bit byte (bits 4) or a
// real byte followed by an imaginary byte (bits 8, paper Sec. 4), two's complement.
__device__ __forceinline__ float2 load_sample(const uint8_t* frame, size_t idx, int bits)
{
    if (bits == 8) {
        const char2 v = *reinterpret_cast<const char2*>(frame + 2 * idx);
        return make_float2((float)v.x, (float)v.y);
    }
    return unpack44(frame[idx]);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b);
__device__ __forceinline__ float2 cfma(float2 w, float2 v, float2 acc);

// Both polarisations of element e of a dual-pol frame, as (X re, X im, Y re, Y im).
// With a polarisation-mixing kernel (Eq. 1 with W_e^{ap}(r) = J_e^{ap} W(r), a
// complex 2x2 J per element and channel) the sample of output polarisation a is
// sum_p conj(J_e^{ap}) E_e^p, which is what gridding with W^{ap*} gives once W*
// is factored out; jm[2 e + a] = (conj J^{a0}, conj J^{a1}).  jm == nullptr: no mixing.
__device__ __forceinline__ float4 load_pair(const uint8_t* frame, int e, int bits, const float4* jm)
{
    const float2 x = load_sample(frame, (size_t)e * 2, bits);
    const float2 y = load_sample(frame, (size_t)e * 2 + 1, bits);
    if (!jm) return make_float4(x.x, x.y, y.x, y.y);
    const float4 r0 = jm[2 * e], r1 = jm[2 * e + 1];
    const float2 mx = cfma(make_float2(r0.z, r0.w), y, cmul(make_float2(r0.x, r0.y), x));
    const float2 my = cfma(make_float2(r1.z, r1.w), y, cmul(make_float2(r1.x, r1.y), x));
    return make_float4(mx.x, mx.y, my.x, my.y);
}

// Element e of a frame with P = 1 or 2 polarisations as (X re, X im, Y re, Y im),
// Y zero for one polarisation; mixed by jm as in load_pair (P == 2 only).
__device__ __forceinline__ float4 load_quad(const uint8_t* frame, int e, int P, int bits, const float4* jm)
{
    if (P == 2) return load_pair(frame, e, bits, jm);
    const float2 x = load_sample(frame, (size_t)e, bits);
    return make_float4(x.x, x.y, 0.f, 0.f);
}

// acc + w * v for complex numbers.
__device__ __forceinline__ float2 cfma(float2 w, float2 v, float2 acc)
{
    acc.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc.x));
    acc.y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc.y));
    return acc;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Stage one frame's samples as float2 [A][P] in shared memory (all threads of the
// block take part), mixed by jm as in load_pair when jm != nullptr (P == 2 only).
__device__ __forceinline__ void stage_frame(float2* dst, const uint8_t* frame, int A, int P, int bits,
                                            const float4* jm)
{
    if (jm) {
        for (int e = threadIdx.x; e < A; e += blockDim.x) {
            const float4 v = load_pair(frame, e, bits, jm);
            dst[2 * e] = make_float2(v.x, v.y);
            dst[2 * e + 1] = make_float2(v.z, v.w);
        }
    } else {
        for (int i = threadIdx.x; i < A * P; i += blockDim.x) dst[i] = load_sample(frame, i, bits);
    }
}

// Stockham autosort FFT with the + sign (Eq. 1), unnormalised, on `batch` transforms of
// length n = 2^logn held in shared memory: element i of transform q is buf[q * bs + i * es].
// Radix-4 stages (spans 1, 4, 16, ...), then one radix-2 stage when logn is odd, so a
// transform takes ceil(logn / 2) passes over shared memory (N = 128: 4 instead of 7).  A
// radix-4 stage of span L turns v_r = a[j + r n/4] w^(r k n / 4L) (k = j mod L, w =
// exp(+2 pi i / n)) into the 4-point DFT y_q = sum_r v_r i^(r q), stored at
// (j / L) 4L + k + q L.  Ping-pongs between a and b; returns the buffer holding the
// natural-order result.  tw[m] = exp(+2 pi i m / n), m < n/2 (w^m = -tw[m - n/2] above).
// Ends with __syncthreads(); all threads of the block must call it.
__device__ __forceinline__ float2* fft_stockham(float2* a, float2* b, int logn, int batch, int es, int bs,
                                                const float2* tw)
{
    const int n = 1 << logn, n4 = n >> 2, half = n >> 1;
    auto W = [&](int m) {
        const float2 t = tw[m < half ? m : m - half];
        return m < half ? t : make_float2(-t.x, -t.y);
    };
    __syncthreads();
    int ls = 0;
    for (; ls + 2 <= logn; ls += 2) {
        const int L = 1 << ls;
        for (int w = threadIdx.x; w < batch * n4; w += blockDim.x) {
            const int q = w >> (logn - 2);
            const int j = w & (n4 - 1);
            const int k = j & (L - 1);
            const int e1 = k << (logn - 2 - ls);
            const float2* src = a + q * bs;
            const float2 v0 = src[j * es];
            const float2 v1 = cmul(src[(j + n4) * es], W(e1));
            const float2 v2 = cmul(src[(j + 2 * n4) * es], W(2 * e1));
            const float2 v3 = cmul(src[(j + 3 * n4) * es], W(3 * e1));
            const float2 s02 = make_float2(v0.x + v2.x, v0.y + v2.y), d02 = make_float2(v0.x - v2.x, v0.y - v2.y);
            const float2 s13 = make_float2(v1.x + v3.x, v1.y + v3.y), d13 = make_float2(v1.x - v3.x, v1.y - v3.y);
            const int idx = ((j >> ls) << (ls + 2)) + k;
            float2* dst = b + q * bs;
            dst[idx * es] = make_float2(s02.x + s13.x, s02.y + s13.y);
            dst[(idx + L) * es] = make_float2(d02.x - d13.y, d02.y + d13.x);      // + i (v1 - v3)
            dst[(idx + 2 * L) * es] = make_float2(s02.x - s13.x, s02.y - s13.y);
            dst[(idx + 3 * L) * es] = make_float2(d02.x + d13.y, d02.y - d13.x);  // - i (v1 - v3)
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
    }
    if (ls < logn) {  // the last factor 2
        const int L = 1 << ls;
        for (int w = threadIdx.x; w < batch * half; w += blockDim.x) {
            const int q = w >> (logn - 1);
            const int j = w & (half - 1);
            const int k = j & (L - 1);
            const float2 v0 = a[q * bs + j * es];
            const float2 v1 = cmul(a[q * bs + (j + half) * es], tw[k << (logn - 1 - ls)]);
            const int idx = ((j >> ls) << (ls + 1)) + k;
            b[q * bs + idx * es] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[q * bs + (idx + L) * es] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace epic
