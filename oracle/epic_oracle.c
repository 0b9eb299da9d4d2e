/*
 * FP64 CPU oracle for the EPIC imaging path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  The CUDA library never includes, links or
 * calls it, and this file uses nothing from the CUDA library (not even its
 * header): geometry, footprints, unpacking, gridding, the transform and the
 * products are all written out again here from the paper's equations.
 *
 * What it computes (paper Sec. 2):
 *   Eq. 1  E^a(s_k) = sum_j d2r_j exp(+i 2pi/lambda s_k . r_j) ( sum_e sum_p W_e^{ap*}(r_j - r_e) E_e^p )
 *          -- "gridding" (the bracket) then a 2-D Fourier sum over grid points
 *          (the outer sum, which the paper implements with an FFT).
 *   Eq. 2  I^{ab}(s_k) = < E^a(s_k) E^{b*}(s_k) >   -- pixelwise outer product
 *          of the polarisations, averaged (here: summed) over the integration.
 *
 * Readings taken where the paper is silent (each is also listed in the design notes):
 *   - W^{ap} = delta_{ap} W (one GCF shared by both pols, no pol mixing) unless a mixing
 *     kernel is given; then W_e^{ap}(r) = J_e^{ap} W(r) with a complex 2x2 J per element
 *     and channel (direction-independent leakage; eo_grid_mix takes Eq. 1's double sum).
 *   - Grid spacing Delta_c = lambda_c/2 unless given; element cell coordinates are
 *     u = (x - xbar)/Delta + N/2, v = (y - ybar)/Delta + N/2 with (xbar, ybar) the
 *     array centroid; grid point j sits at integer cell j.
 *   - Footprint: odd K -> anchor floor(u + 1/2), taps anchor-(K-1)/2 .. anchor+(K-1)/2;
 *     even K -> taps floor(u)-K/2+1 .. floor(u)+K/2.  Any tap outside [0, N) is an
 *     error; taps never wrap.
 *   - Gaussian GCF W(d) = exp(-|d|^2 / (2 sigma_c^2)) in cells, not renormalised;
 *     sigma_c = sigma * f_c / f_ref when frequency scaled.  Tabulated GCF: complex
 *     samples at offsets (i/os - K/2) per axis, nearest sample (ties up).
 *   - Unpack: real part = high nibble, imaginary = low nibble, two's complement; for
 *     8+8-bit input (paper Sec. 4) the real byte precedes the imaginary byte.
 *   - d2r_j = 1, transform sign +, no 1/N; the image index i stores Fourier index
 *     k = (i + N/2) mod N (fftshift), rows = y (m), columns = x (l).
 *   - Products: XX = |E_X|^2, YY = |E_Y|^2, XY = E_X conj(E_Y) stored as Re, Im;
 *     YX = conj(XY) is not stored.  One pol: XX only.
 *   - <.> is the SUM over the block's time samples (the caller divides by T), or over
 *     each interval of `sub` samples when sub-integrations are asked for (Sec. 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EO_OK 0
#define EO_ERR_ARG 1
#define EO_ERR_OVERFLOW 2
#define EO_ERR_OOM 3

static const double EO_C0 = 299792458.0;
static const double EO_PI = 3.14159265358979323846;

/* ---- unpack (4+4-bit two's complement, real in the high nibble) ---------------- */
static int eo_nibble(unsigned v) { return (v & 0x8u) ? (int)v - 16 : (int)v; }

void eo_unpack(uint8_t b, int* re, int* im)
{
    *re = eo_nibble((unsigned)b >> 4);
    *im = eo_nibble((unsigned)b & 0xFu);
}

/* ---- unpack (8+8-bit two's complement: real byte, then imaginary byte) ---------- */
static int eo_byte(unsigned v) { return (v & 0x80u) ? (int)v - 256 : (int)v; }

void eo_unpack8(const uint8_t* b, int* re, int* im)
{
    *re = eo_byte(b[0]);
    *im = eo_byte(b[1]);
}

/* ---- geometry and GCF footprint of one channel (Eq. 1 bracket: W(r_j - r_e)) ---- */
/* tap_x/tap_y: [A][K] first cell index per axis is tap_x[e*K+0]; w: [A][K][K][2]
 * holding conj(W) at (row ty, column tx) for element e.  Returns EO_ERR_OVERFLOW
 * if a tap leaves [0, N). */
int eo_footprint(int n_ant, const double* pos_m, double freq_hz, double cell_m, int N,
                 int gcf_kind, int K, double sigma_cells, double f_ref_hz, int freq_scaled,
                 int oversample, const float* table,
                 int* tap_x, int* tap_y, double* w)
{
    if (n_ant < 1 || N < 2 || K < 1 || freq_hz <= 0.0) return EO_ERR_ARG;
    double lam = EO_C0 / freq_hz;
    double delta = cell_m > 0.0 ? cell_m : 0.5 * lam;
    double xbar = 0.0, ybar = 0.0;
    for (int e = 0; e < n_ant; ++e) { xbar += pos_m[2 * e]; ybar += pos_m[2 * e + 1]; }
    xbar /= n_ant;
    ybar /= n_ant;
    double sig = sigma_cells;
    if (freq_scaled) sig = sigma_cells * freq_hz / f_ref_hz;
    for (int e = 0; e < n_ant; ++e) {
        double u = (pos_m[2 * e] - xbar) / delta + 0.5 * N;
        double v = (pos_m[2 * e + 1] - ybar) / delta + 0.5 * N;
        int fx, fy;
        if (K % 2 == 1) {
            fx = (int)floor(u + 0.5) - (K - 1) / 2;
            fy = (int)floor(v + 0.5) - (K - 1) / 2;
        } else {
            fx = (int)floor(u) - K / 2 + 1;
            fy = (int)floor(v) - K / 2 + 1;
        }
        if (fx < 0 || fy < 0 || fx + K - 1 >= N || fy + K - 1 >= N) return EO_ERR_OVERFLOW;
        for (int k = 0; k < K; ++k) { tap_x[e * K + k] = fx + k; tap_y[e * K + k] = fy + k; }
        for (int ty = 0; ty < K; ++ty) {
            for (int tx = 0; tx < K; ++tx) {
                double dx = (double)(fx + tx) - u;
                double dy = (double)(fy + ty) - v;
                double wr, wi;
                if (gcf_kind == 0) {
                    wr = exp(-(dx * dx + dy * dy) / (2.0 * sig * sig));
                    wi = 0.0;
                } else {
                    int side = K * oversample + 1;
                    int ix = (int)floor((dx + 0.5 * K) * oversample + 0.5);
                    int iy = (int)floor((dy + 0.5 * K) * oversample + 0.5);
                    if (ix < 0) ix = 0;
                    if (iy < 0) iy = 0;
                    if (ix > side - 1) ix = side - 1;
                    if (iy > side - 1) iy = side - 1;
                    wr = table[2 * (iy * side + ix)];
                    wi = -(double)table[2 * (iy * side + ix) + 1]; /* W* */
                }
                double* o = w + (((size_t)e * K + ty) * K + tx) * 2;
                o[0] = wr;
                o[1] = wi;
            }
        }
    }
    return EO_OK;
}

/* ---- 1-D DFT with the + sign, unnormalised: radix-2 decimation in time -------- */
static void eo_fft1(double* re, double* im, int n)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int m = 0; m < half; ++m) {
            double ang = 2.0 * EO_PI * (double)m / (double)len; /* exp(+i ang) */
            double cr = cos(ang), ci = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + m, b = s + m + half;
                double tr = re[b] * cr - im[b] * ci;
                double ti = re[b] * ci + im[b] * cr;
                re[b] = re[a] - tr;
                im[b] = im[a] - ti;
                re[a] += tr;
                im[a] += ti;
            }
        }
    }
}

/* 2-D transform of g[N][N][2] (row y, column x) in place: F[ky][kx] = sum g[y][x] e^{+2pi i (x kx + y ky)/N}. */
int eo_fft2(double* g, int N)
{
    if (N < 1 || (N & (N - 1))) return EO_ERR_ARG;
    double* re = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)malloc(sizeof(double) * (size_t)N);
    if (!re || !im) { free(re); free(im); return EO_ERR_OOM; }
    for (int y = 0; y < N; ++y) {
        for (int x = 0; x < N; ++x) { re[x] = g[(y * N + x) * 2]; im[x] = g[(y * N + x) * 2 + 1]; }
        eo_fft1(re, im, N);
        for (int x = 0; x < N; ++x) { g[(y * N + x) * 2] = re[x]; g[(y * N + x) * 2 + 1] = im[x]; }
    }
    for (int x = 0; x < N; ++x) {
        for (int y = 0; y < N; ++y) { re[y] = g[(y * N + x) * 2]; im[y] = g[(y * N + x) * 2 + 1]; }
        eo_fft1(re, im, N);
        for (int y = 0; y < N; ++y) { g[(y * N + x) * 2] = re[y]; g[(y * N + x) * 2 + 1] = im[y]; }
    }
    free(re);
    free(im);
    return EO_OK;
}

/* ---- gridding of one (t, c, p) frame: G[j] = sum_e w_e(j) E_e^p (Eq. 1 bracket) --- */
static void eo_grid(int n_ant, int K, int N, const int* tap_x, const int* tap_y, const double* w,
                    const uint8_t* frame /* [A][P] samples */, int P, int p, int bits, double* g /* [N][N][2] */)
{
    memset(g, 0, sizeof(double) * 2 * (size_t)N * N);
    for (int e = 0; e < n_ant; ++e) {
        int vr, vi;
        if (bits == 8) eo_unpack8(frame + 2 * ((size_t)e * P + p), &vr, &vi);
        else eo_unpack(frame[e * P + p], &vr, &vi);
        for (int ty = 0; ty < K; ++ty) {
            for (int tx = 0; tx < K; ++tx) {
                const double* c = w + (((size_t)e * K + ty) * K + tx) * 2;
                int jx = tap_x[e * K + tx], jy = tap_y[e * K + ty];
                double* o = g + ((size_t)jy * N + jx) * 2;
                o[0] += c[0] * vr - c[1] * vi;
                o[1] += c[0] * vi + c[1] * vr;
            }
        }
    }
}

/* ---- gridding with a polarisation-mixing kernel (Eq. 1 in full) ----------------
 * Output pol a of one dual-pol frame: G^a[j] = sum_e sum_p conj(W_e^{ap}(r_j - r_e)) E_e^p,
 * the element kernel being W_e^{ap}(r) = J_e^{ap} W(r) with J_e a complex 2x2 matrix
 * (jones_c: [A][2][2][2] doubles, J^{ap} of element e at ((e * 2 + a) * 2 + p) * 2) and w
 * holding conj(W) per tap.  Each tap of each element applies both of its kernel entries
 * conj(J^{ap}) conj(W) to the two input pols, as the double sum reads. */
static void eo_grid_mix(int n_ant, int K, int N, const int* tap_x, const int* tap_y, const double* w,
                        const uint8_t* frame, int a, int bits, const double* jones_c, double* g)
{
    memset(g, 0, sizeof(double) * 2 * (size_t)N * N);
    for (int e = 0; e < n_ant; ++e) {
        int vr[2], vi[2];
        for (int p = 0; p < 2; ++p) {
            if (bits == 8) eo_unpack8(frame + 2 * ((size_t)e * 2 + p), &vr[p], &vi[p]);
            else eo_unpack(frame[e * 2 + p], &vr[p], &vi[p]);
        }
        for (int ty = 0; ty < K; ++ty) {
            for (int tx = 0; tx < K; ++tx) {
                const double* c = w + (((size_t)e * K + ty) * K + tx) * 2;   /* conj(W) */
                int jx = tap_x[e * K + tx], jy = tap_y[e * K + ty];
                double* o = g + ((size_t)jy * N + jx) * 2;
                for (int p = 0; p < 2; ++p) {
                    const double* J = jones_c + (((size_t)e * 2 + a) * 2 + p) * 2;
                    /* conj(J W) = conj(J) conj(W) */
                    const double kr = J[0] * c[0] + J[1] * c[1];
                    const double ki = J[0] * c[1] - J[1] * c[0];
                    o[0] += kr * vr[p] - ki * vi[p];
                    o[1] += kr * vi[p] + ki * vr[p];
                }
            }
        }
    }
}

/* Grid one frame (exposed for transform-level checks such as Parseval). */
int eo_grid_frame(int n_ant, const double* pos_m, int n_pol, int n_chan, const double* freq_hz,
                  const double* cell_m, int N, int gcf_kind, int K, double sigma_cells, double f_ref_hz,
                  int freq_scaled, int oversample, const float* table,
                  const uint8_t* volt, int t, int c, int p, double* g)
{
    if (c < 0 || c >= n_chan || p < 0 || p >= n_pol) return EO_ERR_ARG;
    int* tx = (int*)malloc(sizeof(int) * (size_t)n_ant * K);
    int* ty = (int*)malloc(sizeof(int) * (size_t)n_ant * K);
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n_ant * K * K);
    int rc = EO_ERR_OOM;
    if (tx && ty && w) {
        rc = eo_footprint(n_ant, pos_m, freq_hz[c], cell_m ? cell_m[c] : 0.0, N, gcf_kind, K, sigma_cells,
                          f_ref_hz, freq_scaled, oversample, table, tx, ty, w);
        if (rc == EO_OK) {
            const uint8_t* frame = volt + ((size_t)t * n_chan + c) * (size_t)n_ant * n_pol;
            eo_grid(n_ant, K, N, tx, ty, w, frame, n_pol, p, 4, g);
        }
    }
    free(tx); free(ty); free(w);
    return rc;
}

/* ---- whole path for a set of channels ---------------------------------------- */
/* volt: uint8[T][n_chan][A][P] (bits = 4: one byte per sample) or uint8[T][n_chan][A][P][2]
 * (bits = 8: real byte, imaginary byte); chans: n_sel channel indices (NULL = all);
 * sub: time samples per output image (0 = one image set for the whole block; T a multiple of sub);
 * jones: NULL (W_e^{ap} = delta_ap W) or double[n_chan][A][2][2][2], the complex 2x2 polarisation-
 * mixing matrix J^{ap} of each element and channel (n_pol = 2; see eo_grid_mix);
 * out: double[n_int][n_sel][nprod][N][N] with n_int = T / sub (1 when sub = 0) and nprod = 1
 * (P = 1) or 4 (XX, YY, Re XY, Im XY): Eq. 2's average taken (as a sum) over each interval. */
int eo_image_ext(int n_ant, const double* pos_m, int n_pol, int n_chan, const double* freq_hz,
                 const double* cell_m, int N, int gcf_kind, int K, double sigma_cells, double f_ref_hz,
                 int freq_scaled, int oversample, const float* table,
                 const uint8_t* volt, int T, int bits, int sub, const double* jones, int n_sel, const int* chans,
                 double* out, int n_threads)
{
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_chan < 1 || N < 2 || (N & (N - 1)) || K < 1 ||
        T < 0 || n_sel < 0 || (bits != 4 && bits != 8) || sub < 0 || (sub > 0 && T % sub != 0) ||
        (jones && n_pol != 2))
        return EO_ERR_ARG;
    if (!chans) n_sel = n_chan;
    int nprod = n_pol == 1 ? 1 : 4;
    const int n_int = sub > 0 ? T / sub : 1;
    const int span = sub > 0 ? sub : T;            /* samples per interval */
    const size_t bytes = bits == 8 ? 2 : 1;        /* per complex sample */
    int status = EO_OK;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < n_sel; ++s) {
        int c = chans ? chans[s] : s;
        if (c < 0 || c >= n_chan) { status = EO_ERR_ARG; continue; }
        int* tx = (int*)malloc(sizeof(int) * (size_t)n_ant * K);
        int* ty = (int*)malloc(sizeof(int) * (size_t)n_ant * K);
        double* w = (double*)malloc(sizeof(double) * 2 * (size_t)n_ant * K * K);
        double* g = (double*)malloc(sizeof(double) * 2 * (size_t)N * N * n_pol);
        double* acc = (double*)calloc((size_t)nprod * N * N, sizeof(double));
        if (!tx || !ty || !w || !g || !acc) {
            status = EO_ERR_OOM;
        } else {
            int rc = eo_footprint(n_ant, pos_m, freq_hz[c], cell_m ? cell_m[c] : 0.0, N, gcf_kind, K,
                                  sigma_cells, f_ref_hz, freq_scaled, oversample, table, tx, ty, w);
            if (rc != EO_OK) {
                status = rc;
            } else {
                size_t NN = (size_t)N * N;
                for (int iv = 0; iv < n_int; ++iv) {
                    memset(acc, 0, sizeof(double) * (size_t)nprod * NN);
                    for (int t = iv * span; t < (iv + 1) * span; ++t) {
                        const uint8_t* frame = volt + ((size_t)t * n_chan + c) * (size_t)n_ant * n_pol * bytes;
                        for (int p = 0; p < n_pol; ++p) {
                            if (jones)
                                eo_grid_mix(n_ant, K, N, tx, ty, w, frame, p, bits,
                                            jones + (size_t)c * n_ant * 8, g + p * 2 * NN);
                            else
                                eo_grid(n_ant, K, N, tx, ty, w, frame, n_pol, p, bits, g + p * 2 * NN);
                            eo_fft2(g + p * 2 * NN, N);
                        }
                        for (size_t k = 0; k < NN; ++k) {
                            double xr = g[2 * k], xi = g[2 * k + 1];
                            acc[k] += xr * xr + xi * xi;
                            if (n_pol == 2) {
                                double yr = g[2 * NN + 2 * k], yi = g[2 * NN + 2 * k + 1];
                                acc[NN + k] += yr * yr + yi * yi;
                                acc[2 * NN + k] += xr * yr + xi * yi;   /* Re X conj(Y) */
                                acc[3 * NN + k] += xi * yr - xr * yi;   /* Im X conj(Y) */
                            }
                        }
                    }
                    /* fftshift on output: image index i holds Fourier index (i + N/2) mod N */
                    double* o = out + ((size_t)iv * n_sel + s) * nprod * NN;
                    for (int q = 0; q < nprod; ++q)
                        for (int iy = 0; iy < N; ++iy)
                            for (int ix = 0; ix < N; ++ix) {
                                int ky = (iy + N / 2) % N, kx = (ix + N / 2) % N;
                                o[q * NN + (size_t)iy * N + ix] = acc[q * NN + (size_t)ky * N + kx];
                            }
                }
            }
        }
        free(tx); free(ty); free(w); free(g); free(acc);
    }
    return status;
}

/* The 4+4-bit, whole-block form of eo_image_ext. */
int eo_image(int n_ant, const double* pos_m, int n_pol, int n_chan, const double* freq_hz,
             const double* cell_m, int N, int gcf_kind, int K, double sigma_cells, double f_ref_hz,
             int freq_scaled, int oversample, const float* table,
             const uint8_t* volt, int T, int n_sel, const int* chans, double* out, int n_threads)
{
    return eo_image_ext(n_ant, pos_m, n_pol, n_chan, freq_hz, cell_m, N, gcf_kind, K, sigma_cells, f_ref_hz,
                        freq_scaled, oversample, table, volt, T, 4, 0, NULL, n_sel, chans, out, n_threads);
}

int eo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
