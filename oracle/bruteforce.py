"""Pairwise-correlation brute force of the EPIC image -- TEST INFRASTRUCTURE.

The EPIC image (paper Sec. 2, Eq. 1-2) avoids forming the pairwise products of
element voltages (Sec. 1: the O(N_e^2) correlator it replaces).  Expanding
Eq. 2 with Eq. 1 shows that the two routes give the same image:

    I^{ab}[k] = sum_d exp(+2 pi i d.k / N) sum_{e,e'} V^{ab}_{ee'} R_{ee'}[d],
    V^{ab}_{ee'} = sum_t E^a_e(t) conj(E^b_{e'}(t))          (visibilities, e = e' included)
    R_{ee'}[d]   = sum_j w_e(j + d) conj(w_{e'}(j))           (circular, mod N)

i.e. correlate every pair of elements (an FX correlator), grid each visibility
with the cross-correlation of the two sampled GCF footprints, and take the 2-D
+ sign DFT.  This module evaluates that route directly with numpy, with its
own geometry, footprint and nibble decoding, and with an explicit DFT matrix
(no FFT), so that it shares nothing with ``epic_oracle.c`` but the readings
(centroid origin, anchor rule, Gaussian GCF, fftshifted output).

Cost is O(A^2 N^4): tiny arrays only (A <= 16, N <= 16).
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299_792_458.0


def decode_nibbles(b: np.ndarray) -> np.ndarray:
    """Complex value of each packed byte, two's complement via (v ^ 8) - 8."""
    b = np.asarray(b, dtype=np.int64)
    re = ((b >> 4) ^ 8) - 8
    im = ((b & 15) ^ 8) - 8
    return re + 1j * im


def _table_lookup(table, K, oversample, d):
    """Index of the nearest tabulated sample (ties up) at offsets d (cells)."""
    side = K * oversample + 1
    idx = np.clip(np.floor((d + 0.5 * K) * oversample + 0.5).astype(np.int64), 0, side - 1)
    return idx


def dense_footprints(pos_m, freq_hz, grid_n, gcf_k, sigma_cells, f_ref_hz=1.0, freq_scaled=False,
                     cell_m=None, table=None, oversample=1):
    """complex[A][N][N]: conj(W(r_j - r_e)) on each element's K x K taps, zero elsewhere.

    W is the Gaussian exp(-|d|^2/(2 sigma^2)) or, when ``table`` (complex
    [(K*os+1)][(K*os+1)] as float pairs) is given, its nearest sample."""
    pos = np.asarray(pos_m, dtype=np.float64)
    lam = C0 / freq_hz
    delta = 0.5 * lam if cell_m is None else cell_m
    ctr = pos.mean(axis=0)
    uv = (pos - ctr) / delta + grid_n / 2.0                      # [A][2] continuous cells
    K = gcf_k
    if K % 2:
        first = np.floor(uv + 0.5).astype(np.int64) - (K - 1) // 2
    else:
        first = np.floor(uv).astype(np.int64) - K // 2 + 1
    if (first < 0).any() or (first + K - 1 >= grid_n).any():
        raise ValueError("footprint leaves the grid")
    sig = sigma_cells * freq_hz / f_ref_hz if freq_scaled else sigma_cells
    out = np.zeros((pos.shape[0], grid_n, grid_n), dtype=np.complex128)
    for e in range(pos.shape[0]):
        js = first[e, 0] + np.arange(K)                          # x cells
        iy = first[e, 1] + np.arange(K)                          # y cells
        dx = js - uv[e, 0]
        dy = iy - uv[e, 1]
        if table is None:
            w = np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * sig * sig))
        else:
            tab = np.asarray(table, dtype=np.float64)
            tc = tab[..., 0] + 1j * tab[..., 1]
            w = tc[np.ix_(_table_lookup(tab, K, oversample, dy), _table_lookup(tab, K, oversample, dx))]
        out[e][np.ix_(iy, js)] = np.conj(w)
    return out


def footprint_xcorr(wd: np.ndarray) -> np.ndarray:
    """R[e][f][dy][dx] = sum_j w_e(j + d) conj(w_f(j)), indices mod N."""
    A, N, _ = wd.shape
    flat_conj = np.conj(wd.reshape(A, N * N))
    R = np.zeros((A, A, N, N), dtype=np.complex128)
    for dy in range(N):
        for dx in range(N):
            shifted = np.roll(wd, shift=(-dy, -dx), axis=(1, 2)).reshape(A, N * N)   # w_e(j + d)
            R[:, :, dy, dx] = shifted @ flat_conj.T
    return R


def image(volt: np.ndarray, pos_m, freq_hz, n_pol, grid_n, gcf_k, sigma_cells, f_ref_hz=1.0,
          freq_scaled=False, cell_m=None, table=None, oversample=1, jones=None, input_bits=4) -> np.ndarray:
    """float64[C][nprod][N][N] through visibilities (same output convention as the oracle).

    jones (complex [C][A][2][2], optional): element kernels J_e^{ap} W(r).  Because such a
    kernel factors into a matrix per element and the shared W, the correlator sees the
    element's voltages after mixing, sum_p conj(J^{ap}) E^p, and grids with W as before."""
    v = np.asarray(volt)
    if input_bits == 8:                                          # (real, imaginary) int8 pairs
        b = v.view(np.int8).astype(np.int64)
        E = b[..., 0] + 1j * b[..., 1]
    else:
        E = decode_nibbles(v)                                    # [T][C][A][P]
    T, C, A, P = E.shape
    N = grid_n
    if jones is not None:
        E = np.einsum("caqp,tcap->tcaq", np.conj(np.asarray(jones, dtype=np.complex128)), E)
    kk = np.arange(N)
    D = np.exp(2j * math.pi * np.outer(kk, kk) / N)              # D[k][d], + sign
    shift = (np.arange(N) + N // 2) % N                          # image index -> Fourier index
    nprod = 1 if P == 1 else 4
    out = np.zeros((C, nprod, N, N))
    for c in range(C):
        wd = dense_footprints(pos_m, float(freq_hz[c]), N, gcf_k, sigma_cells, f_ref_hz, freq_scaled,
                              None if cell_m is None else float(cell_m[c]), table, oversample)
        R = footprint_xcorr(wd)
        pairs = [(0, 0)] if P == 1 else [(0, 0), (1, 1), (0, 1)]
        imgs = []
        for a, b in pairs:
            V = np.einsum("te,tf->ef", E[:, c, :, a], np.conj(E[:, c, :, b]))   # correlator
            Vg = np.einsum("ef,efyx->yx", V, R)                                  # gridded visibilities
            I = D @ Vg @ D.T                                                     # I[ky][kx]
            imgs.append(I[np.ix_(shift, shift)])
        out[c, 0] = imgs[0].real
        if P == 2:
            out[c, 1] = imgs[1].real
            out[c, 2] = imgs[2].real
            out[c, 3] = imgs[2].imag
    return out
