"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each check uses an independent
route (hand-written codes, numpy's inverse FFT, a naive DFT matrix, closed
forms, Parseval, the pairwise-correlation brute force, invariants).
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import epic_synth as synth
import oracle
from oracle import bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = synth.C0


# ----------------------------------------------------------------------------- unpack

def test_unpack_hand_codes():
    table = oracle.unpack_table()
    n = 0
    with open(os.path.join(GOLDEN, "unpack_codes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            b, re, im = line.split()
            assert tuple(table[int(b, 16)]) == (int(re), int(im)), b
            n += 1
    assert n >= 16


def test_unpack_exhaustive_bijection_and_roundtrip():
    table = oracle.unpack_table()
    assert table.min() == -8 and table.max() == 7
    pairs = {tuple(r) for r in table}
    assert len(pairs) == 256                                   # every (re, im) in [-8, 7]^2 exactly once
    packed = synth.pack_nibbles(table[:, 0], table[:, 1])
    assert np.array_equal(packed, np.arange(256, dtype=np.uint8))
    assert np.array_equal(bruteforce.decode_nibbles(np.arange(256)),
                          table[:, 0] + 1j * table[:, 1])


# ----------------------------------------------------------------------------- transform

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
def test_fft2_matches_naive_dft_and_numpy(n):
    rng = np.random.default_rng(n)
    g = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    got = oracle.fft2(g)
    k = np.arange(n)
    D = np.exp(2j * math.pi * np.outer(k, k) / n)              # + sign, no 1/N
    naive = D @ g @ D.T
    assert np.abs(got - naive).max() <= 1e-12 * max(1.0, np.abs(naive).max())
    # the + sign unnormalised transform is N^2 times numpy's inverse FFT
    assert np.abs(got - np.fft.ifft2(g) * n * n).max() <= 1e-12 * max(1.0, np.abs(naive).max())


@pytest.mark.parametrize("n", [256, 512])
def test_fft2_large_grids_match_numpy(n):
    # the largest grids the library takes (512 x 512): against numpy's inverse FFT x N^2
    rng = np.random.default_rng(n + 1)
    g = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    got = oracle.fft2(g)
    ref = np.fft.ifft2(g) * n * n
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_fft2_single_impulse_is_plane_wave():
    n = 16
    g = np.zeros((n, n), complex)
    g[3, 5] = 1.0
    got = oracle.fft2(g)
    ky, kx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.allclose(got, np.exp(2j * math.pi * (5 * kx + 3 * ky) / n), atol=1e-13)


# ----------------------------------------------------------------------------- footprint

def test_footprint_anchor_and_weights_hand_cases():
    # two elements symmetric about the centroid, cell spacing 1 m given explicitly
    pos = np.array([[-1.5, 0.25], [1.5, -0.25]])
    N = 16
    # odd K=3: u = -1.5 + 8 = 6.5 -> anchor floor(7.0) = 7 (tie rounds up); v = 8.25 -> 8
    tx, ty, w = oracle.footprint(pos, 100e6, N, 3, 1.0, cell_m=1.0)
    assert list(tx[0]) == [6, 7, 8] and list(ty[0]) == [7, 8, 9]
    assert list(tx[1]) == [9, 10, 11] and list(ty[1]) == [7, 8, 9]     # u = 9.5 -> 10, v = 7.75 -> 8
    # weight of tap (ty=8, tx=7) of element 0: d = (7 - 6.5, 8 - 8.25) = (0.5, -0.25)
    assert w[0, 1, 1] == pytest.approx(math.exp(-(0.25 + 0.0625) / 2.0), rel=1e-14)
    assert np.all(np.imag(w) == 0.0)
    # even K=2 (the paper's 2x2 kernel): taps floor(u) .. floor(u)+1
    tx, ty, _ = oracle.footprint(pos, 100e6, N, 2, 1.0, cell_m=1.0)
    assert list(tx[0]) == [6, 7] and list(ty[0]) == [8, 9]
    assert list(tx[1]) == [9, 10] and list(ty[1]) == [7, 8]
    # K=4: floor(u)-1 .. floor(u)+2
    tx, ty, _ = oracle.footprint(pos, 100e6, N, 4, 1.0, cell_m=1.0)
    assert list(tx[0]) == [5, 6, 7, 8]


def test_footprint_default_spacing_and_frequency_scaling():
    lam = 2.0
    f = C0 / lam
    pos = np.array([[-0.5, 0.0], [0.5, 0.0]])                  # 1 m apart = one half-wavelength cell
    tx, _, w = oracle.footprint(pos, f, 8, 1, 0.5)
    assert tx[1, 0] - tx[0, 0] == 1
    # sigma scaled with frequency: at f = f_ref/2 sigma halves
    pos = np.array([[0.0, 0.0], [0.7, 0.0]])
    _, _, w1 = oracle.footprint(pos, 100e6, 16, 3, 1.2, f_ref_hz=200e6, freq_scaled=True, cell_m=1.0)
    u0 = -0.35 + 8.0                                           # element 0, centroid at x = 0.35
    a0 = math.floor(u0 + 0.5)
    d = (a0 - 1) - u0
    assert w1[0, 1, 0].real == pytest.approx(math.exp(-(d * d) / (2 * 0.6 ** 2)), rel=1e-13)


def test_footprint_overflow_is_an_error():
    pos = np.array([[-10.0, 0.0], [10.0, 0.0]])
    with pytest.raises(oracle.OracleError, match="grid overflow"):
        oracle.footprint(pos, 100e6, 16, 3, 1.0, cell_m=1.0)
    # touching the edge is fine: u = 8 -+ 6 -> anchors 2 and 14, taps 1..3 and 13..15
    pos = np.array([[-6.0, 0.0], [6.0, 0.0]])
    tx, _, _ = oracle.footprint(pos, 100e6, 16, 3, 1.0, cell_m=1.0)
    assert tx[0, 0] == 1 and tx[1, -1] == 15


# ----------------------------------------------------------------------------- whole path

def _closed_cfg(pos, n_pol, N, K=1, sigma=0.5, T=6, seed=5):
    f = np.array([C0 / 2.0])
    return synth.EpicConfig("closed", np.asarray(pos, float), f, n_pol, N, K, sigma, float(f[0]), False, T,
                            np.zeros((0, 2)), np.zeros(0), 2.0, seed)


def test_single_element_on_grid_gives_flat_image():
    cfg = _closed_cfg([[3.0, -1.0]], 2, 16)
    v = synth.random_bytes((cfg.n_time, 1, 1, 2), seed=1)
    img = oracle.image_cfg(cfg, v)[0]
    E = bruteforce.decode_nibbles(v[:, 0, 0, :])
    assert np.allclose(img[0], np.sum(np.abs(E[:, 0]) ** 2), rtol=1e-13)
    assert np.allclose(img[1], np.sum(np.abs(E[:, 1]) ** 2), rtol=1e-13)
    xy = np.sum(E[:, 0] * np.conj(E[:, 1]))
    assert np.allclose(img[2], xy.real, atol=1e-12) and np.allclose(img[3], xy.imag, atol=1e-12)


def test_two_element_fringe_closed_form():
    N = 16
    # 4 cells apart in x, 2 in y (cell = lambda/2 = 1 m), both on grid points: an exact fringe
    cfg = _closed_cfg([[-2.0, -1.0], [2.0, 1.0]], 1, N)
    v = synth.random_bytes((cfg.n_time, 1, 2, 1), seed=2)
    img = oracle.image_cfg(cfg, v)[0, 0]
    E = bruteforce.decode_nibbles(v[:, 0, :, 0])
    k = (np.arange(N) + N // 2) % N                            # image index -> Fourier index
    KY, KX = np.meshgrid(k, k, indexing="ij")
    ph = np.exp(2j * math.pi * ((-4) * KX + (-2) * KY) / N)    # j1 - j2 = (-4, -2)
    cross = np.sum(E[:, 0] * np.conj(E[:, 1]))
    expect = np.sum(np.abs(E) ** 2) + 2.0 * np.real(cross * ph)
    assert np.allclose(img, expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n_pol,K,N,A,freq_scaled", [
    (1, 3, 16, 8, False), (2, 3, 16, 12, False), (2, 2, 16, 10, False), (2, 4, 16, 9, False),
    (2, 5, 16, 6, True), (1, 1, 8, 5, False), (2, 3, 8, 16, False)])
def test_matches_pairwise_correlation_bruteforce(n_pol, K, N, A, freq_scaled):
    cfg = synth.small_config(n_ant=A, n_chan=2, n_pol=n_pol, grid_n=N, gcf_k=K, n_time=4, seed=10 + K + N,
                             diameter_m=5.0 if N == 8 else 10.0, freq_scaled=freq_scaled)
    v = synth.make_voltages(cfg)
    a = oracle.image_cfg(cfg, v)
    b = bruteforce.image(v, cfg.pos_m, cfg.freq_hz, n_pol, N, K, cfg.sigma_cells, cfg.f_ref_hz, freq_scaled)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_parseval_across_transform():
    cfg = synth.small_config(n_ant=14, n_chan=1, n_pol=2, grid_n=16, gcf_k=3, n_time=5, seed=3)
    v = synth.make_voltages(cfg)
    img = oracle.image_cfg(cfg, v)[0]
    N = cfg.grid_n
    gx = [oracle.grid_frame(v, t, 0, 0, cfg.pos_m, cfg.freq_hz, 2, N, 3, cfg.sigma_cells) for t in range(5)]
    gy = [oracle.grid_frame(v, t, 0, 1, cfg.pos_m, cfg.freq_hz, 2, N, 3, cfg.sigma_cells) for t in range(5)]
    assert img[0].sum() == pytest.approx(N * N * sum(np.sum(np.abs(g) ** 2) for g in gx), rel=1e-12)
    assert img[1].sum() == pytest.approx(N * N * sum(np.sum(np.abs(g) ** 2) for g in gy), rel=1e-12)
    xy = N * N * sum(np.sum(a * np.conj(b)) for a, b in zip(gx, gy))
    assert img[2].sum() == pytest.approx(xy.real, rel=1e-11, abs=1e-9 * abs(xy))
    assert img[3].sum() == pytest.approx(xy.imag, rel=1e-11, abs=1e-9 * abs(xy))


def test_grid_frame_is_sum_of_weighted_voltages():
    cfg = synth.small_config(n_ant=7, n_chan=2, n_pol=2, grid_n=16, gcf_k=3, n_time=2, seed=4)
    v = synth.make_voltages(cfg)
    g = oracle.grid_frame(v, 1, 1, 1, cfg.pos_m, cfg.freq_hz, 2, 16, 3, cfg.sigma_cells)
    wd = bruteforce.dense_footprints(cfg.pos_m, cfg.freq_hz[1], 16, 3, cfg.sigma_cells)
    E = bruteforce.decode_nibbles(v[1, 1, :, 1])
    assert np.allclose(g, np.einsum("e,eyx->yx", E, wd), atol=1e-13)


def test_point_sources_peak_at_predicted_pixels():
    spec = json.load(open(os.path.join(GOLDEN, "point_sources.json")))
    for case in spec["cases"]:
        N = case["N"]
        rng = np.random.default_rng(N)
        pos = synth.layout_disc(64, 0.45 * N * 1.0, rng)         # cell = lambda/2 = 1 m
        f = np.array([C0 / 2.0])
        cfg = synth.EpicConfig("pt", pos, f, 1, N, 3, 0.5, float(f[0]), False, 8,
                               np.array([[case["l"], case["m"]]]), np.array([5.0]), 0.0, 9)
        v = synth.make_voltages(cfg)
        img = oracle.image_cfg(cfg, v)[0, 0]
        iy, ix = np.unravel_index(np.argmax(img), img.shape)
        assert ix in case["argmax_ix"] and iy in case["argmax_iy"], case["name"]
        assert case["kappa_x"] == pytest.approx(case["l"] * N / 2) and case["kappa_y"] == pytest.approx(case["m"] * N / 2)


def test_tiny_workload_source_localised():
    cfg = synth.config(1)
    v = synth.make_voltages(cfg)
    img = oracle.image_cfg(cfg, v)
    for c in range(cfg.n_chan):
        iy, ix = np.unravel_index(np.argmax(img[c, 0]), img.shape[2:])
        assert ix in (19, 20) and iy in (14, 15)


def test_transient_appears_only_in_its_frames():
    # one-frame-group transient among a persistent source (paper Sec. 4, Fig. 4 setup)
    N = 32
    rng = np.random.default_rng(77)
    pos = synth.layout_disc(48, 14.0, rng)
    f = np.array([C0 / 2.0])
    base = synth.EpicConfig("persist", pos, f, 2, N, 3, 0.5, float(f[0]), False, 12,
                            np.array([[0.25, 0.25]]), np.array([3.0]), 0.0, 21)
    tran = synth.EpicConfig("transient", pos, f, 2, N, 3, 0.5, float(f[0]), False, 12,
                            np.array([[-0.5, 0.125]]), np.array([4.0]), 0.0, 22)
    vb = synth.make_voltages(base)
    vt = synth.make_voltages(tran)
    Eb = bruteforce.decode_nibbles(vb)
    Et = bruteforce.decode_nibbles(vt)
    E = Eb.copy()
    E[4:8] += Et[4:8]                                            # transient in frames 4..7 only
    v = synth.pack_nibbles(np.clip(E.real, -7, 7), np.clip(E.imag, -7, 7))
    on = oracle.image_cfg(base, v[4:8])[0, 0]
    off = oracle.image_cfg(base, np.concatenate([v[:4], v[8:]]))[0, 0]
    t_pix = (N // 2 + 2, N // 2 - 8)                             # (iy, ix) of (l, m) = (-0.5, 0.125)
    p_pix = (N // 2 + 4, N // 2 + 4)
    assert np.unravel_index(np.argmax(on), on.shape) in (t_pix, p_pix)
    assert on[t_pix] > 10 * off[t_pix] / 2                       # per-frame brightness, 4 vs 8 frames
    assert np.unravel_index(np.argmax(off), off.shape) == p_pix


def test_linearity_in_time():
    cfg = synth.small_config(n_ant=16, n_chan=3, n_pol=2, grid_n=16, gcf_k=3, n_time=9, seed=6)
    v = synth.make_voltages(cfg)
    full = oracle.image_cfg(cfg, v)
    parts = oracle.image_cfg(cfg, v[:4]) + oracle.image_cfg(cfg, v[4:])
    assert np.abs(full - parts).max() <= 1e-12 * np.abs(full).max()
    assert np.all(oracle.image_cfg(cfg, v[:0]) == 0.0)


def test_polarisation_products_are_consistent():
    cfg = synth.small_config(n_ant=16, n_chan=2, n_pol=2, grid_n=16, gcf_k=3, n_time=6, seed=8)
    v = synth.make_voltages(cfg)
    img = oracle.image_cfg(cfg, v)
    xx, yy, rxy, ixy = img[:, 0], img[:, 1], img[:, 2], img[:, 3]
    assert (xx >= 0).all() and (yy >= 0).all()
    assert (rxy ** 2 + ixy ** 2 <= xx * yy * (1 + 1e-12) + 1e-9).all()     # Cauchy-Schwarz per pixel
    # swapping the pols swaps XX/YY and conjugates XY
    sw = oracle.image_cfg(cfg, v[..., ::-1].copy())
    assert np.allclose(sw[:, 0], yy) and np.allclose(sw[:, 1], xx)
    assert np.allclose(sw[:, 2], rxy) and np.allclose(sw[:, 3], -ixy)


def test_channel_selection_matches_full():
    cfg = synth.small_config(n_ant=10, n_chan=4, n_pol=1, grid_n=16, gcf_k=3, n_time=3, seed=9)
    v = synth.make_voltages(cfg)
    full = oracle.image_cfg(cfg, v)
    sel = oracle.image_cfg(cfg, v, chans=[3, 1])
    assert np.array_equal(sel[0], full[3]) and np.array_equal(sel[1], full[1])


def test_table_gcf_constant_equals_scaled_box():
    cfg = synth.small_config(n_ant=9, n_chan=1, n_pol=2, grid_n=16, gcf_k=3, n_time=3, seed=12)
    v = synth.make_voltages(cfg)
    K, os_ = 3, 4
    side = K * os_ + 1
    c = 0.6 - 0.8j
    tab = np.zeros((side, side, 2), np.float32)
    tab[..., 0], tab[..., 1] = c.real, c.imag
    got = oracle.image(v, cfg.pos_m, cfg.freq_hz, 2, 16, K, cfg.sigma_cells, gcf_kind=oracle.GCF_TABLE,
                       oversample=os_, table=tab)
    box = oracle.image(v, cfg.pos_m, cfg.freq_hz, 2, 16, K, 1e9)         # Gaussian with huge sigma = 1
    mag = abs(np.complex64(c)) ** 2
    assert np.allclose(got, mag * box, rtol=1e-6, atol=1e-6 * np.abs(box).max())


@pytest.mark.parametrize("K,os_", [(3, 4), (2, 8), (4, 3)])
def test_table_gcf_matches_bruteforce(K, os_):
    # a complex, position-dependent table: a wrong conjugate, axis order or lookup shows up here
    cfg = synth.small_config(n_ant=8, n_chan=2, n_pol=2, grid_n=16, gcf_k=K, n_time=3, seed=13 + K)
    v = synth.make_voltages(cfg)
    side = K * os_ + 1
    s = (np.arange(side) / os_ - K / 2.0)
    dy, dx = np.meshgrid(s, s, indexing="ij")
    W = np.exp(-(dx ** 2 + 0.5 * dy ** 2)) * np.exp(1j * (0.9 * dx - 0.4 * dy + 0.3 * dx * dy))
    tab = np.stack([W.real, W.imag], axis=-1).astype(np.float32)
    a = oracle.image(v, cfg.pos_m, cfg.freq_hz, 2, 16, K, cfg.sigma_cells, gcf_kind=oracle.GCF_TABLE,
                     oversample=os_, table=tab)
    b = bruteforce.image(v, cfg.pos_m, cfg.freq_hz, 2, 16, K, cfg.sigma_cells, table=tab, oversample=os_)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    assert np.abs(a[:, 3]).max() > 1e-3 * np.abs(a).max()                  # XY carries a real phase


# ----------------------------------------------------------------------------- 8+8-bit input, sub-integrations

def test_unpack8_matches_twos_complement_bytes():
    # every value of the real and of the imaginary byte, against numpy's int8 view
    v = np.arange(256, dtype=np.uint8)
    pairs = np.stack([v, v[::-1]], axis=1)
    got = oracle.unpack8_pairs(pairs)
    assert np.array_equal(got[:, 0], v.view(np.int8).astype(np.int64))
    assert np.array_equal(got[:, 1], v[::-1].view(np.int8).astype(np.int64))


def test_eight_bit_block_images_equal_four_bit_block_with_same_values():
    # the same complex samples written in both formats give identical images
    cfg = synth.small_config(n_ant=12, n_chan=2, n_pol=2, grid_n=16, gcf_k=3, n_time=5, seed=41)
    v4 = synth.make_voltages(cfg)
    E = bruteforce.decode_nibbles(v4)                           # [T][C][A][P] complex, from the pinned table
    v8 = np.stack([E.real, E.imag], axis=-1).astype(np.int8).view(np.uint8)
    a = oracle.image_cfg(cfg, v4)
    cfg8 = dataclasses.replace(cfg, input_bits=8)
    b = oracle.image_cfg(cfg8, v8)
    assert np.array_equal(a, b)


def test_sub_integrations_sum_to_the_block_and_equal_their_sub_blocks():
    cfg = dataclasses.replace(synth.small_config(n_ant=10, n_chan=2, n_pol=2, grid_n=16, gcf_k=3, n_time=12,
                                                 seed=42), input_bits=8)
    v = synth.make_voltages(cfg)
    whole = oracle.image_cfg(cfg, v)
    sub = oracle.image_cfg(dataclasses.replace(cfg, sub_int=4), v)
    assert sub.shape == (3,) + whole.shape
    assert np.abs(sub.sum(axis=0) - whole).max() <= 1e-12 * np.abs(whole).max()
    for k in range(3):
        assert np.array_equal(sub[k], oracle.image_cfg(cfg, v[4 * k:4 * k + 4]))


def test_one_frame_transient_found_in_its_sub_integration():
    # 8+8-bit voltages, 4-frame sub-integrations (paper Sec. 4): a source present in one
    # frame only peaks at its pixel in that frame's sub-integration and nowhere else
    N = 32
    rng = np.random.default_rng(78)
    pos = synth.layout_disc(48, 14.0, rng)
    f = np.array([C0 / 2.0])
    noise = synth.EpicConfig("noise", pos, f, 2, N, 3, 0.5, float(f[0]), False, 12, np.zeros((0, 2)),
                             np.zeros(0), 2.0, 23, input_bits=8)
    tran = synth.EpicConfig("transient", pos, f, 2, N, 3, 0.5, float(f[0]), False, 12,
                            np.array([[-0.5, 0.125]]), np.array([6.0]), 0.0, 24, input_bits=8)
    vn = synth.make_voltages(noise).view(np.int8).astype(np.int32)
    vt = synth.make_voltages(tran).view(np.int8).astype(np.int32)
    x = vn.copy()
    x[6] += vt[6]                                                # one frame (frame 6, interval 1)
    v = np.clip(x, -127, 127).astype(np.int8).view(np.uint8)
    sub = oracle.image_cfg(dataclasses.replace(noise, sub_int=4), v)[:, 0, 0]   # [3][N][N] XX
    t_pix = (N // 2 + 2, N // 2 - 8)                             # (iy, ix) of (l, m) = (-0.5, 0.125)
    assert np.unravel_index(np.argmax(sub[1]), sub[1].shape) == t_pix
    assert sub[1][t_pix] > 5 * max(sub[0][t_pix], sub[2][t_pix])


# ----------------------------------------------------------------------------- polarisation mixing

def _mix_cfg(seed, **kw):
    base = dict(n_ant=14, n_chan=2, n_pol=2, grid_n=16, gcf_k=3, n_time=6, seed=seed, diameter_m=5.0)
    base.update(kw)
    return synth.small_config(**base)


def test_identity_and_swap_kernels_reproduce_the_unmixed_products():
    # W^{ap} = delta_ap W is the unmixed path exactly; J = [[0, 1], [1, 0]] exchanges the
    # polarisations: XX <-> YY, XY -> conj(XY)
    cfg = _mix_cfg(61)
    v = synth.make_voltages(cfg)
    base = oracle.image_cfg(cfg, v)
    eye = np.broadcast_to(np.eye(2, dtype=np.complex128), (cfg.n_chan, cfg.n_ant, 2, 2))
    assert np.array_equal(oracle.image_cfg(dataclasses.replace(cfg, jones=eye), v), base)
    swap = np.broadcast_to(np.array([[0, 1], [1, 0]], dtype=np.complex128), eye.shape)
    sw = oracle.image_cfg(dataclasses.replace(cfg, jones=swap), v)
    assert np.array_equal(sw[:, 0], base[:, 1]) and np.array_equal(sw[:, 1], base[:, 0])
    assert np.array_equal(sw[:, 2], base[:, 2]) and np.array_equal(sw[:, 3], -base[:, 3])


def test_channel_wide_kernel_mixes_the_image_products_linearly():
    # one J for every element of a channel: gridding and the transform are linear, so
    # E'^a = sum_p conj(J^{ap}) E^p per pixel and I'^{ab} = sum_{p,q} conj(J^{ap}) J^{bq} I^{pq}
    # with I^{YX} = conj(I^{XY}); a non-symmetric complex J catches a transposed or
    # unconjugated kernel
    cfg = _mix_cfg(62)
    v = synth.make_voltages(cfg)
    base = oracle.image_cfg(cfg, v)
    Jc = np.array([[[0.9 + 0.3j, 0.2 - 0.1j], [-0.15 + 0.25j, 1.1 - 0.4j]],
                   [[0.7 - 0.2j, -0.3 + 0.05j], [0.1 + 0.2j, 0.8 + 0.6j]]])
    J = np.repeat(Jc[:, None], cfg.n_ant, axis=1)
    got = oracle.image_cfg(dataclasses.replace(cfg, jones=J), v)
    for c in range(cfg.n_chan):
        xy = base[c, 2] + 1j * base[c, 3]
        Ipq = np.array([[base[c, 0], xy], [np.conj(xy), base[c, 1]]])     # [p][q][N][N]
        M = np.einsum("ap,bq,pqyx->abyx", np.conj(Jc[c]), Jc[c], Ipq)
        peak = np.abs(M[0, 0]).max() + np.abs(M[1, 1]).max()
        assert np.abs(got[c, 0] - M[0, 0].real).max() <= 1e-12 * peak
        assert np.abs(got[c, 1] - M[1, 1].real).max() <= 1e-12 * peak
        assert np.abs(got[c, 2] + 1j * got[c, 3] - M[0, 1]).max() <= 1e-12 * peak
        assert np.abs(M[0, 0].imag).max() <= 1e-12 * peak


def test_per_element_kernels_match_the_correlator_route():
    # a different random J per element and channel (8+8-bit input): the oracle's double sum
    # of Eq. 1 against pairwise visibilities of the mixed voltages (no gridding, no FFT shared)
    cfg = dataclasses.replace(_mix_cfg(63, n_ant=10), input_bits=8)
    J = synth.make_jones(cfg, seed=3, gain_rms=0.2, leak_rms=0.3)
    v8 = synth.make_voltages(cfg)
    got = oracle.image_cfg(dataclasses.replace(cfg, jones=J), v8)
    ref = bruteforce.image(v8, cfg.pos_m, cfg.freq_hz, 2, cfg.grid_n, cfg.gcf_k, cfg.sigma_cells, cfg.f_ref_hz,
                           cfg.freq_scaled, jones=J, input_bits=8)
    peak = np.abs(ref[:, :2]).max()
    assert np.abs(got - ref).max() <= 1e-9 * peak


def test_mixing_kernel_rejected_for_one_polarisation():
    cfg = _mix_cfg(64, n_pol=1)
    v = synth.make_voltages(cfg)
    J = np.ones((cfg.n_chan, cfg.n_ant, 2, 2), dtype=np.complex128)
    with pytest.raises(oracle.OracleError):
        oracle.image_cfg(dataclasses.replace(cfg, jones=J), v)
