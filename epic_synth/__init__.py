"""Seeded synthetic inputs for the EPIC imaging path.

This module is shared by the CUDA library's tests/bench and by the CPU
oracle's tests.  It holds NONE of the imaging arithmetic (no gridding, no
transform, no products): only array layouts, the sky model that generates the
antenna voltages, and the 4+4-bit two's-complement packing of those voltages.

Workload shapes follow the arrays the paper images (Sec. 3-4: a 256-element
dual-pol SKA-Low-like station, LWA-like stations, dense large-N arrays).  The
real AAVS2/SKA-Low/LWA layouts are not available, so every layout here is a
seeded synthetic stand-in (uniform disc, uniform ellipse, jittered lattice).

Voltage model (per time sample t, channel c, element e, polarisation p):

    E = n + sum_s a_s(t,c,p) * exp(-2*pi*i*(l_s*x_e + m_s*y_e)/lambda_c)

with n ~ N(0, sigma_n) independently on the real and imaginary parts and
a_s ~ CN(0, amp_s^2) ("sources with intrinsic randomness", Sec. 4), then
rounded half-to-even, clipped to [-7, 7] and packed as one byte with the real
part in the high nibble and the imaginary part in the low nibble.

Every random draw of time sample t comes from its own stream
``default_rng([seed, t])`` so that any time range can be generated on its own
and two calls over different chunkings give identical bytes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

C0 = 299_792_458.0  # speed of light, m/s


@dataclasses.dataclass
class EpicConfig:
    """One imaging workload: geometry, frequencies, grid, GCF and sky."""

    name: str
    pos_m: np.ndarray          # float64 [A][2], x and y in metres
    freq_hz: np.ndarray        # float64 [C]
    n_pol: int
    grid_n: int
    gcf_k: int
    sigma_cells: float         # Gaussian sigma in grid cells at f_ref
    f_ref_hz: float
    freq_scaled: bool          # sigma_c = sigma * f_c / f_ref
    n_time: int
    src_lm: np.ndarray         # float64 [S][2], direction cosines (l, m)
    src_amp: np.ndarray        # float64 [S], rms amplitude of each source
    noise_sigma: float
    seed: int
    input_bits: int = 4        # 4: 4+4-bit bytes; 8: 8+8-bit (real byte, imaginary byte)
    sub_int: int = 0           # time samples per output image (0 = the whole block)
    jones: Optional[np.ndarray] = None  # complex [C][A][2][2] polarisation mixing J^{ap}, None = none

    @property
    def n_ant(self) -> int:
        return int(self.pos_m.shape[0])

    @property
    def n_chan(self) -> int:
        return int(self.freq_hz.shape[0])

    @property
    def n_prod(self) -> int:
        return 1 if self.n_pol == 1 else 4

    def pixel_updates(self, n_time: Optional[int] = None) -> int:
        t = self.n_time if n_time is None else n_time
        return self.grid_n * self.grid_n * self.n_chan * self.n_pol * t

    def voltage_bytes(self, n_time: Optional[int] = None) -> int:
        t = self.n_time if n_time is None else n_time
        return t * self.n_chan * self.n_ant * self.n_pol * (2 if self.input_bits == 8 else 1)

    def image_floats(self) -> int:
        return self.n_chan * self.n_prod * self.grid_n * self.grid_n

    def subset(self, chans: Sequence[int], n_time: Optional[int] = None) -> "EpicConfig":
        """Same array and sky restricted to some channels (and time samples)."""
        c = dataclasses.replace(self)
        c.freq_hz = np.asarray(self.freq_hz)[list(chans)].copy()
        if n_time is not None:
            c.n_time = int(n_time)
        return c


# --------------------------------------------------------------------------- layouts

def layout_disc(n: int, diameter_m: float, rng: np.random.Generator) -> np.ndarray:
    """n points uniform by area in a disc (r = R*sqrt(U)); no minimum spacing."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n))
    th = 2.0 * math.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def layout_ellipse(n: int, axis_x_m: float, axis_y_m: float, rng: np.random.Generator) -> np.ndarray:
    """n points uniform by area in an ellipse with full axes axis_x_m, axis_y_m."""
    p = layout_disc(n, 2.0, rng)
    return p * np.array([0.5 * axis_x_m, 0.5 * axis_y_m])


def layout_lattice(nside: int, pitch_m: float, jitter_frac: float, rng: np.random.Generator) -> np.ndarray:
    """nside x nside square lattice with uniform +-jitter_frac*pitch per axis."""
    g = (np.arange(nside) - 0.5 * (nside - 1)) * pitch_m
    xx, yy = np.meshgrid(g, g, indexing="xy")
    p = np.stack([xx.ravel(), yy.ravel()], axis=1)
    p = p + rng.uniform(-jitter_frac * pitch_m, jitter_frac * pitch_m, size=p.shape)
    return p


# --------------------------------------------------------------------------- configs

def _sky_uniform_box(rng, n, half, amps):
    lm = rng.uniform(-half, half, size=(n, 2))
    return lm, np.asarray(amps, dtype=np.float64)


def config(idx: int) -> EpicConfig:
    """The fixed imaging workloads: 1..4, and 6 (a 512x512 grid; 5 is the streaming mix)."""
    if idx == 1:
        # 64 elements in a 20 m disc, lambda = 2 m, 1 pol, 4 channels, 32x32 grid,
        # 3x3 Gaussian GCF with sigma 0.5 cell, 256 samples, one source at (0.2, -0.1).
        rng = np.random.default_rng([0, 1_000_000])
        pos = layout_disc(64, 20.0, rng)
        f = np.full(4, C0 / 2.0)
        return EpicConfig("tiny-64el-32grid", pos, f, 1, 32, 3, 0.5, float(f[0]), False, 256,
                          np.array([[0.2, -0.1]]), np.array([0.5]), 2.0, 0)
    if idx == 2:
        # LWA-station-like: 256 dual-pol elements in a 100 m x 110 m ellipse, 128 x 25 kHz
        # channels centred on 56 MHz, 128x128 grid, 5x5 GCF, 1000 samples.
        rng = np.random.default_rng([2, 1_000_000])
        pos = layout_ellipse(256, 100.0, 110.0, rng)
        f = 54.4e6 + (np.arange(128) + 0.5) * 25e3
        lm, amp = _sky_uniform_box(rng, 3, 0.5, [0.5, 0.35, 0.25])
        return EpicConfig("lwa-256el-128grid", pos, f, 2, 128, 5, 1.0, float(f.max()), False, 1000,
                          lm, amp, 2.0, 2)
    if idx == 3:
        # SKA-Low-station-like: 256 dual-pol elements in a 38 m disc, 384 x 781.25 kHz
        # channels over 50-350 MHz, 128x128 grid, 7x7 Gaussian GCF with sigma 1.5 cells at
        # 350 MHz scaled with frequency, 512 samples.
        rng = np.random.default_rng([3, 1_000_000])
        pos = layout_disc(256, 38.0, rng)
        f = 50e6 + (np.arange(384) + 0.5) * 781.25e3
        lm, amp = _sky_uniform_box(rng, 3, 0.5, [0.5, 0.35, 0.25])
        return EpicConfig("skalow-256el-128grid", pos, f, 2, 128, 7, 1.5, 350e6, True, 512,
                          lm, amp, 2.0, 3)
    if idx == 4:
        # Dense large-N: 64x64 lattice at 0.5 lambda(150 MHz) pitch with +-5 % jitter,
        # 64 x 781.25 kHz channels from 150 MHz, 256x256 grid, 3x3 GCF, 256 samples,
        # 10 sources with log-uniform flux 0.01-1 inside l^2+m^2 <= 0.64.
        rng = np.random.default_rng([4, 1_000_000])
        lam_ref = C0 / 150e6
        pos = layout_lattice(64, 0.5 * lam_ref, 0.05, rng)
        f = 150e6 + (np.arange(64) + 0.5) * 781.25e3
        n = 10
        rad = 0.8 * np.sqrt(rng.random(n))
        th = 2.0 * math.pi * rng.random(n)
        lm = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
        flux = 10.0 ** rng.uniform(-2.0, 0.0, size=n)
        return EpicConfig("dense-4096el-256grid", pos, f, 2, 256, 3, 0.5, 150e6, False, 256,
                          lm, np.sqrt(flux), 2.0, 4)
    if idx == 6:
        # Large-grid station (the paper's second prototype scale): 20,000 dual-pol elements
        # uniform in a 240 m disc, one 781.25 kHz coarse channel at 159 MHz, 512x512 grid
        # (the aperture fills about half of it at lambda/2 spacing), 2x2 Gaussian GCF,
        # 1000 samples, 3 sources.
        rng = np.random.default_rng([6, 1_000_000])
        pos = layout_disc(20000, 240.0, rng)
        f = np.array([159e6 + 390.625e3])
        lm, amp = _sky_uniform_box(rng, 3, 0.5, [0.5, 0.35, 0.25])
        return EpicConfig("proto2-20000el-512grid", pos, f, 2, 512, 2, 0.5, float(f[0]), False, 1000,
                          lm, amp, 2.0, 6)
    raise ValueError(f"no such config {idx}")


# --------------------------------------------------------------------------- voltages

def pack_nibbles(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer parts in [-8, 7] as one byte: real high nibble, imaginary low."""
    re = np.asarray(re).astype(np.int16)
    im = np.asarray(im).astype(np.int16)
    if re.size and (re.min() < -8 or re.max() > 7 or im.min() < -8 or im.max() > 7):
        raise ValueError("value outside the 4-bit two's-complement range")
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


def source_phases(cfg: EpicConfig) -> np.ndarray:
    """exp(-2 pi i (l x + m y)/lambda_c) for every (channel, element, source)."""
    lam = C0 / np.asarray(cfg.freq_hz)                        # [C]
    proj = cfg.pos_m @ cfg.src_lm.T                             # [A][S]
    return np.exp(-2j * math.pi * proj[None, :, :] / lam[:, None, None])


def make_voltages(cfg: EpicConfig, t0: int = 0, n_time: Optional[int] = None,
                  out: Optional[np.ndarray] = None) -> np.ndarray:
    """uint8[T][C][A][P] packed 4+4-bit voltages for time samples [t0, t0+T), or
    uint8[T][C][A][P][2] 8+8-bit ones (two's complement real, imaginary bytes) when
    cfg.input_bits == 8.

    Noise and source amplitudes are drawn in float32 from the stream of each
    time sample; the source term is a batched (A x S) @ (S x P) product per
    channel.
    """
    T = cfg.n_time - t0 if n_time is None else int(n_time)
    C, A, P = cfg.n_chan, cfg.n_ant, cfg.n_pol
    S = cfg.src_lm.shape[0]
    eight = getattr(cfg, "input_bits", 4) == 8
    if out is None:
        out = np.empty((T, C, A, P, 2) if eight else (T, C, A, P), dtype=np.uint8)
    ph = source_phases(cfg).astype(np.complex64) if S else None       # [C][A][S]
    amp = (cfg.src_amp / math.sqrt(2.0)).astype(np.float32)
    for i in range(T):
        rng = np.random.default_rng([cfg.seed, t0 + i])
        noise = rng.standard_normal(size=(C, A, P, 2), dtype=np.float32)
        noise *= np.float32(cfg.noise_sigma)
        re = noise[..., 0]
        im = noise[..., 1]
        if S:
            g = rng.standard_normal(size=(C, S, P, 2), dtype=np.float32)
            a = (g[..., 0] + 1j * g[..., 1]) * amp[None, :, None]          # [C][S][P]
            src = np.matmul(ph, a.astype(np.complex64))                    # [C][A][P]
            re = re + src.real
            im = im + src.imag
        if eight:  # 8+8-bit: the same signal on a 16x finer scale, clipped to +-127
            q = np.stack([np.clip(np.rint(16.0 * re), -127, 127), np.clip(np.rint(16.0 * im), -127, 127)], axis=-1)
            out[i] = q.astype(np.int8).view(np.uint8)
        else:
            out[i] = pack_nibbles(np.clip(np.rint(re), -7, 7), np.clip(np.rint(im), -7, 7))
    return out


def make_jones(cfg: EpicConfig, seed: int = 0, gain_rms: float = 0.1, leak_rms: float = 0.05) -> np.ndarray:
    """complex128 [C][A][2][2] direction-independent polarisation-mixing matrices per
    element and channel, J = [[g_X, d_XY], [d_YX, g_Y]]: complex gains g_p = (1 + a) e^{i phi}
    with a ~ N(0, gain_rms), phi ~ U(-pi, pi), and leakage terms d ~ CN(0, leak_rms^2),
    drawn independently per (channel, element) from the stream [seed, 9_000_000]."""
    rng = np.random.default_rng([seed, 9_000_000])
    C, A = cfg.n_chan, cfg.n_ant
    J = np.zeros((C, A, 2, 2), dtype=np.complex128)
    amp = 1.0 + gain_rms * rng.standard_normal((C, A, 2))
    phi = rng.uniform(-math.pi, math.pi, (C, A, 2))
    J[:, :, 0, 0] = amp[..., 0] * np.exp(1j * phi[..., 0])
    J[:, :, 1, 1] = amp[..., 1] * np.exp(1j * phi[..., 1])
    d = (rng.standard_normal((C, A, 2)) + 1j * rng.standard_normal((C, A, 2))) * (leak_rms / math.sqrt(2.0))
    J[:, :, 0, 1] = d[..., 0]
    J[:, :, 1, 0] = d[..., 1]
    return J


def random_bytes(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    """Uniform random bytes (all 256 codes, including the -8 nibble) for edge tests."""
    return np.random.default_rng([seed, 7]).integers(0, 256, size=shape, dtype=np.uint8)


def small_config(n_ant: int = 12, n_chan: int = 2, n_pol: int = 2, grid_n: int = 16, gcf_k: int = 3,
                 sigma: float = 0.6, n_time: int = 5, seed: int = 11, diameter_m: float = 10.0,
                 freq_scaled: bool = False, name: str = "small") -> EpicConfig:
    """Tiny array for exact/brute-force checks; frequencies spread 100-140 MHz."""
    rng = np.random.default_rng([seed, 1_000_000])
    pos = layout_disc(n_ant, diameter_m, rng)
    f = np.linspace(100e6, 140e6, n_chan) if n_chan > 1 else np.array([120e6])
    lm = rng.uniform(-0.4, 0.4, size=(2, 2))
    return EpicConfig(name, pos, f, n_pol, grid_n, gcf_k, sigma, float(f.max()), freq_scaled, n_time,
                      lm, np.array([1.0, 0.6]), 1.5, seed)


def mixed_station_types() -> List[EpicConfig]:
    """Station types of the streaming mix: 64, 256, 1024 and 4096 dual-pol elements."""
    c1 = config(1)
    s64 = dataclasses.replace(c1, name="mix-64el-32grid", n_pol=2, seed=51)
    c2 = config(2)
    s256 = dataclasses.replace(c2, name="mix-256el-128grid", seed=52)
    rng = np.random.default_rng([53, 1_000_000])
    lam_ref = C0 / 150e6
    pos = layout_lattice(32, 0.5 * lam_ref, 0.05, rng)
    f = 150e6 + (np.arange(64) + 0.5) * 781.25e3
    lm = rng.uniform(-0.5, 0.5, size=(3, 2))
    s1024 = EpicConfig("mix-1024el-128grid", pos, f, 2, 128, 3, 0.5, 150e6, False, 256,
                       lm, np.array([0.5, 0.35, 0.25]), 2.0, 53)
    c4 = config(4)
    s4096 = dataclasses.replace(c4, name="mix-4096el-256grid", seed=54)
    return [s64, s256, s1024, s4096]


SERVE_CHANNELS = (32, 64, 128, 256, 384)
SERVE_DF_HZ = 25e3


def serving_config(station: EpicConfig, n_chan: int) -> EpicConfig:
    """A block of the streaming mix: `station` (one of mixed_station_types()) with n_chan
    contiguous 25 kHz channels from the station's first frequency (the mix's channel
    plan; the text gives none)."""
    cfg = dataclasses.replace(station, name=f"{station.name}-{n_chan}ch")
    cfg.freq_hz = station.freq_hz[0] + np.arange(n_chan) * SERVE_DF_HZ
    return cfg
