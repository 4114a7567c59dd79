"""Seeded synthetic inputs for the beamformer: array geometry, channel
frequencies, beam directions and channelised antenna voltages.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1412_4907_gb300``): it produces inputs and nothing else.
It holds none of the beamformer's arithmetic (no weights, no beam sums, no
power detection).  The one piece of physics here is the sky model: a plane
wave from unit direction ``s`` reaches antenna ``n`` (position ``r_n``) with
the geometric phase ``exp(+i 2 pi f (r_n . s) / c0)`` (Section 1, Eq. 1 with
the wave arriving along ``s``); the beamformer undoes that phase, the
generator only applies it.

Every random draw comes from numpy's Philox counter-based generator keyed by
``(seed, tag)`` with the channel index in the counter, so any subset of
channels can be regenerated on its own, on any machine, bit for bit.

Workload shapes follow the BEST-2 array of Section 1.1 (32 receivers on a
4 x 8 grid, 1024 channels) and the benchmarks of Section 2.2.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0  # speed of light in vacuum, m/s (exact SI value)

# storage modes of the voltage input (match bf_dtype in include/bf.h)
C32, C16F, C16BF, C8E4M3, CI8, CI4 = 0, 1, 2, 3, 4, 5
MODE_NAMES = {C32: "c32", C16F: "c16f", C16BF: "c16bf", C8E4M3: "c8e4m3",
              CI8: "ci8", CI4: "ci4"}
# bytes per complex sample of each mode
MODE_BYTES = {C32: 8, C16F: 4, C16BF: 4, C8E4M3: 2, CI8: 2, CI4: 1}

_TAG_NOISE = 1
_TAG_SRC_AMP = 1000      # + source index
_TAG_SRC_PARAMS = 7
_TAG_LAYOUT = 11
_TAG_JOBS = 13


def _rng(seed: int, tag: int, counter: int = 0) -> np.random.Generator:
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, tag], dtype=np.uint64)
    ctr = np.array([0, counter, 0, 0], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key, counter=ctr))


# ----------------------------------------------------------------- geometry
def grid_positions(n_cols: int = 4, n_rows: int = 8, dx: float = 10.0,
                   dy: float = 5.0) -> np.ndarray:
    """Regular planar grid, E-W columns spaced ``dx`` m and N-S rows spaced
    ``dy`` m, antenna index ``row * n_cols + col``, z = 0, centred on the
    centroid.  The default is the 4 x 8 BEST-2 layout (Section 1.1)."""
    pos = np.zeros((n_rows * n_cols, 3))
    for row in range(n_rows):
        for col in range(n_cols):
            pos[row * n_cols + col] = (col * dx, row * dy, 0.0)
    pos[:, :2] -= pos[:, :2].mean(axis=0)
    return pos


def random_positions(n_ant: int, extent_m: float, seed: int) -> np.ndarray:
    """``n_ant`` antennas uniform in an ``extent_m`` x ``extent_m`` square,
    z = 0, centred on the centroid."""
    g = _rng(seed, _TAG_LAYOUT)
    pos = np.zeros((n_ant, 3))
    pos[:, :2] = g.uniform(-extent_m / 2, extent_m / 2, size=(n_ant, 2))
    pos[:, :2] -= pos[:, :2].mean(axis=0)
    return pos


def channel_freqs(f_lo_hz: float, bw_hz: float, n_chan: int) -> np.ndarray:
    """Channel centre frequencies f_lo + (c + 1/2) * bw / C."""
    return f_lo_hz + (np.arange(n_chan, dtype=np.float64) + 0.5) * (bw_hz / n_chan)


def direction(theta_x_deg: float, theta_y_deg: float) -> np.ndarray:
    """Unit vector for E-W offset theta_x and N-S offset theta_y from zenith:
    (sin tx, sin ty, sqrt(1 - sin^2 tx - sin^2 ty))."""
    sx = math.sin(math.radians(theta_x_deg))
    sy = math.sin(math.radians(theta_y_deg))
    return np.array([sx, sy, math.sqrt(max(0.0, 1.0 - sx * sx - sy * sy))])


def beam_grid(n_x: int, n_y: int, half_width_deg: float = 10.0) -> np.ndarray:
    """Regular grid of beam directions over +-half_width in each axis,
    beam index ``b = iy * n_x + ix`` (E-W fastest).  Returns (n_x*n_y, 3)."""
    tx = np.linspace(-half_width_deg, half_width_deg, n_x) if n_x > 1 else np.zeros(1)
    ty = np.linspace(-half_width_deg, half_width_deg, n_y) if n_y > 1 else np.zeros(1)
    out = np.zeros((n_x * n_y, 3))
    for iy in range(n_y):
        for ix in range(n_x):
            out[iy * n_x + ix] = direction(tx[ix], ty[iy])
    return out


# ------------------------------------------------------------------ sources
@dataclass
class Source:
    """A noise-like plane-wave source: per-(channel, sample) amplitude drawn
    from CN(0, power), arriving from unit direction ``dir``."""
    dir: np.ndarray
    power: float


@dataclass
class Scene:
    """Everything needed to synthesise voltages ``X[c][t][n]``."""
    pos: np.ndarray                    # (N, 3) metres
    freqs: np.ndarray                  # (C,) Hz
    n_samp: int                        # T
    seed: int
    noise_sigma: float = math.sqrt(0.5)   # std of each real component
    sources: list = field(default_factory=list)

    @property
    def n_ant(self) -> int:
        return self.pos.shape[0]

    @property
    def n_chan(self) -> int:
        return self.freqs.shape[0]


def random_sources(n_src: int, half_width_deg: float, snr_db_lo: float,
                   snr_db_hi: float, noise_power: float, seed: int) -> list:
    """Sources with directions uniform in the +-half_width box and SNR
    (per antenna, per sample, relative to ``noise_power``) uniform in dB."""
    g = _rng(seed, _TAG_SRC_PARAMS)
    out = []
    for _ in range(n_src):
        tx, ty = g.uniform(-half_width_deg, half_width_deg, size=2)
        snr = g.uniform(snr_db_lo, snr_db_hi)
        out.append(Source(direction(tx, ty), noise_power * 10.0 ** (snr / 10.0)))
    return out


def _channel_block(scene: Scene, c: int) -> np.ndarray:
    """Voltages of channel ``c`` as complex64 ``[T][N]``."""
    T, N = scene.n_samp, scene.n_ant
    g = _rng(scene.seed, _TAG_NOISE, c)
    v = g.standard_normal((T, N, 2), dtype=np.float32)
    v *= np.float32(scene.noise_sigma)
    x = v.view(np.complex64)[..., 0]
    f = float(scene.freqs[c])
    for i, src in enumerate(scene.sources):
        ga = _rng(scene.seed, _TAG_SRC_AMP + i, c)
        a = ga.standard_normal((T, 2), dtype=np.float32)
        a *= np.float32(math.sqrt(src.power / 2.0))
        amp = a.view(np.complex64)[:, 0]
        # geometric phase of the incoming plane wave at each antenna
        delay = (scene.pos @ src.dir) / C0
        ph = np.exp(2j * np.pi * f * delay).astype(np.complex64)
        x += amp[:, None] * ph[None, :]
    return x


# ------------------------------------------------------------ quantisation
def _to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u.astype(np.uint64) + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x32)
    if nan.any():
        r[nan] = 0x7FC0
    return r


def _e4m3_table():
    vals = np.zeros(256)
    for code in range(256):
        s = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 7
        if e == 0xF and m == 7:
            vals[code] = np.nan
        elif e == 0:
            vals[code] = s * m * 2.0 ** -9
        else:
            vals[code] = s * (1 + m / 8) * 2.0 ** (e - 7)
    return vals


_E4M3_POS = None


def _to_e4m3_codes(x: np.ndarray) -> np.ndarray:
    """float -> OCP FP8 E4M3FN codes, round to nearest even, saturate at +-448."""
    global _E4M3_POS
    if _E4M3_POS is None:
        _E4M3_POS = _e4m3_table()[:127]  # codes 0..126, ascending, finite
    a = np.minimum(np.abs(x.astype(np.float64)), 448.0)
    idx = np.searchsorted(_E4M3_POS, a)           # first value >= a
    idx = np.clip(idx, 1, 126)
    lo, hi = _E4M3_POS[idx - 1], _E4M3_POS[idx]
    pick_hi = (a - lo > hi - a) | ((a - lo == hi - a) & ((idx & 1) == 0))
    code = np.where(pick_hi, idx, idx - 1)
    code = np.where(a <= 0, 0, code).astype(np.uint8)
    return code | np.where(np.signbit(x), 0x80, 0).astype(np.uint8)


def quantise(x: np.ndarray, mode: int) -> np.ndarray:
    """complex64 ``[..., N]`` -> the mode's storage ``[..., 2N]`` with the real
    and imaginary parts interleaved (antenna fastest).  Round to nearest even;
    FP8 saturates at +-448; int8 rounds to nearest even and clips at +-127."""
    f = x.view(np.float32)
    if mode == C32:
        return f
    if mode == C16F:
        return f.astype(np.float16)
    if mode == C16BF:
        return _to_bf16_bits(f)
    if mode == C8E4M3:
        return _to_e4m3_codes(f)
    if mode == CI8:
        return np.clip(np.rint(f), -127, 127).astype(np.int8)
    if mode == CI4:
        q = np.clip(np.rint(f), -8, 7).astype(np.int8)
        re = q[..., 0::2].astype(np.uint8) & 0xF
        im = q[..., 1::2].astype(np.uint8) & 0xF
        return ((re << 4) | im).astype(np.uint8)
    raise ValueError(f"unknown mode {mode}")


def voltages(scene: Scene, mode: int = C32, channels=None, out=None,
             threads: int | None = None) -> np.ndarray:
    """Voltages in layout ``[c][t][2n]`` (channel, sample, interleaved re/im
    per antenna), quantised to ``mode``.  ``channels`` selects a subset (the
    values of a channel do not depend on which others are generated)."""
    chans = list(range(scene.n_chan)) if channels is None else list(channels)
    T, N = scene.n_samp, scene.n_ant
    width = N if mode == CI4 else 2 * N
    dt = {C32: np.float32, C16F: np.float16, C16BF: np.uint16,
          C8E4M3: np.uint8, CI8: np.int8, CI4: np.uint8}[mode]
    if out is None:
        out = np.empty((len(chans), T, width), dtype=dt)

    def work(i):
        out[i] = quantise(_channel_block(scene, chans[i]), mode)

    n_thr = threads or min(32, os.cpu_count() or 1)
    if len(chans) <= 2 or n_thr == 1:
        for i in range(len(chans)):
            work(i)
    else:
        with ThreadPoolExecutor(max_workers=n_thr) as ex:
            list(ex.map(work, range(len(chans))))
    return out


def to_nct(x_ctn: np.ndarray, mode: int) -> np.ndarray:
    """Re-lay ``[c][t][2n]`` voltages as antenna-major ``[n][c][t][2]``
    (for CI4, ``[n][c][t]`` bytes)."""
    C, T, W = x_ctn.shape
    if mode == CI4:
        return np.ascontiguousarray(x_ctn.transpose(2, 0, 1))
    return np.ascontiguousarray(x_ctn.reshape(C, T, W // 2, 2).transpose(2, 0, 1, 3))


# ----------------------------------------------------------------- configs
def config1() -> tuple[Scene, np.ndarray, int]:
    """Small FP32 case: BEST-2 grid, 64 channels over 400-416 MHz, 128 beams
    (16 E-W x 8 N-S over +-10 deg), T = 1024, unit complex Gaussian noise plus
    one plane wave (SNR 10 dB) from beam 37's direction, T_int = 16."""
    dirs = beam_grid(16, 8, 10.0)
    scene = Scene(pos=grid_positions(), freqs=channel_freqs(400e6, 16e6, 64),
                  n_samp=1024, seed=1,
                  sources=[Source(dirs[37], 10.0 ** (10 / 10.0))])
    return scene, dirs, 16


def config2(sigma: float | None = None) -> tuple[Scene, np.ndarray, int]:
    """Real-time-shaped FP16 case: BEST-2 grid, 1024 channels over 16 MHz,
    1024 beams (32 x 32 over +-10 deg), T = 15625, noise plus 3 sources of
    random direction and SNR 0-20 dB, T_int = 64.  ``sigma``: noise standard
    deviation per component for integer-input variants of the same chunk
    (16 for 8-bit, 2 for 4-bit samples); the default is CN(0, 1) noise."""
    dirs = beam_grid(32, 32, 10.0)
    if sigma is None:
        scene = Scene(pos=grid_positions(), freqs=channel_freqs(400e6, 16e6, 1024),
                      n_samp=15625, seed=2,
                      sources=random_sources(3, 10.0, 0.0, 20.0, 1.0, 2))
    else:
        scene = Scene(pos=grid_positions(), freqs=channel_freqs(400e6, 16e6, 1024),
                      n_samp=15625, seed=2, noise_sigma=sigma,
                      sources=random_sources(3, 10.0, 0.0, 20.0, 2 * sigma ** 2, 2))
    return scene, dirs, 64


def config3(n_chan: int = 4096) -> tuple[Scene, np.ndarray, int]:
    """Precision-sweep case: 256 antennas uniform in 200 m x 200 m, 4096
    channels over 400-416 MHz, 2048 beams (64 x 32 over +-10 deg), T = 8192,
    Gaussian sigma = 16 per component plus one plane wave (SNR 10 dB),
    T_int = 64.  ``n_chan`` < 4096 keeps the first channels of the same band
    layout (per-channel shape unchanged)."""
    dirs = beam_grid(64, 32, 10.0)
    noise_power = 2 * 16.0 ** 2
    freqs = channel_freqs(400e6, 16e6, 4096)[:n_chan]
    src = random_sources(1, 10.0, 10.0, 10.0, noise_power, 3)
    scene = Scene(pos=random_positions(256, 200.0, 3), freqs=freqs,
                  n_samp=8192, seed=3, noise_sigma=16.0, sources=src)
    return scene, dirs, 64


@dataclass
class Job:
    """One sub-array job of the batched workload."""
    ant_idx: np.ndarray     # indices into the parent layout
    scene: Scene
    dirs: np.ndarray
    t_int: int


def config4_jobs(n_jobs: int = 48, n_samp: int = 4096, seed: int = 4,
                 chan_choices=(128, 512, 2048)) -> list:
    """Batched uneven workload: sub-arrays of the 256-antenna random layout
    with N in {16..256}, B log-uniform in 8..4096, C from ``chan_choices``,
    T = 4096, noise plus one plane wave each, T_int = 64."""
    g = _rng(seed, _TAG_JOBS)
    parent = random_positions(256, 200.0, 3)
    jobs = []
    for j in range(n_jobs):
        n = int(g.choice([16, 32, 64, 128, 256]))
        b = int(round(math.exp(g.uniform(math.log(8), math.log(4096)))))
        c = int(g.choice(list(chan_choices)))
        idx = np.sort(g.choice(256, size=n, replace=False))
        nb_x = max(1, int(round(math.sqrt(b))))
        nb_y = max(1, (b + nb_x - 1) // nb_x)
        dirs = beam_grid(nb_x, nb_y, 10.0)[:b]
        f_lo = 400e6
        src_dir = direction(*g.uniform(-10, 10, size=2))
        scene = Scene(pos=parent[idx], freqs=channel_freqs(f_lo, 16e6, c),
                      n_samp=n_samp, seed=seed * 1000 + j,
                      sources=[Source(src_dir, 10.0)])
        jobs.append(Job(idx, scene, dirs, 64))
    return jobs
