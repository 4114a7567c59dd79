"""FP64 CPU oracle of the coherent beamformer — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does, and this
package imports nothing from the product: the two share no code.  The only
module both sides use is ``synth`` (seeded inputs, no beamformer arithmetic).

The arithmetic lives in ``oracle.c`` (plain double-precision loops, see its
header for the definitions and the paper passages they follow).  This module
builds it with gcc, loads it with ctypes and adds the plain definitions of
the storage formats (how a stored code maps to a real number), of the
per-mode weight quantisation, and of the corner turn.

Parity is pinned by ``tests/test_oracle_pins.py`` against closed forms
(N^2 gain, the Eq. 1 array factor of a regular grid as a product of
Dirichlet kernels, the DFT special case through numpy.fft), invariants
(linearity, parallelogram law, single antenna), statistics and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

C32, C16F, C16BF, C8E4M3, CI8, CI4 = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_weights.argtypes = [I, P, P, I, P, I, P, P]
        lib.oracle_beams.argtypes = [I, I, I, I, P, P, I, P, I]
        lib.oracle_power.argtypes = [I, I, I, I, P, P, I, I, P, I]
        lib.oracle_incoherent.argtypes = [I, I, I, P, I, I, P, I]
        for f in (lib.oracle_weights, lib.oracle_beams, lib.oracle_power, lib.oracle_incoherent):
            f.restype = I
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def weights(pos, freqs, dirs, mask=None) -> np.ndarray:
    """W[c][b][n] = exp(-i 2 pi f_c (r_n . s_b) / c0) as complex128
    (Eq. 1; zero where ``mask`` is 0, Section 3.1)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    freqs = np.ascontiguousarray(freqs, dtype=np.float64)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    N, C, B = pos.shape[0], freqs.shape[0], dirs.shape[0]
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.empty((C, B, N, 2))
    rc = _load().oracle_weights(N, _p(pos), None if m is None else _p(m), C, _p(freqs),
                                B, _p(dirs), _p(out))
    if rc:
        raise ValueError("oracle_weights: bad arguments")
    return out.view(np.complex128)[..., 0]


def _cplx_in(x):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    return x.view(np.float64)


def beams(W, X, nct: bool = False, threads: int = 0) -> np.ndarray:
    """B[b][c][t] = sum_n W[c][b][n] X[c][t][n]  (Section 2.1).
    ``X`` is complex ``[C][T][N]`` (or ``[N][C][T]`` with ``nct``)."""
    W = np.ascontiguousarray(W, dtype=np.complex128)
    C, B, N = W.shape
    T = X.shape[2] if nct else X.shape[1]
    xf = _cplx_in(X)
    out = np.empty((B, C, T, 2))
    rc = _load().oracle_beams(N, C, T, B, _p(W.view(np.float64)), _p(xf), int(nct), _p(out), threads)
    if rc:
        raise ValueError("oracle_beams: bad arguments")
    return out.view(np.complex128)[..., 0]


def power(W, X, t_int: int, nct: bool = False, threads: int = 0) -> np.ndarray:
    """P[b][c][j] = sum over window j of |B[b][c][t]|^2  (Section 2.1)."""
    W = np.ascontiguousarray(W, dtype=np.complex128)
    C, B, N = W.shape
    T = X.shape[2] if nct else X.shape[1]
    xf = _cplx_in(X)
    out = np.empty((B, C, T // t_int))
    rc = _load().oracle_power(N, C, T, B, _p(W.view(np.float64)), _p(xf), int(nct), t_int,
                              _p(out), threads)
    if rc:
        raise ValueError("oracle_power: bad arguments")
    return out


def incoherent(X, t_int: int, nct: bool = False, threads: int = 0) -> np.ndarray:
    """P_inc[c][j] = sum over window j of sum_n |X[c][t][n]|^2  (Section 1)."""
    if nct:
        N, C, T = X.shape
    else:
        C, T, N = X.shape
    xf = _cplx_in(X)
    out = np.empty((C, T // t_int))
    rc = _load().oracle_incoherent(N, C, T, _p(xf), int(nct), t_int, _p(out), threads)
    if rc:
        raise ValueError("oracle_incoherent: bad arguments")
    return out


# ---------------------------------------------------------- storage formats
def _e4m3_value(code: int) -> float:
    """OCP FP8 E4M3FN: 1 sign, 4 exponent (bias 7), 3 mantissa bits; no
    infinities; S.1111.111 is NaN; exponent 0 is subnormal (m/8 * 2^-6)."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 7
    if e == 15 and m == 7:
        return float("nan")
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


E4M3_VALUES = np.array([_e4m3_value(c) for c in range(256)])
E4M3_MAX = 448.0


def decode_real(mode: int, a) -> np.ndarray:
    """Stored real components -> float64."""
    a = np.asarray(a)
    if mode == C32:
        return a.astype(np.float32).astype(np.float64)
    if mode == C16F:
        return a.astype(np.float16).astype(np.float64)
    if mode == C16BF:
        return (a.astype(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if mode == C8E4M3:
        return E4M3_VALUES[a.astype(np.uint8)]
    if mode == CI8:
        return a.astype(np.int8).astype(np.float64)
    raise ValueError(f"no real decoding for mode {mode}")


def decode_voltages(mode: int, a) -> np.ndarray:
    """Stored voltages ``[..., 2N]`` (re/im interleaved; for CI4 ``[..., N]``
    bytes with the real part in the high nibble, two's complement, as in the
    4-bit F-engine format of Section 2.1) -> complex128 ``[..., N]``."""
    a = np.asarray(a)
    if mode == CI4:
        b = a.astype(np.uint8).astype(np.int16)
        re = ((b >> 4) & 0xF)
        im = b & 0xF
        re = np.where(re >= 8, re - 16, re)
        im = np.where(im >= 8, im - 16, im)
        return re.astype(np.float64) + 1j * im.astype(np.float64)
    f = decode_real(mode, a)
    return f[..., 0::2] + 1j * f[..., 1::2]


def round_half_even(x):
    return np.rint(x)   # IEEE rint rounds ties to even


def encode_real(mode: int, x) -> np.ndarray:
    """float64 -> nearest stored value (ties to even), as a decoded float64.
    FP8 saturates at +-448; int8 clips at +-127."""
    x = np.asarray(x, dtype=np.float64)
    if mode == C32:
        return x.astype(np.float32).astype(np.float64)
    if mode == C16F:
        return x.astype(np.float16).astype(np.float64)
    if mode == C16BF:
        # round the double to the bf16 grid (8 significant bits), ties to even
        m, e = np.frexp(x)                 # x = m * 2^e, 0.5 <= |m| < 1
        q = round_half_even(m * 256.0) / 256.0
        out = np.ldexp(q, e)
        return np.where(x == 0, 0.0, out)
    if mode == C8E4M3:
        vals = E4M3_VALUES[:127]           # 0 .. 448 ascending
        a = np.minimum(np.abs(x), E4M3_MAX)
        hi_i = np.clip(np.searchsorted(vals, a), 1, 126)
        lo, hi = vals[hi_i - 1], vals[hi_i]
        d_lo, d_hi = a - lo, hi - a
        take_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (hi_i % 2 == 0))
        mag = np.where(take_hi, hi, lo)
        return np.where(x < 0, -mag, mag)
    if mode == CI8:
        return np.clip(round_half_even(x), -127, 127)
    raise ValueError(f"no encoding for mode {mode}")


Q_MAX = {C8E4M3: E4M3_MAX, CI8: 127.0}


def quantised_weights(W, mode: int):
    """The weights a ``mode`` plan multiplies with, as complex128, and the
    per-beam scale.  FP32/FP16/BF16: each component rounded to the format
    (scale 1).  FP8-E4M3 and int8: per beam b a scale
    sigma_b = max_n max(|Re W|, |Im W|) / Qmax, components rounded to the
    format after division by sigma_b; the effective weight is
    sigma_b * stored value.  Returns (effective weights, sigma [C][B],
    stored values)."""
    W = np.asarray(W, dtype=np.complex128)
    if mode in (C32, C16F, C16BF, CI4):
        # 4-bit input is multiplied with FP16 weights
        m = C16F if mode == CI4 else mode
        q = encode_real(m, W.real) + 1j * encode_real(m, W.imag)
        return q, np.ones(W.shape[:2]), q
    qmax = Q_MAX[mode]
    mx = np.maximum(np.abs(W.real), np.abs(W.imag)).max(axis=2)      # [C][B]
    sig = np.where(mx > 0, mx / qmax, 1.0)
    s = sig[..., None]
    q = encode_real(mode, W.real / s) + 1j * encode_real(mode, W.imag / s)
    return q * s, sig, q


def corner_turn(x_nct, perm=None):
    """Antenna-major ``[N][C][T]`` complex -> ``[C][T][N]``, antenna ``n`` of
    the output taken from input row ``perm[n]`` (the F-engine-order lookup
    table of Section 3)."""
    x = np.asarray(x_nct)
    if perm is not None:
        x = x[np.asarray(perm)]
    return np.ascontiguousarray(np.moveaxis(x, 0, 2))


def detect(P, k_sigma: float):
    """Detrend-and-threshold consumer of the integrated powers, the reading of
    the 'detrending' and 'RFI thresholding' stages that follow the beamformer
    in the transient pipeline of Section 3 (Table 3; the paper gives no
    formula for them).  For every beam b and channel c, over the chunk's
    windows j:  mu = mean_j P[b][c][j],  sigma = sqrt(mean_j (P - mu)^2)
    (population), z[b][c][j] = (P - mu) / sigma (0 where sigma = 0), and the
    hits are the (b, c, j) with z > k_sigma.  Returns (z as float64 [B][C][T_o],
    hits as a sorted int array [n][3])."""
    P = np.asarray(P, dtype=np.float64)
    mu = P.mean(axis=2, keepdims=True)
    sd = np.sqrt(((P - mu) ** 2).mean(axis=2, keepdims=True))
    z = np.where(sd > 0, (P - mu) / np.where(sd > 0, sd, 1.0), 0.0)
    hits = np.argwhere(z > k_sigma)
    return z, hits
