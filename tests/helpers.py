"""Shared test helpers: error metrics and oracle references for a plan's mode.

The expected values always come from ``oracle`` (FP64, CPU) applied to the
same seeded inputs the GPU sees; nothing here reads GPU results back into the
oracle.
"""
import numpy as np

import oracle
import synth


def rel_errors(P, P_ref):
    """(max relative error with a floor of 1e-3 x mean, L2 relative error).
    The floor keeps near-null outputs (deep sidelobes) from dominating."""
    P = np.asarray(P, dtype=np.float64)
    P_ref = np.asarray(P_ref, dtype=np.float64)
    if P_ref.size == 0:
        return 0.0, 0.0
    floor = 1e-3 * max(P_ref.mean(), 1e-300)
    mx = float(np.max(np.abs(P - P_ref) / np.maximum(P_ref, floor)))
    l2 = float(np.linalg.norm(P - P_ref) / max(np.linalg.norm(P_ref), 1e-300))
    return mx, l2


def stored_voltages(scene, mode, channels=None):
    """The voltages exactly as stored for ``mode`` ([c][t][2n] or [c][t][n]
    for 4-bit) and their decoded complex128 values for the oracle."""
    x = synth.voltages(scene, mode, channels=channels)
    return x, oracle.decode_voltages(mode, x)


def oracle_power_for_mode(scene, dirs, t_int, mode, X64, channels=None, mask=None):
    """Oracle powers for a plan of ``mode``: the mode's weights are the
    format's rounding of the exact weights (with the per-beam scale of the
    FP8 and int8 readings), inputs are the stored values."""
    freqs = scene.freqs if channels is None else scene.freqs[list(channels)]
    W = oracle.weights(scene.pos, freqs, dirs, mask)
    if mode != oracle.C32:
        W, _, _ = oracle.quantised_weights(W, mode)
    return oracle.power(W, X64, t_int)


def small_scene(n_ant=32, n_chan=3, n_samp=1000, seed=11, grid=True, n_src=2, sigma=0.7071067811865476,
                extent=60.0, snr_lo=5.0, snr_hi=15.0):
    pos = synth.grid_positions() if (grid and n_ant == 32) else synth.random_positions(n_ant, extent, seed)
    freqs = synth.channel_freqs(400e6, 16e6, 64)[:n_chan]
    src = synth.random_sources(n_src, 10.0, snr_lo, snr_hi, 2 * sigma ** 2, seed)
    return synth.Scene(pos=pos, freqs=freqs, n_samp=n_samp, seed=seed, noise_sigma=sigma, sources=src)
