"""bf_execute_nct_static: the antenna-major execute path with its scratch in a
fixed device array, for callers that cannot allocate device memory when they
execute (allocators closed after set-up, real-time loops, fixed budgets).

Its powers must agree with bf_execute's (same kernels, same inputs) within
the tolerance of the other tensor-core tests, and with the FP64 oracle, on
two calls in a row through the shared array.  The second call uses another
scene and fewer samples, so the array still holds the first call's larger
contents when it runs: a leak of stale scratch into the result would show.
Plans with 128 and 256 antennas take the streamed-weight pipeline.  This
file runs last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import synth
from helpers import oracle_power_for_mode, rel_errors, small_scene, stored_voltages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = (2e-5, 5e-6)   # max and L2 relative error, as for the other tensor-core modes


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


def _sigma(mode):
    return {synth.CI8: 16.0, synth.CI4: 2.0, synth.C8E4M3: 16.0}.get(mode, 0.7071)


@pytest.mark.parametrize("n_ant,mode", [
    (32, synth.C16F), (32, synth.CI8), (32, synth.CI4),
    (128, synth.C16F),   # 4 K blocks: streamed weights
    (256, synth.CI8),    # 8 K blocks after widening to FP16: streamed
])
def test_static_scratch_matches_allocating_execute(bf, n_ant, mode):
    dirs = synth.beam_grid(10, 9)
    # first call: 700 samples; second: other noise and sources, 450 samples
    first = small_scene(n_ant=n_ant, n_chan=3, n_samp=700, sigma=_sigma(mode), grid=n_ant == 32)
    second = synth.Scene(pos=first.pos, freqs=first.freqs, n_samp=450, seed=29, noise_sigma=first.noise_sigma,
                         sources=synth.random_sources(2, 10.0, 5.0, 15.0, 2 * first.noise_sigma ** 2, 29))
    plan = bf.Plan(first.pos, first.freqs, dirs, mode, 64, bf.BF_LAYOUT_NCT)
    for scene, T in ((first, 700), (second, 450)):
        x, X64 = stored_voltages(scene, mode)
        xn = torch.from_numpy(synth.to_nct(x, mode)).cuda()
        ref = plan.execute(xn).cpu().numpy()
        out = torch.full((90, 3, T // 64), -1.0, dtype=torch.float32, device="cuda")
        bf.bf_execute_nct_static(plan.handle, xn.data_ptr(), T, out.data_ptr(), plan.stream.cuda_stream)
        plan.sync()
        got = out.cpu().numpy()
        mx, l2 = rel_errors(got, ref)
        assert mx <= TOL[0] and l2 <= TOL[1], ("vs bf_execute", T, mx, l2)
        mx, l2 = rel_errors(got, oracle_power_for_mode(scene, dirs, 64, mode, X64))
        assert mx <= TOL[0] and l2 <= TOL[1], ("vs oracle", T, mx, l2)
    plan.close()


def test_static_scratch_rejects_oversize_input(bf):
    scene = small_scene(n_ant=32, n_chan=64, n_samp=16)
    plan = bf.Plan(scene.pos, scene.freqs, synth.beam_grid(2, 2), synth.C16F, 16, bf.BF_LAYOUT_NCT)
    t = 65536   # 64 channels x 65536 samples x 32 antennas x 4 bytes = 512 MiB > 64 MiB
    with pytest.raises(bf.BFError) as ei:
        bf.bf_execute_nct_static(plan.handle, 256, t, 256, plan.stream.cuda_stream)
    assert ei.value.status == bf.BF_ERR_ARG and "static scratch" in str(ei.value)
    plan.close()


def test_static_scratch_clears_the_last_error(bf):
    """A successful call leaves no message of an earlier failure behind."""
    scene = small_scene(n_ant=32, n_chan=2, n_samp=128)
    plan = bf.Plan(scene.pos, scene.freqs, synth.beam_grid(2, 2), synth.C16F, 64, bf.BF_LAYOUT_NCT)
    with pytest.raises(bf.BFError):
        bf.bf_execute_nct_static(plan.handle, 256, 1 << 20, 256, plan.stream.cuda_stream)
    assert bf.bf_last_error() != ""
    x, _ = stored_voltages(scene, synth.C16F)
    xn = torch.from_numpy(synth.to_nct(x, synth.C16F)).cuda()
    out = torch.empty((4, 2, 2), dtype=torch.float32, device="cuda")
    bf.bf_execute_nct_static(plan.handle, xn.data_ptr(), 128, out.data_ptr(), plan.stream.cuda_stream)
    assert bf.bf_last_error() == ""
    plan.sync()
    plan.close()
