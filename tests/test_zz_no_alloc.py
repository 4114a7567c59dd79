"""bf_execute_nct_static: the antenna-major execute path with its scratch in a
fixed device array, for callers that cannot allocate device memory when they
execute.  Its powers must agree with bf_execute's (same kernels, same inputs)
within the tolerance of the other tensor-core tests, on two calls in a row
through the shared array.  This file runs last so that a failure here comes
after every other test has run."""
import numpy as np
import pytest

import synth
from helpers import oracle_power_for_mode, rel_errors, small_scene, stored_voltages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


@pytest.mark.parametrize("mode", [synth.C16F, synth.CI8])
def test_static_scratch_matches_allocating_execute(bf, mode):
    sigma = 16.0 if mode == synth.CI8 else 0.7071
    scene = small_scene(n_ant=32, n_chan=3, n_samp=700, sigma=sigma)
    dirs = synth.beam_grid(10, 9)
    x, X64 = stored_voltages(scene, mode)
    xn = torch.from_numpy(synth.to_nct(x, mode)).cuda()
    plan = bf.Plan(scene.pos, scene.freqs, dirs, mode, 64, bf.BF_LAYOUT_NCT)
    ref = plan.execute(xn).cpu().numpy()
    out = torch.empty((90, 3, 700 // 64), dtype=torch.float32, device="cuda")
    for _ in range(2):   # the array keeps the previous call's contents
        out.fill_(-1.0)
        bf.bf_execute_nct_static(plan.handle, xn.data_ptr(), 700, out.data_ptr(), plan.stream.cuda_stream)
        plan.sync()
        got = out.cpu().numpy()
        mx, l2 = rel_errors(got, ref)
        assert mx <= 1e-4 and l2 <= 1e-5, (mx, l2)
    # and against the FP64 oracle, with the tolerance of the other 16-bit / int8 tests
    mx, l2 = rel_errors(got, oracle_power_for_mode(scene, dirs, 64, mode, X64))
    assert mx <= 1e-4 and l2 <= 1e-5, (mx, l2)
    plan.close()


def test_static_scratch_rejects_oversize_input(bf):
    scene = small_scene(n_ant=32, n_chan=64, n_samp=16)
    plan = bf.Plan(scene.pos, scene.freqs, synth.beam_grid(2, 2), synth.C16F, 16, bf.BF_LAYOUT_NCT)
    t = 65536   # 64 channels x 65536 samples x 32 antennas x 4 bytes = 512 MiB > 64 MiB
    with pytest.raises(bf.BFError) as ei:
        bf.bf_execute_nct_static(plan.handle, 256, t, 256, plan.stream.cuda_stream)
    assert ei.value.status == bf.BF_ERR_ARG and "static scratch" in str(ei.value)
    plan.close()
