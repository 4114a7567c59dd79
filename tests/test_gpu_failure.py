"""Failure detection on the GPU without a fault: a bounded device wait on a
barrier that nothing signals gives up, reports BF_ERR_TIMEOUT through the
status word, and the context keeps working afterwards."""
import time

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


def test_bounded_wait_reports_timeout_and_context_survives(bf):
    stream = torch.cuda.Stream()
    for limit_ms in (20.0, 100.0):
        t0 = time.perf_counter()
        with pytest.raises(bf.BFError) as ei:
            bf.bf_selftest_timeout(limit_ms, stream.cuda_stream)
        dt = time.perf_counter() - t0
        assert ei.value.status == bf.BF_ERR_TIMEOUT
        assert dt >= 0.5 * limit_ms * 1e-3 and dt < 5.0, dt
    # the context is intact: a beamformer run still matches the oracle
    scene = small_scene(n_ant=32, n_chan=2, n_samp=256)
    dirs = synth.beam_grid(8, 8)
    x, X64 = stored_voltages(scene, synth.C16F)
    plan = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, 64)
    P = plan.execute(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    plan.sync()
    mx, l2 = rel_errors(P.cpu().numpy(), oracle_power_for_mode(scene, dirs, 64, synth.C16F, X64))
    assert mx <= 2e-5 and l2 <= 5e-6   # the tensor-core tolerance of test_gpu_parity
    plan.close()
