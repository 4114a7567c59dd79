"""GPU parity of batched execution (``bf_batch_*``).

A batch step runs the jobs of 4 or more K blocks in one persistent launch and
the others through their plans' resident-weight kernel on forked streams.
Each job of a batch is checked against the FP64 oracle for its own plan (the
tolerances of the single-plan parity tests) and against the same plan run
alone through ``bf_execute``: batching changes where a tile is computed, not
what it computes, so the two agree to FP32 summation order.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import oracle_power_for_mode, rel_errors, small_scene, stored_voltages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tensor-core tolerance of test_gpu_parity (its docstring derives it)
TOL = {m: (2e-5, 5e-6) for m in (synth.C16F, synth.C16BF, synth.CI8, synth.CI4, synth.C8E4M3)}
# batched vs alone: same products and K order; the window sums may group
# the squares differently (tile width), so a few FP32 ulps per sum
ALONE_TOL = 1e-5


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sigma_for(mode):
    return 16.0 if mode in (synth.CI8, synth.C8E4M3) else (2.0 if mode == synth.CI4 else 0.7071)


class Job:
    """One plan of a batch with its seeded scene, stored voltages and the
    oracle's powers."""

    def __init__(self, bf, mode, n_ant, n_beam, n_chan, n_samp, t_int, seed):
        self.mode, self.t_int = mode, t_int
        self.scene = small_scene(n_ant=n_ant, n_chan=n_chan, n_samp=max(n_samp, 1), seed=seed, grid=False,
                                 sigma=sigma_for(mode))
        self.T = n_samp
        self.dirs = synth.beam_grid(13, 13)[seed % 7: seed % 7 + n_beam]
        assert self.dirs.shape[0] == n_beam
        x, X64 = stored_voltages(self.scene, mode)
        self.x_host, self.X64 = x[:, :n_samp], X64[:, :n_samp]
        self.x = dev(self.x_host)
        self.plan = bf.Plan(self.scene.pos, self.scene.freqs, self.dirs, mode, t_int)

    def oracle(self, dirs=None):
        d = self.dirs if dirs is None else dirs
        return oracle_power_for_mode(self.scene, d, self.t_int, self.mode, self.X64)

    def alone(self):
        out = self.plan.execute(self.x, n_samp=self.T)
        self.plan.sync()
        return out.cpu().numpy()


def check_job(name, P, job, P_ref=None):
    P_ref = job.oracle() if P_ref is None else P_ref
    assert P.shape == P_ref.shape, (name, P.shape, P_ref.shape)
    if P.size == 0:
        return
    assert np.all(np.isfinite(P))
    mx, l2 = rel_errors(P, P_ref)
    tmx, tl2 = TOL[job.mode]
    assert mx <= tmx and l2 <= tl2, (name, mx, l2)


def run_batch(bf, jobs, tile_t=0):
    batch = bf.Batch([j.plan for j in jobs], tile_t=tile_t)
    outs = [batch.set(i, j.x, n_samp=j.T) for i, j in enumerate(jobs)]
    batch.execute()
    batch.sync()
    return batch, [o.cpu().numpy() for o in outs]


def streamed(bf, plan):
    """The plan's weights are streamed (4 or more K blocks): its batch jobs
    run in the persistent launch."""
    return bf.bf_plan_query_tiles(plan.handle)["x_stages"] == 0


def test_batch_mixed_fp16_family(bf):
    """FP16, int8 and int4 plans of different antenna counts (1 to 8 K
    blocks), beam counts (partial M tiles), channel counts and sample counts
    (ragged time tiles, a job shorter than one window, an empty job).  The
    int8 job of 36 antennas and the int4 job of 24 have rows TMA cannot read
    raw (72 and 24 bytes): they are widened to FP16 before their
    resident-weight launch; the other 8/4-bit resident jobs are widened in
    the kernel."""
    specs = [(synth.C16F, 64, 100, 3, 640), (synth.C16F, 256, 70, 2, 300), (synth.CI8, 40, 130, 2, 512),
             (synth.CI4, 32, 64, 2, 200), (synth.C16F, 8, 1, 1, 64), (synth.C16F, 16, 20, 1, 30),
             (synth.CI8, 128, 65, 1, 0), (synth.CI8, 36, 30, 1, 256), (synth.CI4, 24, 20, 2, 128),
             (synth.CI8, 160, 40, 2, 384)]
    jobs = [Job(bf, m, n, b, c, t, 64, seed=20 + i) for i, (m, n, b, c, t) in enumerate(specs)]
    batch, outs = run_batch(bf, jobs)
    q = batch.query()
    assert q["tile_t"] == 256
    assert [streamed(bf, j.plan) for j in jobs] == [False, True, False, False, False, False, True, False, False, True]
    # units of the persistent launch; time tiles cover whole windows only (the
    # tail beyond the last window is never read)
    exp_units = sum(j.scene.freqs.size * -(-(j.T // 64 * 64) // 256) * -(-j.dirs.shape[0] // 64)
                    for j in jobs if streamed(bf, j.plan))
    assert q["units"] == exp_units
    for i, (j, P) in enumerate(zip(jobs, outs)):
        check_job(f"job{i}", P, j)
        A = j.alone()
        if P.size:
            assert np.max(np.abs(P - A) / np.maximum(A, 1e-3 * A.mean())) <= ALONE_TOL, i
    batch.close()


@pytest.mark.parametrize("mode", [synth.C16BF, synth.C8E4M3])
def test_batch_formats(bf, mode):
    specs = [(64, 70, 2, 512), (256, 128, 1, 260), (16, 33, 3, 128)]
    jobs = [Job(bf, mode, n, b, c, t, 64, seed=40 + i) for i, (n, b, c, t) in enumerate(specs)]
    batch, outs = run_batch(bf, jobs)
    for i, (j, P) in enumerate(zip(jobs, outs)):
        check_job(f"{synth.MODE_NAMES[mode]}_job{i}", P, j)
    batch.close()


@pytest.mark.parametrize("t_int,tile_t", [(16, 0), (10, 0), (32, 128), (48, 0), (64, 64)])
def test_batch_windows_and_tiles(bf, t_int, tile_t):
    """Compile-time window widths (16, 32), the generic per-column window
    counter (T_int 10 -> 160-sample tiles), lcm tiles (48 -> 240) and a
    requested narrower tile."""
    specs = [(32, 40, 2, 700), (64, 65, 1, 333)]
    jobs = [Job(bf, synth.C16F, n, b, c, t, t_int, seed=60 + i) for i, (n, b, c, t) in enumerate(specs)]
    batch, outs = run_batch(bf, jobs, tile_t=tile_t)
    nt = batch.query()["tile_t"]
    assert nt % t_int == 0 and nt % 16 == 0 and nt // t_int <= 16
    if tile_t:
        assert nt == tile_t
    for i, (j, P) in enumerate(zip(jobs, outs)):
        check_job(f"Ti{t_int}_job{i}", P, j)
    batch.close()


def test_batch_many_small_jobs(bf):
    """More persistent-launch jobs than SMs (and than fit in the launch
    parameters), so CTAs straddle job boundaries and the cost split lands
    inside and between jobs, beside dozens of resident-weight jobs on the
    forked streams; includes empty jobs."""
    rng = np.random.default_rng(5)
    jobs = []
    for i in range(180):
        n = int(rng.choice([4, 8, 12, 32, 68, 100, 132, 200], p=[.05, .05, .05, .05, .1, .3, .2, .2]))
        b = int(rng.integers(1, 90))
        c = int(rng.integers(1, 3))
        t = int(rng.choice([0, 64, 100, 256, 300]))
        jobs.append(Job(bf, synth.C16F, n, b, c, t, 64, seed=100 + i))
    n_streamed = sum(streamed(bf, j.plan) and j.T >= 64 for j in jobs)
    assert n_streamed > 152 // 2 and n_streamed > 64 and len(jobs) - n_streamed > 20
    batch, outs = run_batch(bf, jobs)
    assert batch.query()["units"] > 152
    for i, (j, P) in enumerate(zip(jobs, outs)):
        check_job(f"small{i}", P, j)
    batch.close()


def test_batch_graph_replay_and_weights(bf):
    """A captured step replays on new input contents (same buffers) and picks
    up weights regenerated by bf_weights on a member plan; re-binding a job
    drops the graph."""
    stream = torch.cuda.Stream()
    specs = [(synth.C16F, 64, 64, 2, 512), (synth.CI8, 32, 100, 1, 256), (synth.C16F, 160, 40, 1, 320)]
    jobs = [Job(bf, m, n, b, c, t, 64, seed=80 + i) for i, (m, n, b, c, t) in enumerate(specs)]
    with torch.cuda.stream(stream):
        batch = bf.Batch([j.plan for j in jobs], stream=stream)
        outs = [batch.set(i, j.x, n_samp=j.T) for i, j in enumerate(jobs)]
        batch.capture()
        batch.replay()
        batch.sync()
        for i, (j, o) in enumerate(zip(jobs, outs)):
            check_job(f"replay{i}", o.cpu().numpy(), j)
        # new voltages in the same buffers
        for j in jobs:
            j.scene = synth.Scene(pos=j.scene.pos, freqs=j.scene.freqs, n_samp=j.scene.n_samp, seed=j.scene.seed + 1000,
                                  noise_sigma=j.scene.noise_sigma, sources=j.scene.sources)
            x, X64 = stored_voltages(j.scene, j.mode)
            j.X64 = X64[:, :j.T]
            j.x.copy_(dev(x[:, :j.T]))
        # new pointing of job 0 (same beam count)
        new_dirs = synth.beam_grid(13, 13)[40:40 + jobs[0].dirs.shape[0]]
        jobs[0].plan.weights(new_dirs)
        jobs[0].plan.sync()   # weights are generated on the plan's stream
        batch.replay()
        batch.sync()
        check_job("replay_new0", outs[0].cpu().numpy(), jobs[0], jobs[0].oracle(new_dirs))
        check_job("replay_new1", outs[1].cpu().numpy(), jobs[1])
        check_job("replay_new2", outs[2].cpu().numpy(), jobs[2])
        batch.set(1, jobs[1].x, out=outs[1], n_samp=jobs[1].T)
        with pytest.raises(bf.BFError) as ei:
            batch.replay()
        assert ei.value.status == bf.BF_ERR_STATE
    stream.synchronize()
    batch.close()


def test_batch_rejections(bf):
    scene = small_scene(n_ant=16, n_chan=1, n_samp=128, grid=False)
    dirs = synth.beam_grid(4, 4)
    p16 = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, 64)
    p8 = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C8E4M3, 64)
    p32 = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C32, 64)
    pbf = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16BF, 64)
    pt = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, 32)
    pn = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, 64, bf.BF_LAYOUT_NCT)
    for bad in ([p16, p8], [p16, p32], [p16, pbf], [p16, pt], [pn], [p32]):
        with pytest.raises(bf.BFError) as ei:
            bf.Batch(bad)
        assert ei.value.status == bf.BF_ERR_UNSUPPORTED
    with pytest.raises(bf.BFError) as ei:
        bf.Batch([p16], tile_t=72)   # not a multiple of 16 and T_int
    assert ei.value.status == bf.BF_ERR_UNSUPPORTED
    pdb = bf.Plan(scene.pos, scene.freqs, dirs, bf.BF_C16F, 64)
    pdb.set_weight_buffers(2)        # the batch would hold a weight pointer that moves
    with pytest.raises(bf.BFError) as ei:
        bf.Batch([p16, pdb])
    assert ei.value.status == bf.BF_ERR_UNSUPPORTED
    pdb.close()
    batch = bf.Batch([p16, p16])
    with pytest.raises(bf.BFError) as ei:
        batch.execute()   # jobs not bound
    assert ei.value.status == bf.BF_ERR_STATE
    with pytest.raises(bf.BFError) as ei:
        batch.replay()
    assert ei.value.status == bf.BF_ERR_STATE
    x = torch.zeros((1, 128, 32), dtype=torch.float16, device="cuda")
    with pytest.raises(bf.BFError) as ei:
        bf.bf_batch_set(batch.handle, 2, x.data_ptr(), 128, x.data_ptr())
    assert ei.value.status == bf.BF_ERR_ARG
    with pytest.raises(bf.BFError) as ei:
        bf.bf_batch_set(batch.handle, 0, x.data_ptr() + 2, 128, x.data_ptr())
    assert ei.value.status == bf.BF_ERR_ARG
    # the same plan twice in one batch is allowed: two jobs, two outputs
    xs = [dev(synth.voltages(scene, synth.C16F)), dev(synth.voltages(scene, synth.C16F))]
    o0 = batch.set(0, xs[0])
    o1 = batch.set(1, xs[1])
    batch.execute()
    batch.sync()
    assert torch.equal(o0, o1)
    batch.close()
    for p in (p16, p8, p32, pbf, pt, pn):
        p.close()
