"""Parity at the full sizes of the batched and serving workloads, on sampled
outputs the FP64 oracle can compute one by one (beams and channels are
independent, so a sampled channel and beam subset is exact parity for
those outputs).

- Batched: the 48 sub-array jobs (74 GB of FP16 voltages made on the device
  by the bench's seeded generator) in one graph-captured launch with the
  bench's autotuned tile width; every job is sampled (one channel, 16 beams,
  the first and the last 8 windows) against the oracle fed the same FP16
  values and weights.
- Serving: the six stream configurations at full size, two chunks per stream
  (the second continues the first's open window); sampled beams of one
  channel per stream against the oracle on the concatenated samples.
"""
import numpy as np
import pytest

import bench
import oracle
import synth
from helpers import rel_errors

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {synth.C16F: (2e-5, 5e-6), synth.CI8: (2e-5, 5e-6)}   # as in test_gpu_parity


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


def check(name, P, P_ref, mode):
    assert P.shape == P_ref.shape, (name, P.shape, P_ref.shape)
    mx, l2 = rel_errors(P, P_ref)
    tmx, tl2 = TOL[mode]
    assert mx <= tmx and l2 <= tl2, (name, mx, l2)


def test_batched_jobs_full_size_sampled(bf):
    jobs = synth.config4_jobs()
    stream = torch.cuda.Stream()
    plans, outs = [], []
    for job in jobs:
        B, C, T = job.dirs.shape[0], job.scene.freqs.size, job.scene.n_samp
        plans.append(bf.Plan(job.scene.pos, job.scene.freqs, job.dirs, bf.BF_C16F, job.t_int, stream=stream))
        outs.append(torch.empty((B, C, T // job.t_int), dtype=torch.float32, device="cuda"))
    xs = bench.config4_inputs(jobs, torch)
    batch = bf.Batch(plans, tile_t=256, stream=stream)
    for j, (x, o, job) in enumerate(zip(xs, outs, jobs)):
        batch.set(j, x, o, n_samp=job.scene.n_samp)
    batch.capture()
    batch.replay()
    batch.sync()
    g = np.random.default_rng(44)
    for j, (job, p) in enumerate(zip(jobs, plans)):
        c = int(g.integers(0, p.C))
        beams = np.sort(g.choice(p.B, size=min(p.B, 16), replace=False))
        W = oracle.quantised_weights(oracle.weights(job.scene.pos, job.scene.freqs[c:c + 1], job.dirs[beams]),
                                     synth.C16F)[0]
        n_win = job.scene.n_samp // job.t_int
        bsel = torch.from_numpy(beams).cuda()
        for w0 in (0, n_win - 8):   # the first and the last 8 windows
            t0 = w0 * job.t_int
            X64 = oracle.decode_voltages(synth.C16F, xs[j][c:c + 1, t0:t0 + 8 * job.t_int].cpu().numpy())
            P_ref = oracle.power(W, X64, job.t_int)
            P = outs[j][bsel, c:c + 1, w0:w0 + 8].cpu().numpy()
            check(f"job{j}_c{c}_w{w0}", P, P_ref, synth.C16F)
    batch.close()
    for p in plans:
        p.close()
    del xs, outs
    torch.cuda.empty_cache()


def test_serving_streams_full_size_sampled(bf):
    stream = torch.cuda.Stream()
    plans = bench.serve_plans(bf, stream)
    server = bf.Server(plans, mem_bytes=64 << 30, max_steps=3)
    cuts = (300, 700)   # the first chunk leaves a 44-sample window open
    g = np.random.default_rng(55)
    chunks, samples = [], []
    for i, (N, B, C, mode) in enumerate(bench.SERVE_CONFIGS):
        full = bench.serve_pool(torch, mode, N, C, sum(cuts), 9000 + i)        # [C][1000][2N] pinned
        parts, t0 = [], 0
        for T in cuts:
            h = full[:, t0:t0 + T].contiguous().pin_memory()
            o = torch.zeros(B * C * (-(-T // 64)), dtype=torch.float32).pin_memory()
            parts.append((h, o, T))
            t0 += T
        chunks.append(parts)
        c = int(g.integers(0, C))
        beams = np.sort(g.choice(B, size=min(B, 32), replace=False))
        samples.append((c, beams, full[c:c + 1].numpy().copy()))
    ids = []
    for k in range(len(cuts)):
        for i in range(len(chunks)):
            h, o, T = chunks[i][k]
            ids.append((i, k, server.submit(i, h, o, n_samp=T)))
    server.drain(300000)
    done = {}
    while len(done) < len(ids):
        for r in server.poll(256, 1000):
            done[r["id"]] = r
    server.close()
    for i, (N, B, C, mode) in enumerate(bench.SERVE_CONFIGS):
        c, beams, xc = samples[i]
        parts = []
        for (ii, k, rid) in ids:
            if ii != i:
                continue
            r = done[rid]
            assert r["status"] == 0
            nw = r["n_windows"]
            parts.append(chunks[i][k][1][:B * C * nw].numpy().reshape(B, C, nw)[beams, c:c + 1, :])
        P = np.concatenate(parts, axis=2)
        p = plans[i]
        pos = synth.grid_positions() if N == 32 else synth.random_positions(N, 200.0, 500 + i)
        nx = int(round(np.sqrt(B)))
        dirs = synth.beam_grid(nx, -(-B // nx))[:B]
        freqs = synth.channel_freqs(400e6, 16e6, C)
        W = oracle.quantised_weights(oracle.weights(pos, freqs[c:c + 1], dirs[beams]), mode)[0]
        P_ref = oracle.power(W, oracle.decode_voltages(mode, xc), 64)
        assert P.shape[2] == sum(cuts) // 64
        check(f"stream{i}_c{c}", P, P_ref, mode)
        p.close()
