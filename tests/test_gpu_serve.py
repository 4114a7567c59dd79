"""GPU tests of the serving loop (``bf_server_*``).

- A stream cut into chunks of any length integrates exactly as the same
  samples in one piece: the open window is carried on the device.
- Each chunk's powers are the same alone and in a mix of streams (bitwise:
  a tile is computed by the same code whatever else shares the launch).
- Admission by memory: a small arena serialises the chunks, nothing is lost,
  and a chunk that can never fit is refused.
Expected values come from the FP64 oracle on the same seeded inputs.
"""
import numpy as np
import pytest

import synth
from helpers import oracle_power_for_mode, rel_errors, small_scene, stored_voltages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the tensor-core tolerance of test_gpu_parity (its docstring derives it)
TOL = {m: (2e-5, 5e-6) for m in (synth.C16F, synth.CI8, synth.CI4, synth.C16BF)}


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


class StreamCase:
    """One configuration with a seeded voltage stream of T_total samples."""

    def __init__(self, bf, mode, n_ant, n_beam, n_chan, T_total, seed, t_int=64):
        sigma = 16.0 if mode == synth.CI8 else (2.0 if mode == synth.CI4 else 0.7071)
        self.mode, self.t_int, self.T_total = mode, t_int, T_total
        self.scene = small_scene(n_ant=n_ant, n_chan=n_chan, n_samp=T_total, seed=seed, grid=False, sigma=sigma)
        self.dirs = synth.beam_grid(16, 16)[:n_beam]
        assert self.dirs.shape[0] == n_beam
        self.x, self.X64 = stored_voltages(self.scene, mode)
        self.plan = bf.Plan(self.scene.pos, self.scene.freqs, self.dirs, mode, t_int)
        self.B, self.C = n_beam, n_chan

    def chunks(self, cuts):
        """Pinned host chunks [C][T_k][...] covering the stream in order."""
        assert sum(cuts) == self.T_total
        out, t0 = [], 0
        for T in cuts:
            h = torch.from_numpy(np.ascontiguousarray(self.x[:, t0:t0 + T])).pin_memory()
            o = torch.zeros(self.B * self.C * (-(-T // self.t_int)), dtype=torch.float32).pin_memory()
            out.append((h, o, T))
            t0 += T
        return out

    def oracle(self):
        return oracle_power_for_mode(self.scene, self.dirs, self.t_int, self.mode, self.X64)


def run_stream(server, cfg, chunks):
    ids = [server.submit(cfg, h, o, n_samp=T) for h, o, T in chunks]
    return ids


def collect(server, n, timeout_ms=60000):
    server.drain(timeout_ms)
    done = {}
    while len(done) < n:
        for c in server.poll(256, 1000):
            done[c["id"]] = c
    return done


def assemble(case, chunks, ids, done):
    """Concatenate the windows each chunk completed, in stream order."""
    parts = []
    for (h, o, T), i in zip(chunks, ids):
        c = done[i]
        assert c["status"] == 0, c
        assert c["t_submit"] <= c["t_start"] <= c["t_done"]
        nw = c["n_windows"]
        parts.append(o[:case.B * case.C * nw].numpy().reshape(case.B, case.C, nw))
    return np.concatenate(parts, axis=2)


def check(name, P, P_ref, mode):
    assert P.shape == P_ref.shape, (name, P.shape, P_ref.shape)
    mx, l2 = rel_errors(P, P_ref)
    tmx, tl2 = TOL[mode]
    assert mx <= tmx and l2 <= tl2, (name, mx, l2)


@pytest.mark.parametrize("mode,t_int,cuts", [
    (synth.C16F, 64, [100, 37, 300, 64, 129, 370]),   # windows cut at every offset
    (synth.CI8, 64, [64, 640, 1, 63, 232]),           # a one-sample chunk, a chunk closing a window exactly
    (synth.C16F, 10, [25, 25, 7, 143, 300]),          # generic window width
    (synth.CI4, 32, [31, 33, 500, 436]),
])
def test_stream_chunks_match_one_shot(bf, mode, t_int, cuts):
    case = StreamCase(bf, mode, 32, 70, 3, sum(cuts), seed=7, t_int=t_int)
    server = bf.Server([case.plan], mem_bytes=64 << 20, max_steps=2)
    chunks = case.chunks(cuts)
    ids = run_stream(server, 0, chunks)
    done = collect(server, len(ids))
    P = assemble(case, chunks, ids, done)
    assert P.shape[2] == case.T_total // t_int
    check("stream", P, case.oracle(), mode)
    # the same samples in one piece through bf_execute
    A = case.plan.execute(torch.from_numpy(np.ascontiguousarray(case.x)).cuda(), n_samp=case.T_total)
    case.plan.sync()
    A = A.cpu().numpy()
    assert np.max(np.abs(P - A) / np.maximum(A, 1e-3 * A.mean())) <= 1e-5
    st = server.stats()
    assert st["completed"] == len(cuts) and st["flops"] > 0 and st["kernel_ms"] > 0
    server.close()


def test_alone_vs_mix_identical(bf):
    specs = [(synth.C16F, 32, 100, 4, [700, 90, 210]), (synth.CI8, 64, 64, 2, [300, 300, 100]),
             (synth.C16F, 128, 200, 2, [129, 64, 407]), (synth.C16BF, 16, 30, 1, [1000])]
    # one operand format per server: the BF16 stream gets its own server in both runs
    cases = [StreamCase(bf, m, n, b, c, sum(cuts), seed=30 + i) for i, (m, n, b, c, cuts) in enumerate(specs)]
    cut_list = [s[4] for s in specs]
    alone = []
    for case, cuts in zip(cases, cut_list):
        server = bf.Server([case.plan], mem_bytes=256 << 20, max_steps=3)
        chunks = case.chunks(cuts)
        ids = run_stream(server, 0, chunks)
        alone.append(assemble(case, chunks, ids, collect(server, len(ids))))
        server.close()
    fp16 = [0, 1, 2]
    server = bf.Server([cases[i].plan for i in fp16], mem_bytes=256 << 20, max_steps=1)
    server.pause()   # queue every chunk first, so steps take one chunk of each stream
    all_chunks = [cases[i].chunks(cut_list[i]) for i in fp16]
    ids = [[] for _ in fp16]
    for k in range(3):   # interleave the streams' chunks
        for j, i in enumerate(fp16):
            if k < len(all_chunks[j]):
                h, o, T = all_chunks[j][k]
                ids[j].append(server.submit(j, h, o, n_samp=T))
    server.pause(False)
    done = collect(server, sum(len(x) for x in ids))
    st = server.stats()
    server.close()
    for j, i in enumerate(fp16):
        P = assemble(cases[i], all_chunks[j], ids[j], done)
        assert np.array_equal(P, alone[i]), i
        check(f"mix{i}", P, cases[i].oracle(), cases[i].mode)
    steps_with = {}
    for c in done.values():
        steps_with.setdefault(c["step"], set()).add(c["config"])
    assert st["max_jobs_per_step"] == max(len(v) for v in steps_with.values())
    assert st["max_jobs_per_step"] == 3 and st["steps"] == 3, steps_with   # streams shared every launch
    check("bf16_alone", alone[3], cases[3].oracle(), cases[3].mode)


def test_admission_by_memory(bf):
    case = StreamCase(bf, synth.C16F, 32, 64, 2, 2048, seed=50)
    per_chunk = 2 * 512 * 32 * 4 + 64 * 2 * 8 * 4   # voltages + powers of a 512-sample chunk
    mem = per_chunk + 4096                          # room for one chunk at a time
    server = bf.Server([case.plan], mem_bytes=mem, max_steps=3)
    chunks = case.chunks([512, 512, 512, 512])
    ids = run_stream(server, 0, chunks)
    done = collect(server, len(ids))
    P = assemble(case, chunks, ids, done)
    check("admission", P, case.oracle(), case.mode)
    st = server.stats()
    assert st["arena_peak"] <= mem and st["steps"] == 4
    big = torch.zeros((2, 4096, 64), dtype=torch.float16).pin_memory()
    out = torch.zeros(64 * 2 * 64, dtype=torch.float32).pin_memory()
    with pytest.raises(bf.BFError) as ei:
        server.submit(0, big, out, n_samp=4096)
    assert ei.value.status == bf.BF_ERR_ARG
    server.close()
