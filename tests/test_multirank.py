"""The multi-GPU path on the CPU: two `gloo` ranks (one process each, as
torchrun starts them) run the sharding and timing logic of bench.py.
Channels are independent (Section 2.1: one matrix product per channel), so
the path shards by contiguous channel ranges with no data exchange; the only
collectives are the barrier and the max of the ranks' times.  Each rank
beamforms its channel range with the oracle; rank 0 checks that the union of
the shards equals the whole band computed in one piece."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402
from helpers import small_scene  # noqa: E402


def test_shard_ranges_cover_once():
    for n in (0, 1, 5, 64, 1023, 1024):
        for world in (1, 2, 3, 4, 8):
            ranges = [bench.shard_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scene = small_scene(n_ant=16, n_chan=5, n_samp=128, grid=False)
        dirs = synth.beam_grid(3, 3)
        lo, hi = bench.shard_range(scene.n_chan, world, rank)
        X = oracle.decode_voltages(synth.C32, synth.voltages(scene, synth.C32, channels=range(lo, hi)))
        W = oracle.weights(scene.pos, scene.freqs[lo:hi], dirs)
        P = oracle.power(W, X, 16)
        t = bench.max_over_ranks(float(10 + rank), dist)   # each rank's "time"
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, P, t))
        if rank == 0:
            np.save(os.path.join(out_dir, "ok.npy"), np.array([1]))
            full = oracle.power(oracle.weights(scene.pos, scene.freqs, dirs),
                                oracle.decode_voltages(synth.C32, synth.voltages(scene, synth.C32)), 16)
            got = np.concatenate([p[2] for p in sorted(parts, key=lambda q: q[0])], axis=1)
            assert np.array_equal(got, full)
            assert all(p[3] == 10.0 + world - 1 for p in parts)   # every rank saw the slowest time
            np.save(os.path.join(out_dir, "checked.npy"), np.array([1]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_channels(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert (tmp_path / "checked.npy").exists()
