"""The multi-rank generation step on CPU (gloo, world size 2).

Each rank evaluates its shard of a global population (the oracle stands in
for the GPU evaluator here), the fitness shards are all-gathered, and every
rank's tournament winners must equal those of one process that evaluated
the whole population.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2110_11226_gb300 import synth
from paper_2110_11226_gb300.dist import gather_fitness, max_over_ranks, shard_bounds


def test_shard_bounds_partition():
    for n in (1, 7, 4096, 4097):
        for w in (1, 2, 3, 8):
            spans = [shard_bounds(n, w, r) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir, n_progs):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.pagie_data(512, 3)
    nodes, off = synth.ramped_half_and_half(n_progs, 2, 6, synth.FULL_SET, 2, seed=8)
    progs = synth.unpack(nodes, off)
    a, b = shard_bounds(len(progs), world, rank)
    sn, so = synth.pack(progs[a:b])
    fit_local, _ = oracle.fitness(sn, so, d.X, d.y, None, "rmse")
    fit = gather_fitness(torch.from_numpy(fit_local.astype(np.float32)), n_total=len(progs))
    win = oracle.tournament(fit.numpy(), len(progs), 20, 42)
    t = max_over_ranks(float(rank + 1))
    np.save(os.path.join(out_dir, f"win{rank}.npy"), win)
    np.save(os.path.join(out_dir, f"fit{rank}.npy"), fit.numpy())
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_progs", [64, 65])
def test_two_rank_generation_matches_single_process(tmp_path, n_progs):
    """Even shards (64 programs) and uneven ones (65: 33 and 32)."""
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), n_progs), nprocs=world, join=True)
    d = synth.pagie_data(512, 3)
    nodes, off = synth.ramped_half_and_half(n_progs, 2, 6, synth.FULL_SET, 2, seed=8)
    fit, _ = oracle.fitness(nodes, off, d.X, d.y, None, "rmse")
    want = oracle.tournament(fit.astype(np.float32), n_progs, 20, 42)
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"fit{r}.npy"), fit.astype(np.float32))
        np.testing.assert_array_equal(np.load(tmp_path / f"win{r}.npy"), want)
        assert np.load(tmp_path / f"t{r}.npy")[0] == world
