"""Sharding over ranks, on CPU: whole-element ranges and the rank-ordered reduction of the ln A
gradient (world size 2, gloo).  Each rank evaluates its shard with the oracle; the reduced
gradient must equal the unsharded one."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2409_06404_gb300 import shard, synth


def test_shard_ranges_cover_whole_elements():
    for n in (0, 511, 512, 4096 * 512, 4096 * 512 + 100, 7 * 512 + 3):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            for r, (a, b) in enumerate(ranges):
                assert a % 512 == 0
                if r < world - 1:
                    assert b % 512 == 0
            sizes = [b - a for a, b in ranges[:-1]]
            if sizes:
                assert max(sizes) - min(sizes) <= 512


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mech = synth.mechanism("h2_9sp_21rx")
    st = synth.states_flame(mech.K, 8, seed=5)             # 8 elements, 4096 points
    wbar = synth.normal((mech.K, st.n), 9)
    a, b = shard.shard_range(st.n, world, rank)
    g_local = oracle.grad_lnA(mech, st.T[a:b], st.p[a:b], np.ascontiguousarray(st.Y[:, a:b]),
                              np.ascontiguousarray(wbar[:, a:b]), threads=1)
    g = shard.reduce_in_rank_order(torch.from_numpy(g_local))
    g2 = shard.reduce_in_rank_order(torch.from_numpy(g_local))
    if rank == 0:
        out.put((g.numpy(), bool(torch.equal(g, g2))))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_lnA_gradient_matches_unsharded():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    g, deterministic = q.get()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    assert deterministic
    mech = synth.mechanism("h2_9sp_21rx")
    st = synth.states_flame(mech.K, 8, seed=5)
    wbar = synth.normal((mech.K, st.n), 9)
    g_full = oracle.grad_lnA(mech, st.T, st.p, st.Y, wbar, threads=1)
    fwd, rev = oracle.rates_of_progress(mech, st.T, st.p, st.Y)
    from conftest import nu_matrix
    scale = np.sum(np.abs(nu_matrix(mech).T @ wbar) * (fwd + rev), axis=1)
    assert np.all(np.abs(g - g_full) <= 1e-12 * scale)
