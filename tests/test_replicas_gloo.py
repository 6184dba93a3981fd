"""The multi-process (replica) path on the CPU: two gloo ranks, as ``bench.py --gpus 2``
runs them under torchrun, each with its own seeded catalogue.

Checks the host-side pieces of that path (process-group set-up from the environment,
barrier, max and sum over ranks) and that the replicas' results add up: the estimator is a
sum over centres, so catalogues (or patches) measured on different ranks combine by
summation into the result of measuring them one after the other.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _catalogue(rank):
    import synth
    pos, sh, w = synth.uniform_catalog(150, 20.0, seed=300 + rank)
    return pos, sh, np.random.default_rng(400 + rank).uniform(0.5, 1.5, len(w))


EDGES = np.geomspace(1.0, 6.0, 4)
NMAX = 2


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    w, r, _ = bench.dist_setup(False)
    pos, sh, wt = _catalogue(r)
    ups = oracle.measure(pos, sh, wt, EDGES, NMAX)
    t = torch.tensor(np.stack([ups.real, ups.imag]))
    dist.all_reduce(t)  # combine the replicas' multipoles
    mx = bench.max_over_ranks(float(r + 1), w)
    sm = bench.sum_over_ranks(float(r + 1), w)
    bench.barrier(w)
    if r == 0:
        queue.put((w, mx, sm, t.numpy()))
    dist.destroy_process_group()


def test_two_gloo_replicas(oracle):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(rank, 2, port, queue)) for rank in range(2)]
    for p in procs:
        p.start()
    try:
        world, mx, sm, combined = queue.get(timeout=180)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert world == 2 and mx == 2.0 and sm == 3.0
    serial = sum(oracle.measure(*_catalogue(r), EDGES, NMAX) for r in range(2))
    assert np.abs(serial).max() > 0
    np.testing.assert_allclose(combined[0] + 1j * combined[1], serial, rtol=1e-12,
                               atol=1e-12 * np.abs(serial).max())
