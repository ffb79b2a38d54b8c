"""Multi-process source sharding on CPU (gloo, world size 2).

Each rank owns a disjoint slice of the HP and LP source sets, computes its
per-source loops (here with the oracle on a tiny lattice), and the slices are
gathered in rank order and combined once.  The combined estimate equals the
single-process one exactly, because the per-source values and the combine's
summation order do not depend on the split.
"""
import os
import socket

import numpy as np
import pytest

from paper_1211_0126_gb300 import replicas

DIMS = (2, 2, 2, 4)
KAPPA, MU = 0.124, 0.01


def test_source_ranges_partition():
    for world in (1, 2, 3, 4):
        hp, lp = [], []
        for r in range(world):
            h, l = replicas.source_ranges(4, 10, r, world)
            hp += list(range(*h))
            lp += list(range(*l))
        assert hp == list(range(4 * world))
        assert lp == list(range(4 * world, 14 * world))
        hp, lp = [], []
        for r in range(world):
            h, l = replicas.split_ranges(5, 11, r, world)
            hp += list(range(*h))
            lp += list(range(*l))
        assert hp == list(range(5)) and lp == list(range(5, 16))
    with pytest.raises(ValueError):
        replicas.source_ranges(1, 1, 2, 2)


def _per_source(U, seed, hp_range, lp_range):
    from oracle import loops, philox, solver
    g, q = [0, 5, 8], [(0, 0, 0), (1, 0, 0)]
    corr, lp = [], []
    for j in range(*hp_range):
        eta = philox.noise(seed, j, DIMS, 4)
        s_lp = solver.solve_full(U, eta, DIMS, KAPPA, MU, 0.0, 2)[0]
        s_hp = solver.solve_full(U, eta, DIMS, KAPPA, MU, 1e-12, 3000)[0]
        corr.append(loops.local_loops(eta, s_hp - s_lp, DIMS, g, q))
    for j in range(*lp_range):
        eta = philox.noise(seed, j, DIMS, 4)
        s_lp = solver.solve_full(U, eta, DIMS, KAPPA, MU, 0.0, 2)[0]
        lp.append(loops.local_loops(eta, s_lp, DIMS, g, q))
    shape = (0, 3, 2, DIMS[3])
    return (np.array(corr) if corr else np.zeros(shape, complex)), (np.array(lp) if lp else np.zeros(shape, complex))


def _worker(rank, world, port, U, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h, l = replicas.split_ranges(3, 6, rank, world)
        pc, pl = _per_source(U, 42, h, l)
        gc, gl = replicas.gather_per_source(pc, pl)
        out_q.put((rank, gc, gl))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_gloo_world2_gather_matches_single_process():
    import multiprocessing as mp
    from oracle import loops
    from paper_1211_0126_gb300 import synthetic as S
    U = S.gauge_field(DIMS, 0.3, 9)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, U, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pc, pl = _per_source(U, 42, (0, 3), (3, 9))
    for rank, gc, gl in results:
        assert np.array_equal(gc, pc) and np.array_equal(gl, pl), rank
    est_single, err_single = loops.tsm_combine(pc, pl)
    est_g, err_g = loops.tsm_combine(results[0][1], results[0][2])
    assert np.array_equal(est_single, est_g) and np.array_equal(err_single, err_g)
