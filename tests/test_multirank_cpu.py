"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2, 127.0.0.1):
each rank takes its own view of the weak-scaling workload (its own scene
seed and view id, hence its own STF draws), the step time is the slowest
rank's, and the whole-job value counts every rank's pixels.  The per-rank
filtering here is the CPU oracle; on GPUs it is the library's kernel."""
import os
import socket
import sys
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    dist.init_process_group("gloo", init_method="env://")
    try:
        w, r, _ = bench.dist_setup()
        sc, blocks, Wt, Ht, _ = bench.workload("plane128", r)
        t0 = time.perf_counter()
        out, ev, st = oracle.filter_frame(blocks, Wt, Ht, sc.uv, sc.jac, sc.coverage, view=r, alg=oracle.ALG_MASK,
                                          seed=0, mask_dim=11)
        if r == 1:
            time.sleep(0.2)  # the slower rank sets the step time
        ms = (time.perf_counter() - t0) * 1e3
        m = bench.max_over_ranks(ms, torch.device("cpu"))
        value = bench.weak_scaling_value(w, sc.W * sc.H, m)
        dist.barrier()
        q.put((r, w, ms, m, value, sc.W * sc.H, float(np.abs(sc.uv).sum()), int(ev.sum()), st["pixels_active"]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_filter_their_own_views_and_report_the_slowest():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, w0, ms0, m0, v0, n0, uv0, ev0, act0), (_, w1, ms1, m1, v1, n1, uv1, ev1, act1) = res[0], res[1]
    assert w0 == w1 == 2
    assert ms1 > ms0 + 150  # rank 1 was slowed down
    assert m0 == m1 == max(ms0, ms1)  # every rank sees the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * n0 / (m0 * 1e-3))  # both ranks' pixels over that time
    assert n0 == n1 and act0 > 0 and act1 > 0
    assert uv0 != uv1  # each rank filters its own view
