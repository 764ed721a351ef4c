"""The benchmark's multi-process path on the host: two gloo ranks (no GPU).

bench.py runs one replica per GPU (independent problems, no data-path
collective) and reports the whole job: the units all ranks processed over the
slowest rank's time.  These tests run its gather and that aggregate as two
processes on 127.0.0.1 with the gloo backend, and check that every replica
draws its own inputs.
"""
import multiprocessing as mp
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


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, _, w = bench.dist_env()
        # rank r processed 10 (r + 1) units in 2 + r seconds, and 5 more end to end in 1 + r
        rows = bench.gather_rows([10.0 * (r + 1), 2.0 + r, 5.0, 1.0 + r], w)
        q.put((r, rows.tolist(), bench.weak_rate(rows, 0, 1), bench.weak_rate(rows, 2, 3)))
    finally:
        dist.destroy_process_group()


def _run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_gather_and_weak_rate_two_ranks():
    out = _run(2)
    want_rows = [[10.0, 2.0, 5.0, 1.0], [20.0, 3.0, 5.0, 2.0]]
    for r, rows, value, e2e in out:
        assert rows == want_rows                  # every rank sees all rows, in rank order
        assert value == pytest.approx(30.0 / 3.0)  # units of both ranks / slowest rank
        assert e2e == pytest.approx(10.0 / 2.0)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rows = bench.gather_rows([4.0, 2.0], 1)
    assert rows.shape == (1, 2) and bench.weak_rate(rows, 0, 1) == 2.0


def test_replicas_draw_their_own_inputs():
    sys.path.insert(0, ROOT)
    import synth
    pn = synth.panel(300, 2000, 11)
    y0, c0, _ = synth.config_phenotype(2, pn, which=0)
    y1, c1, _ = synth.config_phenotype(2, pn, which=1)
    assert not np.array_equal(c0, c1) and not np.allclose(y0, y1)


def test_replay_metrics_hand_example():
    """Sec. 3.1 diagnostics on a worked example: support {1,2,3,4} against causal
    {2,4,9}: precision 2/4, recall 2/3; h^2 = var(signal) / var(y) with
    signal (1,2,3) and y (2,4,6): (2/3) / (8/3) = 1/4."""
    import bench
    prec, rec, h2 = bench.replay_metrics(np.array([1, 2, 3, 4]), [2, 4, 9],
                                         np.array([1.0, 2.0, 3.0]), np.array([2.0, 4.0, 6.0]))
    assert prec == 0.5 and rec == 2 / 3 and abs(h2 - 0.25) < 1e-15
    assert bench.replay_metrics([5], [5], np.ones(3) * 2, np.array([1.0, 2.0, 4.0]))[:2] == (1.0, 1.0)
