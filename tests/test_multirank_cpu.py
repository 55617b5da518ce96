"""The multi-rank path on CPU ranks (gloo, world size 2): slicing the starts
over ranks and gathering the matches reproduces the single-rank match set,
and the job timing takes the slowest rank. The CPU oracle stands in for each
rank's scanner (its start-window form is exactly a rank's share of the work)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    import workloads as W
    from paper_1110_1716_gb300 import shard
    res = {}
    for name, (aut, text) in {
        "dfa": W.workload_dna_dfa(1, n=40_000),
        "nfa": W.workload_motif_nfa(2, n=40_000, n_motifs=40, every=500)[:2],
    }.items():
        lo, hi = shard.start_slice(len(text), rank, world)
        mine = oracle.scan(aut, text, lo, hi)
        allm = shard.gather_matches(mine)
        res[name] = oracle.sort_matches(allm)
    step = shard.max_over_ranks(1.0 + rank)
    thr = shard.job_throughput(1000, world, step)
    np.savez(os.path.join(out_dir, "r%d.npz" % rank), dfa=res["dfa"], nfa=res["nfa"],
             step=step, thr=thr)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_single_rank(tmp_path):
    import oracle
    import workloads as W
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    d, t = W.workload_dna_dfa(1, n=40_000)
    n, t2 = W.workload_motif_nfa(2, n=40_000, n_motifs=40, every=500)[:2]
    want = {"dfa": oracle.scan(d, t), "nfa": oracle.scan(n, t2)}
    for r in range(world):
        z = np.load(tmp_path / ("r%d.npz" % r))
        for k in ("dfa", "nfa"):
            assert np.array_equal(z[k], want[k]), (r, k)
        assert float(z["step"]) == 2.0                  # the slowest rank
        assert float(z["thr"]) == 1000 * world / 2.0


def test_start_slices_cover_every_position_once():
    from paper_1110_1716_gb300 import shard
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            cover = []
            for r in range(world):
                lo, hi = shard.start_slice(n, r, world)
                cover.extend(range(lo, hi)) if n < 5000 else None
                assert 0 <= lo <= hi <= n
            if n < 5000:
                assert cover == list(range(n))
