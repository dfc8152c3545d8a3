"""World-size-2 gloo runs of the multi-rank host logic on CPU (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2505_12414_gb300 import dist as gd
    from paper_2505_12414_gb300 import synth

    w, r, lr = gd.env()
    assert (w, r, lr) == (world, rank, rank)
    # weak scaling: independent per-rank samples, the slowest rank's time
    tmax = gd.max_over_ranks(1.0 + rank)
    # event sharding of one sample: per-rank oracle sums added in rank order
    cols = synth.mass1d(5001, stream=3)
    lo, hi = gd.shard(5001, rank, world)
    nll, g, _, _ = oracle.nll_grad(oracle.MASS1D, synth.RANGES_1D, [c[lo:hi] for c in cols], synth.TRUTH_1D)
    tot = gd.sum_in_rank_order(np.concatenate([[nll], g]))
    first = synth.mass1d(4, stream=gd.sample_stream(rank))[0]
    out.put((rank, tmax, tot.tolist(), first.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(2)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2505_12414_gb300 import dist as gd
    from paper_2505_12414_gb300 import synth

    assert res[0][1] == res[1][1] == 2.0
    cols = synth.mass1d(5001, stream=3)
    nll, g, _, _ = oracle.nll_grad(oracle.MASS1D, synth.RANGES_1D, cols, synth.TRUTH_1D)
    for r in res:
        assert abs(r[2][0] - nll) <= 1e-12 * abs(nll)
        np.testing.assert_allclose(r[2][1:], g, rtol=1e-9, atol=1e-9)
    assert res[0][2] == res[1][2]  # every rank holds the same, rank-ordered sum
    assert res[0][3] != res[1][3]  # ranks draw independent samples
    assert gd.whole_job_rate(1_000_000, 2, 0.5) == 4_000_000
