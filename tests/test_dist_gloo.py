"""World-size-2 gloo test of the sharded skyline's exchange logic on CPU.

The local skyline function is the CPU oracle here (test-side); the product
module only gathers and merges. The result must equal the oracle's skyline of
the whole set on every rank."""
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


def _worker(rank, world, port, kind, n, d, q):
    import torch.distributed as dist

    import oracle
    import skydata
    from paper_2107_09993_b300.dist import skyline_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = skydata.generate(kind, n, d, seed=5)
    bounds = np.linspace(0, n, world + 1).astype(int)
    lo, hi = bounds[rank], bounds[rank + 1]
    got = skyline_sharded(P[lo:hi], lo, oracle.skyline_sfs)
    q.put((rank, got.tolist()))
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,n,d", [("anticorrelated", 3000, 4), ("independent", 5000, 3),
                                      ("correlated", 4000, 6)])
def test_sharded_skyline_two_ranks(kind, n, d):
    import oracle
    import skydata

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, n, d, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = oracle.skyline_sfs(skydata.generate(kind, n, d, seed=5)).tolist()
    assert res[0] == want and res[1] == want
