"""The N > 1 sharding of bench.py, run as two gloo ranks on CPU.

Each rank owns a consecutive range of global chain ids (bench.shard_base) and
runs its chains; because every random number is keyed by the global chain id,
the union of the ranks' chains equals one process running all of them, and
the reported time is the max over ranks.  The chains here are the oracle's
(no GPU on this path); the CUDA library follows the same keying.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

C_PER_RANK, STEPS = 4, 3


def _setup():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from helpers import oracle_setup, variant
    from workloads import BASIS_DIS, CONFIGS
    w = variant(CONFIGS["small_fp64"], n_grid=5, r=3, widths=[3, 8, 4],
                basis_kind=BASIS_DIS, noise_frac=0.2)
    return w, oracle_setup(w)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle.chains import OracleChains
    w, (sur, E, D) = _setup()
    base = bench.shard_base(rank, C_PER_RANK)
    ids = np.arange(base, base + C_PER_RANK)
    och = OracleChains(sur, E, D, w.n_grid, w.prior_gamma, w.prior_delta, C_PER_RANK, 0.01,
                       seed=77, chain_ids=ids, noise="cholesky")
    och.step(STEPS)
    mine = torch.tensor(och.m_r)
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((torch.cat(gathered).numpy(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_one_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    m_r, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from oracle.chains import OracleChains
    w, (sur, E, D) = _setup()
    ref = OracleChains(sur, E, D, w.n_grid, w.prior_gamma, w.prior_delta, world * C_PER_RANK,
                       0.01, seed=77, noise="cholesky")
    ref.step(STEPS)
    assert np.allclose(m_r, ref.m_r, rtol=0, atol=1e-12)
    assert tmax == float(world)

