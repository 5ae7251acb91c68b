"""The multi-GPU path on CPU: two gloo ranks, each running the FP64 oracle on
its shard of history ids [r n, (r+1) n) -- the sharding bench.py and
mc_set_history_base use -- then summing the sub-tallies with an all-reduce.
The merged tally must equal one run of 2n histories up to FP64 summation
order (histories are independent and keyed by id; a history's batch is its
id mod B), and the timing reduction must take the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2510_24154_b300 import workloads as W
    p = W.config_water_open(n_histories=n, npx=32, npy=32, pitch=1.2, coupled=True)
    r = oracle.run(p, n_histories=n, hist_begin=rank * n, threads=2)
    q = torch.tensor(r["tally"], dtype=torch.float64)
    dist.all_reduce(q, op=dist.ReduceOp.SUM)
    t = torch.tensor([0.5 + rank])                 # per-rank "time"
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(os.path.join(out_dir, "merged.npy"), q.numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_history_shards_merge_to_one_run(tmp_path):
    import oracle
    from paper_2510_24154_b300 import workloads as W
    oracle.build()
    n = 6000
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, str(tmp_path))) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    merged = np.load(tmp_path / "merged.npy")
    p = W.config_water_open(n_histories=2 * n, npx=32, npy=32, pitch=1.2, coupled=True)
    whole = oracle.run(p, n_histories=2 * n, threads=2)
    want = whole["tally"]
    assert merged.sum() > 0
    # the same per-history deposits, summed in another order (FP64)
    assert np.allclose(merged, want, rtol=1e-12, atol=1e-15 * want.max())
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 1.5
