"""The multi-rank host path on CPU: world_size-2 gloo ranks shard a ragged batch of
instances by work, each steps its shard (FP64 oracle standing in for the GPU),
and the gathered result equals the single-process result; the step time is
reduced with MAX over ranks as the bench does."""
import os
import socket

import numpy as np
import pytest

from paper_2206_02607_gb300.shard import partition_by_work, shard_of


def test_partition_covers_every_instance_once_and_balances_work():
    rng = np.random.default_rng(0)
    sizes = rng.integers(32, 513, size=1000)
    for world in (1, 2, 3, 8):
        parts = partition_by_work(sizes, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(sizes)
        assert all(parts[k][1] == parts[k + 1][0] for k in range(world - 1))
        work = [sizes[a:b].sum() for a, b in parts]
        assert max(work) - min(work) <= 2 * sizes.max()
    assert partition_by_work([5, 5], 4)[-1] == (2, 2)   # more ranks than instances: empty ranges


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import crom_oracle as O
    from workloads import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = gen.heat2d_batched(n_inst=10, m_lo=8, m_hi=40)
    lo, hi, local = shard_of(w.s_off, rank, world)
    dec = O.MLPDecoder(w.params, 2)
    samples = w.samples[w.s_off[lo]:w.s_off[hi]]
    q, st = O.crom_step_batched(dec, w.q0[lo:hi], local, samples, w.alpha[lo:hi], w.dt, w.gn_iters)
    # gather the shards (sizes differ): pad to the largest shard
    n_max = 10
    buf = torch.zeros((n_max, w.spec.r + 1), dtype=torch.float64)
    buf[:hi - lo, :w.spec.r] = torch.tensor(q)
    buf[:hi - lo, w.spec.r] = torch.tensor(st, dtype=torch.float64)
    gathered = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(gathered, buf)
    bounds = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(bounds, torch.tensor([lo, hi]))
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q_all = np.zeros((w.n_inst, w.spec.r))
        for g, b in zip(gathered, bounds):
            a, z = int(b[0]), int(b[1])
            q_all[a:z] = g[:z - a, :w.spec.r].numpy()
        np.save(os.path.join(out_dir, "q_all.npy"), q_all)
        np.save(os.path.join(out_dir, "tmax.npy"), t.numpy())
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather(tmp_path):
    import torch.multiprocessing as mp
    from oracle import crom_oracle as O
    from workloads import gen
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    q_all = np.load(tmp_path / "q_all.npy")
    w = gen.heat2d_batched(n_inst=10, m_lo=8, m_hi=40)
    ref, _ = O.crom_step_batched(O.MLPDecoder(w.params, 2), w.q0, w.s_off, w.samples, w.alpha, w.dt, w.gn_iters)
    np.testing.assert_array_equal(q_all, ref)
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0
