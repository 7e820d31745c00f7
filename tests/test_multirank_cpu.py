"""Row-interval sharding across ranks, on CPU with the gloo backend
(world size 2). Every run here has one GPU, so the sharded product is not
built on the device; this checks the host logic a sharded run would use:
the paper's static partition of the row intervals by block count (section
"Parallelization"), an all-gather of x shards, disjoint row ranges whose
union is y, and the max-over-ranks timing of bench.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


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
    import bench
    import oracle
    from paper_1801_01134_gb300 import inputs

    A = inputs.rmat(12, seed=4)
    r, c = 2, 8
    B = oracle.beta_convert(A, r, c)
    from paper_1801_01134_gb300 import spc5

    bounds = spc5.partition(B.block_rowptr, world)  # the library's partition (host call)
    assert np.array_equal(bounds, oracle.partition(B.block_rowptr, world))
    # this rank's rows and its shard of x
    i0, i1 = int(bounds[rank]), int(bounds[rank + 1])
    row0, row1 = min(i0 * r, A.n), min(i1 * r, A.n)
    x_full = inputs.vec_uniform(A.m, seed=0)
    cuts = np.linspace(0, A.m, world + 1).astype(int)
    x_mine = torch.from_numpy(x_full[cuts[rank]:cuts[rank + 1]].copy())
    shards = [torch.zeros(cuts[k + 1] - cuts[k], dtype=torch.float64) for k in range(world)]
    dist.all_gather(shards, x_mine)
    x = torch.cat(shards).numpy()
    assert np.array_equal(x, x_full)
    # rows [row0, row1) from the rank's own intervals (Algorithm 1 on a slice)
    sub = oracle.Beta(row1 - row0, A.m, r, c, B.block_rowptr[i0:i1 + 1] - B.block_rowptr[i0],
                      B.block_colidx[B.block_rowptr[i0]:B.block_rowptr[i1]],
                      B.block_masks[B.block_rowptr[i0] * 2:B.block_rowptr[i1] * 2],
                      B.values[A.rowptr[row0]:A.rowptr[row1]])
    y_mine = oracle.beta_spmv(sub, x)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([y_mine.size], dtype=torch.int64))
    mx = int(max(s.item() for s in sizes))
    pad = torch.zeros(mx, dtype=torch.float64)
    pad[:y_mine.size] = torch.from_numpy(y_mine)
    parts = [torch.zeros(mx, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, pad)
    if rank == 0:
        y = np.concatenate([parts[k][: int(sizes[k].item())].numpy() for k in range(world)])
        np.save(os.path.join(out_dir, "y.npy"), y)
    # bench's max over ranks
    got = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    assert got == 1.5 * world
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_row_sharded_spmv_equals_the_full_product(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle
    from paper_1801_01134_gb300 import inputs

    A = inputs.rmat(12, seed=4)
    y = np.load(tmp_path / "y.npy")
    # same summation order per row as the plain CSR loop: identical bits
    assert np.array_equal(y, oracle.csr_spmv(A, inputs.vec_uniform(A.m, seed=0)))


def test_partition_is_block_balanced_for_many_ranks():
    import oracle
    from paper_1801_01134_gb300 import inputs

    A = inputs.stencil3d(24, 24, 24, points=27, seed=1)
    B = oracle.beta_convert(A, 4, 8)
    for world in (2, 4, 8):
        b = oracle.partition(B.block_rowptr, world)
        loads = np.diff(B.block_rowptr[b])
        assert loads.sum() == B.nblocks
        assert loads.max() - loads.min() <= np.diff(B.block_rowptr).max() + 1
