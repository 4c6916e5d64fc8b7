"""The sharded multisplit across ranks, on CPU with gloo (world size 2).

The method splits by its own first level (Section 4.3, Eq. 2): rank r owns a
contiguous slice of the input, multisplits it locally and contributes one
column of the m x P histogram matrix.  After an all-gather of that matrix,
every rank knows where each of its bucket runs goes in the global output:
  start(r, b) = sum_{b' < b} total(b') + sum_{r' < r} h(r', b).
The runs are then exchanged (here with point-to-point send/recv) and each rank
writes its share of the output.  The concatenation of the ranks' shares must
equal the single-process multisplit of the whole input.  This checks the
exchange arithmetic of the multi-GPU design on the host; the GPU runs of this
repository use one GPU (replicas only).
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synthetic

N = 20011
M = 13
WORLD = 2


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    keys = synthetic.uniform_u32(N, 77)
    vals = synthetic.index_values(N)
    spec = oracle.Spec(oracle.MOD, M)
    bounds = [N * r // world for r in range(world + 1)]
    lo, hi = bounds[rank], bounds[rank + 1]
    ko, vo, off = oracle.multisplit(keys[lo:hi], vals[lo:hi], spec)  # the local multisplit
    h_local = torch.from_numpy(np.diff(off.astype(np.int64)))
    H = [torch.zeros(M, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(H, h_local)  # the m x P histogram matrix
    H = torch.stack(H, dim=1).numpy()  # [bucket, rank]
    totals = H.sum(axis=1)
    bucket_start = np.concatenate([[0], np.cumsum(totals)[:-1]])
    # global position of this rank's run of bucket b (Eq. 2: earlier buckets + earlier ranks)
    run_start = bucket_start + H[:, :rank].sum(axis=1)
    # output share of rank r: global positions [bounds[r], bounds[r+1])
    local_pos = np.concatenate([run_start[b] + np.arange(H[b, rank]) for b in range(M)])
    sends = {}
    for r in range(world):
        sel = (local_pos >= bounds[r]) & (local_pos < bounds[r + 1])
        sends[r] = (local_pos[sel], ko[sel], vo[sel])
    share_k = np.zeros(bounds[rank + 1] - bounds[rank], np.uint32)
    share_v = np.zeros_like(share_k)
    for r in range(world):
        if r == rank:
            pos, k, v = sends[r]
            share_k[pos - bounds[rank]] = k
            share_v[pos - bounds[rank]] = v
    for step in range(1, world):  # ring exchange of the runs
        to, frm = (rank + step) % world, (rank - step) % world
        pos, k, v = sends[to]
        cnt = torch.tensor([len(pos)], dtype=torch.int64)
        rcnt = torch.zeros(1, dtype=torch.int64)
        reqs = [dist.isend(cnt, to), dist.irecv(rcnt, frm)]
        for q in reqs:
            q.wait()
        payload = torch.from_numpy(np.stack([pos.astype(np.int64), k.astype(np.int64), v.astype(np.int64)]))
        incoming = torch.zeros((3, int(rcnt.item())), dtype=torch.int64)
        reqs = [dist.isend(payload.contiguous(), to), dist.irecv(incoming, frm)]
        for q in reqs:
            q.wait()
        inc = incoming.numpy()
        share_k[inc[0] - bounds[rank]] = inc[1].astype(np.uint32)
        share_v[inc[0] - bounds[rank]] = inc[2].astype(np.uint32)
    np.save(f"{result_path}_{rank}_k.npy", share_k)
    np.save(f"{result_path}_{rank}_v.npy", share_v)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_sharded_multisplit_equals_single(tmp_path):
    port = 29500 + (os.getpid() % 2000)
    path = str(tmp_path / "share")
    mp.start_processes(_worker, args=(WORLD, port, path), nprocs=WORLD, start_method="spawn")
    k = np.concatenate([np.load(f"{path}_{r}_k.npy") for r in range(WORLD)])
    v = np.concatenate([np.load(f"{path}_{r}_v.npy") for r in range(WORLD)])
    keys = synthetic.uniform_u32(N, 77)
    ek, ev, _ = oracle.multisplit(keys, synthetic.index_values(N), oracle.Spec(oracle.MOD, M))
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)
