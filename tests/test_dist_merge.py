"""Image-sharded merge over two processes (gloo on the CPU): each rank merges
its own images, the driver's reduction helper adds the right-hand sides and
Toeplitz kernels over the ranks, and the result equals the merge of all
images (linearity of the type-1 sums, Sec. II-C); the global image count
that scales lambda is the sum of the local counts."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import merge, rotation

WORLD = 2


def _shard(rank):
    pb = synth.make_problem("c1", n_orient=20, n_img=6)
    rng = np.random.default_rng(40)
    quats = pb.quats[rng.integers(0, pb.quats.shape[0], 6)]
    images = rng.poisson(20.0, (6, pb.q_lab.shape[0])).astype(np.float64)
    D = (rng.uniform(size=pb.q_lab.shape[0]) > 0.1).astype(np.float64)
    sel = np.arange(6) % WORLD == rank if rank is not None else np.ones(6, bool)
    N = pb.cfg.N
    t = rotation.nufft_points(quats[sel], pb.q_lab, N, 1.0).reshape(-1, 3)
    Dall = np.tile(D, int(sel.sum()))
    rhs = merge.rhs(images[sel].reshape(-1), t, Dall, N)
    khat = merge.kernel_hat(merge.toeplitz_kernel(t, Dall, N), N)
    return np.ascontiguousarray(rhs), np.ascontiguousarray(khat), int(sel.sum())


def _worker(rank, port, out):
    import torch
    import torch.distributed as dist
    from paper_2109_05339_gb300.dist import allreduce_sum_, global_count
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        rhs, khat, n = _shard(rank)
        t_rhs, t_khat = torch.from_numpy(rhs), torch.from_numpy(khat)
        allreduce_sum_([t_rhs, t_khat])
        total = global_count(n, "cpu")
        if rank == 0:
            np.save(os.path.join(out, "rhs.npy"), t_rhs.numpy())
            np.save(os.path.join(out, "khat.npy"), t_khat.numpy())
            np.save(os.path.join(out, "n.npy"), np.array([total]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_merge_equals_whole(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    rhs, khat, n = _shard(None)
    np.testing.assert_allclose(np.load(tmp_path / "rhs.npy"), rhs, rtol=1e-10, atol=1e-12 * np.abs(rhs).max())
    np.testing.assert_allclose(np.load(tmp_path / "khat.npy"), khat, rtol=1e-10,
                               atol=1e-12 * np.abs(khat).max())
    assert int(np.load(tmp_path / "n.npy")[0]) == n == 6


def test_reduction_helper_rejects_strided_tensors():
    import torch
    from paper_2109_05339_gb300.dist import allreduce_sum_
    with pytest.raises(ValueError):
        allreduce_sum_([torch.zeros(4, 4).t()])
