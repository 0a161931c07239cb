"""The image-sharded M-TIP driver run as two processes (Sec. II-C: per-node
type-1 sums, then a reduction): each process holds half of the images,
matches and merges them, the right-hand sides and Toeplitz kernels are
summed over a gloo group, and both solve the same system. The merged model,
lambda and the matches equal one process merging all images, with the
images on the device and from host buffers (the library's upload into its
device slots, then the steps with the reduction between merge and solve,
three calls so that both slots are used), and with slice-only point sets
(the merge spreading each shard's images at their matched orientations). Both processes share one GPU;
their kernels never wait on each other (the reduction runs on the host
through gloo)."""
import os
import socket
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import synth
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import datetime, os, sys
import numpy as np
sys.path.insert(0, os.environ["SPF_ROOT"])
import torch
import torch.distributed as dist
import synth
from paper_2109_05339_gb300 import MTIP
rank, world, port, out, mode = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3], sys.argv[4], sys.argv[5]
torch.cuda.set_device(0)
dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}",
                        timeout=datetime.timedelta(seconds=120))
d = np.load(os.path.join(out, "inputs.npz"))
n = d["counts"].shape[0]
lo, hi = rank * n // world, (rank + 1) * n // world
dev = torch.device("cuda", 0)
A = torch.from_numpy(d["A"]).to(dev)
q = torch.from_numpy(d["quats"]).to(dev)
ql = torch.from_numpy(d["qlab"]).to(dev)
imgs = torch.from_numpy(d["counts"][lo:hi]).to(dev)
drv = MTIP(A.shape[0], 1.0, ql.shape[0], hi - lo, q.shape[0], orient_chunk=int(d["chunk"]),
           cache_points="slices" if mode == "slices" else True,
           process_group=dist.group.WORLD, host_images="f32" if mode == "host" else None)
if mode == "host":
    # host buffers: the library's upload, then the steps with the reduction
    drv.set_orientations(q, ql)
    A_h = torch.from_numpy(d["A"]).pin_memory()
    img_h = torch.from_numpy(d["counts"][lo:hi]).pin_memory()
    for _ in range(3):
        best, x, lam = drv.iteration_host(A_h, img_h, float(d["scale"]), cg_iters=3)
    torch.cuda.synchronize()
    best, x = best.clone(), x.clone()
else:
    res, x, lam = drv.iteration(A, q, ql, imgs, float(d["scale"]), cg_iters=3)
    best = res["best"]
torch.cuda.synchronize()
drv.status()
np.savez(os.path.join(out, f"rank{rank}.npz"), best=best.cpu().numpy(), x=x.cpu().numpy(), lam=lam)
drv.close()
dist.destroy_process_group()
'''


@pytest.mark.parametrize("mode", ["device", "host", "slices"])
def test_two_image_shards_equal_one_process(mode):
    import torch
    from paper_2109_05339_gb300 import MTIP
    from oracle import slicing
    pb = synth.make_problem("c1", n_orient=80, n_img=24)
    clean = slicing.slice_model(pb.A, pb.img_quats, pb.q_lab, 1.0, method="direct")
    counts, s = pb.image_counts(clean)
    A = pb.A.astype(np.float32)
    quats = pb.quats.astype(np.float32)
    qlab = pb.q_lab.astype(np.float32)
    with tempfile.TemporaryDirectory() as tmp:
        np.savez(os.path.join(tmp, "inputs.npz"), A=A, quats=quats, qlab=qlab, counts=counts.astype(np.float32),
                 scale=np.float32(1.0 / s), chunk=32)
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        env = dict(os.environ, SPF_ROOT=ROOT)
        procs = [subprocess.Popen([sys.executable, "-c", CHILD, str(r), "2", str(port), tmp, mode], env=env)
                 for r in range(2)]
        rcs = []
        for p in procs:
            try:
                rcs.append(p.wait(timeout=600))
            except subprocess.TimeoutExpired:
                p.kill()
                rcs.append(-1)
        assert rcs == [0, 0], rcs
        parts = [np.load(os.path.join(tmp, f"rank{r}.npz")) for r in range(2)]
    # one process over all images
    dev = torch.device("cuda", 0)
    drv = MTIP(A.shape[0], 1.0, qlab.shape[0], counts.shape[0], quats.shape[0], orient_chunk=32,
               cache_points="slices" if mode == "slices" else True)
    res, x, lam = drv.iteration(torch.from_numpy(A).to(dev), torch.from_numpy(quats).to(dev),
                                torch.from_numpy(qlab).to(dev), torch.from_numpy(counts.astype(np.float32)).to(dev),
                                float(np.float32(1.0 / s)), cg_iters=3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np.concatenate([p["best"] for p in parts]), res["best"].cpu().numpy())
    for p in parts:
        assert float(p["lam"]) == lam
        assert rel_l2(p["x"], x.cpu().numpy()) < 1e-6
    assert rel_l2(parts[0]["x"], parts[1]["x"]) < 1e-7
    drv.close()
