"""View sharding across ranks: the partition balances uneven views, and the
gradient sum over two gloo ranks (CPU) equals the single-process gradient
of all views (the oracle supplies the per-rank gradients, so no GPU is
needed)."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2107_12672_b300 import synthetic as syn
from paper_2107_12672_b300.sharding import allreduce_gradients, scatter_camera_gradient, shard_views


def test_partition_is_complete_and_balanced():
    w = syn.workload("tomo_256x64", scale=1 / 16)
    views = w.views
    for world in (1, 2, 3, 8):
        parts = shard_views(views, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(views)))
        loads = [sum(views[i].width * views[i].height for i in p) for p in parts]
        biggest = max(v.width * v.height for v in views)
        assert max(loads) - min(loads) <= biggest


def _case():
    w = syn.workload("tomo_256x64", scale=1 / 32)
    w.views = w.views[:6]
    w.eye = w.eye[:6]
    rng = np.random.default_rng(5)
    G = [rng.normal(size=(v.width * v.height, 1)) for v in w.views]
    return w, G


def _grads(w, G, idx):
    import oracle
    gv = np.zeros(w.volumes[0].shape)
    ge = np.zeros((len(idx), 3))
    for j, k in enumerate(idx):
        g = oracle.backward(w.volumes[0], None, w.model, w.views[k], w.eye[k], w.step_voxels, G[k],
                            want=("volume", "eye"))
        gv += g["volume"]
        ge[j] = g["eye"]
    return gv, ge


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, G = _case()
        owned = shard_views(w.views, world)[rank]
        gv, ge = _grads(w, G, owned)
        grads = {"volume": [torch.from_numpy(gv)],
                 "eye": scatter_camera_gradient(torch.from_numpy(ge), owned, len(w.views))}
        allreduce_gradients(grads)
        if rank == 0:
            np.save(out + "_vol.npy", grads["volume"][0].numpy())
            np.save(out + "_eye.npy", grads["eye"].numpy())
    finally:
        dist.destroy_process_group()


def test_gradient_sum_over_two_gloo_ranks(tmp_path):
    port = 29500 + (os.getpid() % 1000)
    out = str(tmp_path / "g")
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    w, G = _case()
    gv, ge = _grads(w, G, list(range(len(w.views))))
    np.testing.assert_allclose(np.load(out + "_vol.npy"), gv, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.load(out + "_eye.npy"), ge, rtol=1e-12, atol=1e-14)
