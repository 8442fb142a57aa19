"""The named synthetic workloads match the configurations they stand for:
volume size and storage type, TF rows and storage, model, views, step and
the gradients asked for. The bench and the full-size GPU tests build their
inputs from these descriptions, so a drift here (a 16-bit workload built in
binary32, a wrong view count) would mislabel every number measured on it.
CPU only; the large volumes are not generated (the noise generator is
replaced by a stub that records the size it was asked for).
"""
import math

import numpy as np
import pytest

from paper_2107_12672_b300 import synthetic as syn


@pytest.fixture
def sizes(monkeypatch):
    """Record the edge lengths the generators are called with and return
    tiny arrays instead of the full volumes."""
    seen = []

    def fake(n, *a, **k):
        seen.append(n)
        return np.zeros((2, 2, 2), np.float32)

    monkeypatch.setattr(syn, "value_noise", fake)
    monkeypatch.setattr(syn, "gaussian_blobs", fake)
    return seen


# name: (n, volume dtype, R, TF dtype, model, views, view edges, step, grads)
SPEC = {
    "absorption_64": (64, "float32", 0, "float32", "absorption", 1, {64}, 0.5, ("volume",)),
    "ea_256": (256, "float32", 16, "float32", "emission_absorption", 1, {512}, 0.5, ("tf", "camera")),
    "tomo_256x64": (256, "float32", 0, "float32", "absorption", 64, {128, 256, 512, 1024}, 0.5, ("volume",)),
    "ea_bf16_512": (512, "bfloat16", 64, "float16", "emission_absorption", 16, {1024}, 0.25,
                    ("volume", "tf", "camera")),
    "ea_fp16_1024": (1024, "float16", 32, "float32", "emission_absorption", 32, {2048}, 0.25,
                     ("volume", "tf", "camera")),
    "color_256": (256, "float32", 0, "float32", "color", 8, {512}, 0.5, ("volume", "camera")),
}


@pytest.mark.parametrize("name", syn.WORKLOADS)
def test_workload_matches_its_configuration(name, sizes):
    n, vdt, R, tdt, model, nviews, edges, step, grads = SPEC[name]
    w = syn.workload(name)
    assert w.volume_dtype == vdt and w.tf_dtype == tdt
    assert w.model == model
    assert w.step_voxels == step
    assert tuple(w.grads) == grads
    assert len(w.views) == nviews and len(w.eye) == nviews
    assert {v.width for v in w.views} <= edges and all(v.width == v.height for v in w.views)
    if name == "tomo_256x64":
        assert {v.width for v in w.views} == edges     # the seeded draw uses every size
    if R:
        assert w.tf.shape == (R, 4)
        assert 0.0 <= w.tf[:, 3].min() and w.tf[:, 3].max() <= 50.0
    else:
        assert w.tf is None
    if name == "ea_fp16_1024":
        assert w.target["n"] == n and not sizes      # formed on the device by the caller
    else:
        assert sizes[0] == n
    # perspective views at distance 2.5 with a 45 degree field of view,
    # except the orthographic +z view of the 64^3 absorption case
    if name == "absorption_64":
        assert w.views[0].ortho
    else:
        assert not any(v.ortho for v in w.views)
        assert all(math.isclose(v.tan_half_fov_y, math.tan(math.radians(22.5))) for v in w.views)
        eyes = w.eye if w.orbit is None else None
        if eyes is not None:
            assert np.allclose(np.linalg.norm(eyes, axis=1), 2.5, rtol=1e-6)
        else:
            assert np.allclose(w.orbit[:, 2], 2.5)
