"""The bounds-checked library (DVR_DEBUG_BOUNDS, libdvr_bounds.so): on
valid calls its checks never fire and it computes what the release library
computes (images, optical depths, tangents and cell layouts bit for bit,
gradients up to the order of atomic additions); with a site's extent lowered
below the true one (dvr_bounds_cap), in-bounds indices fail their check and
every call reports DVR_ERR_BOUNDS naming that site, with the access skipped,
and passes again once the extent is restored. No index leaves its buffer in
any of these runs: the lowered extents only make the checks stricter."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2107_12672_b300 import _abi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SITES = {_abi.DVR_SITE_VOLUME: "volume", _abi.DVR_SITE_CELLS: "cell layout", _abi.DVR_SITE_PIXEL: "pixel arrays",
         _abi.DVR_SITE_TF: "TF rows", _abi.DVR_SITE_CELL_GRADIENT: "cell-major gradient"}


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    lib = _abi.BOUNDS_LIB_PATH
    if not os.path.exists(lib):
        from paper_2107_12672_b300 import build
        lib = build.build(bounds=True)
    out = str(tmp_path_factory.mktemp("bounds") / "out.npz")
    env = dict(os.environ, DVR_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "tests.bounds_cases", out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_checked_build_matches_release_and_never_fires(checked):
    from tests import bounds_cases
    ref = bounds_cases.cases()
    assert list(checked["status_after_cases"]) == [0, 0, 0, 0, 0]
    for k, v in ref.items():
        got = checked[k]
        assert got.shape == v.shape, k
        if "grad" in k:
            scale = max(float(np.abs(v).max()), 1e-30)
            assert float(np.abs(got - v).max()) <= 1e-4 * scale, k
        else:
            assert np.array_equal(got, v), k


@pytest.mark.parametrize("site", sorted(SITES))
def test_lowered_extent_is_reported_per_site(checked, site):
    r = json.loads(str(checked["caps"]))[str(site)]
    assert r["code"] == _abi.DVR_ERR_BOUNDS, r
    assert f"first: {SITES[site]} index" in r["message"], r
    idx = int(r["message"].split(" index ")[1].split(",")[0])
    ext = int(r["message"].split("extent ")[1].split()[0])
    assert idx >= ext > 0
    assert r["status_after"][:2] == [0, 0]      # the call's own check cleared the records
    assert r["again"] == 0 and r["status_end"][:2] == [0, 0]


def test_graph_replay_is_checked_through_status(checked):
    caps = json.loads(str(checked["caps"]))
    assert caps["graph"]["equal"] and caps["graph"]["status"][:2] == [0, 0]
    st = caps["graph_capped"]["status"]
    assert st[0] == 0 and st[1] > 0 and st[2] == _abi.DVR_SITE_PIXEL and st[3] >= st[4] == 100
    assert caps["graph_capped"]["status_reset"][:2] == [0, 0]
