"""Voxel-grid downsampling with timestamp averaging (Sec. III-C) against the
oracle: output order, counts, mean positions and mean times bit-exact.

The input imitates one rotating scan that sweeps slightly more than a full
turn, so the first and last points of the scan share voxels; their times differ
by about the scan duration and the split (a tenth of it) separates them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_00242_gb300 import api

from test_gpu_parity import cu, dev  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _sweep(n, seed, d_scan=0.1, turns=1.08):
    rng = np.random.default_rng(seed)
    th = 2 * np.pi * turns * np.arange(n) / n
    r = 6.0 + 0.02 * rng.normal(size=n)
    pts = np.column_stack([r * np.cos(th), r * np.sin(th), rng.uniform(-1.0, 2.0, n)])
    t = d_scan * np.arange(n) / n
    return pts.astype(np.float32), t.astype(np.float32)


@pytest.mark.parametrize("n,res", [(20000, 0.25), (5003, 0.5)])
def test_sweep_split_matches_oracle(dev, n, res):  # noqa: F811
    pts, t = _sweep(n, seed=n)
    split = 0.1 / 10
    gp, gt, gc, oo = api.downsample(cu(pts), res, times=cu(t), split=split)
    rp, rt, rc = oracle.downsample(pts, t, res, split)
    assert oo[-1] == len(rc)
    assert np.array_equal(gc.cpu().numpy(), rc)
    assert np.array_equal(gp.cpu().numpy(), rp)
    assert np.array_equal(gt.cpu().numpy(), rt)
    _, _, rc0 = oracle.downsample(pts, None, res)
    assert len(rc) > len(rc0)  # the split separated the two ends of the sweep


def test_batched_clouds_and_no_times(dev):  # noqa: F811
    clouds = [_sweep(n, seed=s) for n, s in ((3000, 1), (0, 2), (4500, 3), (7, 4))]
    pts = np.concatenate([c[0] for c in clouds])
    t = np.concatenate([c[1] for c in clouds])
    offs = np.concatenate([[0], np.cumsum([len(c[0]) for c in clouds])])
    gp, gt, gc, oo = api.downsample(cu(pts), 0.3, times=cu(t), split=0.01, offsets=offs)
    gp, gt, gc = gp.cpu().numpy(), gt.cpu().numpy(), gc.cpu().numpy()
    for k, (p, tt) in enumerate(clouds):
        rp, rt, rc = oracle.downsample(p, tt, 0.3, 0.01)
        a, b = oo[k], oo[k + 1]
        assert b - a == len(rc)
        assert np.array_equal(gp[a:b], rp) and np.array_equal(gt[a:b], rt)
        assert np.array_equal(gc[a:b], rc)
    # without timestamps: the voxel means of the voxel map, in its order
    hp, ht, hc, _ = api.downsample(cu(clouds[0][0]), 0.3)
    rp, _, rc = oracle.downsample(clouds[0][0], None, 0.3)
    assert ht is None
    assert np.array_equal(hp.cpu().numpy(), rp) and np.array_equal(hc.cpu().numpy(), rc)
