"""Admission scheduling (host logic, no GPU): every pair lands in exactly one
batch and every batch's working set fits the budget."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def api():
    from paper_2202_00242_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("budget_maps", [2, 3, 7, 1000])
def test_schedule_fits_budget(api, budget_maps):
    rng = np.random.default_rng(budget_maps)
    n = 40
    mb = rng.integers(10, 20, size=n) * 1000
    pairs = np.array([[j, i] for i in range(n) for j in rng.choice(n, 4, replace=False) if j != i])
    budget = int(budget_maps * 20000)
    batch, nb = api.admission_schedule(mb, pairs, budget)
    assert batch.shape[0] == pairs.shape[0] and batch.min() == 0 and batch.max() == nb - 1
    for b in range(nb):
        items = np.unique(pairs[batch == b].ravel())
        assert mb[items].sum() <= budget
    if budget_maps >= 1000:
        assert nb == 1


def test_schedule_rejects_oversized_pair(api):
    from paper_2202_00242_gb300._lib import VGICPError
    with pytest.raises(VGICPError):
        api.admission_schedule([10, 10], [[0, 1]], 15)
    assert api.voxelmap_bytes(100000) > 100000 * 36
