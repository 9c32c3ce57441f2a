"""The oracle still reproduces its stored regression fixture (written by
tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_fixture(oracle_lib):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden",
                                                  os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "golden", "oracle_room_small.json")) as f:
        ref = json.load(f)
    now = mg.compute()
    assert now["num_voxels"] == ref["num_voxels"] and now["counts_sum"] == ref["counts_sum"]
    for name in ("planted", "identity", "planted_27"):
        a, b = now[name], ref[name]
        assert a["inliers"] == b["inliers"]
        # generator trig may differ by an ulp between hosts: tight, not bitwise
        np.testing.assert_allclose(a["H"], b["H"], rtol=1e-9, atol=1e-9 * np.abs(b["H"]).max())
        np.testing.assert_allclose(a["b"], b["b"], rtol=1e-7, atol=1e-9 * np.abs(b["H"]).max())
        np.testing.assert_allclose(a["err"], b["err"], rtol=1e-9)
