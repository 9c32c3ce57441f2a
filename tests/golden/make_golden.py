"""Write oracle_room_small.json: FP64 oracle outputs for a small seeded room case.

Calls only the oracle and the seeded input generator."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2202_00242_gb300 import synth  # noqa: E402


def case():
    w = synth.room_pair(seed=21, n_target=1024, n_source=1024)
    tp, _ = w.clouds.cloud(0)
    sp, _ = w.clouds.cloud(1)
    tc = oracle.knn_covariances(tp).astype(np.float32)
    sc = oracle.knn_covariances(sp).astype(np.float32)
    return tp, tc, sp, sc, w.true_poses[0], 0.5


def compute():
    tp, tc, sp, sc, T, r = case()
    vm = oracle.build_voxelmap(tp, tc, r)
    out = {"resolution": r, "num_voxels": vm.num_voxels, "counts_sum": int(vm.counts.sum())}
    for name, neighbours, pose in (("planted", 1, T), ("identity", 1, np.eye(4)),
                                   ("planted_27", 27, T)):
        lin = oracle.linearize(vm, sp, sc, pose, neighbours=neighbours)
        out[name] = {"H": lin.H.tolist(), "b": lin.b.tolist(), "err": lin.err,
                     "inliers": lin.inliers}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_room_small.json"), "w") as f:
        json.dump(compute(), f, indent=1)
