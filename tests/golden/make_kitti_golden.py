"""Write tests/golden/kitti_1242x375x128.json from the CPU oracle alone.

The full 1242x375x128 frame (10 Dual MM iterations, 100 primal-dual
iterations) takes the oracle tens of minutes, too long for a test, so its
results are stored: hashes of the inputs, the cost volume and the labels, the
lower bound of every iteration, a sample of labels and of the refined
disparity, and the final continuous energy.  Run:  python tests/golden/make_kitti_golden.py
"""

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1601_06274_gb300 import synthetic as S  # noqa: E402


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    spec = S.KITTI
    sp = S.make_workload(spec, seed=0)
    H, W, L = spec["H"], spec["W"], spec["L"]
    t0 = time.time()
    res = O.solve(sp.left, sp.right, L, spec["dmm_iters"], spec["pd_iters"],
                  nthreads=os.cpu_count())
    rng = np.random.default_rng(2024)
    ys = rng.integers(0, H, size=4096)
    xs = rng.integers(0, W, size=4096)
    out = {
        "workload": "kitti-1242x375x128", "seed": 0, "H": H, "W": W, "L": L,
        "dmm_iters": spec["dmm_iters"], "pd_iters": spec["pd_iters"],
        "left_sha256": sha(sp.left), "right_sha256": sha(sp.right),
        "cost_sha256": sha(res["cost"].astype(np.uint8)),
        "labels_sha256": sha(res["labels"].astype(np.uint16)),
        "lower_bounds": [int(v) for v in res["lb"]],
        "sample_y": ys.tolist(), "sample_x": xs.tolist(),
        "sample_labels": res["labels"][ys, xs].astype(int).tolist(),
        "sample_u": [float(v) for v in res["u"][ys, xs]],
        "energy": float(res["energy"][-1]),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kitti_1242x375x128.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print("wrote", path, "in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
