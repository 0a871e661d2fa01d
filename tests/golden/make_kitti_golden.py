"""Write tests/golden/kitti_1242x375x128.json from the CPU oracle alone.

The full 1242x375x128 frame (10 Dual MM iterations, 100 primal-dual
iterations) takes the oracle tens of minutes, too long for a test, so its
results are stored: hashes of the inputs, the cost volume and the labels, the
lower bound of every iteration, a sample of labels and of the refined
disparity, and the final continuous energy (kitti_1242x375x128.json), and, in
kitti_1242x375x128_u.npz, the whole refined disparity rounded to float32 (the
rounding error is below 1e-5 px) with its float32 spread: per pixel, the
largest move of the double-precision result when the state is perturbed by
float32-sized relative noise after every iteration (oracle.fp32_spread, eight
seeds), stored as float16 rounded up and at least 1e-5.
Run:  python tests/golden/make_kitti_golden.py
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


def round_up_f16(a, floor):
    """max(a, floor) as float16, rounded up (the stored spread never
    understates the computed one; the floor keeps the file small)"""
    a = np.maximum(a, floor)
    h = a.astype(np.float16)
    low = h.astype(np.float64) < a
    h[low] = np.nextafter(h[low], np.float16(np.inf))
    return h


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
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "kitti_1242x375x128.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    spread = O.fp32_spread(res["cost"].astype(np.float64), res["wh"], res["wv"],
                           res["labels"].astype(np.float64), spec["pd_iters"])
    np.savez_compressed(os.path.join(here, "kitti_1242x375x128_u.npz"),
                        u=res["u"].astype(np.float32), spread=round_up_f16(spread, 1e-5))
    print("wrote", path, "in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
