"""Full-size parity on the 1242x375x128 benchmark frame.

The CPU oracle needs minutes for this frame, so its results were stored by
tests/golden/make_kitti_golden.py (which calls only the oracle and the input
generator): input and cost-volume hashes, the lower bound after each of the
10 Dual MM iterations, the label hash, 4096 sampled labels, the final energy,
the whole refined disparity (float32) and its float32 spread.  The GPU runs the
frame through the same C ABI calls as bench.py.

The refinement's difference-of-convex iteration (Sec. 2.4) amplifies rounding
where the concave part is active: the q step adds tau A u and the u step
subtracts tau A^T(-q), a pair with growth factor above one until a prox
saturates.  On this frame the double-precision result moves by up to about two
pixels at a few hundred pixels when the state carries float32-sized relative
noise (2^-24) after every iteration, so no float32 computation determines it
there to 1e-3.  The check is therefore made at every pixel against the
oracle's own spread: |u - u_oracle| <= 1e-3 + spread, where spread is the
largest move of the oracle under that noise over eight seeds; at the pixels
with spread <= 1e-4 (more than 99 % of them) this is the plain 1e-3 bar.
"""

import hashlib
import json
import os

import numpy as np
import pytest

from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kitti_1242x375x128.json")
GOLDEN_U = os.path.join(os.path.dirname(__file__), "golden", "kitti_1242x375x128_u.npz")
U_TOL = 1e-3
E_TOL = 1e-5


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm
    build.build()
    g = json.load(open(GOLDEN))
    sp = S.make_workload(S.KITTI, seed=g["seed"])
    return dm, g, sp


def test_inputs_match_the_stored_frame(setup):
    _, g, sp = setup
    assert _sha(sp.left) == g["left_sha256"] and _sha(sp.right) == g["right_sha256"]


@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_full_frame_discrete_bit_exact(setup, path):
    dm, g, sp = setup
    H, W, L = g["H"], g["W"], g["L"]
    ctx = dm.Context(H, W, L, dm.default_params(dmm_path=path))
    ctx.cost_volume(sp.left, sp.right)
    c, _, _ = ctx.cost()
    lb = ctx.discrete(g["dmm_iters"], lower_bounds=True)
    labels = dm.labels_u16(ctx.labels())
    assert _sha(c.cpu().numpy()) == g["cost_sha256"]
    assert lb.tolist() == g["lower_bounds"]
    assert _sha(labels) == g["labels_sha256"]
    assert labels[g["sample_y"], g["sample_x"]].astype(int).tolist() == g["sample_labels"]


def test_full_frame_solve_matches_oracle(setup):
    dm, g, sp = setup
    H, W, L = g["H"], g["W"], g["L"]
    ctx = dm.Context(H, W, L)
    u = ctx.solve(sp.left, sp.right, g["dmm_iters"], g["pd_iters"]).cpu().numpy().astype(np.float64)
    e = ctx.energy()
    ref = np.array(g["sample_u"])
    assert np.abs(u[g["sample_y"], g["sample_x"]] - ref).max() <= U_TOL
    # every pixel against the oracle's whole refined disparity, within the
    # oracle's own float32 spread
    z = np.load(GOLDEN_U)
    u_ref, spread = z["u"].astype(np.float64), z["spread"].astype(np.float64)
    assert u_ref.shape == (H, W) and spread.shape == (H, W)
    err = np.abs(u - u_ref)
    assert (err - spread).max() <= U_TOL
    stable = spread <= 1e-4
    assert stable.mean() >= 0.99
    assert err[stable].max() <= U_TOL
    assert abs(e - g["energy"]) <= E_TOL * abs(g["energy"])
    # invariants that hold at any size: the refined disparity stays within the
    # warps' boxes around the labels and inside the label range
    labels = dm.labels_u16(ctx.labels()).astype(np.float64)
    assert np.all(u >= 0) and np.all(u <= L - 1)
    assert np.all(np.abs(u - labels) <= 5.0 + 1e-4)
