"""Memory safety of the packed Dual MM kernels, lane groups and one warp per
chain (compute-sanitizer is not available): the checked build (libdm_checked.so, -DDM_CHECKED) verifies every
node, edge and message position before each global access and reports a
position outside its chain through the device error word.  Ragged, tiny and
large-label shapes, uint8 and uint16 costs, the batched kernel: no index
check may fire, and the results stay bit-exact against the oracle."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, ".")
from oracle import oracle as O
from paper_1601_06274_gb300 import build, dm, synthetic as S
assert dm.LIB_PATH.endswith("libdm_checked.so")
build.build(checked=True)

def passes(ctx, cost, wh, wv, iters):
    lam_v = np.zeros(cost.shape, dtype=np.int64)
    for it in range(iters):
        for which in (0, 1):
            ctx.discrete_pass(which)
            ref = O.dmm_pass(cost, wh, wv, which, lam_v if which == 0 else lam_h)
            lh, lv = ctx.duals()
            got = (lh if which == 0 else lv).cpu().numpy().astype(np.int64)
            assert np.array_equal(got, ref), (cost.shape, it, which)
            if which == 0:
                lam_h = ref
            else:
                lam_v = ref
    ctx.sync()   # raises if an index check fired

for (H, W, L) in [(1, 37, 16), (23, 1, 16), (2, 3, 16), (5, 6, 32), (13, 29, 48), (9, 21, 64),
                  (7, 19, 128), (4, 9, 256), (3, 1000, 16), (600, 2, 32), (5, 777, 128), (300, 3, 256)]:
    for cb, path in ((1, 0), (2, 0), (1, 2), (2, 2), (1, 3)):
        sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=H * W + L)
        ctx = dm.Context(H, W, L, dm.default_params(cost_bytes=cb, dmm_path=path))
        ctx.cost_volume(sp.left, sp.right)
        assert ctx.path()[0] == (16 if path == 2 else 8)
        cost = O.cost_volume(sp.left, sp.right, L)
        wh, wv = O.edge_weights(sp.left)
        passes(ctx, cost, wh, wv, 2)
        ctx.reset_duals()
        lb = ctx.discrete(3, lower_bounds=True)
        rl, rlb, _, _ = O.dmm(cost, wh, wv, 3)
        assert np.array_equal(lb, rlb) and np.array_equal(dm.labels_u16(ctx.labels()), rl)

shapes = [(24, 32, 32), (40, 48, 64), (30, 70, 128), (1, 50, 32), (45, 1, 64)]
pairs = [S.make_pair(H, W, L, planes=3, seed=k) for k, (H, W, L) in enumerate(shapes)]
b = dm.Batch(shapes)
b.solve([p.left for p in pairs], [p.right for p in pairs], 3, 10)
b.sync()
for k, ((H, W, L), sp) in enumerate(zip(shapes, pairs)):
    cost = O.cost_volume(sp.left, sp.right, L)
    wh, wv = O.edge_weights(sp.left)
    rl, rlb, _, _ = O.dmm(cost, wh, wv, 3)
    assert np.array_equal(dm.labels_u16(b.pairs[k].labels()), rl)
print("checked ok")
'''


def test_checked_build_no_index_out_of_range_and_bit_exact():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    env = dict(os.environ, DM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:] + r.stderr[-4000:])
