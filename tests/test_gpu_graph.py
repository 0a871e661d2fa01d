"""A single-pair solve captured as a CUDA graph (dm_capture / dm_replay):
every replay on new images is bit-identical to a plain solve of those images,
which the parity tests tie to the oracle."""

import numpy as np
import pytest

from paper_1601_06274_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1601_06274_gb300 import build, dm as _dm
    build.build()
    return _dm


@pytest.mark.parametrize("shape", [(40, 64, 32), (37, 71, 128), (375, 1242, 128)])
def test_replays_match_plain_solves(dm, shape):
    import torch
    H, W, L = shape
    ctx = dm.Context(H, W, L, stream=torch.cuda.Stream())
    ref = dm.Context(H, W, L)
    left = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    right = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    first = S.make_pair(H, W, L, planes=3, seed=0)
    ctx.solve(first.left, first.right, 5, 30)
    ctx.capture(left, right, 5, 30, out)
    for seed in (1, 2):
        sp = S.make_pair(H, W, L, planes=3, noise_sigma=2.0, seed=seed)
        left.copy_(torch.from_numpy(sp.left))
        right.copy_(torch.from_numpy(sp.right))
        ctx.replay()
        u = ref.solve(sp.left, sp.right, 5, 30)
        torch.cuda.synchronize()
        assert torch.equal(out, u)
        assert np.array_equal(dm.labels_u16(ctx.labels()), dm.labels_u16(ref.labels()))
    ctx.sync()


def test_capture_needs_its_own_stream(dm):
    import torch
    ctx = dm.Context(8, 16, 16)            # torch's current (legacy) stream
    t = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
    o = torch.empty((8, 16), dtype=torch.float32, device="cuda")
    if torch.cuda.current_stream().cuda_stream == 0:
        with pytest.raises(dm.DMError):
            ctx.capture(t, t, 2, 2, o)
