"""Seeded synthetic stereo pairs shaped like the paper's workloads.

This module holds no arithmetic of the matching method: it only draws input
images (and the ground truth used to make them).  Both the CUDA path and the
CPU oracle are fed from here, so the generator is written with integer
arithmetic wherever a platform-dependent float rounding could change a pixel:
the same seed gives the same bytes on x86_64 and aarch64.

Recipe (per pair):
  * left image: uniform integer noise, blurred by a separable integer kernel
    approximating a Gaussian with sigma = 1.5 px (taps exp(-k^2/4.5) * 1000,
    rounded), rescaled to 0..255 with integer arithmetic;
  * ground truth: P slanted planes d = a*x + b*y + c0, one per Voronoi cell of
    P random seed points, clipped to [0, L-1];
  * right image: every left pixel is forward-splatted to x - round(d) (the
    larger disparity wins), holes (occlusions) are filled with fresh blurred
    noise, optional extra occlusion blobs are painted until a minimum fraction
    of pixels is occluded, then N(0, sigma_n^2) noise is added, rounded and
    clipped to 0..255.

The paper's own inputs (KITTI-like driving stereo, Middlebury, a live 640x480
camera) are not available here; these pairs stand in for them with the same
shapes, label counts and image statistics (band-limited texture, piecewise
planar disparity, occlusions, sensor noise).

Sequences (the streaming workload): one band-limited scene texture, wider than
a frame, pans one pixel per frame; the planes drift by a small random walk;
each frame's right view is made as above with its own noise.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# exp(-k^2 / (2 * 1.5^2)) * 1000 for k = 0..4, rounded: a fixed integer kernel
_BLUR_TAPS = np.array([29, 135, 411, 801, 1000, 801, 411, 135, 29], dtype=np.int64)


@dataclass
class StereoPair:
    left: np.ndarray        # uint8 [H, W]
    right: np.ndarray       # uint8 [H, W]
    gt: np.ndarray          # float64 [H, W], ground-truth disparity of the left image
    occluded: np.ndarray    # bool [H, W], right-image pixels with no left correspondence
    seed: int


def _blur_int(img: np.ndarray) -> np.ndarray:
    """Separable integer blur with clamp-to-edge borders (int64 in, int64 out)."""
    r = len(_BLUR_TAPS) // 2
    H, W = img.shape
    pad = np.pad(img, ((0, 0), (r, r)), mode="edge")
    tmp = np.zeros((H, W), dtype=np.int64)
    for k, t in enumerate(_BLUR_TAPS):
        tmp += t * pad[:, k:k + W]
    pad = np.pad(tmp, ((r, r), (0, 0)), mode="edge")
    out = np.zeros((H, W), dtype=np.int64)
    for k, t in enumerate(_BLUR_TAPS):
        out += t * pad[k:k + H, :]
    return out


def _texture(rng: np.random.Generator, H: int, W: int) -> np.ndarray:
    """Band-limited noise rescaled to 0..255 (uint8)."""
    noise = rng.integers(0, 1 << 16, size=(H, W), dtype=np.int64)
    b = _blur_int(noise)
    lo, hi = int(b.min()), int(b.max())
    if hi == lo:
        return np.zeros((H, W), dtype=np.uint8)
    return ((b - lo) * 255 // (hi - lo)).astype(np.uint8)


def _plane_params(rng: np.random.Generator, H: int, W: int, L: int, P: int) -> dict:
    """P slanted planes: seed points, the value at each seed in [0, L-1], gentle slopes."""
    sy = rng.integers(0, H, size=P)
    sx = rng.integers(0, W, size=P)
    c_at_seed = rng.uniform(0.0, L - 1.0, size=P)
    slope = (L - 1.0) / max(W, H)
    a = rng.uniform(-0.5 * slope, 0.5 * slope, size=P)
    b = rng.uniform(-0.5 * slope, 0.5 * slope, size=P)
    return dict(sy=sy, sx=sx, c=c_at_seed, a=a, b=b)


def _render_planes(pp: dict, H: int, W: int, L: int) -> np.ndarray:
    """Piecewise-planar disparity: one slanted plane per Voronoi cell of the seeds."""
    sy, sx = pp["sy"], pp["sx"]
    yy, xx = np.mgrid[0:H, 0:W]
    best = np.full((H, W), np.iinfo(np.int64).max, dtype=np.int64)
    cell = np.zeros((H, W), dtype=np.int64)
    for p in range(len(sy)):
        d2 = (yy - sy[p]).astype(np.int64) ** 2 + (xx - sx[p]).astype(np.int64) ** 2
        closer = d2 < best
        best[closer] = d2[closer]
        cell[closer] = p
    dx = xx - sx[cell]
    dy = yy - sy[cell]
    d = pp["c"][cell] + pp["a"][cell] * dx + pp["b"][cell] * dy
    return np.clip(d, 0.0, L - 1.0)


def _planes(rng: np.random.Generator, H: int, W: int, L: int, P: int) -> np.ndarray:
    return _render_planes(_plane_params(rng, H, W, L, P), H, W, L)


def _right_image(rng: np.random.Generator, left: np.ndarray, gt: np.ndarray, noise_sigma: float,
                 min_occluded: float):
    """The right view of `left` under disparity `gt` (see the module docstring)."""
    H, W = left.shape
    d_int = np.rint(gt).astype(np.int64)
    right = np.zeros((H, W), dtype=np.int64)
    zbuf = np.full((H, W), -1, dtype=np.int64)
    ys, xs = np.mgrid[0:H, 0:W]
    xr = xs - d_int
    ok = xr >= 0
    # painter's order: ascending disparity so that the nearest surface wins
    order = np.argsort(d_int[ok], kind="stable")
    yv, xv, xrv, dv = ys[ok][order], xs[ok][order], xr[ok][order], d_int[ok][order]
    right[yv, xrv] = left[yv, xv]
    zbuf[yv, xrv] = dv
    occluded = zbuf < 0
    fill = _texture(rng, H, W)
    right[occluded] = fill[occluded]
    if min_occluded > 0.0:
        # paint occlusion blobs (discs of fresh texture) until enough is occluded
        target = int(np.ceil(min_occluded * H * W))
        rmax = max(2, min(H, W) // 20)
        while int(occluded.sum()) < target:
            cy, cx = int(rng.integers(0, H)), int(rng.integers(0, W))
            rad = int(rng.integers(2, rmax + 1))
            disc = (ys - cy) ** 2 + (xs - cx) ** 2 <= rad * rad
            fresh = _texture(rng, H, W)
            right[disc] = fresh[disc]
            occluded |= disc
    if noise_sigma > 0:
        right = right + np.rint(rng.normal(0.0, noise_sigma, size=(H, W))).astype(np.int64)
    return np.clip(right, 0, 255).astype(np.uint8), occluded


def make_pair(H: int, W: int, L: int, *, planes: int = 4, noise_sigma: float = 2.0,
              min_occluded: float = 0.0, seed: int = 0) -> StereoPair:
    """One synthetic rectified stereo pair; see the module docstring."""
    rng = np.random.default_rng(seed)
    left = _texture(rng, H, W)
    gt = _planes(rng, H, W, L, planes)
    right, occluded = _right_image(rng, left, gt, noise_sigma, min_occluded)
    return StereoPair(left=left, right=right, gt=gt, occluded=occluded, seed=seed)


def make_sequence(H: int, W: int, L: int, frames: int, *, planes: int = 12,
                  noise_sigma: float = 3.0, drift: float = 0.25, pan: int = 1, seed: int = 0):
    """A sequence of pairs: the scene texture pans `pan` pixels per frame and the
    ground-truth planes drift (a random walk of `drift` labels in each plane's
    offset and drift / max(H, W) in its slopes per frame).  Yields StereoPair."""
    rng = np.random.default_rng(seed)
    scene = _texture(rng, H, W + pan * frames)
    pp = _plane_params(rng, H, W, L, planes)
    for f in range(frames):
        if f > 0:
            P = len(pp["c"])
            pp = dict(pp, c=np.clip(pp["c"] + rng.uniform(-drift, drift, size=P), 0.0, L - 1.0),
                      a=pp["a"] + rng.uniform(-drift, drift, size=P) / max(H, W),
                      b=pp["b"] + rng.uniform(-drift, drift, size=P) / max(H, W))
        left = np.ascontiguousarray(scene[:, pan * f:pan * f + W])
        gt = _render_planes(pp, H, W, L)
        right, occluded = _right_image(np.random.default_rng((seed, f)), left, gt, noise_sigma, 0.0)
        yield StereoPair(left=left, right=right, gt=gt, occluded=occluded, seed=seed)


# ---------------------------------------------------------------------------
# The workloads (shapes, label counts and iteration counts)
# ---------------------------------------------------------------------------

#: 64x48 pair, 16 labels, 4 planes, sigma_n = 2: the small parity case
SMALL = dict(H=48, W=64, L=16, planes=4, noise_sigma=2.0, min_occluded=0.0,
             dmm_iters=5, pd_iters=50)
#: KITTI-shaped 1242x375 pair, 128 labels, 12 planes, 5% occluded, sigma_n = 3
KITTI = dict(H=375, W=1242, L=128, planes=12, noise_sigma=3.0, min_occluded=0.05,
             dmm_iters=10, pd_iters=100)
#: streaming: 60 frames of 1920x1080 with 256 labels (uint16 cost volume), drifting planes
STREAM = dict(H=1080, W=1920, L=256, planes=12, noise_sigma=3.0, frames=60, drift=0.25,
              dmm_iters=10, pd_iters=100)


def make_workload(spec: dict, seed: int = 0) -> StereoPair:
    return make_pair(spec["H"], spec["W"], spec["L"], planes=spec["planes"],
                     noise_sigma=spec["noise_sigma"], min_occluded=spec["min_occluded"],
                     seed=seed)


def batch_specs(n_pairs: int = 32, seed: int = 0) -> list[dict]:
    """Mixed-size batch: sizes uniform over {320x240, 640x480, 1242x375}, L in {32, 64, 128}."""
    rng = np.random.default_rng(seed)
    sizes = [(240, 320), (480, 640), (375, 1242)]
    labels = [32, 64, 128]
    out = []
    for k in range(n_pairs):
        H, W = sizes[int(rng.integers(0, 3))]
        L = labels[int(rng.integers(0, 3))]
        out.append(dict(H=H, W=W, L=L, planes=4, noise_sigma=2.0, min_occluded=0.0,
                        dmm_iters=5, pd_iters=50, seed=seed * 1000 + k))
    return out


@dataclass
class FlowPair:
    img1: np.ndarray        # uint8 [H, W]
    img2: np.ndarray        # uint8 [H, W]
    gt1: np.ndarray         # int64 [H, W], horizontal displacement of every img1 pixel
    gt2: np.ndarray         # int64 [H, W], vertical displacement
    seed: int


def make_flow_pair(H: int, W: int, lo1: int, K1: int, lo2: int, K2: int, *, objects: int = 6,
                   noise_sigma: float = 2.0, seed: int = 0) -> FlowPair:
    """Two frames of a moving scene: a textured background displaced by one integer
    vector and `objects` textured rectangles on top, each displaced by its own
    (later rectangles occlude earlier ones, in both frames).  Every displacement
    lies in [lo1, lo1 + K1) x [lo2, lo2 + K2); img2(y + d2, x + d1) = img1(y, x)
    wherever that pixel stays visible; uncovered img2 pixels show fresh texture
    and img2 gets N(0, noise_sigma^2) noise."""
    rng = np.random.default_rng(seed)
    M = max(abs(lo1), abs(lo1 + K1 - 1), abs(lo2), abs(lo2 + K2 - 1)) + 1
    canvas = _texture(rng, H + 2 * M, W + 2 * M)
    draw = lambda: (int(rng.integers(lo1, lo1 + K1)), int(rng.integers(lo2, lo2 + K2)))
    b1, b2 = draw()
    img1 = canvas[M:M + H, M:M + W].copy()
    ys, xs = np.mgrid[0:H, 0:W]
    img2 = canvas[np.clip(ys - b2 + M, 0, H + 2 * M - 1), np.clip(xs - b1 + M, 0, W + 2 * M - 1)]
    gt1 = np.full((H, W), b1, dtype=np.int64)
    gt2 = np.full((H, W), b2, dtype=np.int64)
    for _ in range(objects):
        h = min(H, int(rng.integers(max(4, H // 10), max(5, H // 3))))
        w = min(W, int(rng.integers(max(4, W // 10), max(5, W // 3))))
        y0 = int(rng.integers(0, max(1, H - h)))
        x0 = int(rng.integers(0, max(1, W - w)))
        f1, f2 = draw()
        patch = _texture(rng, h, w)
        img1[y0:y0 + h, x0:x0 + w] = patch
        gt1[y0:y0 + h, x0:x0 + w] = f1
        gt2[y0:y0 + h, x0:x0 + w] = f2
        ya, xa = max(0, y0 + f2), max(0, x0 + f1)
        yb, xb = min(H, y0 + f2 + h), min(W, x0 + f1 + w)
        if ya < yb and xa < xb:
            img2[ya:yb, xa:xb] = patch[ya - y0 - f2:yb - y0 - f2, xa - x0 - f1:xb - x0 - f1]
    noise = np.rint(rng.normal(0.0, noise_sigma, size=(H, W))).astype(np.int64)
    img2 = np.clip(img2.astype(np.int64) + noise, 0, 255).astype(np.uint8)
    return FlowPair(img1=img1, img2=img2, gt1=gt1, gt2=gt2, seed=seed)


# 640x480 frames (the paper's live camera size) with displacements in [-32, 32)^2
FLOW = dict(H=480, W=640, lo1=-32, K1=64, lo2=-32, K2=64, objects=6, noise_sigma=2.0,
            dmm_iters=10, pd_iters=100)


def make_flow_workload(spec: dict, seed: int = 0) -> FlowPair:
    return make_flow_pair(spec["H"], spec["W"], spec["lo1"], spec["K1"], spec["lo2"], spec["K2"],
                          objects=spec["objects"], noise_sigma=spec["noise_sigma"], seed=seed)


def random_image(H: int, W: int, seed: int) -> np.ndarray:
    """Plain uniform uint8 noise (edge-case tests)."""
    return np.random.default_rng(seed).integers(0, 256, size=(H, W), dtype=np.uint8)
