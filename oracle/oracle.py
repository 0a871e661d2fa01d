"""Python front end of the CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It compiles ``dm_oracle.c`` with gcc into ``_build/`` next to
this file and exposes numpy-level wrappers.  Nothing here touches the CUDA
library or the package that wraps it.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdm_oracle.so")
_lib = None

i64p = ctypes.POINTER(ctypes.c_int64)
i32p = ctypes.POINTER(ctypes.c_int32)
u32p = ctypes.POINTER(ctypes.c_uint32)
u16p = ctypes.POINTER(ctypes.c_uint16)
u8p = ctypes.POINTER(ctypes.c_uint8)
f64p = ctypes.POINTER(ctypes.c_double)
f32p = ctypes.POINTER(ctypes.c_float)


class ContParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("delta", ctypes.c_double), ("C", ctypes.c_double),
                ("lambda_r", ctypes.c_double), ("tau", ctypes.c_double),
                ("sigma", ctypes.c_double), ("h", ctypes.c_double), ("warps", ctypes.c_int)]


class FlowGeo(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("lo1", ctypes.c_int),
                ("K1", ctypes.c_int), ("lo2", ctypes.c_int), ("K2", ctypes.c_int),
                ("maxc", ctypes.c_int), ("c1", u32p), ("c2", u32p)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path: str):
    """Open a build of dm_oracle.c at `path` with every signature declared (the
    tests also load copies with planted mistakes this way)."""
    L = ctypes.CDLL(path)
    L.or_census.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int, u32p]
    L.or_cost_volume.argtypes = [ctypes.c_int] * 3 + [u32p, u32p, ctypes.c_int, i32p]
    G = ctypes.POINTER(FlowGeo)
    L.or_flow_cost_projected.argtypes = [G, i32p, i32p]
    L.or_flow_D.argtypes = [G, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.or_flow_D.restype = ctypes.c_double
    L.or_flow_fit_samples.argtypes = [f64p, ctypes.c_double, f64p, f64p]
    L.or_psd2.argtypes = [f64p]
    L.or_flow_linearise_px.argtypes = [G, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 \
        + [f64p, f64p, f64p]
    L.or_flow_prox.argtypes = [ctypes.c_double] * 4 + [f64p, f64p, f64p, ctypes.c_double,
                                                       f64p, f64p]
    L.or_flow_energy.argtypes = [G, ctypes.c_double, f64p, f64p, ctypes.POINTER(ContParams),
                                 f64p, f64p]
    L.or_flow_energy.restype = ctypes.c_double
    L.or_flow_refine.argtypes = [G, ctypes.c_double, f64p, f64p, ctypes.c_int,
                                 ctypes.POINTER(ContParams), f64p, f64p, f64p, ctypes.c_int,
                                 f64p]
    L.or_cost_volume_right.argtypes = [ctypes.c_int] * 3 + [u32p, u32p, ctypes.c_int, i32p]
    L.or_lr_check.argtypes = [ctypes.c_int, ctypes.c_int, f32p, f32p, ctypes.c_float, u8p,
                              f32p]
    L.or_edge_weights.argtypes = [ctypes.c_int, ctypes.c_int, u8p] + [ctypes.c_int] * 3 + [i32p, i32p]
    L.or_r.argtypes = [ctypes.c_double] * 4
    L.or_r.restype = ctypes.c_double
    L.or_r_ab.argtypes = [ctypes.c_double] * 3
    L.or_r_ab.restype = ctypes.c_double
    L.or_penalty_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, i64p]
    L.or_msg.argtypes = [ctypes.c_int, i64p, i64p, i64p]
    L.or_min_marginals.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
    L.or_hier_minorant.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
    L.or_naive_minorant.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
    L.or_iterative_minorant.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p] + \
        [ctypes.c_int] * 3 + [i64p]
    L.or_uniform_minorant.argtypes = [ctypes.c_int, ctypes.c_int, i64p, i64p, ctypes.c_double,
                                      ctypes.c_int, f64p]
    L.or_pmm_majorant.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p] + [ctypes.c_double] * 3
                                  + [ctypes.c_int, u16p, f64p])
    L.or_primal_mm.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p] + [ctypes.c_double] * 3
                               + [ctypes.c_int, u16p, i64p])
    L.or_dmm_pass_kind.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p]
                                   + [ctypes.c_double] * 3 + [ctypes.c_int, i64p, i64p]
                                   + [ctypes.c_int] * 5)
    L.or_dmm_kind.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p] + [ctypes.c_double] * 3
                              + [ctypes.c_int, i64p, i64p, i64p, u16p] + [ctypes.c_int] * 5)
    L.or_dmm_pass.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p] + [ctypes.c_double] * 3
                              + [ctypes.c_int, i64p, i64p, ctypes.c_int])
    L.or_dmm_outputs.argtypes = [ctypes.c_int] * 3 + [i64p, i64p, u16p]
    L.or_dmm_outputs.restype = ctypes.c_int64
    L.or_dmm.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p] + [ctypes.c_double] * 3
                         + [ctypes.c_int, i64p, i64p, i64p, u16p, ctypes.c_int])
    L.or_discrete_energy.argtypes = ([ctypes.c_int] * 3 + [i32p, i32p, i32p]
                                     + [ctypes.c_double] * 3 + [u16p])
    L.or_discrete_energy.restype = ctypes.c_int64
    L.or_interp.argtypes = [ctypes.c_int, f64p, ctypes.c_double]
    L.or_interp.restype = ctypes.c_double
    L.or_linearise_px.argtypes = [ctypes.c_int, f64p] + [ctypes.c_double] * 3 + [f64p] * 4
    L.or_prox_data.argtypes = [ctypes.c_double] * 7
    L.or_prox_data.restype = ctypes.c_double
    L.or_prox_conj.argtypes = [ctypes.c_double] * 5
    L.or_prox_conj.restype = ctypes.c_double
    L.or_conj.argtypes = [ctypes.c_double] * 4
    L.or_conj.restype = ctypes.c_double
    L.or_cont_energy.argtypes = ([ctypes.c_int] * 3 + [f64p] * 4
                                 + [ctypes.POINTER(ContParams), f64p])
    L.or_cont_energy.restype = ctypes.c_double
    L.or_refine.argtypes = ([ctypes.c_int] * 3 + [f64p] * 4 + [ctypes.c_int,
                            ctypes.POINTER(ContParams)] + [f64p] * 5 + [ctypes.c_int, f64p])
    L.or_refine_perturbed.argtypes = ([ctypes.c_int] * 3 + [f64p] * 4 + [ctypes.c_int,
                                      ctypes.POINTER(ContParams)] + [f64p] * 5
                                      + [ctypes.c_int, ctypes.c_double, ctypes.c_uint64])
    L.or_convex_gap.argtypes = ([ctypes.c_int] * 3 + [f64p] * 4
                                + [ctypes.POINTER(ContParams)] + [f64p] * 4 + [f64p, f64p])
    L.or_refine_grad.argtypes = ([ctypes.c_int] * 3 + [f64p] * 5 + [ctypes.c_int,
                                 ctypes.POINTER(ContParams)] + [f64p] * 7)
    return L


def _p(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


def _chk(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------------------
# Parameters (the readings of the paper; see the C file header)
# ---------------------------------------------------------------------------

@dataclass
class Params:
    census_win: int = 5
    edge_T: int = 16
    w_hi: int = 8
    w_lo: int = 4
    eps: float = 0.25
    delta: float = 1.0
    C: float = 2.0
    lambda_r: float = 1.0
    alpha: float = 1.0
    tau: float = 0.35
    sigma: float = 0.35
    h: float = 1.0
    warps: int = 5

    def cont(self) -> ContParams:
        return ContParams(self.eps, self.delta, self.C, self.lambda_r, self.tau, self.sigma,
                          self.h, self.warps)


# ---------------------------------------------------------------------------
# Wrappers
# ---------------------------------------------------------------------------

def census(img: np.ndarray, win: int = 5) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), dtype=np.uint32)
    _chk(lib().or_census(H, W, _p(img, u8p), win, _p(out, u32p)), "census")
    return out


def cost_volume(left: np.ndarray, right: np.ndarray, L: int, win: int = 5) -> np.ndarray:
    cl, cr = census(left, win), census(right, win)
    H, W = cl.shape
    out = np.zeros((H, W, L), dtype=np.int32)
    _chk(lib().or_cost_volume(H, W, L, _p(cl, u32p), _p(cr, u32p), win * win - 1,
                              _p(out, i32p)), "cost_volume")
    return out


def cost_volume_right(left: np.ndarray, right: np.ndarray, L: int, win: int = 5) -> np.ndarray:
    """Right-view cost volume (the right image as reference, matched l pixels to
    the right in the left image), written from its definition."""
    cl, cr = census(left, win), census(right, win)
    H, W = cl.shape
    out = np.zeros((H, W, L), dtype=np.int32)
    _chk(lib().or_cost_volume_right(H, W, L, _p(cl, u32p), _p(cr, u32p), win * win - 1,
                                    _p(out, i32p)), "cost_volume_right")
    return out


def lr_check(u_left: np.ndarray, u_right: np.ndarray, max_diff: float = 1.0):
    """Two-sided consistency check of a left-view and a right-view disparity
    (both float32 [H, W], each in its own view's coordinates); returns
    (ok uint8 [H, W], checked disparity float32 [H, W], -1 where it fails)."""
    ul = np.ascontiguousarray(u_left, dtype=np.float32)
    ur = np.ascontiguousarray(u_right, dtype=np.float32)
    assert ul.shape == ur.shape and ul.ndim == 2
    H, W = ul.shape
    ok = np.zeros((H, W), dtype=np.uint8)
    out = np.zeros((H, W), dtype=np.float32)
    _chk(lib().or_lr_check(H, W, _p(ul, f32p), _p(ur, f32p), float(max_diff), _p(ok, u8p),
                           _p(out, f32p)), "lr_check")
    return ok, out


def edge_weights(img: np.ndarray, P: Params = Params()):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    wh = np.zeros((H, W), dtype=np.int32)
    wv = np.zeros((H, W), dtype=np.int32)
    _chk(lib().or_edge_weights(H, W, _p(img, u8p), P.edge_T, P.w_hi, P.w_lo, _p(wh, i32p),
                               _p(wv, i32p)), "edge_weights")
    return wh, wv


def r(t: float, P: Params = Params()) -> float:
    return lib().or_r(float(t), P.eps, P.delta, P.C)


def penalty_table(omega: int, K: int, P: Params = Params()) -> np.ndarray:
    V = np.zeros(K, dtype=np.int64)
    _chk(lib().or_penalty_table(int(omega), P.eps, P.delta, P.C, K, _p(V, i64p)), "penalty_table")
    return V


def msg(a: np.ndarray, V: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int64)
    V = np.ascontiguousarray(V, dtype=np.int64)
    out = np.zeros_like(a)
    lib().or_msg(len(a), _p(a, i64p), _p(V, i64p), _p(out, i64p))
    return out


def min_marginals(theta: np.ndarray, V: np.ndarray) -> np.ndarray:
    """theta: [n, K]; V: [n-1, K] (table of edge k, k+1)."""
    theta = np.ascontiguousarray(theta, dtype=np.int64)
    n, K = theta.shape
    V = np.ascontiguousarray(V, dtype=np.int64).reshape(max(n - 1, 1), K) if n > 1 else np.zeros((1, K), np.int64)
    out = np.zeros_like(theta)
    lib().or_min_marginals(n, K, _p(theta, i64p), _p(V, i64p), _p(out, i64p))
    return out


def hier_minorant(theta: np.ndarray, V: np.ndarray) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.int64)
    n, K = theta.shape
    V = np.ascontiguousarray(V, dtype=np.int64).reshape(max(n - 1, 1), K) if n > 1 else np.zeros((1, K), np.int64)
    out = np.zeros_like(theta)
    lib().or_hier_minorant(n, K, _p(theta, i64p), _p(V, i64p), _p(out, i64p))
    return out


def _chain_args(theta, V):
    theta = np.ascontiguousarray(theta, dtype=np.int64)
    n, K = theta.shape
    V = np.ascontiguousarray(V, dtype=np.int64).reshape(max(n - 1, 1), K) if n > 1 else np.zeros((1, K), np.int64)
    return theta, V, n, K


def naive_minorant(theta: np.ndarray, V: np.ndarray) -> np.ndarray:
    """floor(min-marginal / n) at every node of the chain (theta [n, K], V [n-1, K])."""
    theta, V, n, K = _chain_args(theta, V)
    out = np.zeros_like(theta)
    lib().or_naive_minorant(n, K, _p(theta, i64p), _p(V, i64p), _p(out, i64p))
    return out


def iterative_minorant(theta: np.ndarray, V: np.ndarray, max_pass: int = 3,
                       gamma=(1, 4)) -> np.ndarray:
    """Alg. iterative-minorant with gamma = gamma[0] / gamma[1] (1 on the last pass)."""
    theta, V, n, K = _chain_args(theta, V)
    out = np.zeros_like(theta)
    _chk(lib().or_iterative_minorant(n, K, _p(theta, i64p), _p(V, i64p), int(max_pass),
                                     int(gamma[0]), int(gamma[1]), _p(out, i64p)),
         "iterative_minorant")
    return out


def uniform_minorant(theta: np.ndarray, V: np.ndarray, tol: float = 1e-9,
                     max_rounds: int = 10000):
    """Alg. uniform-minorant (minimum ratios by Dinkelbach's iteration), float64;
    returns (lam, rounds)."""
    theta, V, n, K = _chain_args(theta, V)
    out = np.zeros((n, K), dtype=np.float64)
    r = lib().or_uniform_minorant(n, K, _p(theta, i64p), _p(V, i64p), float(tol), int(max_rounds),
                                  _p(out, f64p))
    if r < 0:
        raise RuntimeError("oracle uniform_minorant did not converge")
    return out, r


def primal_mm(cost, wh, wv, iters: int, labels0, P: Params = Params()):
    """Alg. Primal_MM from labels0; returns (labels, energy after each iteration)."""
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    H, W, L = cost.shape
    labels = np.array(labels0, dtype=np.uint16, order="C")
    en = np.zeros(max(iters, 1), dtype=np.int64)
    _chk(lib().or_primal_mm(H, W, L, _p(cost, i32p), _p(np.ascontiguousarray(wh, np.int32), i32p),
                            _p(np.ascontiguousarray(wv, np.int32), i32p), P.eps, P.delta, P.C,
                            int(iters), _p(labels, u16p), _p(en, i64p)), "primal_mm")
    return labels, en[:iters]


def pmm_majorant(cost, wh, wv, half: int, labels, P: Params = Params()):
    """The modular majorant of Primal_MM exact at `labels` for the family `half`
    (0: data + horizontal edges, 1: vertical edges), float64 [H, W, L]."""
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    H, W, L = cost.shape
    lab = np.ascontiguousarray(labels, dtype=np.uint16)
    bar = np.zeros((H, W, L), dtype=np.float64)
    _chk(lib().or_pmm_majorant(H, W, L, _p(cost, i32p), _p(np.ascontiguousarray(wh, np.int32), i32p),
                               _p(np.ascontiguousarray(wv, np.int32), i32p), P.eps, P.delta, P.C,
                               int(half), _p(lab, u16p), _p(bar, f64p)), "pmm_majorant")
    return bar


MINORANTS = {"hier": 0, "naive": 1, "iterative": 2}


def dmm_pass(cost, wh, wv, which: int, lam_in, P: Params = Params(), nthreads: int = 0,
             minorant: str = "hier", max_pass: int = 3, gamma=(1, 4)):
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    H, W, L = cost.shape
    lam_in = np.ascontiguousarray(lam_in, dtype=np.int64)
    out = np.zeros((H, W, L), dtype=np.int64)
    _chk(lib().or_dmm_pass_kind(H, W, L, _p(cost, i32p),
                                _p(np.ascontiguousarray(wh, np.int32), i32p),
                                _p(np.ascontiguousarray(wv, np.int32), i32p), P.eps, P.delta, P.C,
                                which, _p(lam_in, i64p), _p(out, i64p), nthreads,
                                MINORANTS[minorant], int(max_pass), int(gamma[0]),
                                int(gamma[1])), "dmm_pass")
    return out


def dmm_outputs(lam_h, lam_v):
    lam_h = np.ascontiguousarray(lam_h, dtype=np.int64)
    lam_v = np.ascontiguousarray(lam_v, dtype=np.int64)
    H, W, L = lam_h.shape
    labels = np.zeros((H, W), dtype=np.uint16)
    lb = lib().or_dmm_outputs(H, W, L, _p(lam_h, i64p), _p(lam_v, i64p), _p(labels, u16p))
    return labels, int(lb)


def dmm(cost, wh, wv, iters: int, P: Params = Params(), lam_v0=None, nthreads: int = 0,
        minorant: str = "hier", max_pass: int = 3, gamma=(1, 4)):
    """Dual MM with the chosen chain minorant; returns (labels, lb per
    iteration, lam_h, lam_v)."""
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    H, W, L = cost.shape
    lam_h = np.zeros((H, W, L), dtype=np.int64)
    lam_v = np.zeros((H, W, L), dtype=np.int64) if lam_v0 is None else np.array(lam_v0, dtype=np.int64)
    lb = np.zeros(max(iters, 1), dtype=np.int64)
    labels = np.zeros((H, W), dtype=np.uint16)
    _chk(lib().or_dmm_kind(H, W, L, _p(cost, i32p), _p(np.ascontiguousarray(wh, np.int32), i32p),
                           _p(np.ascontiguousarray(wv, np.int32), i32p), P.eps, P.delta, P.C,
                           iters, _p(lam_h, i64p), _p(lam_v, i64p), _p(lb, i64p),
                           _p(labels, u16p), nthreads, MINORANTS[minorant], int(max_pass),
                           int(gamma[0]), int(gamma[1])), "dmm")
    return labels, lb[:iters], lam_h, lam_v


def discrete_energy(cost, wh, wv, labels, P: Params = Params()) -> int:
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    H, W, L = cost.shape
    labels = np.ascontiguousarray(labels, dtype=np.uint16)
    return int(lib().or_discrete_energy(H, W, L, _p(cost, i32p),
                                        _p(np.ascontiguousarray(wh, np.int32), i32p),
                                        _p(np.ascontiguousarray(wv, np.int32), i32p),
                                        P.eps, P.delta, P.C, _p(labels, u16p)))


def interp(c: np.ndarray, u: float) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return lib().or_interp(len(c), _p(c, f64p), float(u))


def linearise_px(c, alpha, u0, h):
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(4)]
    lib().or_linearise_px(len(c), _p(c, f64p), float(alpha), float(u0), float(h),
                          *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def prox_data(uh, u0, s1, s2, lo, hi, tau):
    return lib().or_prox_data(uh, u0, s1, s2, lo, hi, tau)


def prox_conj(t, omega, a, b, step):
    return lib().or_prox_conj(t, omega, a, b, step)


def conj(s, omega, a, b):
    return lib().or_conj(s, omega, a, b)


def cont_energy(cost, wh, wv, u, P: Params = Params(), alpha=None) -> float:
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    H, W, L = cost.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    al = np.ascontiguousarray(np.broadcast_to(P.alpha if alpha is None else alpha, (H, W)), np.float64)
    cp = P.cont()
    return lib().or_cont_energy(H, W, L, _p(cost, f64p), _p(al, f64p),
                                _p(np.ascontiguousarray(wh, np.float64), f64p),
                                _p(np.ascontiguousarray(wv, np.float64), f64p),
                                ctypes.byref(cp), _p(u, f64p))


def refine(cost, wh, wv, u0, iters: int, P: Params = Params(), alpha=None, state=None):
    """Primal-dual refinement; returns (u, (ph, pv, qh, qv), energy per warp)."""
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    H, W, L = cost.shape
    u = np.array(u0, dtype=np.float64).reshape(H, W).copy()
    if state is None:
        ph, pv, qh, qv = (np.zeros((H, W)) for _ in range(4))
        init = 1
    else:
        ph, pv, qh, qv = (np.array(s, dtype=np.float64).copy() for s in state)
        init = 0
    al = np.ascontiguousarray(np.broadcast_to(P.alpha if alpha is None else alpha, (H, W)), np.float64)
    energy = np.zeros(P.warps)
    cp = P.cont()
    _chk(lib().or_refine(H, W, L, _p(cost, f64p), _p(al, f64p),
                         _p(np.ascontiguousarray(wh, np.float64), f64p),
                         _p(np.ascontiguousarray(wv, np.float64), f64p), iters, ctypes.byref(cp),
                         _p(u, f64p), _p(ph, f64p), _p(pv, f64p), _p(qh, f64p), _p(qv, f64p),
                         init, _p(energy, f64p)), "refine")
    return u, (ph, pv, qh, qv), energy


def refine_perturbed(cost, wh, wv, u0, iters: int, noise: float, seed: int,
                     P: Params = Params(), alpha=None):
    """The refinement with the state (u, p, q) multiplied by 1 + noise * U
    (U uniform in [-1, 1), splitmix64 from seed) after every iteration; noise =
    2^-24 models keeping the state in float32.  Returns u."""
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    H, W, L = cost.shape
    u = np.array(u0, dtype=np.float64).reshape(H, W).copy()
    ph, pv, qh, qv = (np.zeros((H, W)) for _ in range(4))
    al = np.ascontiguousarray(np.broadcast_to(P.alpha if alpha is None else alpha, (H, W)), np.float64)
    cp = P.cont()
    _chk(lib().or_refine_perturbed(H, W, L, _p(cost, f64p), _p(al, f64p),
                                   _p(np.ascontiguousarray(wh, np.float64), f64p),
                                   _p(np.ascontiguousarray(wv, np.float64), f64p), iters,
                                   ctypes.byref(cp), _p(u, f64p), _p(ph, f64p), _p(pv, f64p),
                                   _p(qh, f64p), _p(qv, f64p), 1, float(noise), int(seed)),
         "refine_perturbed")
    return u


def fp32_spread(cost, wh, wv, u0, iters: int, P: Params = Params(), seeds=range(8), alpha=None):
    """Per pixel, the largest distance between the refinement and its float32
    noise model (refine_perturbed with noise 2^-24) over the given seeds: how
    far the double-precision result is determined at float32 precision."""
    u = refine(cost, wh, wv, u0, iters, P, alpha=alpha)[0]
    spread = np.zeros_like(u)
    for s in seeds:
        spread = np.maximum(spread, np.abs(
            refine_perturbed(cost, wh, wv, u0, iters, 2.0 ** -24, s, P, alpha=alpha) - u))
    return spread


def convex_gap(cost, wh, wv, u0, u, ph, pv, P: Params, alpha=None):
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    H, W, L = cost.shape
    al = np.ascontiguousarray(np.broadcast_to(P.alpha if alpha is None else alpha, (H, W)), np.float64)
    pr, du = ctypes.c_double(), ctypes.c_double()
    cp = P.cont()
    lib().or_convex_gap(H, W, L, _p(cost, f64p), _p(al, f64p),
                        _p(np.ascontiguousarray(wh, np.float64), f64p),
                        _p(np.ascontiguousarray(wv, np.float64), f64p), ctypes.byref(cp),
                        _p(np.ascontiguousarray(u0, np.float64), f64p),
                        _p(np.ascontiguousarray(u, np.float64), f64p),
                        _p(np.ascontiguousarray(ph, np.float64), f64p),
                        _p(np.ascontiguousarray(pv, np.float64), f64p),
                        ctypes.byref(pr), ctypes.byref(du))
    return pr.value, du.value


def refine_grad(cost, wh, wv, u0, iters: int, gt, P: Params = Params(), alpha=None,
                want_u0: bool = False):
    """Reverse mode of the refinement: loss = mean |u - gt| and its gradient with
    respect to the cost samples, the per-pixel data weights and lambda_r (and,
    with want_u0, the start u0: a sixth result)."""
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    H, W, L = cost.shape
    al = np.ascontiguousarray(np.broadcast_to(P.alpha if alpha is None else alpha, (H, W)), np.float64)
    u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(H, W)
    gt = np.ascontiguousarray(gt, dtype=np.float64).reshape(H, W)
    u = np.zeros((H, W))
    loss = np.zeros(1)
    gc = np.zeros((H, W, L))
    ga = np.zeros((H, W))
    gl = np.zeros(1)
    g0 = np.zeros((H, W))
    cp = P.cont()
    _chk(lib().or_refine_grad(H, W, L, _p(cost, f64p), _p(al, f64p),
                              _p(np.ascontiguousarray(wh, np.float64), f64p),
                              _p(np.ascontiguousarray(wv, np.float64), f64p), _p(u0, f64p), iters,
                              ctypes.byref(cp), _p(gt, f64p), _p(u, f64p), _p(loss, f64p),
                              _p(gc, f64p), _p(ga, f64p), _p(gl, f64p), _p(g0, f64p)),
         "refine_grad")
    if want_u0:
        return u, float(loss[0]), gc, ga, float(gl[0]), g0
    return u, float(loss[0]), gc, ga, float(gl[0])


def solve(left, right, L: int, dmm_iters: int, pd_iters: int, P: Params = Params(),
          nthreads: int = 0):
    """Whole path on the CPU: cost volume, Dual MM, refinement."""
    cost = cost_volume(left, right, L, P.census_win)
    wh, wv = edge_weights(left, P)
    labels, lb, lam_h, lam_v = dmm(cost, wh, wv, dmm_iters, P, nthreads=nthreads)
    u, st, en = refine(cost.astype(np.float64), wh.astype(np.float64), wv.astype(np.float64),
                       labels.astype(np.float64), pd_iters, P)
    return dict(cost=cost, wh=wh, wv=wv, labels=labels, lb=lb, lam_h=lam_h, lam_v=lam_v, u=u,
                state=st, energy=en)


def solve_lr(left, right, L: int, dmm_iters: int, pd_iters: int, P: Params = Params(),
             max_diff: float = 1.0, nthreads: int = 0):
    """Two-view path with the consistency check (Sec. 4.1.1; readings R25-R28).
    The left view is solve(left, right).  The right view is the same path on
    the mirrored pair (mirrored right image as reference, mirrored left image
    as the other view), whose cost volume is the right-view cost volume with
    columns reversed; its disparity is mirrored back.  The check runs on the
    two disparities rounded to float32."""
    sl = solve(left, right, L, dmm_iters, pd_iters, P, nthreads)
    sm = solve(np.ascontiguousarray(right[:, ::-1]), np.ascontiguousarray(left[:, ::-1]), L,
               dmm_iters, pd_iters, P, nthreads)
    u_left = sl["u"].astype(np.float32)
    u_right = np.ascontiguousarray(sm["u"][:, ::-1]).astype(np.float32)
    ok, out = lr_check(u_left, u_right, max_diff)
    return dict(left=sl, mirrored=sm, u_left=u_left, u_right=u_right, ok=ok, u=out)


# ---------------------------------------------------------------------------
# Optical flow (Sec. 2.2 "Flow"; the appendix's quadratic data model)
# ---------------------------------------------------------------------------

class Flow:
    """Flow geometry: images I1, I2 (uint8 [H, W]), displacement d_k = lo_k + label,
    labels 0..K_k-1 (d1 horizontal, d2 vertical)."""

    def __init__(self, img1, img2, lo1: int, K1: int, lo2: int, K2: int, win: int = 5):
        self.img1 = np.ascontiguousarray(img1, dtype=np.uint8)
        self.img2 = np.ascontiguousarray(img2, dtype=np.uint8)
        self.H, self.W = self.img1.shape
        self.lo1, self.K1, self.lo2, self.K2 = int(lo1), int(K1), int(lo2), int(K2)
        self.c1, self.c2 = census(self.img1, win), census(self.img2, win)
        self.geo = FlowGeo(self.H, self.W, self.lo1, self.K1, self.lo2, self.K2, win * win - 1,
                           _p(self.c1, u32p), _p(self.c2, u32p))

    def projected_costs(self):
        p1 = np.zeros((self.H, self.W, self.K1), dtype=np.int32)
        p2 = np.zeros((self.H, self.W, self.K2), dtype=np.int32)
        _chk(lib().or_flow_cost_projected(ctypes.byref(self.geo), _p(p1, i32p), _p(p2, i32p)),
             "flow_cost_projected")
        return p1, p2

    def D(self, y: int, x: int, v1: float, v2: float) -> float:
        return lib().or_flow_D(ctypes.byref(self.geo), int(y), int(x), float(v1), float(v2))

    def linearise_px(self, y, x, u01, u02, h=1.0, alpha=1.0):
        L = np.zeros(2)
        Q = np.zeros(3)
        box = np.zeros(4)
        lib().or_flow_linearise_px(ctypes.byref(self.geo), int(y), int(x), float(alpha),
                                   float(u01), float(u02), float(h), _p(L, f64p), _p(Q, f64p),
                                   _p(box, f64p))
        return L, Q, box

    def energy(self, u1, u2, wh, wv, P: Params = Params()) -> float:
        u1 = np.ascontiguousarray(u1, dtype=np.float64)
        u2 = np.ascontiguousarray(u2, dtype=np.float64)
        cp = P.cont()
        return lib().or_flow_energy(ctypes.byref(self.geo), float(P.alpha),
                                    _p(np.ascontiguousarray(wh, np.float64), f64p),
                                    _p(np.ascontiguousarray(wv, np.float64), f64p),
                                    ctypes.byref(cp), _p(u1, f64p), _p(u2, f64p))

    def refine(self, u1, u2, wh, wv, iters: int, P: Params = Params(), duals=None):
        """Primal-dual refinement from (u1, u2) (label coordinates); returns (u1, u2,
        duals [8, H, W], energy per warp)."""
        u1 = np.array(u1, dtype=np.float64, order="C")
        u2 = np.array(u2, dtype=np.float64, order="C")
        D = (np.zeros((8, self.H, self.W)) if duals is None
             else np.array(duals, dtype=np.float64, order="C"))
        en = np.zeros(P.warps)
        cp = P.cont()
        _chk(lib().or_flow_refine(ctypes.byref(self.geo), float(P.alpha),
                                  _p(np.ascontiguousarray(wh, np.float64), f64p),
                                  _p(np.ascontiguousarray(wv, np.float64), f64p), int(iters),
                                  ctypes.byref(cp), _p(u1, f64p), _p(u2, f64p), _p(D, f64p),
                                  1 if duals is None else 0, _p(en, f64p)), "flow_refine")
        return u1, u2, D, en


def flow_fit_samples(S, h: float = 1.0):
    """L [2], Q [q11, q12, q22] from the 3x3 samples S[j][i] = D(u0 + (i-1)h e1 + (j-1)h e2)."""
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(9)
    L = np.zeros(2)
    Q = np.zeros(3)
    lib().or_flow_fit_samples(_p(S, f64p), float(h), _p(L, f64p), _p(Q, f64p))
    return L, Q


def psd2(Q):
    Q = np.array(Q, dtype=np.float64).reshape(3)
    lib().or_psd2(_p(Q, f64p))
    return Q


def flow_prox(uh, u0, L, Q, box, tau):
    L = np.ascontiguousarray(L, np.float64)
    Q = np.ascontiguousarray(Q, np.float64)
    box = np.ascontiguousarray(box, np.float64)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_flow_prox(float(uh[0]), float(uh[1]), float(u0[0]), float(u0[1]), _p(L, f64p),
                       _p(Q, f64p), _p(box, f64p), float(tau), ctypes.byref(a), ctypes.byref(b))
    return np.array([a.value, b.value])


def solve_flow(img1, img2, lo1: int, K1: int, lo2: int, K2: int, dmm_iters: int, pd_iters: int,
               P: Params = Params(), nthreads: int = 0):
    """Whole flow path: decoupled costs, Dual MM on each layer (edge weights of I1),
    refinement of both components from the labels."""
    fl = Flow(img1, img2, lo1, K1, lo2, K2, P.census_win)
    p1, p2 = fl.projected_costs()
    wh, wv = edge_weights(fl.img1, P)
    l1, lb1, _, _ = dmm(p1, wh, wv, dmm_iters, P, nthreads=nthreads)
    l2, lb2, _, _ = dmm(p2, wh, wv, dmm_iters, P, nthreads=nthreads)
    u1, u2, D, en = fl.refine(l1.astype(np.float64), l2.astype(np.float64), wh, wv, pd_iters, P)
    return dict(flow=fl, p1=p1, p2=p2, wh=wh, wv=wv, labels1=l1, labels2=l2, lb1=lb1, lb2=lb2,
                u1=u1, u2=u2, duals=D, energy=en)
