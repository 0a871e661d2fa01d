"""Python binding of libdm.so: argument marshalling only.

Every function maps one-to-one onto an entry point of include/dm.h.  torch
supplies device memory (the workspace, inputs, outputs) and the stream; all
computation happens in the CUDA library.  There is no fallback: if libdm.so
is missing or no GPU is present the calls raise.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DM_CHECKED=1 selects the checked build (index checks in the kernels)
LIB_PATH = os.path.join(_HERE, "libdm_checked.so" if os.environ.get("DM_CHECKED") == "1"
                        else "libdm.so")

DM_OK, DM_ERR_ARG, DM_ERR_CUDA, DM_ERR_RANGE, DM_ERR_TIMEOUT = 0, 1, 2, 3, 4
DM_ERR_STATE, DM_ERR_WORKSPACE, DM_ERR_DEVICE = 5, 6, 7


class DMError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {error_string(code)} (status {code})")


class DmParams(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("census_win", ctypes.c_int32),
                ("edge_threshold", ctypes.c_int32), ("w_hi", ctypes.c_int32),
                ("w_lo", ctypes.c_int32), ("eps", ctypes.c_double), ("delta", ctypes.c_double),
                ("C", ctypes.c_double), ("lambda_r", ctypes.c_double),
                ("alpha", ctypes.c_double), ("tau", ctypes.c_double),
                ("sigma", ctypes.c_double), ("h", ctypes.c_double), ("warps", ctypes.c_int32),
                ("dmm_path", ctypes.c_int32), ("cost_bytes", ctypes.c_int32),
                ("pd_launch", ctypes.c_int32), ("wait_test", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int


def lib() -> ctypes.CDLL:
    """Load libdm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1601_06274_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "dm_default_params": [ctypes.POINTER(DmParams)],
            "dm_create": [_i, _i, _i, ctypes.POINTER(DmParams), ctypes.POINTER(_vp)],
            "dm_destroy": [_vp],
            "dm_workspace_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
            "dm_bind_workspace": [_vp, _vp, ctypes.c_size_t],
            "dm_set_stream": [_vp, _vp],
            "dm_cost_volume": [_vp, _vp, _vp],
            "dm_set_cost_volume": [_vp, _vp, _vp, _vp],
            "dm_reset_duals": [_vp],
            "dm_discrete_pass": [_vp, _i],
            "dm_discrete": [_vp, _i, _vp],
            "dm_refine": [_vp, _i, _vp],
            "dm_solve": [_vp, _vp, _vp, _i, _i, _vp],
            "dm_solve_host": [_vp, _vp, _vp, _i, _i, _vp, _vp],
            "dm_get_labels": [_vp, _vp],
            "dm_get_disparity": [_vp, _vp],
            "dm_get_duals": [_vp, _vp, _vp],
            "dm_get_cost_volume": [_vp, _vp, _vp, _vp],
            "dm_get_lower_bounds": [_vp, _vp, _i],
            "dm_energy": [_vp, ctypes.POINTER(ctypes.c_double)],
            "dm_sync": [_vp],
            "dm_launch_count": [_vp, ctypes.POINTER(ctypes.c_uint64)],
            "dm_get_path": [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
            "dm_batch_create": [_i, _vp, _vp, _vp, ctypes.POINTER(DmParams), ctypes.POINTER(_vp)],
            "dm_batch_destroy": [_vp],
            "dm_batch_workspace_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
            "dm_batch_bind_workspace": [_vp, _vp, ctypes.c_size_t],
            "dm_batch_set_stream": [_vp, _vp],
            "dm_batch_context": [_vp, _i, ctypes.POINTER(_vp)],
            "dm_batch_solve": [_vp, _vp, _vp, _i, _i, _vp],
            "dm_batch_capture": [_vp, _vp, _vp, _i, _i, _vp],
            "dm_batch_replay": [_vp],
            "dm_batch_sync": [_vp],
            "dm_batch_tune": [_vp, _vp, _vp, ctypes.c_char_p, _vp],
            "dm_batch_set_tuning": [_vp, _vp],
            "dm_batch_get_tuning": [_vp, _vp],
            "dm_batch_launch_count": [_vp, ctypes.POINTER(ctypes.c_uint64)],
            "dm_batch_discrete_pass": [_vp, _i],
            "dm_discrete_pass_noalloc": [_i, _i, _i, ctypes.POINTER(DmParams), _i, _vp, _vp,
                                         _vp, _vp, _vp, _vp],
            "dm_set_cost_volume_f32": [_vp, _vp, _vp, _vp],
            "dm_set_cost_volume_u16": [_vp, _vp, _vp, _vp, _i],
            "dm_cost_volume_warm": [_vp, _vp, _vp],
            "dm_solve_next": [_vp, _vp, _vp, _i, _i, _vp],
            "dm_cost_volume_mirrored": [_vp, _vp, _vp],
            "dm_set_minorant": [_vp, _i, _i, _i, _i],
            "dm_capture": [_vp, _vp, _vp, _i, _i, _vp],
            "dm_replay": [_vp],
            "dm_flow_cost_volumes": [_vp, _vp, _vp, _vp, _i, _i],
            "dm_flow_refine_bytes": [_i, _i, ctypes.POINTER(ctypes.c_size_t)],
            "dm_flow_refine": [_vp, _vp, _i, _vp, ctypes.c_size_t, _vp, _vp],
            "dm_lr_check": [_vp, _vp, _i, _i, ctypes.c_float, _vp, _vp, _vp, _vp],
            "dm_solve_lr": [_vp, _vp, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp, _vp],
            "dm_set_data_weights": [_vp, _vp],
            "dm_set_lambda_r": [_vp, ctypes.c_double],
            "dm_tape_bytes": [_vp, _i, _i, ctypes.POINTER(ctypes.c_size_t)],
            "dm_refine_tape": [_vp, _i, _i, _vp, _vp, ctypes.c_size_t],
            "dm_refine_backward": [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp],
            "dm_jvp_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
            "dm_refine_jvp": [_vp, _i, _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp,
                              ctypes.c_size_t],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.dm_error_string.argtypes = [_i]
        L.dm_error_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().dm_error_string(int(code)).decode()


def _ck(rc: int, what: str):
    if rc != DM_OK:
        raise DMError(rc, what)


def default_params(**overrides) -> DmParams:
    p = DmParams()
    _ck(lib().dm_default_params(ctypes.byref(p)), "dm_default_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


MINORANTS = {"hier": 0, "naive": 1, "iterative": 2}


class Context:
    """One dm_ctx with its workspace (a torch uint8 tensor on the GPU)."""

    def __init__(self, H: int, W: int, L: int, params: DmParams | None = None,
                 device: str = "cuda", stream=None):
        import torch
        self._torch = torch
        self.H, self.W, self.L = H, W, L
        self.params = params if params is not None else default_params()
        h = _vp()
        _ck(lib().dm_create(H, W, L, ctypes.byref(self.params), ctypes.byref(h)), "dm_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _ck(lib().dm_workspace_bytes(self._h, ctypes.byref(nbytes)), "dm_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        self._tape = None
        # the workspace may be a block that work still queued on torch's stream
        # writes (the caching allocator orders reuse on that stream only)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _ck(lib().dm_set_stream(self._h, _vp(self.stream.cuda_stream)), "dm_set_stream")
        _ck(lib().dm_bind_workspace(self._h, self._ws.data_ptr(), self.workspace_bytes),
            "dm_bind_workspace")

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().dm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------------
    def _empty(self, shape, dtype):
        return self._torch.empty(shape, dtype=dtype, device=self.device)

    def _fork(self):
        # a context on its own stream reads what torch's stream produced
        cur = self._torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def _join(self):
        # ... and torch's stream reads what the context produced
        cur = self._torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def _dev_u8(self, a):
        t = self._torch.as_tensor(np.ascontiguousarray(a)) if isinstance(a, np.ndarray) else a
        t = t.to(self.device, self._torch.uint8).contiguous()
        self._fork()
        return t

    # -- entry points ------------------------------------------------------------
    def cost_volume(self, left, right):
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        _ck(lib().dm_cost_volume(self._h, self._left.data_ptr(), self._right.data_ptr()),
            "dm_cost_volume")

    def set_cost_volume(self, cost, wh, wv):
        self._c, self._wh, self._wv = self._dev_u8(cost), self._dev_u8(wh), self._dev_u8(wv)
        _ck(lib().dm_set_cost_volume(self._h, self._c.data_ptr(), self._wh.data_ptr(),
                                     self._wv.data_ptr()), "dm_set_cost_volume")

    def set_cost_volume_u16(self, cost, wh, wv, cost_max: int):
        torch = self._torch
        c = torch.as_tensor(np.ascontiguousarray(cost).view(np.int16)) \
            if isinstance(cost, np.ndarray) else cost
        self._c = c.to(self.device).contiguous()
        self._wh, self._wv = self._dev_u8(wh), self._dev_u8(wv)
        _ck(lib().dm_set_cost_volume_u16(self._h, self._c.data_ptr(), self._wh.data_ptr(),
                                         self._wv.data_ptr(), int(cost_max)),
            "dm_set_cost_volume_u16")

    def set_minorant(self, kind: str = "hier", max_pass: int = 3, gamma=(1, 4)):
        """Chain minorant of the Dual MM passes: "hier" (default), "naive" or
        "iterative" (max_pass passes, gamma = gamma[0] / gamma[1] but the last)."""
        _ck(lib().dm_set_minorant(self._h, MINORANTS[kind], int(max_pass), int(gamma[0]),
                                  int(gamma[1])), "dm_set_minorant")

    def cost_volume_mirrored(self, left, right):
        """The right view's problem of (left, right), in mirrored columns."""
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        _ck(lib().dm_cost_volume_mirrored(self._h, self._left.data_ptr(), self._right.data_ptr()),
            "dm_cost_volume_mirrored")

    def cost_volume_warm(self, left, right):
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        _ck(lib().dm_cost_volume_warm(self._h, self._left.data_ptr(), self._right.data_ptr()),
            "dm_cost_volume_warm")

    def solve_next(self, left, right, dmm_iters: int, pd_iters: int, out=None):
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        out = out if out is not None else self._empty((self.H, self.W), self._torch.float32)
        self._fork()
        _ck(lib().dm_solve_next(self._h, self._left.data_ptr(), self._right.data_ptr(), dmm_iters,
                                pd_iters, out.data_ptr()), "dm_solve_next")
        self._join()
        return out

    def reset_duals(self):
        _ck(lib().dm_reset_duals(self._h), "dm_reset_duals")

    def discrete_pass(self, which: int):
        _ck(lib().dm_discrete_pass(self._h, int(which)), "dm_discrete_pass")

    def discrete(self, iters: int, lower_bounds: bool = False):
        if lower_bounds:
            lb = np.zeros(iters, dtype=np.int64)
            _ck(lib().dm_discrete(self._h, iters, lb.ctypes.data), "dm_discrete")
            return lb
        _ck(lib().dm_discrete(self._h, iters, None), "dm_discrete")
        return None

    def refine(self, iters: int, u0=None):
        if u0 is not None:
            u0 = self._torch.as_tensor(u0).to(self.device, self._torch.float32).contiguous()
            self._u0 = u0
        _ck(lib().dm_refine(self._h, iters, _ptr(u0)), "dm_refine")

    def solve(self, left, right, dmm_iters: int, pd_iters: int, out=None):
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        out = out if out is not None else self._empty((self.H, self.W), self._torch.float32)
        self._fork()
        _ck(lib().dm_solve(self._h, self._left.data_ptr(), self._right.data_ptr(), dmm_iters,
                           pd_iters, out.data_ptr()), "dm_solve")
        self._join()
        return out

    def capture(self, left, right, dmm_iters: int, pd_iters: int, out):
        """Record a solve on these device tensors (which stay alive and in place)
        as a CUDA graph of the context's stream (create the context with its own
        stream)."""
        self._graph_keep = (left, right, out)
        self._torch.cuda.synchronize(self.device)
        _ck(lib().dm_capture(self._h, left.data_ptr(), right.data_ptr(), int(dmm_iters),
                             int(pd_iters), out.data_ptr()), "dm_capture")

    def replay(self):
        """Launch the captured solve after the work queued on torch's stream (new
        images copied into the captured buffers); torch's stream then waits for it."""
        self._fork()
        _ck(lib().dm_replay(self._h), "dm_replay")
        self._join()

    def solve_host(self, left, right, dmm_iters: int, pd_iters: int, u_out=None, labels_out=None):
        """Host buffers in and out (pinned torch CPU tensors or numpy arrays)."""
        torch = self._torch
        lt = torch.as_tensor(left) if isinstance(left, np.ndarray) else left
        rt = torch.as_tensor(right) if isinstance(right, np.ndarray) else right
        u_out = u_out if u_out is not None else torch.empty((self.H, self.W), dtype=torch.float32)
        _ck(lib().dm_solve_host(self._h, lt.data_ptr(), rt.data_ptr(), dmm_iters, pd_iters,
                                u_out.data_ptr(), _ptr(labels_out)), "dm_solve_host")
        return u_out

    def labels(self):
        out = self._empty((self.H, self.W), self._torch.int16)
        self._fork()
        _ck(lib().dm_get_labels(self._h, out.data_ptr()), "dm_get_labels")
        self._join()
        return out

    def disparity(self):
        out = self._empty((self.H, self.W), self._torch.float32)
        self._fork()
        _ck(lib().dm_get_disparity(self._h, out.data_ptr()), "dm_get_disparity")
        self._join()
        return out

    def duals(self):
        lh = self._empty((self.H, self.W, self.L), self._torch.int32)
        lv = self._empty((self.H, self.W, self.L), self._torch.int32)
        self._fork()
        _ck(lib().dm_get_duals(self._h, lh.data_ptr(), lv.data_ptr()), "dm_get_duals")
        self._join()
        return lh, lv

    def cost(self):
        """(cost volume, wh, wv); the cost is int16 holding uint16 samples when
        params.cost_bytes = 2 (numpy: .view(np.uint16))."""
        dt = self._torch.int16 if self.params.cost_bytes == 2 else self._torch.uint8
        c = self._empty((self.H, self.W, self.L), dt)
        wh = self._empty((self.H, self.W), self._torch.uint8)
        wv = self._empty((self.H, self.W), self._torch.uint8)
        self._fork()
        _ck(lib().dm_get_cost_volume(self._h, c.data_ptr(), wh.data_ptr(), wv.data_ptr()),
            "dm_get_cost_volume")
        self._join()
        return c, wh, wv

    def lower_bounds(self, n: int):
        lb = np.zeros(n, dtype=np.int64)
        _ck(lib().dm_get_lower_bounds(self._h, lb.ctypes.data, n), "dm_get_lower_bounds")
        return lb

    def energy(self) -> float:
        e = ctypes.c_double()
        _ck(lib().dm_energy(self._h, ctypes.byref(e)), "dm_energy")
        return e.value

    # -- differentiable refinement ---------------------------------------------
    def _dev_f32(self, a):
        t = self._torch.as_tensor(a) if isinstance(a, np.ndarray) else a
        return t.to(self.device, self._torch.float32).contiguous()

    def set_cost_volume_f32(self, cost, wh=None, wv=None):
        """Borrow a float32 [H][W][L] cost volume (the reference is kept here)."""
        self._cf = self._dev_f32(cost)
        if wh is not None:
            self._wh, self._wv = self._dev_u8(wh), self._dev_u8(wv)
        _ck(lib().dm_set_cost_volume_f32(self._h, self._cf.data_ptr(),
                                         _ptr(self._wh) if wh is not None else None,
                                         _ptr(self._wv) if wh is not None else None),
            "dm_set_cost_volume_f32")
        self._tape = None

    def set_data_weights(self, alpha=None):
        self._alpha = None if alpha is None else self._dev_f32(alpha)
        _ck(lib().dm_set_data_weights(self._h, _ptr(self._alpha)), "dm_set_data_weights")
        self._tape = None

    def set_lambda_r(self, value: float):
        _ck(lib().dm_set_lambda_r(self._h, float(value)), "dm_set_lambda_r")
        self.params.lambda_r = float(value)
        self._tape = None

    def tape_bytes(self, iters: int, ckpt_every: int) -> int:
        n = ctypes.c_size_t()
        _ck(lib().dm_tape_bytes(self._h, iters, ckpt_every, ctypes.byref(n)), "dm_tape_bytes")
        return n.value

    def refine_tape(self, iters: int, ckpt_every: int, u0=None, tape=None):
        """dm_refine with checkpoints; returns the tape (a device uint8 tensor)."""
        if u0 is not None:
            self._u0 = self._dev_f32(u0)
            u0 = self._u0
        nb = self.tape_bytes(iters, ckpt_every)
        if tape is None or tape.numel() < nb:
            tape = self._empty(nb, self._torch.uint8)
        _ck(lib().dm_refine_tape(self._h, iters, ckpt_every, _ptr(u0), tape.data_ptr(),
                                 tape.numel()), "dm_refine_tape")
        self._tape = tape
        return tape

    def refine_backward(self, gu, tape, cost=True, alpha=True, lam=True, u0=False):
        """Reverse mode of the last refine_tape: (d cost, d alpha, d lambda_r, d u0),
        each None unless asked for."""
        torch = self._torch
        gu = self._dev_f32(gu)
        gc = self._empty((self.H, self.W, self.L), torch.float32) if cost else None
        ga = self._empty((self.H, self.W), torch.float32) if alpha else None
        gl = self._empty((1,), torch.float64) if lam else None
        g0 = self._empty((self.H, self.W), torch.float32) if u0 else None
        _ck(lib().dm_refine_backward(self._h, gu.data_ptr(), tape.data_ptr(), tape.numel(),
                                     _ptr(gc), _ptr(ga), _ptr(gl), _ptr(g0)),
            "dm_refine_backward")
        return gc, ga, gl, g0

    def refine_jvp(self, iters: int, u0=None, du0=None, dcost=None, dalpha=None,
                   dlambda: float = 0.0):
        """dm_refine_jvp: refined u (read with disparity()) and its directional
        derivative in (du0, dcost, dalpha, dlambda)."""
        n = ctypes.c_size_t()
        _ck(lib().dm_jvp_bytes(self._h, ctypes.byref(n)), "dm_jvp_bytes")
        scratch = self._empty(n.value, self._torch.uint8)
        keep = [None if a is None else self._dev_f32(a) for a in (u0, du0, dcost, dalpha)]
        du = self._empty((self.H, self.W), self._torch.float32)
        _ck(lib().dm_refine_jvp(self._h, iters, *[_ptr(a) for a in keep], float(dlambda),
                                du.data_ptr(), scratch.data_ptr(), n.value), "dm_refine_jvp")
        self._jvp_keep = (keep, scratch)
        return du

    def path(self):
        """(Dual MM kernel: 8 lane groups, 16 one warp per chain, 32 int32;
        bytes per dual delta)"""
        k, d = ctypes.c_int(), ctypes.c_int()
        _ck(lib().dm_get_path(self._h, ctypes.byref(k), ctypes.byref(d)), "dm_get_path")
        return k.value, d.value

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _ck(lib().dm_launch_count(self._h, ctypes.byref(n)), "dm_launch_count")
        return n.value

    def sync(self):
        _ck(lib().dm_sync(self._h), "dm_sync")


class _PairView(Context):
    """The context of one pair of a Batch (owned by the batch)."""

    def __init__(self, batch, i, H, W, L, params):
        self._torch = batch._torch
        self.H, self.W, self.L = H, W, L
        self.params = params
        self.device = batch.device
        self.stream = batch.stream
        self._tape = None
        h = _vp()
        _ck(lib().dm_batch_context(batch._h, i, ctypes.byref(h)), "dm_batch_context")
        self._h = h
        self._batch = batch

    def close(self):
        self._h = None

    # the getters enqueue copies on the batch's stream: wait for them before torch
    # (on its own stream) reads the results
    def labels(self):
        out = super().labels()
        self.stream.synchronize()
        return out

    def disparity(self):
        out = super().disparity()
        self.stream.synchronize()
        return out

    def cost(self):
        out = super().cost()
        self.stream.synchronize()
        return out


class Batch:
    """dm_batch: pairs of mixed sizes solved by persistent kernels, optionally
    as one captured CUDA graph.  shapes: list of (H, W, L)."""

    def __init__(self, shapes, params: DmParams | None = None, device: str = "cuda"):
        import torch
        self._torch = torch
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.n = len(self.shapes)
        self.params = params if params is not None else default_params()
        arr = lambda k: (ctypes.c_int * self.n)(*[s[k] for s in self.shapes])
        h = _vp()
        _ck(lib().dm_batch_create(self.n, arr(0), arr(1), arr(2), ctypes.byref(self.params),
                                  ctypes.byref(h)), "dm_batch_create")
        self._h = h
        nb = ctypes.c_size_t()
        _ck(lib().dm_batch_workspace_bytes(self._h, ctypes.byref(nb)), "dm_batch_workspace_bytes")
        self.workspace_bytes = nb.value
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)   # capturable (not the legacy stream)
        self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        # the block may still be written by work queued on torch's stream: bind after it
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _ck(lib().dm_batch_set_stream(self._h, _vp(self.stream.cuda_stream)), "dm_batch_set_stream")
        _ck(lib().dm_batch_bind_workspace(self._h, self._ws.data_ptr(), self.workspace_bytes),
            "dm_batch_bind_workspace")
        self.pairs = [_PairView(self, i, *self.shapes[i], self.params) for i in range(self.n)]
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            lib().dm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, ts):
        return (ctypes.c_void_p * self.n)(*[None if t is None else t.data_ptr() for t in ts])

    def _inputs(self, lefts, rights):
        torch = self._torch
        dev = lambda a: (torch.as_tensor(np.ascontiguousarray(a)) if isinstance(a, np.ndarray)
                         else a).to(self.device, torch.uint8).contiguous()
        ls, rs = [dev(a) for a in lefts], [dev(a) for a in rights]
        # the copies ran on torch's stream; the batch reads them on its own
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        return ls, rs

    def outputs(self):
        return [self._torch.empty((H, W), dtype=self._torch.float32, device=self.device)
                for H, W, _ in self.shapes]

    def solve(self, lefts, rights, dmm_iters: int, pd_iters: int, outs=None):
        ls, rs = self._inputs(lefts, rights)
        outs = outs if outs is not None else self.outputs()
        self._keep = (ls, rs, outs)
        _ck(lib().dm_batch_solve(self._h, self._ptrs(ls), self._ptrs(rs), dmm_iters, pd_iters,
                                 self._ptrs(outs)), "dm_batch_solve")
        self._join()
        return outs

    def _join(self):
        # torch's stream continues after the batch's work: the outputs are ready for
        # torch, and blocks the allocator hands out again are no longer in use
        self._torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def capture(self, lefts, rights, dmm_iters: int, pd_iters: int, outs):
        """Record one solve on these device buffers (torch tensors that stay
        alive and in place) into the batch's CUDA graph."""
        self._graph_keep = (list(lefts), list(rights), list(outs))
        self._torch.cuda.synchronize(self.device)
        _ck(lib().dm_batch_capture(self._h, self._ptrs(lefts), self._ptrs(rights), dmm_iters,
                                   pd_iters, self._ptrs(outs)), "dm_batch_capture")

    def replay(self):
        """Launch the captured graph after the work queued on torch's stream
        (e.g. new inputs copied into the captured buffers)."""
        self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        _ck(lib().dm_batch_replay(self._h), "dm_batch_replay")
        self._join()

    def sync(self):
        _ck(lib().dm_batch_sync(self._h), "dm_batch_sync")

    def tune(self, lefts, rights, cache_path: str | None = None):
        ls, rs = self._inputs(lefts, rights)
        out = (ctypes.c_int * 5)()
        _ck(lib().dm_batch_tune(self._h, self._ptrs(ls), self._ptrs(rs),
                                cache_path.encode() if cache_path else None, out), "dm_batch_tune")
        self._join()
        return tuple(out)

    def set_tuning(self, choice):
        _ck(lib().dm_batch_set_tuning(self._h, (ctypes.c_int * 5)(*choice)), "dm_batch_set_tuning")

    def tuning(self):
        out = (ctypes.c_int * 5)()
        _ck(lib().dm_batch_get_tuning(self._h, out), "dm_batch_get_tuning")
        return tuple(out)

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _ck(lib().dm_batch_launch_count(self._h, ctypes.byref(n)), "dm_batch_launch_count")
        return n.value

    def discrete_pass(self, which: int):
        """One Dual MM pass over every pair (instrumentation; after a solve)."""
        _ck(lib().dm_batch_discrete_pass(self._h, int(which)), "dm_batch_discrete_pass")


class StereoLR:
    """Two views and the two-sided consistency check (dm_solve_lr): a context
    per view, each on its own stream, so that the right view (the mirrored
    pair) runs concurrently with the left one."""

    def __init__(self, H: int, W: int, L: int, params: DmParams | None = None,
                 device: str = "cuda"):
        import torch
        self._torch = torch
        self.H, self.W, self.L = H, W, L
        self.device = torch.device(device)
        self.left = Context(H, W, L, params, device, stream=torch.cuda.Stream(self.device))
        self.right = Context(H, W, L, params, device, stream=torch.cuda.Stream(self.device))

    def outputs(self):
        t = self._torch
        return (t.empty((self.H, self.W), dtype=t.float32, device=self.device),
                t.empty((self.H, self.W), dtype=t.uint8, device=self.device),
                t.empty((self.H, self.W), dtype=t.float32, device=self.device))

    def solve(self, left, right, dmm_iters: int, pd_iters: int, max_diff: float = 1.0,
              outs=None):
        """(u: checked left-view disparity, -1 where the check fails; ok: uint8
        mask; u_right: the right view's disparity), float32 / uint8 [H, W]."""
        torch = self._torch
        cur = torch.cuda.current_stream(self.device)
        lt, rt = self.left._dev_u8(left), self.left._dev_u8(right)
        u, ok, ur = outs if outs is not None else self.outputs()
        self._keep = (lt, rt, u, ok, ur)
        self.left.stream.wait_stream(cur)        # inputs and outputs in torch's order
        _ck(lib().dm_solve_lr(self.left._h, self.right._h, lt.data_ptr(), rt.data_ptr(),
                              int(dmm_iters), int(pd_iters), float(max_diff), ok.data_ptr(),
                              u.data_ptr(), _ptr(ur)), "dm_solve_lr")
        cur.wait_stream(self.left.stream)        # the left stream joined the right one
        return u, ok, ur

    def sync(self):
        self.left.sync()
        self.right.sync()


class Flow:
    """Optical flow (dm_flow_*): two layer contexts, the second on its own stream
    so that the two discrete stages run concurrently, and the refinement
    scratch.  Displacement d_k = lo_k + label_k, label_k in [0, K_k)."""

    def __init__(self, H: int, W: int, lo1: int, K1: int, lo2: int, K2: int,
                 params: DmParams | None = None, device: str = "cuda"):
        import torch
        self._torch = torch
        self.H, self.W = H, W
        self.lo1, self.K1, self.lo2, self.K2 = lo1, K1, lo2, K2
        self.device = torch.device(device)
        self.layer1 = Context(H, W, K1, params, device)
        self.layer2 = Context(H, W, K2, params, device, stream=torch.cuda.Stream(self.device))
        nb = ctypes.c_size_t()
        _ck(lib().dm_flow_refine_bytes(H, W, ctypes.byref(nb)), "dm_flow_refine_bytes")
        self.scratch_bytes = nb.value
        self._scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=self.device)

    def cost_volumes(self, img1, img2):
        l1 = self.layer1
        self._i1, self._i2 = l1._dev_u8(img1), l1._dev_u8(img2)
        _ck(lib().dm_flow_cost_volumes(l1._h, self.layer2._h, self._i1.data_ptr(),
                                       self._i2.data_ptr(), int(self.lo1), int(self.lo2)),
            "dm_flow_cost_volumes")

    def discrete(self, iters: int, lower_bounds: bool = False):
        b1 = self.layer1.discrete(iters, lower_bounds)
        b2 = self.layer2.discrete(iters, lower_bounds)
        return (b1, b2) if lower_bounds else None

    def refine(self, iters: int, outs=None):
        """(d1, d2) float32 [H, W] displacements after `iters` iterations."""
        t = self._torch
        d1, d2 = outs if outs is not None else (
            t.empty((self.H, self.W), dtype=t.float32, device=self.device),
            t.empty((self.H, self.W), dtype=t.float32, device=self.device))
        _ck(lib().dm_flow_refine(self.layer1._h, self.layer2._h, int(iters),
                                 self._scratch.data_ptr(), self.scratch_bytes, d1.data_ptr(),
                                 d2.data_ptr()), "dm_flow_refine")
        return d1, d2

    def solve(self, img1, img2, dmm_iters: int, pd_iters: int, outs=None):
        self.cost_volumes(img1, img2)
        self.discrete(dmm_iters)
        return self.refine(pd_iters, outs)

    def sync(self):
        self.layer1.sync()
        self.layer2.sync()


def solve_flow(img1, img2, lo1: int, K1: int, lo2: int, K2: int, dmm_iters: int = 10,
               pd_iters: int = 100, params: DmParams | None = None, device: str = "cuda"):
    """Optical flow of one pair: (d1, d2) float32 displacements [H, W]."""
    H, W = np.asarray(img1).shape if isinstance(img1, np.ndarray) else tuple(img1.shape)
    f = Flow(H, W, lo1, K1, lo2, K2, params, device)
    out = f.solve(img1, img2, dmm_iters, pd_iters)
    f.sync()
    return out


def lr_check(u_left, u_mirrored, max_diff: float = 1.0, outs=None):
    """dm_lr_check on torch's current stream: (u_out, ok, u_right) for a left-view
    disparity and the disparity of the mirrored (right-view) problem; outs:
    optional preallocated (u_out, ok, u_right)."""
    import torch
    ul = u_left.contiguous()
    um = u_mirrored.contiguous()
    assert ul.dtype == torch.float32 and um.dtype == torch.float32 and ul.shape == um.shape
    H, W = ul.shape
    if outs is None:
        outs = (torch.empty_like(ul), torch.empty((H, W), dtype=torch.uint8, device=ul.device),
                torch.empty_like(ul))
    out, ok, ur = outs
    assert out.shape == ok.shape == ur.shape == (H, W) and ok.dtype == torch.uint8
    st = torch.cuda.current_stream(ul.device).cuda_stream
    _ck(lib().dm_lr_check(ul.data_ptr(), um.data_ptr(), H, W, float(max_diff), ok.data_ptr(),
                          out.data_ptr(), ur.data_ptr(), _vp(st)), "dm_lr_check")
    return out, ok, ur


def solve_lr(left, right, L: int, dmm_iters: int = 10, pd_iters: int = 100,
             max_diff: float = 1.0, params: DmParams | None = None, device: str = "cuda"):
    """Both views of one pair and the consistency check: (u checked, ok, u_left,
    u_right), the first three for the left view, -1 in u where the check fails."""
    H, W = np.asarray(left).shape if isinstance(left, np.ndarray) else tuple(left.shape)
    s = StereoLR(H, W, L, params, device)
    u, ok, ur = s.solve(left, right, dmm_iters, pd_iters, max_diff)
    s.sync()
    return u, ok, s.left.disparity(), ur


def discrete_pass_noalloc(params: DmParams, which: int, cost, wedge, lam_in, lam_out,
                          err=None, stream=None):
    """dm_discrete_pass_noalloc: one Dual MM pass with no workspace and no
    allocation inside the library (inputs/outputs are caller tensors, all
    contiguous on the current device: cost uint8 [H, W, L] (which = 0), wedge
    uint8 [H, W], lam_in and lam_out int32 [H, W, L], distinct; err a zeroed
    int32 tensor)."""
    import torch
    H, W, L = lam_in.shape
    dev = torch.device("cuda", torch.cuda.current_device())

    def need(t, dtype, shape, what):
        if not (isinstance(t, torch.Tensor) and t.dtype == dtype and tuple(t.shape) == shape
                and t.is_contiguous() and t.device == dev):
            raise DMError(DM_ERR_ARG, f"dm_discrete_pass_noalloc: {what} must be a contiguous "
                                      f"{dtype} tensor of shape {shape} on {dev}")
    if which == 0 or cost is not None:
        need(cost, torch.uint8, (H, W, L), "cost")
    need(wedge, torch.uint8, (H, W), "wedge")
    need(lam_in, torch.int32, (H, W, L), "lam_in")
    need(lam_out, torch.int32, (H, W, L), "lam_out")
    if err is None or not (isinstance(err, torch.Tensor) and err.dtype == torch.int32
                           and err.numel() >= 1 and err.device == dev):
        raise DMError(DM_ERR_ARG, "dm_discrete_pass_noalloc: err must be an int32 tensor on the "
                                  "current device")
    if lam_out.data_ptr() == lam_in.data_ptr():
        raise DMError(DM_ERR_ARG, "dm_discrete_pass_noalloc: lam_out must not be lam_in")
    st = stream.cuda_stream if stream is not None else None
    _ck(lib().dm_discrete_pass_noalloc(H, W, L, ctypes.byref(params), int(which), _ptr(cost),
                                       _ptr(wedge), _ptr(lam_in), _ptr(lam_out), _ptr(err),
                                       _vp(st) if st else None),
        "dm_discrete_pass_noalloc")


_REFINE_FN = None


def _refine_function():
    """torch.autograd.Function over refine_tape / refine_backward (built on first use)."""
    global _REFINE_FN
    if _REFINE_FN is not None:
        return _REFINE_FN
    import torch

    class RefineFunction(torch.autograd.Function):
        @staticmethod
        def forward(fctx, cost, alpha, lambda_r, u0, dmctx, iters, ckpt_every):
            lam = float(lambda_r)
            dmctx.set_cost_volume_f32(cost.detach())
            dmctx.set_data_weights(None if alpha is None else alpha.detach())
            dmctx.set_lambda_r(lam)
            tape = dmctx.refine_tape(iters, ckpt_every, None if u0 is None else u0.detach())
            fctx.dm, fctx.tape, fctx.iters, fctx.ckpt = dmctx, tape, iters, ckpt_every
            fctx.inputs = (cost.detach(), None if alpha is None else alpha.detach(), lam,
                           None if u0 is None else u0.detach())
            fctx.lam_like = lambda_r if torch.is_tensor(lambda_r) else None
            return dmctx.disparity()

        @staticmethod
        def backward(fctx, gu):
            dmctx = fctx.dm
            if dmctx._tape is not fctx.tape:
                # another forward ran on this context since: rebuild this tape
                cost, alpha, lam, u0 = fctx.inputs
                dmctx.set_cost_volume_f32(cost)
                dmctx.set_data_weights(alpha)
                dmctx.set_lambda_r(lam)
                dmctx.refine_tape(fctx.iters, fctx.ckpt, u0, fctx.tape)
            need = fctx.needs_input_grad
            gc, ga, gl, g0 = dmctx.refine_backward(gu, fctx.tape, cost=need[0],
                                                   alpha=need[1], lam=need[2], u0=need[3])
            if gl is not None and fctx.lam_like is not None:
                gl = gl.reshape(()).to(fctx.lam_like.device, fctx.lam_like.dtype)
            elif gl is not None:
                gl = None
            return gc, ga, gl, g0, None, None, None

    _REFINE_FN = RefineFunction
    return _REFINE_FN


def refine_differentiable(dmctx: Context, cost, alpha, lambda_r, u0, iters: int,
                          ckpt_every: int = 20):
    """Refined disparity u(cost, alpha, lambda_r, u0) as a differentiable torch op.

    cost: [H][W][L] float32 (CUDA), alpha: [H][W] float32 or None (scalar
    params.alpha), lambda_r: float or 0-d tensor, u0: [H][W] float32 or None
    (the labels of the last discrete stage).  The edge weights are those already
    in dmctx.  Gradients come from dm_refine_backward with a checkpoint every
    ckpt_every iterations."""
    return _refine_function().apply(cost, alpha, lambda_r, u0, dmctx, iters, ckpt_every)


def solve(left, right, L: int, dmm_iters: int = 10, pd_iters: int = 100,
          params: DmParams | None = None, device: str = "cuda"):
    """One pair through the whole path: (refined u [H][W] float32 tensor, labels
    [H][W] uint16 numpy, lower bound of every Dual MM iteration numpy int64)."""
    H, W = np.asarray(left).shape if isinstance(left, np.ndarray) else tuple(left.shape)
    ctx = Context(H, W, L, params, device=device)
    u = ctx.solve(left, right, dmm_iters, pd_iters)
    return u, labels_u16(ctx.labels()), ctx.lower_bounds(dmm_iters)


def batch_solve(pairs, labels, dmm_iters: int = 5, pd_iters: int = 50,
                params: DmParams | None = None, device: str = "cuda", tune: bool = True):
    """Many pairs [(left, right), ...] with label counts `labels` (one per pair)
    through the batched kernels: a list of (u, labels, lower bounds) as in solve."""
    shapes = [(np.asarray(l).shape[0], np.asarray(l).shape[1], int(n))
              for (l, _), n in zip(pairs, labels)]
    b = Batch(shapes, params, device=device)
    lefts, rights = [p[0] for p in pairs], [p[1] for p in pairs]
    if tune:
        b.tune(lefts, rights)
    outs = b.solve(lefts, rights, dmm_iters, pd_iters)
    b.sync()
    return [(outs[i], labels_u16(b.pairs[i].labels()), b.pairs[i].lower_bounds(dmm_iters))
            for i in range(b.n)]


def DMRefine():
    """The torch.autograd.Function behind refine_differentiable (built on first use)."""
    return _refine_function()


def labels_u16(t) -> np.ndarray:
    """int16 tensor holding uint16 labels -> numpy uint16."""
    return t.cpu().numpy().view(np.uint16)
