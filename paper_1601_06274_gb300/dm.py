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
LIB_PATH = os.path.join(_HERE, "libdm.so")

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
                ("dmm_path", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


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
            "dm_discrete_pass_noalloc": [_i, _i, _i, ctypes.POINTER(DmParams), _i, _vp, _vp,
                                         _vp, _vp, _vp, _vp],
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

    def _dev_u8(self, a):
        t = self._torch.as_tensor(np.ascontiguousarray(a)) if isinstance(a, np.ndarray) else a
        return t.to(self.device, self._torch.uint8).contiguous()

    # -- entry points ------------------------------------------------------------
    def cost_volume(self, left, right):
        self._left, self._right = self._dev_u8(left), self._dev_u8(right)
        _ck(lib().dm_cost_volume(self._h, self._left.data_ptr(), self._right.data_ptr()),
            "dm_cost_volume")

    def set_cost_volume(self, cost, wh, wv):
        self._c, self._wh, self._wv = self._dev_u8(cost), self._dev_u8(wh), self._dev_u8(wv)
        _ck(lib().dm_set_cost_volume(self._h, self._c.data_ptr(), self._wh.data_ptr(),
                                     self._wv.data_ptr()), "dm_set_cost_volume")

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
        _ck(lib().dm_solve(self._h, self._left.data_ptr(), self._right.data_ptr(), dmm_iters,
                           pd_iters, out.data_ptr()), "dm_solve")
        return out

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
        _ck(lib().dm_get_labels(self._h, out.data_ptr()), "dm_get_labels")
        return out

    def disparity(self):
        out = self._empty((self.H, self.W), self._torch.float32)
        _ck(lib().dm_get_disparity(self._h, out.data_ptr()), "dm_get_disparity")
        return out

    def duals(self):
        lh = self._empty((self.H, self.W, self.L), self._torch.int32)
        lv = self._empty((self.H, self.W, self.L), self._torch.int32)
        _ck(lib().dm_get_duals(self._h, lh.data_ptr(), lv.data_ptr()), "dm_get_duals")
        return lh, lv

    def cost(self):
        c = self._empty((self.H, self.W, self.L), self._torch.uint8)
        wh = self._empty((self.H, self.W), self._torch.uint8)
        wv = self._empty((self.H, self.W), self._torch.uint8)
        _ck(lib().dm_get_cost_volume(self._h, c.data_ptr(), wh.data_ptr(), wv.data_ptr()),
            "dm_get_cost_volume")
        return c, wh, wv

    def lower_bounds(self, n: int):
        lb = np.zeros(n, dtype=np.int64)
        _ck(lib().dm_get_lower_bounds(self._h, lb.ctypes.data, n), "dm_get_lower_bounds")
        return lb

    def energy(self) -> float:
        e = ctypes.c_double()
        _ck(lib().dm_energy(self._h, ctypes.byref(e)), "dm_energy")
        return e.value

    def launch_count(self) -> int:
        n = ctypes.c_uint64()
        _ck(lib().dm_launch_count(self._h, ctypes.byref(n)), "dm_launch_count")
        return n.value

    def sync(self):
        _ck(lib().dm_sync(self._h), "dm_sync")


def discrete_pass_noalloc(params: DmParams, which: int, cost, wedge, lam_in, lam_out,
                          err=None, stream=None):
    """dm_discrete_pass_noalloc: one Dual MM pass with no workspace and no
    allocation inside the library (inputs/outputs are caller tensors)."""
    H, W, L = lam_in.shape
    st = stream.cuda_stream if stream is not None else None
    _ck(lib().dm_discrete_pass_noalloc(H, W, L, ctypes.byref(params), int(which), _ptr(cost),
                                       _ptr(wedge), _ptr(lam_in), _ptr(lam_out), _ptr(err),
                                       _vp(st) if st else None),
        "dm_discrete_pass_noalloc")


def labels_u16(t) -> np.ndarray:
    """int16 tensor holding uint16 labels -> numpy uint16."""
    return t.cpu().numpy().view(np.uint16)
