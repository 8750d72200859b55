"""Thin ctypes binding of libnufft_radon (include/nufft_radon.h).

Argument marshalling only: every step of the Radon operators and of MBIR runs
in the CUDA library.  Tensors are torch CUDA float32, contiguous; torch supplies
device memory and the current stream.  If the library cannot be loaded the
calls raise -- there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import torch

from . import build as _build

_LIB = None

TC_OK = 0
_STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
           -4: "device wait timed out", -5: "unsupported parameters"}


class TcError(RuntimeError):
    def __init__(self, fn, code, detail=""):
        super().__init__(f"{fn} failed: {_STATUS.get(code, code)} ({code}) {detail}".strip())
        self.code = code


class _Geom(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_det", ctypes.c_int),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("oversample", ctypes.c_int),
                ("kernel_width", ctypes.c_int), ("center_offset", ctypes.c_double)]


class _Prior(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double), ("sigma", ctypes.c_double), ("c", ctypes.c_double),
                ("lam", ctypes.c_double), ("dims", ctypes.c_int)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("step", ctypes.c_double), ("restart", ctypes.c_int),
                ("normal", ctypes.c_int), ("power_iter", ctypes.c_int)]


class _SolveState(ctypes.Structure):
    _fields_ = [("z", ctypes.c_void_p), ("g", ctypes.c_void_p), ("t", ctypes.c_double),
                ("k", ctypes.c_int), ("n_restarts", ctypes.c_int),
                ("obj", ctypes.c_double * 2), ("atb", ctypes.c_void_p), ("step", ctypes.c_double),
                ("dots", ctypes.c_double * 2)]


# every symbol the C header declares
SYMBOLS = ("tc_status_string", "tc_last_error_detail", "tc_plan_create", "tc_plan_destroy",
           "tc_plan_device_bytes", "radon_fwd", "radon_adj", "mbir_grad",
           "mbir_power_norm", "mbir_solve", "mbir_solve_host", "tc_profile_enable",
           "tc_profile_collect", "tc_profile_kernel_name", "tc_launch_count",
           "tc_plan_autotune", "tc_plan_set_launch", "tc_prior_grad_noalloc",
           "tc_plan_status", "tc_selftest_wait_timeout", "radon_normal", "tc_plan_prepare_normal",
           "tc_checkpoint_save", "tc_checkpoint_load", "tc_test_fail_copy_after",
           "tc_plan_group_create", "tc_plan_group_destroy", "tc_plan_group_device_bytes",
           "radon_fwd_group", "radon_adj_group", "mbir_grad_group", "tc_plan_set_spread_chunk",
           "tc_plan_get_spread_chunk", "tc_plan_autotune_spread", "tc_sfu_throughput")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first if asked)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libnufft_radon not found at {path}; run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.tc_status_string.argtypes = [i]
    L.tc_status_string.restype = ctypes.c_char_p
    L.tc_last_error_detail.argtypes = []
    L.tc_last_error_detail.restype = ctypes.c_char_p
    L.tc_plan_create.argtypes = [ctypes.POINTER(_Geom), i, ctypes.POINTER(vp)]
    L.tc_plan_destroy.argtypes = [vp]
    L.tc_plan_device_bytes.argtypes = [vp]
    L.tc_plan_device_bytes.restype = ctypes.c_longlong
    L.radon_fwd.argtypes = [vp, vp, vp, i, vp]
    L.radon_adj.argtypes = [vp, vp, vp, i, vp]
    L.mbir_grad.argtypes = [vp, vp, vp, vp, ctypes.POINTER(_Prior), vp, vp, i, vp]
    L.mbir_power_norm.argtypes = [vp, vp, vp, vp, i, i, ctypes.POINTER(d), vp]
    L.mbir_solve.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(_Prior),
                             ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveState), vp]
    L.mbir_solve_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, ctypes.POINTER(_Prior),
                                  ctypes.POINTER(_SolveOpts), ctypes.POINTER(_SolveState), vp]
    L.tc_profile_enable.argtypes = [i]
    L.tc_profile_collect.argtypes = [i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d)]
    L.tc_profile_kernel_name.argtypes = [i]
    L.tc_profile_kernel_name.restype = ctypes.c_char_p
    L.tc_launch_count.argtypes = []
    L.tc_launch_count.restype = ctypes.c_longlong
    L.tc_plan_autotune.argtypes = [vp, vp, vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), vp]
    L.tc_plan_set_launch.argtypes = [vp, i, i]
    L.tc_prior_grad_noalloc.argtypes = [vp, vp, i, i, ctypes.POINTER(_Prior), vp, vp]
    L.tc_plan_status.argtypes = [vp]
    L.tc_selftest_wait_timeout.argtypes = [vp]
    L.radon_normal.argtypes = [vp, vp, vp, i, vp]
    L.tc_plan_prepare_normal.argtypes = [vp, vp]
    L.tc_checkpoint_save.argtypes = [ctypes.c_char_p, vp, vp, i, ctypes.POINTER(_SolveState), vp]
    L.tc_checkpoint_load.argtypes = [ctypes.c_char_p, vp, vp, i, ctypes.POINTER(_SolveState), vp]
    L.tc_test_fail_copy_after.argtypes = [i]
    L.tc_plan_group_create.argtypes = [ctypes.POINTER(_Geom), ctypes.POINTER(i), i, ctypes.POINTER(vp)]
    L.tc_plan_group_destroy.argtypes = [vp]
    L.tc_plan_group_device_bytes.argtypes = [vp]
    L.tc_plan_group_device_bytes.restype = ctypes.c_longlong
    L.radon_fwd_group.argtypes = [vp, vp, vp, vp]
    L.radon_adj_group.argtypes = [vp, vp, vp, vp]
    L.mbir_grad_group.argtypes = [vp, vp, vp, vp, ctypes.POINTER(_Prior), vp, vp, vp]
    L.tc_plan_set_spread_chunk.argtypes = [vp, i]
    L.tc_plan_get_spread_chunk.argtypes = [vp]
    L.tc_plan_autotune_spread.argtypes = [vp, vp, vp, i, i, ctypes.POINTER(i), vp]
    L.tc_sfu_throughput.argtypes = [i, ctypes.POINTER(d), vp]
    for fn in ("tc_profile_enable", "tc_profile_collect", "tc_plan_create", "tc_plan_destroy",
               "radon_fwd", "radon_adj", "mbir_grad", "mbir_power_norm", "mbir_solve",
               "mbir_solve_host", "tc_plan_autotune", "tc_plan_set_launch",
               "tc_prior_grad_noalloc", "radon_normal", "tc_plan_prepare_normal",
               "tc_checkpoint_save", "tc_checkpoint_load", "tc_test_fail_copy_after",
           "tc_plan_group_create", "tc_plan_group_destroy", "tc_plan_group_device_bytes",
           "radon_fwd_group", "radon_adj_group", "mbir_grad_group", "tc_plan_set_spread_chunk",
           "tc_plan_get_spread_chunk", "tc_plan_autotune_spread", "tc_sfu_throughput"):
        getattr(L, fn).restype = i
    _LIB = L
    return L


def _check(fn, rc):
    if rc != TC_OK:
        detail = load().tc_last_error_detail().decode()
        raise TcError(fn, rc, detail)


def _stream(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


@dataclass
class Prior:
    """qGGMRF prior parameters (Sec. 3 Eqs. reg2/reg3; defaults from Sec. 5)."""
    p: float = 1.2
    sigma: float = 1.0 / 0.7
    c: float = 1e-4
    lam: float = 1.0
    dims: int = 2

    def _c(self):
        return _Prior(self.p, self.sigma, self.c, self.lam, self.dims)


class Plan:
    """Geometry + tables + scratch for max_batch slices per launch (tc_plan_create)."""

    def __init__(self, n, n_angles, n_det, angles=None, oversample=2, kernel_width=7,
                 max_batch=1, device=None, center_offset=0.0):
        L = load()
        self.n, self.n_angles, self.n_det = int(n), int(n_angles), int(n_det)
        self.kernel_width, self.max_batch = int(kernel_width), int(max_batch)
        self.center_offset = float(center_offset)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self._angles = None
        aptr = ctypes.POINTER(ctypes.c_double)()
        if angles is not None:
            import numpy as np
            self._angles = np.ascontiguousarray(angles, dtype=np.float64)
            assert self._angles.shape == (self.n_angles,)
            aptr = self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        g = _Geom(self.n, self.n_angles, self.n_det, aptr, int(oversample), self.kernel_width,
                  self.center_offset)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check("tc_plan_create", L.tc_plan_create(ctypes.byref(g), self.max_batch, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    @property
    def device_bytes(self) -> int:
        return int(load().tc_plan_device_bytes(self.handle))

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().tc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def autotune(self, batch=None, reps=2, stream=None):
        """Pick slices per launch and column pairs per CTA by timing (tc_plan_autotune).

        Uses scratch buffers of `batch` slices (default max_batch); returns (chunk, col_pairs)."""
        B = self.max_batch if batch is None else int(batch)
        x = torch.rand(self.image_shape(B), device=self.device)
        y = torch.empty(self.sino_shape(B), device=self.device)
        ch, cp = ctypes.c_int(), ctypes.c_int()
        _check("tc_plan_autotune", load().tc_plan_autotune(self.handle, _ptr(x), _ptr(y), B, int(reps),
                                                           ctypes.byref(ch), ctypes.byref(cp),
                                                           _stream(stream, self.device)))
        return ch.value, cp.value

    def prepare_normal(self, stream=None):
        """Build the spectra of radon_normal's Toeplitz-plus-Hankel kernels now
        (otherwise the first radon_normal call does; needed before graph capture)."""
        _check("tc_plan_prepare_normal", load().tc_plan_prepare_normal(self.handle,
                                                                       _stream(stream, self.device)))

    @property
    def spread_chunk(self) -> int:
        """Entries per spreading chunk of A^T (256, 512 or 1024)."""
        return int(load().tc_plan_get_spread_chunk(self.handle))

    @spread_chunk.setter
    def spread_chunk(self, entries):
        _check("tc_plan_set_spread_chunk", load().tc_plan_set_spread_chunk(self.handle, int(entries)))

    def autotune_spread(self, batch=None, reps=2, stream=None) -> int:
        """Pick the spreading chunk by timing radon_adj (tc_plan_autotune_spread)."""
        B = self.max_batch if batch is None else int(batch)
        y = torch.rand(self.sino_shape(B), device=self.device)
        x = torch.empty(self.image_shape(B), device=self.device)
        ch = ctypes.c_int()
        _check("tc_plan_autotune_spread", load().tc_plan_autotune_spread(self.handle, _ptr(y), _ptr(x), B, int(reps),
                                                                         ctypes.byref(ch),
                                                                         _stream(stream, self.device)))
        return ch.value

    def set_launch(self, chunk, col_pairs=0):
        """Slices per launch (1..max_batch) and column pairs per CTA (1, 2, 4; 0 keeps)."""
        _check("tc_plan_set_launch", load().tc_plan_set_launch(self.handle, int(chunk), int(col_pairs)))

    def image_shape(self, batch):
        return (batch, self.n, self.n)

    def sino_shape(self, batch):
        return (batch, self.n_angles, self.n_det)


class PlanGroup:
    """Several geometries in one batch (tc_plan_group_create): geoms is a list of
    (n, n_angles, n_det) or dicts with the Plan keywords; counts the slices of
    each.  Arrays are the geometries' slices concatenated in that order
    (flat float32 CUDA tensors, see image_numel / sino_numel)."""

    def __init__(self, geoms, counts, device=None):
        L = load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self._keep = []
        cg = (_Geom * len(geoms))()
        self.geoms = []
        for k, gm in enumerate(geoms):
            d = dict(gm) if isinstance(gm, dict) else dict(zip(("n", "n_angles", "n_det"), gm))
            aptr = ctypes.POINTER(ctypes.c_double)()
            if d.get("angles") is not None:
                import numpy as np
                arr = np.ascontiguousarray(d["angles"], dtype=np.float64)
                self._keep.append(arr)
                aptr = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            cg[k] = _Geom(int(d["n"]), int(d["n_angles"]), int(d["n_det"]), aptr, int(d.get("oversample", 2)),
                          int(d.get("kernel_width", 7)), float(d.get("center_offset", 0.0)))
            self.geoms.append((int(d["n"]), int(d["n_angles"]), int(d["n_det"])))
        self.counts = [int(c) for c in counts]
        cc = (ctypes.c_int * len(self.counts))(*self.counts)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check("tc_plan_group_create", L.tc_plan_group_create(cg, cc, len(self.geoms), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan group is closed")
        return self._h

    @property
    def image_numel(self):
        return sum(c * n * n for (n, _, _), c in zip(self.geoms, self.counts))

    @property
    def sino_numel(self):
        return sum(c * a * d for (_, a, d), c in zip(self.geoms, self.counts))

    def split_images(self, flat):
        """Views [counts[i], N_i, N_i] of a concatenated image array."""
        out, o = [], 0
        for (n, _, _), c in zip(self.geoms, self.counts):
            out.append(flat[o:o + c * n * n].view(c, n, n))
            o += c * n * n
        return out

    def split_sinos(self, flat):
        out, o = [], 0
        for (_, a, d), c in zip(self.geoms, self.counts):
            out.append(flat[o:o + c * a * d].view(c, a, d))
            o += c * a * d
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().tc_plan_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _need_flat(t, numel, name, device):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of {numel} elements")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, group is on {device}")


def radon_fwd_group(group: PlanGroup, x, y=None, stream=None):
    """y = A x for every slice of the group (concatenated layouts)."""
    _need_flat(x, group.image_numel, "x", group.device)
    if y is None:
        y = torch.empty(group.sino_numel, device=group.device, dtype=torch.float32)
    _need_flat(y, group.sino_numel, "y", group.device)
    _check("radon_fwd_group", load().radon_fwd_group(group.handle, _ptr(x), _ptr(y), _stream(stream, group.device)))
    return y


def radon_adj_group(group: PlanGroup, y, x=None, stream=None):
    """x = A^T y for every slice of the group (concatenated layouts)."""
    _need_flat(y, group.sino_numel, "y", group.device)
    if x is None:
        x = torch.empty(group.image_numel, device=group.device, dtype=torch.float32)
    _need_flat(x, group.image_numel, "x", group.device)
    _check("radon_adj_group", load().radon_adj_group(group.handle, _ptr(y), _ptr(x), _stream(stream, group.device)))
    return x


def mbir_grad_group(group: PlanGroup, x, b, w=None, prior: Prior | None = None, grad=None, obj=None,
                    stream=None):
    """grad = A^T W (A x - b) + lam grad H(x) over the group; obj (device float64
    [n_geoms, 2]) = (data, lam H) per geometry."""
    _need_flat(x, group.image_numel, "x", group.device)
    _need_flat(b, group.sino_numel, "b", group.device)
    if w is not None:
        _need_flat(w, group.sino_numel, "w", group.device)
    if grad is None:
        grad = torch.empty_like(x)
    _need_flat(grad, group.image_numel, "grad", group.device)
    if obj is None:
        obj = torch.zeros((len(group.counts), 2), dtype=torch.float64, device=group.device)
    pr = prior._c() if prior is not None else None
    _check("mbir_grad_group", load().mbir_grad_group(group.handle, _ptr(x), _ptr(b), _ptr(w),
                                                     ctypes.byref(pr) if pr is not None else None,
                                                     _ptr(grad), _ptr(obj), _stream(stream, group.device)))
    return grad, obj


def _need(t, shape, name, device):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, plan is on {device}")


def _batch_of(t, trailing):
    """(batch, squeezed) for a tensor of shape trailing or (B,) + trailing."""
    shp = tuple(t.shape)
    if shp == tuple(trailing):
        return 1, True
    if len(shp) == len(trailing) + 1 and shp[1:] == tuple(trailing):
        return shp[0], False
    raise ValueError(f"tensor of shape {shp} does not match {tuple(trailing)} or (B,)+that")


def radon_fwd(plan: Plan, x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """y = A x (Sec. 2.2 NUFFT in reverse order).  x: [B,N,N] or [N,N]."""
    B, sq = _batch_of(x, plan.image_shape(1)[1:])
    xb = x.reshape(plan.image_shape(B))
    _need(xb, plan.image_shape(B), "x", plan.device)
    if y is None:
        y = torch.empty(plan.sino_shape(B), device=plan.device, dtype=torch.float32)
    yb = y.reshape(plan.sino_shape(B))
    _need(yb, plan.sino_shape(B), "y", plan.device)
    _check("radon_fwd", load().radon_fwd(plan.handle, _ptr(xb), _ptr(yb), B, _stream(stream, plan.device)))
    return y.reshape(plan.sino_shape(B)[1:]) if sq else y


def radon_adj(plan: Plan, y: torch.Tensor, x: torch.Tensor | None = None, stream=None):
    """x = A^T y (Sec. 3 Eq. transpose).  y: [B,A,D] or [A,D]."""
    B, sq = _batch_of(y, plan.sino_shape(1)[1:])
    yb = y.reshape(plan.sino_shape(B))
    _need(yb, plan.sino_shape(B), "y", plan.device)
    if x is None:
        x = torch.empty(plan.image_shape(B), device=plan.device, dtype=torch.float32)
    xb = x.reshape(plan.image_shape(B))
    _need(xb, plan.image_shape(B), "x", plan.device)
    _check("radon_adj", load().radon_adj(plan.handle, _ptr(yb), _ptr(xb), B, _stream(stream, plan.device)))
    return x.reshape(plan.image_shape(B)[1:]) if sq else x


def radon_normal(plan: Plan, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """out = A^T A x by Toeplitz-plus-Hankel embedding (no gridding).  x: [B,N,N] or [N,N]."""
    B, sq = _batch_of(x, plan.image_shape(1)[1:])
    xb = x.reshape(plan.image_shape(B))
    _need(xb, plan.image_shape(B), "x", plan.device)
    if out is None:
        out = torch.empty(plan.image_shape(B), device=plan.device, dtype=torch.float32)
    ob = out.reshape(plan.image_shape(B))
    _need(ob, plan.image_shape(B), "out", plan.device)
    _check("radon_normal", load().radon_normal(plan.handle, _ptr(xb), _ptr(ob), B, _stream(stream, plan.device)))
    return out.reshape(plan.image_shape(B)[1:]) if sq else out


def mbir_grad(plan: Plan, x, b, w=None, prior: Prior | None = None, grad=None, obj=None, stream=None):
    """grad = A^T W (A x - b) + lam grad H(x); obj (device float64 [2]) = (data, lam H)."""
    B = x.shape[0]
    _need(x, plan.image_shape(B), "x", plan.device)
    _need(b, plan.sino_shape(B), "b", plan.device)
    if w is not None:
        _need(w, plan.sino_shape(B), "w", plan.device)
    if grad is None:
        grad = torch.empty_like(x)
    _need(grad, plan.image_shape(B), "grad", plan.device)
    if obj is None:
        obj = torch.zeros(2, dtype=torch.float64, device=plan.device)
    pr = prior._c() if prior is not None else None
    _check("mbir_grad", load().mbir_grad(plan.handle, _ptr(x), _ptr(b), _ptr(w),
                                         ctypes.byref(pr) if pr is not None else None,
                                         _ptr(grad), _ptr(obj), B, _stream(stream, plan.device)))
    return grad, obj


def mbir_power_norm(plan: Plan, v, w=None, n_iter=30, work=None, stream=None) -> float:
    """Largest eigenvalue of A^T W A by power iteration from v (v is overwritten)."""
    B = v.shape[0]
    _need(v, plan.image_shape(B), "v", plan.device)
    if work is None:
        work = torch.empty_like(v)
    lam = ctypes.c_double()
    _check("mbir_power_norm", load().mbir_power_norm(plan.handle, _ptr(w), _ptr(v), _ptr(work), B,
                                                     int(n_iter), ctypes.byref(lam),
                                                     _stream(stream, plan.device)))
    return lam.value


class SolveState:
    """Resumable solver state: device z, g buffers plus FP64 scalars.

    step: the step the iteration used (the caller's, or the one the library
    derived on the first call when none was given)."""

    def __init__(self, x):
        self.z = torch.empty_like(x)
        self.g = torch.empty_like(x)
        self.t = 1.0
        self.k = 0
        self.n_restarts = 0
        self.obj = (0.0, 0.0)
        self.atb = None  # A^T b, allocated by a normal-operator solve
        self.step = 0.0
        self.dots = (0.0, 0.0)  # restart-test inner products of the last iteration

    def _c(self):
        s = _SolveState(self.z.data_ptr(), self.g.data_ptr(), self.t, self.k, self.n_restarts)
        s.obj[0], s.obj[1] = self.obj
        s.atb = self.atb.data_ptr() if self.atb is not None else None
        s.step = self.step
        return s

    def _load(self, s):
        # the solve may hand back z and g exchanged: s.z names the buffer of z_k
        if s.z != self.z.data_ptr():
            if s.z != self.g.data_ptr():
                raise RuntimeError("solver state: z points to neither of the state's buffers")
            self.z, self.g = self.g, self.z
        self.t, self.k, self.n_restarts = s.t, s.k, s.n_restarts
        self.obj = (s.obj[0], s.obj[1])
        self.step = s.step
        self.dots = (s.dots[0], s.dots[1])


def _restart_code(restart) -> int:
    """True -> 1 (gradient restart), False -> 0 (none), "monotone" -> 2."""
    if restart == "monotone":
        return 2
    if restart is True or restart is False:
        return 1 if restart else 0
    raise ValueError(f"restart must be True, False or 'monotone', not {restart!r}")


def mbir_solve(plan: Plan, b, w, x, n_iter, step=None, prior: Prior | None = None, restart=True,
               state: SolveState | None = None, stream=None, normal=False, power_iter=0) -> SolveState:
    """Run n_iter accelerated-gradient iterations on device buffers (x in/out).

    step: the constant step 1/L, or None for the library's own (a power
    iteration of power_iter steps, 0 = 30, on the first call; state.step then
    holds it and later calls with the same state reuse it).

    restart: True (gradient test), "monotone" (function-value test: Phi(x_k)
    never increases; state.obj is then the objective at the returned x) or
    False (plain momentum).
    normal: unweighted data term (w must be None) through the Toeplitz-plus-Hankel
    normal operator (radon_normal) instead of the gridded A and A^T."""
    B = x.shape[0]
    _need(x, plan.image_shape(B), "x", plan.device)
    _need(b, plan.sino_shape(B), "b", plan.device)
    if w is not None:
        _need(w, plan.sino_shape(B), "w", plan.device)
    st = state if state is not None else SolveState(x)
    if normal and st.atb is None:
        st.atb = torch.empty_like(x)
    cs = st._c()
    pr = prior._c() if prior is not None else None
    opts = _SolveOpts(int(n_iter), 0.0 if step is None else float(step), _restart_code(restart),
                      int(bool(normal)), int(power_iter))
    _check("mbir_solve", load().mbir_solve(plan.handle, _ptr(b), _ptr(w), _ptr(x), B,
                                           ctypes.byref(pr) if pr is not None else None,
                                           ctypes.byref(opts), ctypes.byref(cs),
                                           _stream(stream, plan.device)))
    st._load(cs)
    return st


def mbir_solve_host(plan: Plan, b_host, w_host, x_host, n_iter, step=None, prior: Prior | None = None,
                    restart=True, state: SolveState | None = None, dev=None, stream=None, normal=False,
                    power_iter=0):
    """End-to-end solve from host (ideally pinned) tensors: copies in, iterates, copies x back.

    dev: optional dict of reusable device buffers {"b", "w", "x"}.
    normal: as in mbir_solve (w_host must be None).
    """
    B = x_host.shape[0]
    for t, shp, nm in ((b_host, plan.sino_shape(B), "b_host"), (x_host, plan.image_shape(B), "x_host")):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"{nm} must be a contiguous host float32 tensor of shape {shp}")
    dev = dev if dev is not None else {}
    db = dev.setdefault("b", torch.empty(plan.sino_shape(B), device=plan.device))
    dx = dev.setdefault("x", torch.empty(plan.image_shape(B), device=plan.device))
    dw = None
    if w_host is not None:
        dw = dev.setdefault("w", torch.empty(plan.sino_shape(B), device=plan.device))
    st = state if state is not None else SolveState(dx)
    if normal and st.atb is None:
        st.atb = torch.empty_like(dx)
    cs = st._c()
    pr = prior._c() if prior is not None else None
    opts = _SolveOpts(int(n_iter), 0.0 if step is None else float(step), _restart_code(restart),
                      int(bool(normal)), int(power_iter))
    _check("mbir_solve_host", load().mbir_solve_host(
        plan.handle, _ptr(b_host), _ptr(w_host), _ptr(x_host), _ptr(db), _ptr(dw), _ptr(dx), B,
        ctypes.byref(pr) if pr is not None else None, ctypes.byref(opts), ctypes.byref(cs),
        _stream(stream, plan.device)))
    st._load(cs)
    return st


def checkpoint_save(path, plan: Plan, x, state: SolveState, stream=None):
    """Write x, state.z and the scalar state to `path` (tc_checkpoint_save)."""
    B = x.shape[0]
    _need(x, plan.image_shape(B), "x", plan.device)
    cs = state._c()
    _check("tc_checkpoint_save", load().tc_checkpoint_save(os.fsencode(path), plan.handle, _ptr(x), B,
                                                           ctypes.byref(cs), _stream(stream, plan.device)))


def checkpoint_load(path, plan: Plan, x, state: SolveState | None = None, stream=None) -> SolveState:
    """Read a checkpoint into x (device, [B,N,N]) and a state (tc_checkpoint_load)."""
    B = x.shape[0]
    _need(x, plan.image_shape(B), "x", plan.device)
    st = state if state is not None else SolveState(x)
    cs = st._c()
    _check("tc_checkpoint_load", load().tc_checkpoint_load(os.fsencode(path), plan.handle, _ptr(x), B,
                                                           ctypes.byref(cs), _stream(stream, plan.device)))
    st._load(cs)
    return st


def fail_copy_after(after: int):
    """Testing hook: the copy of mbir_solve_host after `after` more copies
    reports a CUDA failure instead of running (negative: off)."""
    _check("tc_test_fail_copy_after", load().tc_test_fail_copy_after(int(after)))


def sfu_throughput(op: str, device=None) -> float:
    """Lane operations per second of the special-function unit for op in
    ("lg2", "ex2", "rcp"), measured on the device (tc_sfu_throughput)."""
    code = {"lg2": 0, "ex2": 1, "rcp": 2}[op]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        _check("tc_sfu_throughput", load().tc_sfu_throughput(code, ctypes.byref(out),
                                                             _stream(None, dev)))
    return out.value


def profile_enable(on: bool = True):
    """Start (or stop) per-kernel event timing inside the library."""
    _check("tc_profile_enable", load().tc_profile_enable(1 if on else 0))


def profile_collect() -> dict:
    """{kernel name: (launches, summed ms)} for the launches since profile_enable."""
    L = load()
    n = 64
    counts = (ctypes.c_longlong * n)()
    ms = (ctypes.c_double * n)()
    k = L.tc_profile_collect(n, counts, ms)
    if k < 0:
        _check("tc_profile_collect", k)
    return {L.tc_profile_kernel_name(i).decode(): (int(counts[i]), float(ms[i]))
            for i in range(min(k, n)) if counts[i]}


def launch_count() -> int:
    """Kernel launches issued by the library since it was loaded."""
    return int(load().tc_launch_count())


class RadonFwd(torch.autograd.Function):
    """Differentiable y = A x whose backward is the hand-written A^T kernel."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return radon_fwd(plan, x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return radon_adj(ctx.plan, gy.contiguous()), None


def radon(x, plan):
    """Autograd entry: A x with gradient A^T (dL/dy)."""
    return RadonFwd.apply(x, plan)
