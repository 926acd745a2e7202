"""ctypes binding of liblfbp.so (include/lfbp.h): argument marshalling only.

Every step of H -> H' runs in the CUDA library; this module converts torch
tensors to device pointers and streams, and turns error codes into
exceptions.  There is no fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import torch

from . import build as _build

F32, F16 = 0, 1
MAP_TRANSPOSE, MAP_PAPER_WINDOW = 0, 1

ERRORS = {
    -1: "LFBP_ERR_BAD_SHAPE", -2: "LFBP_ERR_NULL", -3: "LFBP_ERR_ALIGN", -4: "LFBP_ERR_ALIAS",
    -5: "LFBP_ERR_DTYPE", -6: "LFBP_ERR_CUDA", -7: "LFBP_ERR_TIMEOUT", -8: "LFBP_ERR_NOMEM",
    -9: "LFBP_ERR_INVALID",
}

# name -> (argtypes, restype), mirroring include/lfbp.h
_P, _I, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "lfbp_plan_create": ([ctypes.POINTER(_P), _I, _I, _P, _I, _I], _I),
    "lfbp_plan_create2": ([ctypes.POINTER(_P), _I, _I, _I, _P, _P, _I, _I], _I),
    "lfbp_plan_destroy": ([_P], None),
    "lfbp_plan_elems": ([_P], _S),
    "lfbp_plan_depth_offset": ([_P, _I], _S),
    "lfbp_plan_esize": ([_P], _I),
    "lfbp_plan_partition": ([_P, _I, _I, _P, _P], _I),
    "lfbp_backproject_array": ([_P, _P, _P, _P], _I),
    "lfbp_backproject_array_host": ([_P, _P, _P, _P, _P, _P], _I),
    "lfbp_backproject_batched": ([_I, _P, _P, _P, _P], _I),
    "lfbp_adjoint": ([_P, _P, _P, _P], _I),
    "lfbp_tune_batched": ([_I, _P, _P, _P, _P, _I, _P], _I),
    "lfbp_backproject_batched_noalloc": ([_I, _P, _P, _P, _P], _I),
    "lfbp_backproject_volume": ([_P, _P, _P, _I, _I, _P, _P], _I),
    "lfbp_forward_project": ([_P, _P, _P, _I, _I, _P, _P], _I),
    "lfbp_backproject_volume_grad": ([_P, _P, _P, _I, _I, _P, _P], _I),
    "lfbp_backproject_volume_from_h": ([_P, _P, _P, _I, _I, _P, _P], _I),
    "lfbp_rl_step": ([_P, _P, _P, _P, _P, _I, _I, _P, _P, _P, _P], _I),
    "lfbp_rl_step_fused": ([_P, _P, _P, _P, _I, _I, _P, _P, _P, _P], _I),
    "lfbp_rl_normaliser": ([_P, _P, _P, _I, _I, _P, _P, _P], _I),
    "lfbp_sync_status": ([_P], _I),
    "lfbp_last_error": ([], ctypes.c_char_p),
    "lfbp_version": ([], ctypes.c_char_p),
}

_lib = None


class LfbpError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = _lib.lfbp_last_error().decode() if _lib is not None else ""
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({msg})")
        self.code = code


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblfbp.so (optionally building it first); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    check = os.environ.get("LFBP_CHECK", "") == "1"  # the self-checking build
    path = _build.LIB_CHECK if check else _build.LIB
    if build_if_missing:
        path = _build.build(check=check)
    if not os.path.exists(path):
        raise RuntimeError(
            f"lfbp CUDA library not built ({path} missing); run "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise LfbpError(rc, what)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """Shape of one ragged PSF array (a handle of ``lfbp_plan``).

    Nx, Ny: cell sizes (odd); Ks, Kt: per-depth cut-out sizes (odd);
    dtype: torch.float32 or torch.float16; mode: MAP_TRANSPOSE (default)
    or MAP_PAPER_WINDOW.
    """

    def __init__(self, Nx: int, Ny: int, Ks: Sequence[int], Kt: Sequence[int] = None,
                 dtype=torch.float32, mode: int = MAP_TRANSPOSE):
        lib = load()
        Kt = Ks if Kt is None else Kt
        if len(Ks) != len(Kt):
            raise ValueError("Ks and Kt must have the same length")
        self.Nx, self.Ny = int(Nx), int(Ny)
        self.Ks, self.Kt = [int(k) for k in Ks], [int(k) for k in Kt]
        self.Nz = len(self.Ks)
        self.dtype = dtype
        self.mode = int(mode)
        dt = {torch.float32: F32, torch.float16: F16}.get(dtype)
        if dt is None:
            raise ValueError(f"unsupported dtype {dtype}")
        ks = (ctypes.c_int * max(1, self.Nz))(*self.Ks)
        kt = (ctypes.c_int * max(1, self.Nz))(*self.Kt)
        h = _P()
        self._h = None
        _check(lib.lfbp_plan_create2(ctypes.byref(h), self.Nx, self.Ny, self.Nz,
                                     ctypes.cast(ks, _P), ctypes.cast(kt, _P), dt, self.mode),
               "lfbp_plan_create2")
        self._h = h
        self._lib = lib

    @property
    def handle(self):
        return self._h

    @property
    def elems(self) -> int:
        return int(self._lib.lfbp_plan_elems(self._h))

    @property
    def esize(self) -> int:
        return int(self._lib.lfbp_plan_esize(self._h))

    @property
    def nbytes(self) -> int:
        return self.elems * self.esize

    def depth_offset(self, z: int) -> int:
        return int(self._lib.lfbp_plan_depth_offset(self._h, int(z)))

    def partition(self, nparts: int, part: int):
        """Depth range [z0, z1) of part `part` of `nparts` (``lfbp_plan_partition``)."""
        z0, z1 = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lfbp_plan_partition(self._h, int(nparts), int(part), ctypes.byref(z0),
                                             ctypes.byref(z1)), "lfbp_plan_partition")
        return int(z0.value), int(z1.value)

    def sub_plan(self, z0: int, z1: int) -> "Plan":
        """A plan of depths z0 .. z1-1 alone; its arrays are the slice
        [depth_offset(z0), depth_offset(z1)) of this plan's arrays."""
        return Plan(self.Nx, self.Ny, self.Ks[z0:z1], self.Kt[z0:z1], self.dtype, self.mode)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.lfbp_plan_destroy(h)
            self._h = None


def _check_tensor(plan: Plan, t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != plan.dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, plan expects {plan.dtype}")
    if t.numel() != plan.elems:
        raise ValueError(f"{name} has {t.numel()} elements, plan expects {plan.elems}")


def backproject_array(plan: Plan, H: torch.Tensor, out: torch.Tensor = None, stream=None):
    """H -> H' with one launch per depth (``lfbp_backproject_array``)."""
    _check_tensor(plan, H, "H")
    if out is None:
        out = torch.empty_like(H)
    _check_tensor(plan, out, "out")
    with torch.cuda.device(H.device):
        _check(plan._lib.lfbp_backproject_array(plan.handle, H.data_ptr(), out.data_ptr(),
                                                _stream_ptr(stream)), "lfbp_backproject_array")
    return out


def backproject_array_host(plan: Plan, H_host: torch.Tensor, out_host: torch.Tensor = None,
                           work=None, stream=None):
    """H -> H' from host to host with copies overlapping the map (``lfbp_backproject_array_host``).

    ``H_host`` should be a pinned CPU tensor; ``work`` = (dH, dHp) device tensors
    of the plan's size (allocated on the current device when omitted).
    """
    if not isinstance(H_host, torch.Tensor) or H_host.is_cuda:
        raise ValueError("H_host must be a CPU tensor")
    if H_host.dtype != plan.dtype or H_host.numel() != plan.elems or not H_host.is_contiguous():
        raise ValueError("H_host does not match the plan")
    if out_host is None:
        out_host = torch.empty_like(H_host, pin_memory=H_host.is_pinned())
    if work is None:
        work = (torch.empty(plan.elems, dtype=plan.dtype, device="cuda"),
                torch.empty(plan.elems, dtype=plan.dtype, device="cuda"))
    dH, dHp = work
    _check_tensor(plan, dH, "dH_work")
    _check_tensor(plan, dHp, "dHp_work")
    with torch.cuda.device(dH.device):
        _check(plan._lib.lfbp_backproject_array_host(plan.handle, H_host.data_ptr(),
                                                     out_host.data_ptr(), dH.data_ptr(),
                                                     dHp.data_ptr(), _stream_ptr(stream)),
               "lfbp_backproject_array_host")
    return out_host


def backproject_batched(plans: Sequence[Plan], Hs: Sequence[torch.Tensor],
                        outs: Sequence[torch.Tensor] = None, stream=None):
    """H -> H' for several arrays in one persistent launch (``lfbp_backproject_batched``)."""
    n = len(plans)
    if len(Hs) != n:
        raise ValueError("one input per plan")
    if outs is None:
        outs = [torch.empty_like(h) for h in Hs]
    for p, h, o in zip(plans, Hs, outs):
        _check_tensor(p, h, "H")
        _check_tensor(p, o, "out")
    lib = load()
    hp = (_P * max(1, n))(*[p.handle for p in plans])
    ip = (_P * max(1, n))(*[h.data_ptr() for h in Hs])
    op = (_P * max(1, n))(*[o.data_ptr() for o in outs])
    dev = Hs[0].device if n else torch.device("cuda")
    with torch.cuda.device(dev):
        _check(lib.lfbp_backproject_batched(n, ctypes.cast(hp, _P), ctypes.cast(ip, _P),
                                            ctypes.cast(op, _P), _stream_ptr(stream)),
               "lfbp_backproject_batched")
    return outs


def tune_batched(plans: Sequence[Plan], Hs: Sequence[torch.Tensor],
                 outs: Sequence[torch.Tensor] = None, reps: int = 3, stream=None):
    """Pick the fastest batched launch shape for these plans (``lfbp_tune_batched``).

    Returns (tile_bytes, ctas_per_sm, stages, pair_consumer, form), form 0 for
    persistent CTAs and 1 for one tile per CTA; later ``backproject_batched``
    calls with the same plans use it.
    """
    n = len(plans)
    if outs is None:
        outs = [torch.empty_like(h) for h in Hs]
    for p, h, o in zip(plans, Hs, outs):
        _check_tensor(p, h, "H")
        _check_tensor(p, o, "out")
    lib = load()
    hp = (_P * max(1, n))(*[p.handle for p in plans])
    ip = (_P * max(1, n))(*[h.data_ptr() for h in Hs])
    op = (_P * max(1, n))(*[o.data_ptr() for o in outs])
    res = (ctypes.c_int * 5)()
    with torch.cuda.device(Hs[0].device):
        _check(lib.lfbp_tune_batched(n, ctypes.cast(hp, _P), ctypes.cast(ip, _P), ctypes.cast(op, _P),
                                     _stream_ptr(stream), int(reps), ctypes.cast(res, _P)),
               "lfbp_tune_batched")
    return tuple(res)


def adjoint(plan: Plan, dHp: torch.Tensor, out: torch.Tensor = None, stream=None):
    """Gradient w.r.t. H from a gradient w.r.t. H' (``lfbp_adjoint``)."""
    _check_tensor(plan, dHp, "dHp")
    if out is None:
        out = torch.empty_like(dHp)
    _check_tensor(plan, out, "out")
    with torch.cuda.device(dHp.device):
        _check(plan._lib.lfbp_adjoint(plan.handle, dHp.data_ptr(), out.data_ptr(),
                                      _stream_ptr(stream)), "lfbp_adjoint")
    return out


def _check_f32(t: torch.Tensor, shape, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def backproject_volume(plan: Plan, Hp: torch.Tensor, f: torch.Tensor, out: torch.Tensor = None,
                       stream=None):
    """g = H' f on a finite sensor (``lfbp_backproject_volume``): f [Wx, Wy] -> g [Nz, Wx, Wy]."""
    _check_tensor(plan, Hp, "Hp")
    Wx, Wy = f.shape
    _check_f32(f, (Wx, Wy), "f")
    if out is None:
        out = torch.empty((plan.Nz, Wx, Wy), dtype=torch.float32, device=f.device)
    _check_f32(out, (plan.Nz, Wx, Wy), "out")
    with torch.cuda.device(f.device):
        _check(plan._lib.lfbp_backproject_volume(plan.handle, Hp.data_ptr(), f.data_ptr(), Wx, Wy,
                                                 out.data_ptr(), _stream_ptr(stream)),
               "lfbp_backproject_volume")
    return out


def forward_project(plan: Plan, H: torch.Tensor, g: torch.Tensor, out: torch.Tensor = None,
                    stream=None):
    """f = H g, Eq. (1) (``lfbp_forward_project``): g [Nz, Wx, Wy] -> f [Wx, Wy]."""
    _check_tensor(plan, H, "H")
    Nz, Wx, Wy = g.shape
    _check_f32(g, (plan.Nz, Wx, Wy), "g")
    if out is None:
        out = torch.empty((Wx, Wy), dtype=torch.float32, device=g.device)
    _check_f32(out, (Wx, Wy), "out")
    with torch.cuda.device(g.device):
        _check(plan._lib.lfbp_forward_project(plan.handle, H.data_ptr(), g.data_ptr(), Wx, Wy,
                                              out.data_ptr(), _stream_ptr(stream)),
               "lfbp_forward_project")
    return out


def backproject_volume_grad(plan: Plan, f: torch.Tensor, grad_g: torch.Tensor,
                            out: torch.Tensor = None, stream=None):
    """dL/dH' from dL/dg for g = H' f (``lfbp_backproject_volume_grad``)."""
    Wx, Wy = f.shape
    _check_f32(f, (Wx, Wy), "f")
    _check_f32(grad_g, (plan.Nz, Wx, Wy), "grad_g")
    if out is None:
        out = torch.empty(plan.elems, dtype=torch.float32, device=f.device)
    _check_tensor(plan, out, "out")
    with torch.cuda.device(f.device):
        _check(plan._lib.lfbp_backproject_volume_grad(plan.handle, f.data_ptr(), grad_g.data_ptr(),
                                                      Wx, Wy, out.data_ptr(), _stream_ptr(stream)),
               "lfbp_backproject_volume_grad")
    return out


def backproject_volume_from_h(plan: Plan, H: torch.Tensor, f: torch.Tensor,
                              out: torch.Tensor = None, stream=None):
    """g = H' f read straight from H, H' never built (``lfbp_backproject_volume_from_h``)."""
    _check_tensor(plan, H, "H")
    Wx, Wy = f.shape
    _check_f32(f, (Wx, Wy), "f")
    if out is None:
        out = torch.empty((plan.Nz, Wx, Wy), dtype=torch.float32, device=f.device)
    _check_f32(out, (plan.Nz, Wx, Wy), "out")
    with torch.cuda.device(f.device):
        _check(plan._lib.lfbp_backproject_volume_from_h(plan.handle, H.data_ptr(), f.data_ptr(),
                                                        Wx, Wy, out.data_ptr(),
                                                        _stream_ptr(stream)),
               "lfbp_backproject_volume_from_h")
    return out


def rl_normaliser(plan: Plan, H: torch.Tensor, Hp: torch.Tensor = None, Wx: int = None,
                  Wy: int = None, out: torch.Tensor = None, work: torch.Tensor = None,
                  stream=None):
    """H' 1 on a Wx x Wy sensor (``lfbp_rl_normaliser``); with Hp None, from H directly."""
    _check_tensor(plan, H, "H")
    if Hp is not None:
        _check_tensor(plan, Hp, "Hp")
    dev = H.device
    if out is None:
        out = torch.empty((plan.Nz, Wx, Wy), dtype=torch.float32, device=dev)
    _check_f32(out, (plan.Nz, Wx, Wy), "out")
    if work is None:
        work = torch.empty((Wx, Wy), dtype=torch.float32, device=dev)
    _check_f32(work, (Wx, Wy), "work")
    with torch.cuda.device(dev):
        _check(plan._lib.lfbp_rl_normaliser(plan.handle, H.data_ptr(),
                                            Hp.data_ptr() if Hp is not None else None, Wx, Wy,
                                            out.data_ptr(), work.data_ptr(), _stream_ptr(stream)),
               "lfbp_rl_normaliser")
    return out


def rl_step(plan: Plan, H: torch.Tensor, Hp: torch.Tensor, norm: torch.Tensor, f: torch.Tensor,
            g: torch.Tensor, out: torch.Tensor = None, work: torch.Tensor = None, stream=None):
    """One Richardson-Lucy update, Eq. (2) (``lfbp_rl_step``; with Hp None
    ``lfbp_rl_step_fused``, H' never built).  ``out`` may be ``g`` itself."""
    _check_tensor(plan, H, "H")
    Wx, Wy = f.shape
    _check_f32(f, (Wx, Wy), "f")
    _check_f32(g, (plan.Nz, Wx, Wy), "g")
    _check_f32(norm, (plan.Nz, Wx, Wy), "norm")
    if out is None:
        out = torch.empty_like(g)
    _check_f32(out, (plan.Nz, Wx, Wy), "out")
    if work is None:
        work = torch.empty((Wx, Wy), dtype=torch.float32, device=f.device)
    _check_f32(work, (Wx, Wy), "work")
    with torch.cuda.device(f.device):
        if Hp is not None:
            _check_tensor(plan, Hp, "Hp")
            _check(plan._lib.lfbp_rl_step(plan.handle, H.data_ptr(), Hp.data_ptr(),
                                          norm.data_ptr(), f.data_ptr(), Wx, Wy, g.data_ptr(),
                                          out.data_ptr(), work.data_ptr(), _stream_ptr(stream)),
                   "lfbp_rl_step")
        else:
            _check(plan._lib.lfbp_rl_step_fused(plan.handle, H.data_ptr(), norm.data_ptr(),
                                                f.data_ptr(), Wx, Wy, g.data_ptr(),
                                                out.data_ptr(), work.data_ptr(),
                                                _stream_ptr(stream)),
                   "lfbp_rl_step_fused")
    return out


def sync_status(stream=None):
    """Synchronise the stream and raise if an in-kernel wait timed out."""
    _check(load().lfbp_sync_status(_stream_ptr(stream)), "lfbp_sync_status")
