"""CPU oracle for the H -> H' backprojection-array construction -- TEST INFRASTRUCTURE.

Plain, slow, obviously correct statements of what the method computes
(arXiv 2003.09133), used only to check the CUDA path: the test-suite, the
smoke check and the benchmark's CPU-baseline leg may import this package;
the product library never does.  The arithmetic lives in ``lfbp_oracle.c``
(plain C, built with gcc); this module loads it with ctypes and adds the
small numpy constructions the oracle's own tests use as independent pins
(a dense measurement matrix built by pattern placement).

Each function names the passage it follows.  Layout of every array: flat,
depth-major, ragged; depth z is row-major [a][b][s][t] with
Nx*Ny*Ks[z]*Kt[z] elements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfbp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile lfbp_oracle.c into _build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_long
        for name, args in {
            "oracle_transpose": [P, P, I, I, I, I, P, P, I],
            "oracle_transpose_adjoint": [P, P, I, I, I, I, P, P, I],
            "oracle_paper_window": [P, P, I, I, I, I, P, P],
            "oracle_forward_f64": [P, I, I, I, P, P, P, I, I, P],
            "oracle_backproject_f64": [P, I, I, I, P, P, P, I, I, P],
            "oracle_backproject_points": [P, I, I, I, P, P, P, I, I, L, P, P, I],
            "oracle_grad_hp_f64": [P, P, I, I, I, P, P, I, I, P, I],
            "oracle_grad_hp_points": [P, P, I, I, I, P, P, I, I, L, P, P, I],
            "oracle_threads": [I],
        }.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ints(xs: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(xs, dtype=np.int32))


_CPU_SRC = os.path.join(_HERE, "lfbp_cpu_rearrange.c")
_CPU_LIB_PATH = os.path.join(_HERE, "_build", "libcpu_rearrange.so")
_cpu_lib = None


def build_cpu_baseline(force: bool = False) -> str:
    """Compile lfbp_cpu_rearrange.c into _build/libcpu_rearrange.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_CPU_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_CPU_LIB_PATH) or \
            os.path.getmtime(_CPU_LIB_PATH) < os.path.getmtime(_CPU_SRC):
        tmp = _CPU_LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _CPU_SRC])
        os.replace(tmp, _CPU_LIB_PATH)
    return _CPU_LIB_PATH


def cpu_rearrange(H: np.ndarray, Nx: int, Ny: int, Ks, Kt=None, nthreads: int = 0) -> np.ndarray:
    """The paper's closed-form rearrangement (Sec. 4) on the host cores: the CPU
    baseline the benchmark times beside the oracle (not part of the oracle;
    checked against ``transpose`` by the tests).  Odd cut-outs, 2- or 4-byte
    elements."""
    global _cpu_lib
    if _cpu_lib is None:
        lib = ctypes.CDLL(build_cpu_baseline())
        P, I = ctypes.c_void_p, ctypes.c_int
        lib.cpu_rearrange.argtypes = [P, P, I, I, I, I, P, P, I]
        lib.cpu_rearrange.restype = I
        lib.cpu_rearrange_threads.argtypes = [I]
        lib.cpu_rearrange_threads.restype = I
        _cpu_lib = lib
    Kt = Ks if Kt is None else Kt
    H = np.ascontiguousarray(H)
    out = np.empty_like(H)
    ks, kt = _ints(Ks), _ints(Kt)
    _check(_cpu_lib.cpu_rearrange(_ptr(H), _ptr(out), H.itemsize, Nx, Ny, len(ks), _ptr(ks),
                                  _ptr(kt), nthreads), "cpu_rearrange")
    return out


def cpu_rearrange_threads(n: int = 0) -> int:
    """Threads the CPU baseline uses (n > 0 sets it)."""
    cpu_rearrange(np.zeros(1, np.float32), 1, 1, [1], [1])  # loads the library
    return _cpu_lib.cpu_rearrange_threads(int(n))


def threads(n: int = 0) -> int:
    """Worker threads the oracle's OpenMP loops use (n > 0 sets it)."""
    return _load().oracle_threads(int(n))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def transpose(H: np.ndarray, Nx: int, Ny: int, Ks, Kt=None, nthreads: int = 0) -> np.ndarray:
    """H' as the transpose of the measurement operator of Eq. (1), pixel-centred.

    Element-for-element copy of raw bytes (any 1/2/4/8-byte dtype).
    """
    Kt = Ks if Kt is None else Kt
    H = np.ascontiguousarray(H)
    out = np.empty_like(H)
    ks, kt = _ints(Ks), _ints(Kt)
    _check(_load().oracle_transpose(_ptr(H), _ptr(out), H.itemsize, Nx, Ny, len(ks),
                                    _ptr(ks), _ptr(kt), nthreads), "oracle_transpose")
    return out


def transpose_adjoint(dHp: np.ndarray, Nx: int, Ny: int, Ks, Kt=None, nthreads: int = 0):
    """Adjoint (scatter back) of ``transpose``: gradient of a loss on H' w.r.t. H."""
    Kt = Ks if Kt is None else Kt
    dHp = np.ascontiguousarray(dHp)
    out = np.empty_like(dHp)
    ks, kt = _ints(Ks), _ints(Kt)
    _check(_load().oracle_transpose_adjoint(_ptr(dHp), _ptr(out), dHp.itemsize, Nx, Ny,
                                            len(ks), _ptr(ks), _ptr(kt), nthreads),
           "oracle_transpose_adjoint")
    return out


def paper_window(H: np.ndarray, Nx: int, Ny: int, Ks, Kt=None) -> np.ndarray:
    """Eqs. (4)-(9) with the paper's loop ranges (Sec. 4); unreached entries are 0."""
    Kt = Ks if Kt is None else Kt
    H = np.ascontiguousarray(H)
    out = np.empty_like(H)
    ks, kt = _ints(Ks), _ints(Kt)
    _check(_load().oracle_paper_window(_ptr(H), _ptr(out), H.itemsize, Nx, Ny, len(ks),
                                       _ptr(ks), _ptr(kt)), "oracle_paper_window")
    return out


def forward(H: np.ndarray, Nx, Ny, Ks, Kt, g: np.ndarray) -> np.ndarray:
    """f = H g, Eq. (1), FP64, on a finite sensor/volume; g is [Nz][Wx][Wy]."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    Nz, Wx, Wy = g.shape
    f = np.empty((Wx, Wy))
    ks, kt = _ints(Ks), _ints(Kt)
    _check(_load().oracle_forward_f64(_ptr(H), Nx, Ny, Nz, _ptr(ks), _ptr(kt), _ptr(g),
                                      Wx, Wy, _ptr(f)), "oracle_forward_f64")
    return f


def backproject(Hp: np.ndarray, Nx, Ny, Ks, Kt, f: np.ndarray) -> np.ndarray:
    """g = H' f (the backprojection of Eq. 2), FP64; returns [Nz][Wx][Wy]."""
    Hp = np.ascontiguousarray(Hp, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    Wx, Wy = f.shape
    ks, kt = _ints(Ks), _ints(Kt)
    g = np.empty((len(ks), Wx, Wy))
    _check(_load().oracle_backproject_f64(_ptr(Hp), Nx, Ny, len(ks), _ptr(ks), _ptr(kt),
                                          _ptr(f), Wx, Wy, _ptr(g)), "oracle_backproject_f64")
    return g


def backproject_points(Hp: np.ndarray, Nx, Ny, Ks, Kt, f: np.ndarray, pts: np.ndarray,
                       nthreads: int = 0) -> np.ndarray:
    """g = H' f at voxels pts[i] = (z, X, Y), each computed on its own, FP64."""
    Hp = np.ascontiguousarray(Hp, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    Wx, Wy = f.shape
    ks, kt = _ints(Ks), _ints(Kt)
    out = np.empty(len(pts))
    _check(_load().oracle_backproject_points(_ptr(Hp), Nx, Ny, len(ks), _ptr(ks), _ptr(kt),
                                             _ptr(f), Wx, Wy, len(pts), _ptr(pts), _ptr(out),
                                             nthreads), "oracle_backproject_points")
    return out


def grad_hp(f: np.ndarray, r: np.ndarray, Nx, Ny, Ks, Kt, nthreads: int = 0) -> np.ndarray:
    """dL/dH' for L = sum (H' f - g_ref)^2, given the residual r = 2 (H' f - g_ref)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    Nz, Wx, Wy = r.shape
    ks, kt = _ints(Ks), _ints(Kt)
    n = int(sum(Nx * Ny * a * b for a, b in zip(Ks, Kt)))
    out = np.empty(n)
    _check(_load().oracle_grad_hp_f64(_ptr(f), _ptr(r), Nx, Ny, Nz, _ptr(ks), _ptr(kt),
                                      Wx, Wy, _ptr(out), nthreads), "oracle_grad_hp_f64")
    return out


def grad_hp_points(f: np.ndarray, r: np.ndarray, Nx, Ny, Ks, Kt, pts: np.ndarray,
                   nthreads: int = 0) -> np.ndarray:
    """``grad_hp`` at entries pts[i] = (z, p, q, u, v), each computed on its own."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    Nz, Wx, Wy = r.shape
    ks, kt = _ints(Ks), _ints(Kt)
    out = np.empty(len(pts))
    _check(_load().oracle_grad_hp_points(_ptr(f), _ptr(r), Nx, Ny, Nz, _ptr(ks), _ptr(kt), Wx, Wy,
                                         len(pts), _ptr(pts), _ptr(out), nthreads),
           "oracle_grad_hp_points")
    return out


def rl_step(H: np.ndarray, Hp: np.ndarray, Nx, Ny, Ks, Kt, g: np.ndarray, f: np.ndarray,
            norm: np.ndarray = None) -> np.ndarray:
    """One Richardson-Lucy update, Eq. (2), in FP64:

        g_next = g / (H' 1) * [H' (f / (H g))]

    The forward projection H g (Eq. 1) is compared with the measured image f
    by an elementwise quotient, the quotient is backprojected with H', and the
    estimate is scaled by it and divided by the backprojection of a ones
    image.  The paper is silent on zeros; readings: a pixel where H g = 0
    contributes 0 to the quotient, and a voxel where H' 1 = 0 gets 0.  ``norm``
    (H' 1 over the W_x x W_y sensor, [Nz][Wx][Wy]) may be passed in.
    """
    g = np.asarray(g, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    fe = forward(H, Nx, Ny, Ks, Kt, g)
    r = np.divide(f, fe, out=np.zeros_like(fe), where=fe != 0)
    bp = backproject(Hp, Nx, Ny, Ks, Kt, r)
    if norm is None:
        norm = backproject(Hp, Nx, Ny, Ks, Kt, np.ones_like(f))
    scaled = np.divide(g, norm, out=np.zeros_like(g), where=norm != 0)
    return scaled * bp


# --------------------------------------------------------------------------
# numpy constructions used as independent pins
# --------------------------------------------------------------------------

def measurement_matrix(Hz: np.ndarray, Mx: int, My: int, periodic: bool = True) -> np.ndarray:
    """Dense matrix A[pixel][voxel] of Eq. (1) for one depth, by pattern placement.

    ``Hz`` is one depth of H as [Nx][Ny][Ks][Kt].  The domain is Mx x My
    lenslets (Wx = Mx*Nx by Wy = My*Ny pixels; one voxel per pixel position).
    Each voxel X adds its cut-out H[X mod N] onto the sensor with the
    cut-out's centre on X (Sec. 2.1).  With ``periodic`` the sensor wraps
    around (lenslet-periodic domain); otherwise entries off the sensor drop.
    """
    Nx, Ny, Ks, Kt = Hz.shape
    Wx, Wy = Mx * Nx, My * Ny
    cs, ct = (Ks - 1) // 2, (Kt - 1) // 2
    A = np.zeros((Wx * Wy, Wx * Wy))
    for X in range(Wx):
        for Y in range(Wy):
            pat = Hz[X % Nx, Y % Ny].astype(np.float64)
            for s in range(Ks):
                Sx = X + s - cs
                if periodic:
                    Sx %= Wx
                elif not 0 <= Sx < Wx:
                    continue
                for t in range(Kt):
                    Sy = Y + t - ct
                    if periodic:
                        Sy %= Wy
                    elif not 0 <= Sy < Wy:
                        continue
                    A[Sx * Wy + Sy, X * Wy + Y] += pat[s, t]
    return A
