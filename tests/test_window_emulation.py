"""The literal paper-window map's index arithmetic (csrc/lfbp_window.cuh, the
one the CUDA kernel uses), run on the CPU over whole arrays and compared with
the oracle's literal evaluation of Eqs. (4)-(9): odd and even cut-outs, the map
and its adjoint (CPU only)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def win(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("win") / "libwin.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-w", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_2003_09133_gb300", "csrc"),
                           "-o", so, os.path.join(HERE, "host_emu", "window_emu.cpp")])
    lib = ctypes.CDLL(so)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.window_apply.argtypes = [P, P, I, I, I, I, P, P, I]
    lib.window_apply.restype = I
    return lib


SHAPES = [  # Nx, Ny, Ks, Kt: even, odd and mixed cut-outs, K < N and K > N
    (3, 1, [4], [1]), (3, 1, [6], [1]), (3, 3, [6, 4], [4, 9]), (5, 3, [14, 15], [15, 6]),
    (1, 1, [2, 8], [6, 3]), (7, 5, [2, 21, 16], [10, 5, 3]), (5, 5, [15, 5], [15, 25]),
    (9, 13, [26, 3], [40, 12]),
    (19, 19, [76, 57], [76, 58]), (95, 55, [12, 96], [10, 7]),  # the GPU test's cells
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2]}x{s[3]}")
def test_literal_window_index_map(win, shape):
    Nx, Ny, Ks, Kt = shape
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    H = np.random.default_rng(5).uniform(-1, 1, n)
    ks, kt = np.asarray(Ks, np.int32), np.asarray(Kt, np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    out = np.empty_like(H)
    assert win.window_apply(p(H), p(out), 8, Nx, Ny, len(Ks), p(ks), p(kt), 0) == 0
    np.testing.assert_array_equal(out, oracle.paper_window(H, Nx, Ny, Ks, Kt))
    # adjoint: each written entry back at its source, zero elsewhere
    src = oracle.paper_window(np.arange(1, n + 1, dtype=np.int64), Nx, Ny, Ks, Kt)
    want = np.zeros(n)
    w = src > 0
    want[src[w] - 1] = H[w]
    adj = np.empty_like(H)
    assert win.window_apply(p(H), p(adj), 8, Nx, Ny, len(Ks), p(ks), p(kt), 1) == 0
    np.testing.assert_array_equal(adj, want)
