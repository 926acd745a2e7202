"""The kernel's tile code, run on the CPU with every memory access checked.

tests/host_emu/lfbp_emu.cpp compiles the device tile functions of
lfbp_device.cuh as host C++ with checked stand-ins for TMA bulk copies,
mbarrier transactions and global stores.  These CPU tests show, before any
GPU run, that each launch shape keeps all copies aligned and inside their
buffers, writes every output byte exactly once, and reproduces the oracle.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host_emu", "lfbp_emu.cpp")


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("emu") / "libemu.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-w", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_2003_09133_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", so, SRC])
    lib = ctypes.CDLL(so)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.emu_run.argtypes = [P, P, P, I, I, I, P, P, I, I, I, I, P]
    lib.emu_run.restype = ctypes.c_long
    lib.emu_message.restype = ctypes.c_char_p
    return lib


def _aligned(nbytes, offset=0):
    """uint8 view of nbytes starting `offset` bytes after a 64-byte boundary."""
    raw = np.zeros(nbytes + 128, dtype=np.uint8)
    base = (-raw.ctypes.data) % 64 + offset
    return raw[base:base + nbytes]


def _run(emu, H, Nx, Ny, Ks, Kt, mode=0, target=32768, nthr=8):
    es = H.itemsize
    nbytes = H.nbytes
    hin = _aligned(nbytes)
    hin[:] = H.view(np.uint8)
    out = _aligned(nbytes)
    out[:] = 0x5A
    counts = np.zeros(nbytes, dtype=np.uint8)
    ks = np.asarray(Ks, dtype=np.int32)
    kt = np.asarray(Kt, dtype=np.int32)
    stats = np.zeros(6, dtype=np.uint64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    nerr = emu.emu_run(p(hin), p(out), p(counts), Nx, Ny, len(ks), p(ks), p(kt), es, mode,
                       target, nthr, p(stats))
    assert nerr == 0, emu.emu_message().decode()
    np.testing.assert_array_equal(counts, 1)
    return out.view(H.dtype), stats


def _random_bits(n, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == np.float32:
        return rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
    return rng.integers(0, 2 ** 16, n, dtype=np.uint32).astype(np.uint16).view(np.float16)


SHAPES = [
    # Nx, Ny, Ks, Kt, tile target (small targets force partial tiles and column splits)
    (5, 5, [15, 15, 15], [15, 15, 15], 32768),
    (5, 5, [15, 5, 25], [15, 5, 25], 600),
    (3, 5, [9, 3, 15], [15, 5, 5], 32768),
    (1, 1, [5, 1, 9], [7, 1, 3], 32768),
    (7, 3, [21, 7], [9, 33], 1500),
    (19, 19, [95, 57], [95, 57], 32768),
    (19, 19, [133], [133], 4096),
    (11, 11, [99, 33], [99, 33], 20000),
    (15, 15, [45, 75], [45, 75], 32768),
    (9, 13, [27, 3, 1], [39, 13, 5], 2048),
    (9, 9, [27, 45], [27, 45], 32768),       # short rows: pairs and sectors straddle rows
    (5, 3, [3, 5, 7], [5, 7, 3], 32768),     # rows shorter than a sector
    (3, 3, [1, 1], [1, 1], 32768),
    (17, 17, [255], [255], 32768),
    (15, 15, [45, 75], [45, 75], 65536),  # the plain form's tile target: up to 64 rows
    # wide cells as in the large Table 1 sizes and the 95 x 55 cell (cut-outs scaled down)
    (5, 55, [181], [181], 32768),         # a row of 55 x 181 fp32 exceeds the stage: column split
    (51, 51, [53], [53], 32768),
    (95, 3, [19, 21], [97, 9], 32768),    # Ny below a chunk: element walk
    (3, 95, [11], [191], 32768),
    # the stripe consumer: run blocks of 4 runs, 1 to 5 per stripe, bands beyond
    (11, 11, [33, 55], [33, 55], 32768),  # 3 run blocks
    (13, 13, [39, 65], [39, 65], 32768),  # 4
    (19, 19, [57, 399], [57, 399], 32768),  # 5, and a one-row tile per stage in fp32
    (3, 7, [9, 21], [9, 21], 32768),      # 1 and 2
    (7, 27, [21, 35], [21, 35], 32768),   # 7 run blocks: bands of 4
    (5, 3, [13, 21], [9, 17], 8192),      # Ks*Kt = 1 mod 4 with Ks != Kt, multi-row tiles
    (3, 3, [461], [461], 8192),           # one-row fp32 tiles with runs of >= 1800 B: run ends
                                          # stored inside the main loop (shorter: edge pass)
]


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}_t{s[4]}")
def test_tiles_transpose(emu, shape, dtype):
    Nx, Ny, Ks, Kt, target = shape
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    H = _random_bits(n, dtype, 1)
    got, stats = _run(emu, H, Nx, Ny, Ks, Kt, 0, target)
    want = oracle.transpose(H, Nx, Ny, Ks, Kt)
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    E = 16 // H.itemsize
    # the chunk path's context fits every tile whose rows and cells are at least a chunk long
    if Ny >= E and min(Kt) >= E and target >= 32768:
        assert stats[3] == stats[0]
    # the pair path takes the tiles whose run stride Ks*Kt is 1 mod E (odd Ny >= E,
    # rows longer than a chunk); the stripe path the other fp16 tiles with Ks*Kt = 1 mod 4
    pair_ok = [(a * b) % E == 1 and Ny % 2 == 1 and Ny >= E and b > E for a, b in zip(Ks, Kt)]
    if all(pair_ok) and target >= 32768:
        assert stats[5] == stats[0]
    if not any(pair_ok):
        assert stats[5] == 0
    if H.itemsize == 2 and Ny >= 3 and not any(pair_ok) and target >= 32768 and \
            all((a * b) % 4 == 1 and b >= 8 for a, b in zip(Ks, Kt)):
        assert stats[4] == stats[0]
    if H.itemsize == 4:
        assert stats[4] == 0


def _stripe_shape(Ny, Ks, Kt):
    return Ny >= 3 and any((a * b) % 4 == 1 and b >= 8 for a, b in zip(Ks, Kt))


def test_stripe_shapes_are_covered():
    """The shape list reaches the stripe consumer with every run-block count
    per stripe (1 to 5) and with bands of several stripes (Ny > 20)."""
    nrb = sorted({(Ny + 3) // 4 for _, Ny, Ks, Kt, _ in SHAPES if _stripe_shape(Ny, Ks, Kt)})
    assert {1, 2, 3, 4, 5} <= set(nrb) and max(nrb) > 5


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}_t{s[4]}")
def test_tiles_paper_window_and_adjoint(emu, shape, dtype):
    Nx, Ny, Ks, Kt, target = shape
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    H = _random_bits(n, dtype, 2)
    got, stats = _run(emu, H, Nx, Ny, Ks, Kt, 1, target)
    want = oracle.paper_window(H, Nx, Ny, Ks, Kt)
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    # the paper-window mask runs on the chunk path too
    if Ny >= 16 // H.itemsize and min(Kt) >= 16 // H.itemsize and target >= 32768:
        assert stats[3] == stats[0]
    # adjoint of the windowed map: keep only the entries the forward map writes
    keep = oracle.paper_window(np.ones(n), Nx, Ny, Ks, Kt) != 0
    Y = H.copy()
    Y[~keep] = 0
    got2, _ = _run(emu, H, Nx, Ny, Ks, Kt, 2, target)
    want2 = oracle.transpose_adjoint(Y, Nx, Ny, Ks, Kt)
    np.testing.assert_array_equal(got2.view(np.uint8), want2.view(np.uint8))


EVEN_SHAPES = [
    # even cut-outs in the paper-window mode (the literal Eq. 8): even, odd and
    # mixed parities, K < N, non-square cells, multi-row tiles, column splits
    # (small targets) and the zero column alone in a column block
    (3, 3, [4, 6], [4, 6], 32768),
    (5, 3, [14, 15], [15, 6], 32768),
    (19, 19, [96, 20], [96, 20], 32768),
    (11, 7, [90, 12], [34, 89], 4096),
    (5, 5, [16, 2], [16, 2], 600),
    (95, 5, [182], [18], 32768),
    (19, 19, [400], [400], 32768),
    (3, 5, [10], [10], 300),
]


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("shape", EVEN_SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}x{s[3][0]}_t{s[4]}")
def test_tiles_even_cutouts(emu, shape, dtype):
    """Even cut-outs on the tiled gather: the map as the cropped odd cut-out
    under the loop ranges' window, and its adjoint, against the oracle's
    evaluation of Eqs. 4-9."""
    Nx, Ny, Ks, Kt, target = shape
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    H = _random_bits(n, dtype, 4)
    got, _ = _run(emu, H, Nx, Ny, Ks, Kt, 1, target)
    want = oracle.paper_window(H, Nx, Ny, Ks, Kt)
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    # the adjoint moves every written entry back to its source, zero elsewhere
    idx = np.arange(1, n + 1, dtype=np.int64)
    fwd = oracle.paper_window(idx, Nx, Ny, Ks, Kt)
    want2 = np.zeros_like(H)
    written = fwd != 0
    want2[fwd[written] - 1] = H[written]
    got2, _ = _run(emu, H, Nx, Ny, Ks, Kt, 2, target)
    np.testing.assert_array_equal(got2.view(np.uint8), want2.view(np.uint8))


def test_warp_count_does_not_matter(emu):
    Nx, Ny, Ks, Kt = 5, 3, [15, 9], [9, 21]
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    for dtype in (np.float32, np.float16):
        H = _random_bits(n, dtype, 3)
        want = oracle.transpose(H, Nx, Ny, Ks, Kt)
        for nwarps in (1, 3, 8, 9):
            got, _ = _run(emu, H, Nx, Ny, Ks, Kt, 0, 2048, nwarps)
            np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
