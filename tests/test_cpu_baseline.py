"""The benchmark's CPU baseline -- the paper's closed-form rearrangement of
Sec. 4 on the host cores (oracle/lfbp_cpu_rearrange.c) -- gives the oracle's
H' bit for bit (CPU only), on one thread and on all."""
import numpy as np
import pytest

import oracle

SHAPES = [(5, 5, [15, 3, 25], [15, 3, 25]), (3, 7, [9, 21], [21, 5]), (1, 1, [5], [7]),
          (19, 19, [95], [95]), (11, 11, [89], [89]), (95, 55, [11], [13])]


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}")
def test_closed_form_matches_the_oracle(shape, dtype):
    Nx, Ny, Ks, Kt = shape
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    rng = np.random.default_rng(9)
    if dtype == np.float16:
        H = rng.integers(0, 2 ** 16, n, dtype=np.uint32).astype(np.uint16).view(np.float16)
    else:
        H = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
    want = oracle.transpose(H, Nx, Ny, Ks, Kt)
    w = np.uint16 if dtype == np.float16 else np.uint32
    for nthreads in (1, 0):
        got = oracle.cpu_rearrange(H, Nx, Ny, Ks, Kt, nthreads)
        assert np.array_equal(got.view(w), want.view(w))
    assert oracle.cpu_rearrange_threads(0) >= 1
