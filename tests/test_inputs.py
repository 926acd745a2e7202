"""The synthetic input recipe (CPU only): workload shapes, the ragged batch's
draws and the Gaussian-spot cut-outs that stand in for the paper's PSFs."""
import numpy as np
import pytest
import torch

import lfgen


def test_workload_shapes():
    tiny = lfgen.config_specs("tiny")[0]
    assert (tiny.Nx, tiny.Ny, tiny.Ks, tiny.radius) == (5, 5, (15, 15, 15), (2, 1, 2))
    assert lfgen.array_elems(tiny) == 3 * 5 * 5 * 15 * 15
    mid = lfgen.config_specs("mid")[0]
    assert mid.Nx == 15 and mid.Nz == 51 and set(mid.Ks) == {45, 75, 105, 135, 165}
    assert mid.Ks[25] == 45 and mid.Ks[0] == mid.Ks[50] == 165
    hr = lfgen.config_specs("highres")[0]
    assert hr.Nx == 19 and hr.Nz == 41 and hr.Ks[20] == 95 and hr.Ks[0] == hr.Ks[40] == 399
    assert list(hr.Ks) == list(reversed(hr.Ks))  # symmetric about the focal plane
    assert lfgen.array_elems(hr) == 946_782_065
    ag = lfgen.config_specs("autograd")[0]
    assert ag.Nx == 11 and ag.Nz == 21 and max(ag.Ks) == 99 and min(ag.Ks) == 33
    for s in (tiny, mid, hr, ag):
        assert s.Ks == s.Kt and all(k % 2 == 1 and k % s.Nx == 0 for k in s.Ks)
        assert s.dtype == "f32"


def test_ragged_batch_draws():
    specs = lfgen.config_specs("ragged")
    assert [s.seed for s in specs] == list(range(2, 18))
    for s in specs:
        assert s.Nx == s.Ny and s.Nx in (9, 11, 13, 15, 17, 19)
        assert 11 <= s.Nz <= 61
        L = [k // s.Nx for k in s.Ks]
        assert all(k == l * s.Nx and l in (3, 5, 7, 9, 11, 13, 15) for k, l in zip(s.Ks, L))
        assert s.dtype == ("f16" if s.seed % 2 == 0 else "f32")
    assert sum(lfgen.array_elems(s) for s in specs) == 5_059_797_922
    assert lfgen.config_specs("ragged") == specs  # deterministic


def _small_spec(N=5, Ls=(3, 5), r=(1, 2), seed=7):
    Ks = tuple(L * N for L in Ls)
    return lfgen.ArraySpec(N, N, Ks, Ks, tuple(r), "f32", seed, "small")


def test_cutouts_are_normalised_nonnegative_and_seeded():
    spec = _small_spec()
    H = lfgen.generate(spec).numpy().astype(np.float64)
    assert np.isfinite(H).all() and (H >= 0).all()
    off = lfgen.depth_offsets(spec) + [H.size]
    for z, K in enumerate(spec.Ks):
        cut = H[off[z]:off[z + 1]].reshape(spec.Nx * spec.Ny, K * K)
        # unit sum before the fp32 cast and the 1e-6 cut (at most K^2 values of < 1e-6 dropped)
        assert np.abs(cut.sum(axis=1) - 1).max() <= K * K * 1e-6 + 1e-5
        # values that survive the cut are at least 1e-6 (fp32 rounding aside)
        nz = cut[cut > 0]
        assert nz.min() >= 1e-6 * (1 - 2 ** -23)
    assert torch.equal(lfgen.generate(spec), lfgen.generate(spec))
    other = lfgen.generate(_small_spec(seed=8))
    assert not torch.equal(lfgen.generate(spec), other)


def test_spots_sit_on_the_lattice_offset_by_the_source_position():
    """Reading of the recipe: spots of source (a, b) lie at
    (c + jN + (a - h), c + kN + (b - h)) from the cut-out's corner, so the
    pixel residues mod N that hold most of the mass are (c + a - h) mod N
    along s and (c + b - h) mod N along t."""
    spec = _small_spec(N=7, Ls=(3, 5), r=(1, 2))
    H = lfgen.generate(spec).numpy().astype(np.float64)
    off = lfgen.depth_offsets(spec)
    N, h = spec.Nx, (spec.Nx - 1) // 2
    for z, K in enumerate(spec.Ks):
        c = (K - 1) // 2
        D = H[off[z]:off[z] + N * N * K * K].reshape(N, N, K, K)
        for a in range(N):
            for b in range(N):
                ms = np.bincount(np.arange(K) % N, weights=D[a, b].sum(axis=1), minlength=N)
                mt = np.bincount(np.arange(K) % N, weights=D[a, b].sum(axis=0), minlength=N)
                assert int(np.argmax(ms)) == (c + a - h) % N, (z, a, b)
                assert int(np.argmax(mt)) == (c + b - h) % N, (z, a, b)
        # the central source's central spot is the cut-out's centre pixel
        assert D[h, h, c, c] > 0.5 * D[h, h].max()


@pytest.mark.parametrize("r", [0, 1, 2])
def test_spot_count_follows_the_radius(r):
    """(2r+1)^2 amplitudes are drawn, those with j^2 + k^2 > r^2 masked out:
    the number of distinct spots of a cut-out is the disk's lattice count."""
    N = 9
    spec = lfgen.ArraySpec(N, N, ((2 * r + 1) * N,), ((2 * r + 1) * N,), (r,), "f32", 3, "disk")
    K = spec.Ks[0]
    D = lfgen.generate(spec).numpy().reshape(N, N, K, K)
    h = (N - 1) // 2
    cut = D[h, h]
    c = (K - 1) // 2
    lattice = [(c + j * N, c + k * N) for j in range(-r, r + 1) for k in range(-r, r + 1)]
    inside = [(j * j + k * k <= r * r) for j in range(-r, r + 1) for k in range(-r, r + 1)]
    for (s, t), keep in zip(lattice, inside):
        assert (cut[s, t] > 1e-3) == keep, (s, t)
