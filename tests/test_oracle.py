"""Pins of the CPU oracle against things other than itself (CPU only).

Each pin targets a plausible mistake: a hand evaluation of Eqs. (4)-(9)
(wrong sign or offset in the index map, a dropped flip), a dense measurement
matrix built by pattern placement and transposed by numpy (wrong pairing of
axes, wrong centring, non-square mix-ups), closed special cases (N = 1 is a
180-degree kernel rotation, shift-invariant PSFs), invariants the paper
states (reversibility, Sec. 4; summed slices rotated by 180 degrees, Sec. 4),
the adjoint identity of the projectors and central finite differences.
"""
import os

import numpy as np
import pytest

import lfgen
import oracle


def _read_golden(path):
    rows = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            p, u = int(tok[0]), int(tok[1])
            if tok[2] == "-":
                paper, trans = None, (int(tok[3]), int(tok[4]))
            else:
                paper = (int(tok[2]), int(tok[3]))
                trans = (int(tok[4]), int(tok[5]))
            rows[(p, u)] = (paper, trans)
    return rows


def _tagged_1d(N, K):
    """1-D array (Ny = Kt = 1) whose value encodes its own (a, s) position."""
    H = np.zeros(N * K)
    for a in range(N):
        for s in range(K):
            H[a * K + s] = 100 * a + s + 1
    return H


def _tag(a, s):
    return 100 * a + s + 1


@pytest.mark.parametrize("fname,N,K", [("eqs4to9_nx3_ns5.txt", 3, 5),
                                       ("eqs4to9_nx3_ns3.txt", 3, 3)])
def test_golden_hand_evaluation(golden_dir, fname, N, K):
    rows = _read_golden(os.path.join(golden_dir, fname))
    assert len(rows) == N * K
    H = _tagged_1d(N, K)
    pw = oracle.paper_window(H, N, 1, [K], [1])
    tr = oracle.transpose(H, N, 1, [K], [1])
    for (p, u), (paper, trans) in rows.items():
        i = p * K + u
        assert tr[i] == _tag(*trans), (p, u)
        assert pw[i] == (0 if paper is None else _tag(*paper)), (p, u)


SHAPES = [  # Nx, Ny, Ks, Kt
    (3, 3, 9, 9), (5, 3, 15, 9), (3, 5, 5, 3), (1, 3, 5, 7), (5, 5, 5, 5),
    (3, 3, 3, 3), (7, 5, 7, 11),
]


def _rand(shape_elems, seed):
    return np.random.default_rng(seed).uniform(-1, 1, shape_elems)


@pytest.mark.parametrize("Nx,Ny,Ks,Kt", SHAPES)
def test_dense_measurement_matrix_transpose(Nx, Ny, Ks, Kt):
    """H' read off the numpy transpose of the dense Eq. (1) matrix, every pixel."""
    Hz = _rand((Nx, Ny, Ks, Kt), 1)
    Mx = -(-Ks // Nx) + 2
    My = -(-Kt // Ny) + 2
    Wx, Wy = Mx * Nx, My * Ny
    B = oracle.measurement_matrix(Hz, Mx, My, periodic=True).T  # [voxel][pixel]
    Hp = oracle.transpose(Hz.reshape(-1), Nx, Ny, [Ks], [Kt]).reshape(Nx, Ny, Ks, Kt)
    cs, ct = (Ks - 1) // 2, (Kt - 1) // 2
    for Sx in range(Wx):
        for Sy in range(Wy):
            col = B[:, Sx * Wy + Sy].reshape(Wx, Wy).copy()
            win = np.empty((Ks, Kt))
            for u in range(Ks):
                for v in range(Kt):
                    X, Y = (Sx + u - cs) % Wx, (Sy + v - ct) % Wy
                    win[u, v] = col[X, Y]
                    col[X, Y] = 0.0
            np.testing.assert_array_equal(win, Hp[Sx % Nx, Sy % Ny])
            # nothing outside the pixel-centred window reaches this pixel
            assert not np.any(col)


PW_SHAPES = SHAPES + [(11, 11, 89, 89), (5, 7, 15, 21), (7, 3, 5, 3), (9, 9, 27, 45)]


@pytest.mark.parametrize("Nx,Ny,Ks,Kt", PW_SHAPES)
def test_paper_window_is_masked_transpose(Nx, Ny, Ks, Kt):
    """Eqs. (4)-(9) write exactly the transpose, except on the overhang entries."""
    H = _rand(Nx * Ny * Ks * Kt, 2)
    pw = oracle.paper_window(H, Nx, Ny, [Ks], [Kt]).reshape(Nx, Ny, Ks, Kt)
    tr = oracle.transpose(H, Nx, Ny, [Ks], [Kt]).reshape(Nx, Ny, Ks, Kt)
    hx, hy = (Nx - 1) // 2, (Ny - 1) // 2
    p = np.arange(Nx)[:, None, None, None]
    q = np.arange(Ny)[None, :, None, None]
    u = np.arange(Ks)[None, None, :, None]
    v = np.arange(Kt)[None, None, None, :]
    keep = (p + u >= hx) & (p + u <= Ks - 1 + hx) & (q + v >= hy) & (q + v <= Kt - 1 + hy)
    np.testing.assert_array_equal(pw, np.where(keep, tr, 0.0))
    if Ks >= Nx:
        keep_x = (np.arange(Nx)[:, None] + np.arange(Ks)[None, :])
        dropped = np.sum((keep_x < hx) | (keep_x > Ks - 1 + hx))
        assert dropped == hx * (hx + 1)


@pytest.mark.parametrize("dtype", [np.float32, np.float16, np.float64, np.uint8])
def test_involution_and_adjoint(dtype):
    """Reversibility (Sec. 4): mapping H' again returns H; the adjoint is the map."""
    Nx, Ny, Ks, Kt = 5, 3, [15, 5, 9], [9, 3, 21]
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    rng = np.random.default_rng(3)
    if dtype == np.uint8:
        H = rng.integers(0, 256, n).astype(np.uint8)
    else:
        H = rng.uniform(-1, 1, n).astype(dtype)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    assert not np.array_equal(Hp, H)
    np.testing.assert_array_equal(oracle.transpose(Hp, Nx, Ny, Ks, Kt), H)
    np.testing.assert_array_equal(oracle.transpose_adjoint(H, Nx, Ny, Ks, Kt), Hp)


def test_multisets_and_summed_slices():
    """Each depth's values are preserved; Sec. 4's summed-slice identity holds."""
    spec = lfgen.config_specs("tiny")[0]
    H = lfgen.generate(spec).numpy()
    Hp = oracle.transpose(H, spec.Nx, spec.Ny, spec.Ks, spec.Kt)
    off = lfgen.depth_offsets(spec)
    for z, (ks, kt) in enumerate(zip(spec.Ks, spec.Kt)):
        n = spec.Nx * spec.Ny * ks * kt
        a = H[off[z]:off[z] + n].reshape(spec.Nx, spec.Ny, ks, kt)
        b = Hp[off[z]:off[z] + n].reshape(spec.Nx, spec.Ny, ks, kt)
        np.testing.assert_array_equal(np.sort(a.view(np.uint32), axis=None),
                                      np.sort(b.view(np.uint32), axis=None))
        # for each (u, v): the N^2 summands of H' equal those of H at (K-1-u, K-1-v)
        lhs = np.sort(b.reshape(-1, ks, kt), axis=0)
        rhs = np.sort(a[:, :, ::-1, ::-1].reshape(-1, ks, kt), axis=0)
        np.testing.assert_array_equal(lhs, rhs)
        # the summed image of H' is the summed image of H rotated by 180 degrees
        s_hp = b.astype(np.float64).sum(axis=(0, 1))
        s_h = np.rot90(a.astype(np.float64).sum(axis=(0, 1)), 2)
        np.testing.assert_allclose(s_hp, s_h, rtol=1e-13, atol=1e-15)


def test_single_position_is_rot180():
    """N = 1 (shift-invariant imaging): H' is the 180-degree rotation of each kernel."""
    Ks, Kt = [5, 9, 3], [7, 9, 1]
    H = _rand(sum(a * b for a, b in zip(Ks, Kt)), 4)
    Hp = oracle.transpose(H, 1, 1, Ks, Kt)
    off = 0
    for ks, kt in zip(Ks, Kt):
        k = H[off:off + ks * kt].reshape(ks, kt)
        np.testing.assert_array_equal(Hp[off:off + ks * kt].reshape(ks, kt), np.rot90(k, 2))
        off += ks * kt


def test_shift_invariant_kernel():
    """All cell positions share one kernel: every H' slice is that kernel rotated."""
    Nx, Ny, K = 5, 3, 15
    k = _rand((K, K), 5)
    Hz = np.broadcast_to(k, (Nx, Ny, K, K)).copy()
    Hp = oracle.transpose(Hz.reshape(-1), Nx, Ny, [K], [K]).reshape(Nx, Ny, K, K)
    for p in range(Nx):
        for q in range(Ny):
            np.testing.assert_array_equal(Hp[p, q], np.rot90(k, 2))


def test_special_bit_patterns_survive():
    """The map moves bits: NaN payloads, -0, inf and subnormals come through."""
    Nx, Ny, Ks, Kt = 3, 3, [9], [9]
    n = 81 * 9
    bits = np.random.default_rng(6).integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0x7fc00001, 0x7f800001, 0xffc12345, 0x80000000, 0x7f800000,
                         0xff800000, 0x00000001, 0x807fffff], dtype=np.uint32)
    bits[:len(specials)] = specials
    H = bits.view(np.float32)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    np.testing.assert_array_equal(np.sort(Hp.view(np.uint32)), np.sort(bits))
    np.testing.assert_array_equal(oracle.transpose(Hp, Nx, Ny, Ks, Kt).view(np.uint32), bits)


def _proj_case(seed=7):
    Nx, Ny, Ks, Kt = 3, 5, [9, 3, 15], [15, 5, 5]
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    rng = np.random.default_rng(seed)
    H = rng.uniform(0, 1, n)
    Wx, Wy = 13, 17
    g = rng.uniform(0, 1, (len(Ks), Wx, Wy))
    f = rng.uniform(0, 1, (Wx, Wy))
    return Nx, Ny, Ks, Kt, H, g, f


def test_adjoint_identity_fp64():
    """<H g, f> = <g, H' f> on a finite zero-padded domain (FP64)."""
    Nx, Ny, Ks, Kt, H, g, f = _proj_case()
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    lhs = np.sum(oracle.forward(H, Nx, Ny, Ks, Kt, g) * f)
    rhs = np.sum(g * oracle.backproject(Hp, Nx, Ny, Ks, Kt, f))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_projectors_match_dense_matrix():
    """Forward = A g and backprojection = A^T f with A built by pattern placement."""
    Nx, Ny, K = 3, 3, 9
    rng = np.random.default_rng(8)
    Hz = rng.uniform(0, 1, (Nx, Ny, K, K))
    Mx = My = 4
    A = oracle.measurement_matrix(Hz, Mx, My, periodic=False)
    W = Mx * Nx
    g = rng.uniform(0, 1, (1, W, W))
    f = rng.uniform(0, 1, (W, W))
    np.testing.assert_allclose(oracle.forward(Hz.reshape(-1), Nx, Ny, [K], [K], g).reshape(-1),
                               A @ g.reshape(-1), rtol=1e-13, atol=1e-13)
    Hp = oracle.transpose(Hz.reshape(-1), Nx, Ny, [K], [K])
    np.testing.assert_allclose(oracle.backproject(Hp, Nx, Ny, [K], [K], f).reshape(-1),
                               A.T @ f.reshape(-1), rtol=1e-13, atol=1e-13)


def test_backproject_points_match_full():
    Nx, Ny, Ks, Kt, H, g, f = _proj_case(9)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    full = oracle.backproject(Hp, Nx, Ny, Ks, Kt, f)
    rng = np.random.default_rng(10)
    pts = np.stack([rng.integers(0, len(Ks), 200), rng.integers(0, f.shape[0], 200),
                    rng.integers(0, f.shape[1], 200)], axis=1)
    got = oracle.backproject_points(Hp, Nx, Ny, Ks, Kt, f, pts)
    np.testing.assert_allclose(got, full[pts[:, 0], pts[:, 1], pts[:, 2]], rtol=1e-14, atol=1e-14)


def test_gradient_central_differences():
    """dL/dH for L = sum (H'(H) f - g_ref)^2 against FP64 central differences."""
    Nx, Ny, Ks, Kt = 3, 3, [9, 3], [9, 3]
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    rng = np.random.default_rng(11)
    H = rng.uniform(0, 1, n)
    W = 2 * Nx
    f = rng.uniform(0, 1, (W, W))
    gref = rng.uniform(0, 1, (len(Ks), W, W))

    def loss(Hv):
        g = oracle.backproject(oracle.transpose(Hv, Nx, Ny, Ks, Kt), Nx, Ny, Ks, Kt, f)
        return np.sum((g - gref) ** 2)

    g = oracle.backproject(oracle.transpose(H, Nx, Ny, Ks, Kt), Nx, Ny, Ks, Kt, f)
    dhp = oracle.grad_hp(f, 2.0 * (g - gref), Nx, Ny, Ks, Kt)
    dh = oracle.transpose_adjoint(dhp, Nx, Ny, Ks, Kt)
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        Hplus, Hminus = H.copy(), H.copy()
        Hplus[i] += h
        Hminus[i] -= h
        fd = (loss(Hplus) - loss(Hminus)) / (2 * h)
        assert abs(fd - dh[i]) <= 1e-6 * max(1.0, abs(dh[i])), (i, fd, dh[i])


def test_grad_points_match_full():
    Nx, Ny, Ks, Kt = 3, 5, [9, 15], [5, 25]
    rng = np.random.default_rng(12)
    Wx, Wy = 14, 23
    f = rng.uniform(0, 1, (Wx, Wy))
    r = rng.uniform(-1, 1, (2, Wx, Wy))
    full = oracle.grad_hp(f, r, Nx, Ny, Ks, Kt)
    off = [0, Nx * Ny * Ks[0] * Kt[0]]
    pts, want = [], []
    for _ in range(100):
        z = int(rng.integers(0, 2))
        p, q = int(rng.integers(0, Nx)), int(rng.integers(0, Ny))
        u, v = int(rng.integers(0, Ks[z])), int(rng.integers(0, Kt[z]))
        pts.append((z, p, q, u, v))
        want.append(full[off[z] + ((p * Ny + q) * Ks[z] + u) * Kt[z] + v])
    got = oracle.grad_hp_points(f, r, Nx, Ny, Ks, Kt, np.array(pts))
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- Eq. (2) --

def _rl_case(seed=13):
    """Two depths with different cut-outs, a non-negative volume and image."""
    Nx, Ny, Ks, Kt = 3, 3, [9, 3], [9, 3]
    rng = np.random.default_rng(seed)
    Hz = [rng.uniform(0, 1, (Nx, Ny, k, t)) for k, t in zip(Ks, Kt)]
    H = np.concatenate([h.reshape(-1) for h in Hz])
    Mx = My = 4
    W = Mx * Nx
    g = rng.uniform(0.1, 1, (len(Ks), W, W))
    f = rng.uniform(0.1, 1, (W, W))
    return Nx, Ny, Ks, Kt, Hz, H, g, f, Mx, My


def test_rl_step_matches_dense_matrix():
    """Eq. (2) against the dense measurement matrix A = [A_0 | A_1] (pattern
    placement, zero outside the sensor): g' = g / (A^T 1) * A^T (f / (A g))."""
    Nx, Ny, Ks, Kt, Hz, H, g, f, Mx, My = _rl_case()
    A = np.concatenate([oracle.measurement_matrix(h, Mx, My, periodic=False) for h in Hz], axis=1)
    fe = A @ g.reshape(-1)
    r = f.reshape(-1) / fe
    want = g.reshape(-1) / (A.T @ np.ones(A.shape[0])) * (A.T @ r)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    got = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, f)
    np.testing.assert_allclose(got.reshape(-1), want, rtol=1e-12, atol=0)


def test_rl_step_fixed_point_and_flux():
    """f = H g*  makes g* a fixed point of Eq. (2); and every update conserves
    sum_X (H'1)(X) g'(X) = sum_S f(S) (over pixels where H g > 0)."""
    Nx, Ny, Ks, Kt, Hz, H, g, f, Mx, My = _rl_case(14)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    g_true = g.copy()
    g_true[:, ::3, ::2] = 0.0  # some empty voxels
    f_true = oracle.forward(H, Nx, Ny, Ks, Kt, g_true)
    got = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g_true, f_true)
    np.testing.assert_allclose(got, g_true, rtol=1e-12, atol=1e-14)
    norm = oracle.backproject(Hp, Nx, Ny, Ks, Kt, np.ones_like(f))
    g1 = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, f)
    assert abs(np.sum(norm * g1) - np.sum(f)) <= 1e-12 * np.sum(f)


def test_rl_step_homogeneity_and_zeros():
    """Eq. (2) is linear in f and invariant to scaling g; zero voxels stay zero;
    pixels with H g = 0 and voxels with H' 1 = 0 follow the stated readings."""
    Nx, Ny, Ks, Kt, Hz, H, g, f, Mx, My = _rl_case(15)
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    g1 = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, f)
    np.testing.assert_allclose(oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, 2.5 * f), 2.5 * g1,
                               rtol=1e-13)
    np.testing.assert_allclose(oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, 3.0 * g, f), g1, rtol=1e-13)
    assert (g1 >= 0).all()
    gz = g.copy()
    gz[1] = 0.0
    assert (oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, gz, f)[1] == 0).all()
    # an all-zero volume: H g = 0 everywhere, the quotient is 0, so is g'
    assert (oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, np.zeros_like(g), f) == 0).all()
    # a depth whose PSF is zero: H' 1 = 0 there, g' = 0 there
    H0 = H.copy()
    H0[Nx * Ny * Ks[0] * Kt[0]:] = 0.0
    Hp0 = oracle.transpose(H0, Nx, Ny, Ks, Kt)
    assert (oracle.rl_step(H0, Hp0, Nx, Ny, Ks, Kt, g, f)[1] == 0).all()


@pytest.mark.parametrize("Nx,Ny,K,Kt,m,mt", [(5, 3, 15, 9, 3, 1), (3, 5, 21, 25, 9, 10),
                                              (7, 7, 9, 9, 4, 4)])
def test_centred_cropping_commutes_with_the_map(Nx, Ny, K, Kt, m, mt):
    """Reading A6: a centred crop of the cut-outs (m entries off each end of s,
    mt off each end of t) taken before the map equals the same crop of H'
    taken after it, so ragged per-depth storage loses nothing.  A centre
    offset taken from the uncropped size, or a flip about the wrong centre,
    breaks it (for m = (K-1)/2 the crop is the central entry alone)."""
    H = _rand(Nx * Ny * K * Kt, 9).reshape(Nx, Ny, K, Kt)
    crop = lambda A: A[:, :, m:K - m, mt:Kt - mt]
    Hp = oracle.transpose(H.reshape(-1), Nx, Ny, [K], [Kt]).reshape(Nx, Ny, K, Kt)
    Hc = np.ascontiguousarray(crop(H))
    Hpc = oracle.transpose(Hc.reshape(-1), Nx, Ny, [K - 2 * m], [Kt - 2 * mt])
    np.testing.assert_array_equal(Hpc.reshape(Hc.shape), crop(Hp))
    # the ragged array of both sizes maps depth by depth
    both = np.concatenate([H.reshape(-1), Hc.reshape(-1)])
    Hb = oracle.transpose(both, Nx, Ny, [K, K - 2 * m], [Kt, Kt - 2 * mt])
    np.testing.assert_array_equal(Hb[:H.size], Hp.reshape(-1))
    np.testing.assert_array_equal(Hb[H.size:], Hpc)
    # the central entry alone: H'[p, q, 0, 0] = H[p, q, 0, 0] for a 1 x 1 cut-out
    c = np.ascontiguousarray(H[:, :, (K - 1) // 2:(K + 1) // 2, (Kt - 1) // 2:(Kt + 1) // 2])
    np.testing.assert_array_equal(oracle.transpose(c.reshape(-1), Nx, Ny, [1], [1]), c.reshape(-1))


@pytest.mark.parametrize("fname,N,K", [("eqs4to9_nx3_ns4_even.txt", 3, 4),
                                       ("eqs4to9_nx3_ns6_even.txt", 3, 6)])
def test_golden_even_cutout_literal_equations(golden_dir, fname, N, K):
    """Even n_s (reading A2): the literal Eqs. (4)-(9) drop s = n_s and never
    write s' = n_s.  The oracle's paper-window evaluation must give the hand
    evaluations in tests/golden/ (n_s = 4: no offset; n_s = 6: offset 1)
    entry by entry."""
    rows = {}
    with open(os.path.join(golden_dir, fname)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            rows[(int(tok[0]), int(tok[1]))] = None if tok[2] == "-" else (int(tok[2]), int(tok[3]))
    assert len(rows) == N * K
    pw = oracle.paper_window(_tagged_1d(N, K), N, 1, [K], [1])
    for (p, u), src in rows.items():
        assert pw[p * K + u] == (0 if src is None else _tag(*src)), (p, u)


@pytest.mark.parametrize("Nx,Ny,K,Kt", [(3, 1, 4, 1), (5, 3, 2, 9), (5, 5, 4, 4), (3, 5, 10, 7),
                                        (7, 3, 8, 12), (1, 1, 4, 6), (9, 5, 6, 15), (5, 7, 16, 2)])
def test_even_cutout_loop_is_a_cropped_odd_transpose(Nx, Ny, K, Kt):
    """Even n_s (reading A2) against the brute-force transpose.  Solving
    Eqs. (4)-(8) for even n_s = K (0-based p = x'-1, u = s'-1, s0 = s-1):
    Eq. (8) gives u = K-2-s0, so s0 = K-1 is dropped and u = K-1 never
    written; Eqs. (4)-(6) give a = p+u-(K/2-1+n) = p+u-(K/2-1) (mod n), using
    dS = (K-n-1)/2 for odd n, and m = p+u+1-h.  That is the transpose of the
    odd (K-1)-pixel cut-out s0 < K-1 (centre (K-2)/2 = K/2-1), written at
    u < K-1, with the loop's range 1 <= m <= K as the usual window
    h <= p+u <= K-1+h.  An odd axis keeps its own transpose and window.  The
    two sides are separate oracle functions: the literal loop and the
    measurement-matrix transpose."""
    rng = np.random.default_rng(Nx * 1000 + K * 10 + Kt)
    H = rng.uniform(0.5, 1.0, Nx * Ny * K * Kt)
    H4 = H.reshape(Nx, Ny, K, Kt)
    Ke, Kte = K - 1 + K % 2, Kt - 1 + Kt % 2
    sub = np.ascontiguousarray(H4[:, :, :Ke, :Kte]).reshape(-1)
    T = oracle.transpose(sub, Nx, Ny, [Ke], [Kte]).reshape(Nx, Ny, Ke, Kte)
    want = np.zeros_like(H4)
    want[:, :, :Ke, :Kte] = T
    hx, hy = (Nx - 1) // 2, (Ny - 1) // 2
    p = np.arange(Nx)[:, None, None, None]
    q = np.arange(Ny)[None, :, None, None]
    u = np.arange(K)[None, None, :, None]
    v = np.arange(Kt)[None, None, None, :]
    keep = (p + u >= hx) & (p + u <= K - 1 + hx) & (q + v >= hy) & (q + v <= Kt - 1 + hy)
    want = np.where(keep, want, 0.0).reshape(-1)
    np.testing.assert_array_equal(oracle.paper_window(H, Nx, Ny, [K], [Kt]), want)
