"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case copies lfbp_oracle.c with one plausible slip (wrong sign, dropped
flip, off-by-one, swapped axis), builds the copy into a temporary directory
and checks that the hand-evaluated Eqs. (4)-(9) tables or the dense
measurement-matrix transpose reject it.  Every slip keeps all indices in
range, so the mutated code cannot read or write outside its arrays.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "lfbp_oracle.c")

MUTATIONS = {
    "transpose_sign": ("long Xx = Sx + u - cs, Xy = Sy + v - ct;",
                       "long Xx = Sx - u + cs, Xy = Sy + v - ct;"),
    "cutout_flip": ("long k = S - X + (K - 1) / 2;", "long k = X - S + (K - 1) / 2;"),
    "transpose_cell_offset": ("int a = (int)floor_mod(Xx, Nx);      /* voxel's cell position */",
                              "int a = (int)floor_mod(Xx + 1, Nx);"),
    "transpose_axes": ("int b = (int)floor_mod(Xy, Ny);\n                    int s = cutout_index(Sx, Xx, ks);",
                       "int b = (int)floor_mod(Xx, Ny);\n                    int s = cutout_index(Sx, Xx, ks);"),
    "eq8_no_flip": ("*sp = K - s + (K % 2);", "*sp = s;"),
    "eq6_offset": ("long xp = s - n + alpha + floor_div(n - 1, 2) - dS;",
                   "long xp = s - n + alpha + floor_div(n - 1, 2) - dS + 1;"),
    "eq5_wrap": ("if (alpha <= 0) return alpha + ceil_div(1 - alpha, n) * n;",
                 "if (alpha <= 0) return alpha + floor_div(1 - alpha, n) * n + n;"),
    "eq4_alpha": ("long dS = floor_div(K - n, 2);", "long dS = floor_div(K - n + 2, 2);"),
    # slips that only even cut-outs see (reading A2): the odd-K form of Eq. (8),
    # and Eq. (4)'s floor taken as a ceiling (equal when n_s - n_x is even)
    "eq8_even_as_odd": ("*sp = K - s + (K % 2);", "*sp = K - s + 1;"),
    "eq4_even_ceil": ("long dS = floor_div(K - n, 2);", "long dS = ceil_div(K - n, 2);"),
}


def _build_variant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.oracle_transpose.argtypes = [P, P, I, I, I, I, P, P, I]
    lib.oracle_paper_window.argtypes = [P, P, I, I, I, I, P, P]
    return lib


def _run(fn, H, Nx, Ny, Ks, Kt, *extra):
    out = np.zeros_like(H)
    ks = np.asarray(Ks, dtype=np.int32)
    kt = np.asarray(Kt, dtype=np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = fn(p(H), p(out), H.itemsize, Nx, Ny, len(ks), p(ks), p(kt), *extra)
    return rc, out


def _read_golden_even(path):
    """(p, u) -> source (a, s) or None, from a hand-evaluated even-n_s table."""
    rows = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                tok = line.split()
                rows[(int(tok[0]), int(tok[1]))] = (None if tok[2] == "-"
                                                    else (int(tok[2]), int(tok[3])))
    return rows


def _pins_pass(lib):
    """True iff the variant passes the golden tables (odd and even n_s) and the
    dense-matrix pin."""
    from test_oracle import _read_golden, _tagged_1d, _tag
    gold = os.path.join(os.path.dirname(__file__), "golden")
    for fname, N, K in [("eqs4to9_nx3_ns5.txt", 3, 5), ("eqs4to9_nx3_ns3.txt", 3, 3)]:
        rows = _read_golden(os.path.join(gold, fname))
        H = _tagged_1d(N, K)
        rc_t, tr = _run(lib.oracle_transpose, H, N, 1, [K], [1], 1)
        rc_p, pw = _run(lib.oracle_paper_window, H, N, 1, [K], [1])
        if rc_t != 0 or rc_p != 0:
            return False
        for (p, u), (paper, trans) in rows.items():
            if tr[p * K + u] != _tag(*trans):
                return False
            if pw[p * K + u] != (0 if paper is None else _tag(*paper)):
                return False
    for fname, N, K in [("eqs4to9_nx3_ns4_even.txt", 3, 4), ("eqs4to9_nx3_ns6_even.txt", 3, 6)]:
        rc_p, pw = _run(lib.oracle_paper_window, _tagged_1d(N, K), N, 1, [K], [1])
        if rc_p != 0:
            return False
        for (p, u), src in _read_golden_even(os.path.join(gold, fname)).items():
            if pw[p * K + u] != (0 if src is None else _tag(*src)):
                return False
    Nx, Ny, Ks, Kt = 5, 3, 15, 9
    Hz = np.random.default_rng(1).uniform(-1, 1, (Nx, Ny, Ks, Kt))
    rc, Hp = _run(lib.oracle_transpose, Hz.reshape(-1), Nx, Ny, [Ks], [Kt], 1)
    if rc != 0:
        return False
    Hp = Hp.reshape(Nx, Ny, Ks, Kt)
    Mx, My = 5, 5
    B = oracle.measurement_matrix(Hz, Mx, My).T
    Wy = My * Ny
    for Sx, Sy in [(0, 0), (3, 7), (11, 2)]:
        col = B[:, Sx * Wy + Sy].reshape(Mx * Nx, Wy)
        for u in range(Ks):
            for v in range(Kt):
                X, Y = (Sx + u - 7) % (Mx * Nx), (Sy + v - 4) % Wy
                if col[X, Y] != Hp[Sx % Nx, Sy % Ny, u, v]:
                    return False
    # Eqs. (4)-(9) with several added slices (alpha reaches -2 and below):
    # the paper's loop must equal the transpose on the entries it writes
    for Nx, Ny, Ks, Kt in [(3, 5, 9, 15), (5, 3, 25, 9)]:
        H = np.random.default_rng(2).uniform(-1, 1, Nx * Ny * Ks * Kt)
        rc_t, tr = _run(lib.oracle_transpose, H, Nx, Ny, [Ks], [Kt], 1)
        rc_p, pw = _run(lib.oracle_paper_window, H, Nx, Ny, [Ks], [Kt])
        if rc_t != 0 or rc_p != 0:
            return False
        hx, hy = (Nx - 1) // 2, (Ny - 1) // 2
        p = np.arange(Nx)[:, None, None, None]
        q = np.arange(Ny)[None, :, None, None]
        u = np.arange(Ks)[None, None, :, None]
        v = np.arange(Kt)[None, None, None, :]
        keep = ((p + u >= hx) & (p + u <= Ks - 1 + hx) & (q + v >= hy) & (q + v <= Kt - 1 + hy))
        want = np.where(keep, tr.reshape(Nx, Ny, Ks, Kt), 0.0)
        if not np.array_equal(pw.reshape(Nx, Ny, Ks, Kt), want):
            return False
    return True


def test_unmutated_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "plain.c"
    path.write_text(src)
    so = tmp_path / "plain.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.oracle_transpose.argtypes = [P, P, I, I, I, I, P, P, I]
    lib.oracle_paper_window.argtypes = [P, P, I, I, I, I, P, P]
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not _pins_pass(_build_variant(tmp_path, name))


# ------------------------------------------------- Eq. (2) composition slips --

def _rl_variant(kind):
    """oracle.rl_step with one plausible slip in how Eq. (2) is composed."""
    def step(H, Hp, Nx, Ny, Ks, Kt, g, f):
        fe = oracle.forward(H, Nx, Ny, Ks, Kt, g)
        r = fe / f if kind == "quotient_inverted" else f / fe
        bp_op = H if kind == "backproject_with_H" else Hp
        bp = oracle.backproject(bp_op, Nx, Ny, Ks, Kt, r)
        if kind == "no_normaliser":
            return g * bp
        norm = oracle.backproject(Hp, Nx, Ny, Ks, Kt, np.ones_like(f))
        if kind == "normaliser_of_H":
            norm = oracle.backproject(H, Nx, Ny, Ks, Kt, np.ones_like(f))
        return g / norm * bp
    return step


@pytest.mark.parametrize("kind", ["quotient_inverted", "backproject_with_H", "no_normaliser",
                                  "normaliser_of_H"])
def test_rl_composition_slip_is_caught(kind):
    """The dense-matrix pin of Eq. (2) rejects each slip (and accepts the oracle)."""
    Nx, Ny, K = 3, 3, 9
    rng = np.random.default_rng(16)
    Hz = rng.uniform(0, 1, (Nx, Ny, K, K))
    H = Hz.reshape(-1)
    Mx = My = 4
    W = Mx * Nx
    g = rng.uniform(0.1, 1, (1, W, W))
    f = rng.uniform(0.1, 1, (W, W))
    A = oracle.measurement_matrix(Hz, Mx, My, periodic=False)
    want = g.reshape(-1) / (A.T @ np.ones(A.shape[0])) * (A.T @ (f.reshape(-1) / (A @ g.reshape(-1))))
    Hp = oracle.transpose(H, Nx, Ny, [K], [K])
    ok = oracle.rl_step(H, Hp, Nx, Ny, [K], [K], g, f).reshape(-1)
    np.testing.assert_allclose(ok, want, rtol=1e-12)
    bad = _rl_variant(kind)(H, Hp, Nx, Ny, [K], [K], g, f).reshape(-1)
    assert not np.allclose(bad, want, rtol=1e-6)


# ------------------------------------------------------- projector slips --

PROJ_MUTATIONS = {
    # forward model, Eq. (1): the cut-out flipped, or the wrong voxel's pattern
    "forward_flip": ("long Sx = X + s - cs;                 /* pixel of entry s */",
                     "long Sx = X - s + cs;"),
    "forward_cell": ("int a = (int)(X % Nx), b = (int)(Y % Ny);",
                     "int a = (int)((X + 1) % Nx), b = (int)(Y % Ny);"),
    # backprojection: the window walked the wrong way, or the wrong pixel's slice
    "backproject_window_sign": (
        "                const double* win = Hp + off + ((size_t)p * Ny + q) * ks * kt;\n"
        "                for (int u = 0; u < ks; ++u) {\n"
        "                    long X = Sx + u - cs;",
        "                const double* win = Hp + off + ((size_t)p * Ny + q) * ks * kt;\n"
        "                for (int u = 0; u < ks; ++u) {\n"
        "                    long X = Sx - u + cs;"),
    "backproject_cell": ("                int p = (int)(Sx % Nx), q = (int)(Sy % Ny);\n"
                         "                const double* win",
                         "                int p = (int)(Sx % Nx), q = (int)((Sy + 1) % Ny);\n"
                         "                const double* win"),
    # gradient with respect to H': the voxel offset with the wrong sign
    "grad_offset_sign": ("                for (long Sx = p; Sx < Wx; Sx += Nx) {\n"
                         "                    long X = Sx + u - cs;",
                         "                for (long Sx = p; Sx < Wx; Sx += Nx) {\n"
                         "                    long X = Sx - u + cs;"),
}


def _build_proj_variant(tmp_path, name):
    src = open(SRC).read()
    if name is not None:
        old, new = PROJ_MUTATIONS[name]
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    path = tmp_path / f"{name or 'plain'}_proj.c"
    path.write_text(src)
    so = tmp_path / f"{name or 'plain'}_proj.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.oracle_transpose.argtypes = [P, P, I, I, I, I, P, P, I]
    lib.oracle_forward_f64.argtypes = [P, I, I, I, P, P, P, I, I, P]
    lib.oracle_backproject_f64.argtypes = [P, I, I, I, P, P, P, I, I, P]
    lib.oracle_grad_hp_f64.argtypes = [P, P, I, I, I, P, P, I, I, P, I]
    return lib


def _proj_pins_pass(lib):
    """True iff the variant's projectors pass the dense-matrix pins (forward =
    A g, backprojection = A^T f, A built by pattern placement) and the gradient
    passes the bilinear identity <dL/dH', dH'> = <r, dH' f> against the pinned
    backprojection."""
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    Nx, Ny, K = 3, 3, 9
    rng = np.random.default_rng(8)
    Hz = rng.uniform(0, 1, (Nx, Ny, K, K))
    Mx = My = 4
    A = oracle.measurement_matrix(Hz, Mx, My, periodic=False)
    W = Mx * Nx
    g = rng.uniform(0, 1, (1, W, W))
    f = rng.uniform(0, 1, (W, W))
    ks = np.array([K], np.int32)
    H = np.ascontiguousarray(Hz.reshape(-1))
    fo = np.zeros((W, W))
    if lib.oracle_forward_f64(p(H), Nx, Ny, 1, p(ks), p(ks), p(g), W, W, p(fo)) != 0:
        return False
    if not np.allclose(fo.reshape(-1), A @ g.reshape(-1), rtol=1e-12, atol=1e-12):
        return False
    Hp = np.zeros_like(H)
    if lib.oracle_transpose(p(H), p(Hp), 8, Nx, Ny, 1, p(ks), p(ks), 1) != 0:
        return False
    go = np.zeros((1, W, W))
    if lib.oracle_backproject_f64(p(Hp), Nx, Ny, 1, p(ks), p(ks), p(f), W, W, p(go)) != 0:
        return False
    if not np.allclose(go.reshape(-1), A.T @ f.reshape(-1), rtol=1e-12, atol=1e-12):
        return False
    # gradient: L(H') = <r, H' f> is linear in H', so <dL/dH', dH'> = <r, dH' f>
    r = rng.uniform(-1, 1, (1, W, W))
    dHp = rng.uniform(-1, 1, H.size)
    gr = np.zeros_like(H)
    if lib.oracle_grad_hp_f64(p(f), p(r), Nx, Ny, 1, p(ks), p(ks), W, W, p(gr), 1) != 0:
        return False
    bd = np.zeros((1, W, W))
    lib.oracle_backproject_f64(p(dHp), Nx, Ny, 1, p(ks), p(ks), p(f), W, W, p(bd))
    lhs, rhs = float(gr @ dHp), float((r * bd).sum())
    return abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs))


def test_unmutated_projectors_pass(tmp_path):
    assert _proj_pins_pass(_build_proj_variant(tmp_path, None))


@pytest.mark.parametrize("name", sorted(PROJ_MUTATIONS))
def test_planted_projector_mistake_is_caught(tmp_path, name):
    assert not _proj_pins_pass(_build_proj_variant(tmp_path, name))
