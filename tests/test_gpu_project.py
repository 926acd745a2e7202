"""GPU projectors and the differentiation workload against the CPU oracle.

The projectors sum in fp32; the oracle sums in FP64.  Tolerance per output
(recursive fp32 summation of n products of fp32 inputs):
    |gpu - oracle| <= n * 2^-23 * sum_k |term_k|
with n the number of products in that output and sum |term| computed by the
oracle on absolute values.  The map H -> H' and its adjoint stay bit-exact.
"""
import numpy as np
import pytest
import torch

import lfgen
import oracle

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def lf():
    import paper_2003_09133_gb300 as m
    m.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return m


def _within(got, want, abs_terms, n, what):
    tol = n * EPS32 * abs_terms + 1e-30
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.flatnonzero(bad.reshape(-1))[:5]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside n*eps*sum|t|; "
                             f"first {i}: got {got.reshape(-1)[i]} want {want.reshape(-1)[i]}")


CASES = [  # Nx, Ny, Ks, Kt, Wx, Wy
    (3, 5, [9, 15], [5, 25], 14, 23),
    (5, 5, [15, 5, 25], [15, 5, 25], 37, 40),
    (1, 1, [3], [5], 9, 7),
    (11, 11, [33, 99], [33, 99], 66, 77),
    (95, 55, [95], [165], 190, 110),   # the R29 elementary cell (Sec. 5), two cells per axis
    (31, 31, [249], [249], 62, 93),     # a Table 1 size: K not a multiple of N (S = 9)
    (3, 3, [9, 15], [9, 3], 200, 151),  # cells of 67 x 51 pixels: two gradient tiles per cell
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_W{c[4]}")
def test_backproject_forward_grad_small(lf, case):
    Nx, Ny, Ks, Kt, Wx, Wy = case
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    rng = np.random.default_rng(3)
    H = rng.uniform(-1, 1, plan.elems).astype(np.float32)
    f = rng.uniform(-1, 1, (Wx, Wy)).astype(np.float32)
    g = rng.uniform(-1, 1, (len(Ks), Wx, Wy)).astype(np.float32)
    Hd, fd, gd = (torch.from_numpy(a).cuda() for a in (H, f, g))
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    Hpd = lf.backproject_array(plan, Hd)
    assert np.array_equal(Hpd.cpu().numpy().view(np.uint32), Hp.view(np.uint32))
    kk = max(a * b for a, b in zip(Ks, Kt))
    # g = H' f
    got = lf.backproject_volume_raw(plan, Hpd, fd).cpu().numpy()
    want = oracle.backproject(Hp, Nx, Ny, Ks, Kt, f)
    absum = oracle.backproject(np.abs(Hp), Nx, Ny, Ks, Kt, np.abs(f))
    _within(got, want, absum, kk, "backproject")
    # f = H g (Eq. 1)
    got = lf.forward_project(plan, Hd, gd).cpu().numpy()
    want = oracle.forward(H, Nx, Ny, Ks, Kt, g)
    absum = oracle.forward(np.abs(H), Nx, Ny, Ks, Kt, np.abs(g))
    _within(got, want, absum, kk * len(Ks), "forward")
    # dL/dH' for a given dL/dg
    got = lf.backproject_volume_grad(plan, fd, gd).cpu().numpy()
    want = oracle.grad_hp(f, g, Nx, Ny, Ks, Kt)
    absum = oracle.grad_hp(np.abs(f), np.abs(g), Nx, Ny, Ks, Kt)
    n_pix = -(-Wx // Nx) * -(-Wy // Ny)
    _within(got, want, absum, n_pix, "grad")
    lf.sync_status()


def test_autograd_chain_small_finite_differences(lf):
    """dL/dH through H -> H' -> g = H' f -> L = sum (g - g_ref)^2 against FP64
    central differences (2 x 2-lenslet sensor, the autograd workload's cell and
    first three cut-out sizes), entry by entry within a bound derived from the
    GPU's fp32 sums:
      g = H' f       : |dg| <= n1 eps G,      G  = sum |H'| |f|   (n1 products)
      r = 2 (g - gr) : |dr| <= 2 n1 eps G + eps |r|               (one rounding)
      dL/dH' = f * r : |d|  <= n2 eps sum |f| |r| + sum |f| |dr|  (n2 products)
    and dL/dH is the exact adjoint gather of dL/dH'.  The differences of the
    FP64 chain add their own rounding, bounded by err(L) / h."""
    spec = lfgen.config_specs("autograd")[0]
    Nx, Ny = spec.Nx, spec.Ny
    Ks, Kt = list(spec.Ks[:3]), list(spec.Kt[:3])
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    rng = np.random.default_rng(5)
    H = rng.uniform(0, 1, plan.elems).astype(np.float32)
    W = 2 * Nx
    f = rng.uniform(0, 1, (W, W)).astype(np.float32)
    gref = rng.uniform(0, 1, (len(Ks), W, W))
    Hd = torch.from_numpy(H).cuda().requires_grad_(True)
    g = lf.backproject_volume(lf.backprojection_array(Hd, plan), torch.from_numpy(f).cuda(), plan)
    loss = ((g.double() - torch.from_numpy(gref).cuda()) ** 2).sum()
    loss.backward()
    dH = Hd.grad.cpu().numpy().astype(np.float64)

    # the fp32 bound per entry, from the FP64 chain on absolute values
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt).astype(np.float64)
    g64 = oracle.backproject(Hp, Nx, Ny, Ks, Kt, f)
    r64 = 2 * (g64 - gref)
    n1 = np.array([a * b for a, b in zip(Ks, Kt)], dtype=np.float64)[:, None, None]
    G = oracle.backproject(np.abs(Hp), Nx, Ny, Ks, Kt, np.abs(f))
    r_abs = np.abs(r64) + 2 * n1 * EPS32 * G
    dr = 2 * n1 * EPS32 * G + EPS32 * r_abs
    n2 = -(-W // Nx) * -(-W // Ny)
    bound_hp = (n2 * EPS32 * oracle.grad_hp(np.abs(f), r_abs, Nx, Ny, Ks, Kt)
                + oracle.grad_hp(np.abs(f), dr, Nx, Ny, Ks, Kt))
    bound = oracle.transpose_adjoint(bound_hp, Nx, Ny, Ks, Kt)

    def g_of(Hv):
        return oracle.backproject(oracle.transpose(Hv, Nx, Ny, Ks, Kt), Nx, Ny, Ks, Kt, f)

    # L(H + h e) - L(H - h e) summed voxel by voxel as (g+ - g-)(g+ + g- - 2 g_ref):
    # no cancellation between two large sums.  Voxels the entry does not reach
    # get identical FP64 sums on both sides (d = 0 exactly); the others carry
    # the rounding of g's n1-term sums and of the final sum.
    eps64 = 2.0 ** -52
    H64 = H.astype(np.float64)
    h = 1e-3  # L is quadratic in H: central differences are exact up to rounding
    # entries that reach the sensor (nonzero bound), and a few that do not
    reach = np.flatnonzero(bound > 0)
    assert reach.size > 100
    sample = np.concatenate([rng.choice(reach, 50, replace=False),
                             rng.choice(np.flatnonzero(bound == 0), 10, replace=False)])
    for i in sample:
        Hp_, Hm_ = H64.copy(), H64.copy()
        Hp_[i] += h
        Hm_[i] -= h
        gp, gm = g_of(Hp_), g_of(Hm_)
        d, t = gp - gm, gp + gm - 2 * gref
        fd = np.sum(d * t) / (2 * h)
        m = d != 0
        err_fd = (np.sum((4 * n1 * eps64 * G * (np.abs(t) + np.abs(d)))[m])
                  + (m.sum() + 1) * eps64 * np.sum(np.abs(d * t))) / (2 * h)
        tol = bound[i] + err_fd
        assert abs(fd - dH[i]) <= tol, (i, fd, dH[i], bound[i], err_fd)


def test_autograd_workload(lf):
    """Full-size differentiation workload: N=11, 21 depths, K_z up to 99, 704 x 704 sensor."""
    spec = lfgen.config_specs("autograd")[0]
    Nx, Ny, Ks, Kt = spec.Nx, spec.Ny, list(spec.Ks), list(spec.Kt)
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    H = lfgen.generate(spec, device="cuda")
    f = torch.from_numpy(lfgen.raw_image(64, Nx, 19).astype(np.float32)).cuda()
    W = f.shape[0]
    gref = torch.from_numpy(lfgen.blob_volume(W, spec.Nz, 200, 20).astype(np.float32)).cuda()
    Hg = H.clone().requires_grad_(True)
    Hp = lf.backprojection_array(Hg, plan)
    Hp.retain_grad()
    g = lf.backproject_volume(Hp, f, plan)
    g.retain_grad()
    loss = ((g - gref) ** 2).sum()
    loss.backward()
    lf.sync_status()
    Hn = H.cpu().numpy()
    Hp_want = oracle.transpose(Hn, Nx, Ny, Ks, Kt)
    assert np.array_equal(Hp.detach().cpu().numpy().view(np.uint32), Hp_want.view(np.uint32))
    fn = f.cpu().numpy()
    rng = np.random.default_rng(7)
    # g at sampled voxels, each computed on its own by the oracle in FP64
    pts = np.stack([rng.integers(0, spec.Nz, 400), rng.integers(0, W, 400),
                    rng.integers(0, W, 400)], axis=1)
    gw = oracle.backproject_points(Hp_want, Nx, Ny, Ks, Kt, fn, pts)
    ga = oracle.backproject_points(np.abs(Hp_want), Nx, Ny, Ks, Kt, np.abs(fn), pts)
    gg = g.detach().cpu().numpy()[pts[:, 0], pts[:, 1], pts[:, 2]]
    _within(gg, gw, ga, max(Ks) ** 2, "g samples")
    # dL/dH' at sampled entries, for the dL/dg autograd handed to the kernel
    r = g.grad.cpu().numpy()
    off = lfgen.depth_offsets(spec)
    zs = rng.integers(0, spec.Nz, 300)
    ent = np.array([(z, rng.integers(0, Nx), rng.integers(0, Ny), rng.integers(0, Ks[z]),
                     rng.integers(0, Kt[z])) for z in zs])
    dw = oracle.grad_hp_points(fn, r, Nx, Ny, Ks, Kt, ent)
    da = oracle.grad_hp_points(np.abs(fn), np.abs(r), Nx, Ny, Ks, Kt, ent)
    idx = [off[z] + ((p * Ny + q) * Ks[z] + u) * Kt[z] + v for z, p, q, u, v in ent]
    dHp = Hp.grad.cpu().numpy()
    _within(dHp[idx], dw, da, 64 * 64, "dL/dH' samples")
    # dL/dH is the adjoint of the map applied to dL/dH', bit for bit
    assert np.array_equal(Hg.grad.cpu().numpy().view(np.uint32),
                          oracle.transpose_adjoint(dHp, Nx, Ny, Ks, Kt).view(np.uint32))


def test_projector_validation(lf):
    plan16 = lf.Plan(5, 5, [15], [15], torch.float16)
    x = torch.zeros(plan16.elems, dtype=torch.float16, device="cuda")
    f = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(lf.LfbpError, match="DTYPE"):
        lf.backproject_volume_raw(plan16, x, f)
