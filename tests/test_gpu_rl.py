"""The Richardson-Lucy update (Eq. 2) and the backprojection read straight
from H, on the GPU, against the CPU oracle.

All data are non-negative (a PSF, a volume, an image), so every fp32 sum has
a relative error of at most n * 2^-23 for n products, and the errors of the
update's parts add up (first order) to

    |gpu - oracle| <= (n1 + 2 n2 + 4) * 2^-23 * |oracle|

per voxel: n1 products in the forward sum of a pixel (all depths), n2 in
the backprojection of a voxel (its depth), once for H' (f / Hg) and once for
the normaliser H' 1, plus the quotient, the division by the normaliser and
the product (one rounding each, and one spare).
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


def _close(got, want, rtol, what):
    tol = rtol * np.abs(want) + 1e-30
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.flatnonzero(bad.reshape(-1))[:5]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside the bound; first {i}: "
                             f"got {got.reshape(-1)[i]} want {want.reshape(-1)[i]}")


def _rl_rtol(Ks, Kt):
    n1 = sum(a * b for a, b in zip(Ks, Kt))
    n2 = np.array([a * b for a, b in zip(Ks, Kt)], dtype=np.float64)
    return ((n1 + 2 * n2 + 4) * EPS32)[:, None, None]


CASES = [  # Nx, Ny, Ks, Kt, Wx, Wy
    (3, 3, [9, 3], [9, 3], 12, 12),
    (3, 5, [9, 15], [5, 25], 14, 23),
    (5, 5, [15, 5, 25], [15, 5, 25], 37, 40),
    (1, 1, [3], [5], 9, 7),
    (11, 11, [33, 99], [33, 99], 66, 77),
    (3, 5, [9] * 5 + [15], [15] * 5 + [5], 30, 41),  # five equal cut-outs: several depths per block
    (3, 3, [9, 15, 9, 9], [9, 3, 9, 9], 200, 151),  # 67 x 51 pixels per cell: several tiles per phase
    # groups of equal cut-outs whose blocks have one or three sub-problems
    # (phases; a product of odd numbers), so the staging ring of the grouped
    # backprojection starts with nothing or one sub-problem behind the first;
    # three, four and ten depths go three, four and two per block
    (1, 1, [5, 5, 5], [3, 3, 3], 9, 11),
    (1, 1, [3] * 4, [3] * 4, 10, 7),
    (1, 3, [5] * 10, [7] * 10, 8, 40),
]


def _case_data(plan, case, seed):
    Nx, Ny, Ks, Kt, Wx, Wy = case
    rng = np.random.default_rng(seed)
    H = rng.uniform(0, 1, plan.elems).astype(np.float32)
    g = rng.uniform(0.1, 1, (len(Ks), Wx, Wy)).astype(np.float32)
    f = rng.uniform(0.1, 1, (Wx, Wy)).astype(np.float32)
    return H, g, f


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_W{c[4]}x{c[5]}")
def test_backproject_from_h_and_normaliser(lf, case):
    Nx, Ny, Ks, Kt, Wx, Wy = case
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    H, g, f = _case_data(plan, case, 21)
    Hd, fd = torch.from_numpy(H).cuda(), torch.from_numpy(f).cuda()
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    rtol = (np.array([a * b for a, b in zip(Ks, Kt)]) * EPS32)[:, None, None]
    want = oracle.backproject(Hp, Nx, Ny, Ks, Kt, f)
    got = lf.backproject_volume_from_h(plan, Hd, fd).cpu().numpy()
    _close(got, want, rtol, "H' f from H")
    ones = oracle.backproject(Hp, Nx, Ny, Ks, Kt, np.ones_like(f))
    Hpd = lf.backproject_array(plan, Hd)
    for hp in (Hpd, None):
        n = lf.rl_normaliser(plan, Hd, hp, Wx, Wy).cpu().numpy()
        _close(n, ones, rtol, f"H' 1 ({'H prime' if hp is not None else 'from H'})")
    lf.sync_status()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_W{c[4]}x{c[5]}")
def test_rl_step_against_oracle(lf, case):
    Nx, Ny, Ks, Kt, Wx, Wy = case
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    H, g, f = _case_data(plan, case, 22)
    Hd, gd, fd = (torch.from_numpy(a).cuda() for a in (H, g, f))
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    want = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, f)
    rtol = _rl_rtol(Ks, Kt)
    Hpd = lf.backproject_array(plan, Hd)
    norm = lf.rl_normaliser(plan, Hd, Hpd, Wx, Wy)
    got = lf.rl_step(plan, Hd, Hpd, norm, fd, gd).cpu().numpy()
    _close(got, want, rtol, "rl_step with H'")
    norm_h = lf.rl_normaliser(plan, Hd, None, Wx, Wy)
    got_f = lf.rl_step(plan, Hd, None, norm_h, fd, gd).cpu().numpy()
    _close(got_f, want, rtol, "rl_step_fused (H' never built)")
    # in place: the update may overwrite the estimate it reads (the forward
    # sum then runs inside each block instead of through per-depth partials)
    for hp in (Hpd, None):
        g2 = gd.clone()
        lf.rl_step(plan, Hd, hp, norm if hp is not None else norm_h, fd, g2, out=g2)
        _close(g2.cpu().numpy(), want, rtol, "rl_step in place")
    lf.sync_status()


def test_rl_zero_readings(lf):
    """H g = 0 pixels give a zero quotient; H' 1 = 0 voxels give 0 (oracle's readings)."""
    Nx, Ny, Ks, Kt, Wx, Wy = 3, 3, [9, 3], [9, 3], 12, 12
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    H, g, f = _case_data(plan, (Nx, Ny, Ks, Kt, Wx, Wy), 23)
    H[Nx * Ny * 81:] = 0.0      # depth 1 has an all-zero PSF: its normaliser is 0
    g[0, :, :6] = 0.0           # half the volume of depth 0 empty: some pixels see H g = 0
    g[1] = 0.0
    Hd, gd, fd = (torch.from_numpy(a).cuda() for a in (H, g, f))
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    want = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g, f)
    norm = lf.rl_normaliser(plan, Hd, None, Wx, Wy)
    got = lf.rl_step(plan, Hd, None, norm, fd, gd).cpu().numpy()
    assert (got[1] == 0).all() and (want[1] == 0).all()
    assert ((got[0] == 0) == (want[0] == 0)).all()
    _close(got, want, _rl_rtol(Ks, Kt), "rl_step zeros")


def test_rl_iterations_autograd_workload_crop(lf):
    """Three updates on the differentiation workload's PSF (N = 11, 21 depths,
    K up to 99), an 8 x 8-lenslet crop of its raw image, starting from ones:
    the fused and the H' forms against the oracle after each update, and the
    oracle's flux identity sum (H'1) g' = sum f on the GPU's result."""
    spec = lfgen.config_specs("autograd")[0]
    Nx, Ny, Ks, Kt = spec.Nx, spec.Ny, list(spec.Ks), list(spec.Kt)
    Wx = Wy = 8 * Nx
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    Hd = lfgen.generate(spec, device="cuda")
    H = Hd.cpu().numpy()
    f = lfgen.raw_image(64, Nx, 19)[:Wx, :Wy].astype(np.float32).copy()  # the workload's image, cropped
    fd = torch.from_numpy(f).cuda()
    Hp = oracle.transpose(H, Nx, Ny, Ks, Kt)
    norm_o = oracle.backproject(Hp, Nx, Ny, Ks, Kt, np.ones_like(f))
    Hpd = lf.backproject_array(plan, Hd)
    norm = lf.rl_normaliser(plan, Hd, Hpd, Wx, Wy)
    norm_h = lf.rl_normaliser(plan, Hd, None, Wx, Wy)
    g_o = np.ones((len(Ks), Wx, Wy))
    g_a = torch.ones((len(Ks), Wx, Wy), device="cuda")
    g_b = g_a.clone()
    rtol1 = _rl_rtol(Ks, Kt)
    for it in range(3):
        # each update starts from the oracle's previous estimate rounded to
        # fp32, so the bound of one update applies
        g32 = g_o.astype(np.float32)
        g_in = torch.from_numpy(g32).cuda()
        g_o = oracle.rl_step(H, Hp, Nx, Ny, Ks, Kt, g32, f, norm=norm_o)
        got_a = lf.rl_step(plan, Hd, Hpd, norm, fd, g_in, out=g_a).cpu().numpy()
        got_b = lf.rl_step(plan, Hd, None, norm_h, fd, g_in, out=g_b).cpu().numpy()
        _close(got_a, g_o, rtol1, f"update {it} with H'")
        _close(got_b, g_o, rtol1, f"update {it} fused")
        flux = float(np.sum(norm.cpu().numpy().astype(np.float64) * got_a))
        assert abs(flux - float(np.sum(f, dtype=np.float64))) <= 1e-3 * float(np.sum(f))
    lf.sync_status()


def test_rl_validation(lf):
    plan16 = lf.Plan(3, 3, [9], [9], torch.float16)
    H = torch.zeros(plan16.elems, dtype=torch.float16, device="cuda")
    f = torch.ones((12, 12), device="cuda")
    g = torch.ones((1, 12, 12), device="cuda")
    with pytest.raises(lf.LfbpError):
        lf.rl_step(plan16, H, None, g, f, g)
    plan = lf.Plan(3, 3, [9], [9], torch.float32)
    H32 = torch.zeros(plan.elems, device="cuda")
    work = torch.empty((12, 12), device="cuda")
    with pytest.raises(lf.LfbpError):  # the scratch image may not be the measured image
        lf.rl_step(plan, H32, None, g, f, g, work=f)
    lib = lf.load()
    rc = lib.lfbp_rl_step(plan.handle, H32.data_ptr(), None, g.data_ptr(), f.data_ptr(), 12, 12,
                          g.data_ptr(), g.data_ptr(), work.data_ptr(), None)
    assert rc == -2


def test_projectors_are_deterministic(lf):
    """Fixed-order fp32 sums, no atomics: repeated calls give identical bits."""
    spec = lfgen.config_specs("autograd")[0]
    Nx, Ny, Ks, Kt = spec.Nx, spec.Ny, list(spec.Ks), list(spec.Kt)
    W = 6 * Nx
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    Hd = lfgen.generate(spec, device="cuda")
    f = torch.from_numpy(lfgen.raw_image(64, Nx, 19)[:W, :W].astype(np.float32).copy()).cuda()
    g = torch.rand((len(Ks), W, W), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    norm = lf.rl_normaliser(plan, Hd, None, W, W)
    outs = [lf.rl_step(plan, Hd, None, norm, f, g).cpu().numpy() for _ in range(2)]
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    grads = [lf.backproject_volume_grad(plan, f, g).cpu().numpy() for _ in range(2)]
    assert np.array_equal(grads[0].view(np.uint32), grads[1].view(np.uint32))
    fw = [lf.forward_project(plan, Hd, g).cpu().numpy() for _ in range(2)]
    assert np.array_equal(fw[0].view(np.uint32), fw[1].view(np.uint32))
    lf.sync_status()


def test_tma_and_cpasync_staging_agree_bitwise(lf, monkeypatch):
    """The projectors and the H'-gradient stage their input tiles either by
    TMA tensor copies from the inputs laid out by phase (default; the
    single-depth projector as a producer/consumer pipeline, or with block
    barriers under LFBP_PROJ_PIPE=0) or by 4-byte cp.async copies
    (LFBP_PROJ_TMA=0).  Both feed the same products in the same
    order, so the normaliser, both forms of the update, the backprojection and
    the gradient agree bit for bit; rows and columns outside the sensor arrive
    as zeros either way."""
    spec = lfgen.config_specs("autograd")[0]
    cases = CASES + [(spec.Nx, spec.Ny, list(spec.Ks), list(spec.Kt), 7 * spec.Nx + 5, 6 * spec.Ny)]
    for Nx, Ny, Ks, Kt, Wx, Wy in cases:
        plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
        H, g, f = _case_data(plan, (Nx, Ny, Ks, Kt, Wx, Wy), 24)
        Hd, gd, fd = (torch.from_numpy(a).cuda() for a in (H, g, f))
        res = {}
        for mode in ("1", "0", "1-nopipe"):
            monkeypatch.setenv("LFBP_PROJ_TMA", mode[0])
            monkeypatch.setenv("LFBP_PROJ_PIPE", "0" if mode.endswith("nopipe") else "1")
            norm = lf.rl_normaliser(plan, Hd, None, Wx, Wy)
            out = lf.rl_step(plan, Hd, None, norm, fd, gd)
            g2 = gd.clone()
            lf.rl_step(plan, Hd, None, norm, fd, g2, out=g2)
            vol = lf.backproject_volume_from_h(plan, Hd, fd)
            grad = lf.backproject_volume_grad(plan, fd, gd)
            lf.sync_status()
            res[mode] = [x.cpu().numpy() for x in (norm, out, g2, vol, grad)]
        for other in ("0", "1-nopipe"):
            for what, a, b in zip(("normaliser", "update", "update in place", "backprojection",
                                   "gradient"), res["1"], res[other]):
                assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), \
                    (Nx, Ny, Ks, Wx, Wy, what, other)


def test_gradient_output_right_after_the_gradient_volume(lf):
    """dL/dg sized as an Nz x Wx x Wy volume (smaller than the plan here): an
    output placed right after it in one allocation is accepted and correct."""
    Nx, Ny, Ks, W = 3, 3, [9, 15], 12
    plan = lf.Plan(Nx, Ny, Ks, Ks, torch.float32)
    nvol = len(Ks) * W * W
    buf = torch.zeros(nvol + plan.elems, device="cuda")
    dg, out = buf[:nvol].view(len(Ks), W, W), buf[nvol:]
    dg.copy_(torch.rand((len(Ks), W, W), device="cuda", generator=torch.Generator("cuda").manual_seed(3)))
    f = torch.rand((W, W), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    lf.backproject_volume_grad(plan, f, dg, out=out)
    want = lf.backproject_volume_grad(plan, f, dg.clone())
    lf.sync_status()
    assert torch.equal(out, want)
