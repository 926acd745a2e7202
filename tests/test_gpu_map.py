"""GPU parity of H -> H' against the CPU oracle, bit for bit (needs a GB300).

Every comparison is on raw bit patterns: the map only moves values, so fp32
and fp16 results must equal the oracle's exactly, NaN payloads included.
"""
import numpy as np
import pytest
import torch

import lfgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_2003_09133_gb300 as m
    m.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return m


def _bits(a: np.ndarray):
    return a.view(np.uint32 if a.itemsize == 4 else np.uint16)


def _assert_same_bits(got: torch.Tensor, want: np.ndarray, what=""):
    g = got.cpu().numpy()
    gb, wb = _bits(g), _bits(want)
    if not np.array_equal(gb, wb):
        bad = np.flatnonzero(gb != wb)
        raise AssertionError(f"{what}: {bad.size} of {gb.size} elements differ, first at {bad[:8]}")


def _random_bits(n, dtype, seed, device="cuda"):
    g = torch.Generator(device="cpu").manual_seed(seed)
    if dtype == torch.float32:
        x = torch.randint(-2 ** 31, 2 ** 31 - 1, (n,), generator=g, dtype=torch.int64)
        return x.to(torch.int32).view(torch.float32).to(device)
    x = torch.randint(-2 ** 15, 2 ** 15 - 1, (n,), generator=g, dtype=torch.int32)
    return x.to(torch.int16).view(torch.float16).to(device)


SHAPES = [
    (5, 5, [15, 15, 15], [15, 15, 15]),
    (3, 5, [9, 3, 15], [15, 5, 5]),
    (1, 1, [5, 1, 9], [7, 1, 3]),
    (7, 3, [21, 7], [9, 33]),
    (19, 19, [95, 57, 19], [95, 57, 19]),
    (11, 11, [99, 33, 11], [99, 33, 11]),
    (9, 13, [27, 3, 1], [39, 13, 5]),
    (51, 51, [153], [153]),           # rows larger than one stage: column-split tiles
    (31, 31, [249], [249]),
    (95, 55, [181], [181]),           # the non-square R29 cell shape (Table 1, Sec. 5)
    (11, 11, [89], [89]),             # K not a multiple of N (Table 1 shapes)
]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}")
def test_random_bits_plain_batched_adjoint(lf, shape, dtype):
    Nx, Ny, Ks, Kt = shape
    plan = lf.Plan(Nx, Ny, Ks, Kt, dtype)
    H = _random_bits(plan.elems, dtype, 11)
    Hn = H.cpu().numpy()
    want = oracle.transpose(Hn, Nx, Ny, Ks, Kt)
    _assert_same_bits(lf.backproject_array(plan, H), want, "plain")
    _assert_same_bits(lf.backproject_batched([plan], [H])[0], want, "batched")
    _assert_same_bits(lf.adjoint(plan, H), oracle.transpose_adjoint(Hn, Nx, Ny, Ks, Kt), "adjoint")
    lf.sync_status()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}")
def test_random_bits_batched_lsu_copies(lf, shape, dtype, monkeypatch):
    """The persistent kernel with its segments moved by 16-byte cp.async copies
    (LFBP_LOADS=lsu) instead of TMA bulk copies: the same bits, both modes."""
    monkeypatch.setenv("LFBP_LOADS", "lsu")
    Nx, Ny, Ks, Kt = shape
    plan = lf.Plan(Nx, Ny, Ks, Kt, dtype)
    H = _random_bits(plan.elems, dtype, 14)
    Hn = H.cpu().numpy()
    _assert_same_bits(lf.backproject_batched([plan], [H])[0],
                      oracle.transpose(Hn, Nx, Ny, Ks, Kt), "batched lsu")
    pw = lf.Plan(Nx, Ny, Ks, Kt, dtype, mode=lf.MAP_PAPER_WINDOW)
    _assert_same_bits(lf.backproject_batched([pw], [H])[0],
                      oracle.paper_window(Hn, Nx, Ny, Ks, Kt), "batched lsu, paper window")
    lf.sync_status()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("shape", SHAPES[:7], ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}")
def test_paper_window_mode(lf, shape, dtype):
    Nx, Ny, Ks, Kt = shape
    plan = lf.Plan(Nx, Ny, Ks, Kt, dtype, mode=lf.MAP_PAPER_WINDOW)
    H = _random_bits(plan.elems, dtype, 12)
    Hn = H.cpu().numpy()
    _assert_same_bits(lf.backproject_array(plan, H), oracle.paper_window(Hn, Nx, Ny, Ks, Kt), "plain")
    _assert_same_bits(lf.backproject_batched([plan], [H])[0],
                      oracle.paper_window(Hn, Nx, Ny, Ks, Kt), "batched")
    keep = oracle.paper_window(np.ones(plan.elems), Nx, Ny, Ks, Kt) != 0
    Y = Hn.copy()
    Y[~keep] = 0
    _assert_same_bits(lf.adjoint(plan, H), oracle.transpose_adjoint(Y, Nx, Ny, Ks, Kt), "adjoint")
    lf.sync_status()


def test_guard_bands_untouched(lf):
    """Canaries around the output catch any write outside it."""
    Nx, Ny, Ks, Kt = 7, 5, [21, 9, 35], [15, 5, 45]
    for dtype in (torch.float32, torch.float16):
        plan = lf.Plan(Nx, Ny, Ks, Kt, dtype)
        n = plan.elems
        H = _random_bits(n, dtype, 13)
        pad = 64 // plan.esize  # 64 bytes on each side, keeps 16-byte alignment
        buf = torch.full((n + 2 * pad,), float("nan"), dtype=dtype, device="cuda")
        canary = buf.clone()
        out = buf[pad:pad + n]
        lf.backproject_array(plan, H, out)
        lf.backproject_batched([plan], [H], [out])
        torch.cuda.synchronize()
        assert torch.equal(buf[:pad].view(torch.int16 if dtype == torch.float16 else torch.int32),
                           canary[:pad].view(torch.int16 if dtype == torch.float16 else torch.int32))
        assert torch.equal(buf[pad + n:].view(torch.int16 if dtype == torch.float16 else torch.int32),
                           canary[pad + n:].view(torch.int16 if dtype == torch.float16 else torch.int32))
        _assert_same_bits(out, oracle.transpose(H.cpu().numpy(), Nx, Ny, Ks, Kt), "guarded")


def test_special_bit_patterns(lf):
    Nx, Ny, Ks, Kt = 5, 5, [15], [15]
    plan = lf.Plan(Nx, Ny, Ks, Kt, torch.float32)
    bits = np.random.default_rng(14).integers(0, 2 ** 32, plan.elems, dtype=np.uint64).astype(np.uint32)
    bits[:8] = [0x7fc00001, 0x7f800001, 0xffc12345, 0x80000000, 0x7f800000, 0xff800000,
                0x00000001, 0x807fffff]
    H = torch.from_numpy(bits.view(np.float32).copy()).cuda()
    want = oracle.transpose(bits.view(np.float32), Nx, Ny, Ks, Kt)
    _assert_same_bits(lf.backproject_array(plan, H), want, "plain")
    _assert_same_bits(lf.backproject_batched([plan], [H])[0], want, "batched")


@pytest.mark.parametrize("form", ["0", "1", "2"])
def test_batched_mixed_dtypes_and_pointer_changes(lf, form, monkeypatch):
    """One batched launch over fp32 and fp16 arrays, replayed with new buffers (the
    graph's node parameters patched), in each batched form: persistent CTAs, one
    tile per CTA, per-depth grids (one graph node per depth of every array)."""
    monkeypatch.setenv("LFBP_FORM", form)
    shapes = [(5, 5, [15, 25], [15, 25], torch.float32), (3, 7, [9, 27, 3], [21, 7, 35], torch.float16),
              (19, 19, [57], [57], torch.float16), (11, 11, [33, 55], [33, 55], torch.float32)]
    plans = [lf.Plan(a, b, c, d, t) for a, b, c, d, t in shapes]
    for rep in range(3):
        Hs = [_random_bits(p.elems, p.dtype, 20 + rep * 10 + i) for i, p in enumerate(plans)]
        outs = lf.backproject_batched(plans, Hs)
        for p, H, o in zip(plans, Hs, outs):
            _assert_same_bits(o, oracle.transpose(H.cpu().numpy(), p.Nx, p.Ny, p.Ks, p.Kt), f"rep{rep}")
    lf.sync_status()


def test_tiny_workload(lf):
    spec = lfgen.config_specs("tiny")[0]
    H = lfgen.generate(spec).cuda()
    want = oracle.transpose(H.cpu().numpy(), spec.Nx, spec.Ny, spec.Ks, spec.Kt)
    for dtype in (torch.float32, torch.float16):
        Hd = H.to(dtype)
        wd = want.astype(np.float32).astype(np.float16) if dtype == torch.float16 else want
        plan = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, dtype)
        _assert_same_bits(lf.backproject_array(plan, Hd), wd, "plain")
        _assert_same_bits(lf.backproject_batched([plan], [Hd])[0], wd, "batched")
    pw = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float32, mode=lf.MAP_PAPER_WINDOW)
    _assert_same_bits(lf.backproject_array(pw, H),
                      oracle.paper_window(H.cpu().numpy(), spec.Nx, spec.Ny, spec.Ks, spec.Kt), "window")


def test_autograd_backward_is_the_adjoint(lf):
    spec = lfgen.config_specs("tiny")[0]
    plan = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float32)
    H = lfgen.generate(spec).cuda().requires_grad_(True)
    Hp = lf.backprojection_array(H, plan)
    w = torch.randn_like(Hp)
    (Hp * w).sum().backward()
    want = oracle.transpose_adjoint(w.cpu().numpy(), spec.Nx, spec.Ny, spec.Ks, spec.Kt)
    _assert_same_bits(H.grad, want, "grad")


def test_sync_status_ok(lf):
    lf.sync_status()


def _full_workload(lf, name, dtype=None, forms=("batched", "plain")):
    specs = lfgen.config_specs(name)
    plans, Hs = [], []
    for s in specs:
        dt = dtype or s.torch_dtype
        plans.append(lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, dt))
        Hs.append(lfgen.generate(s, device="cuda").to(dt))
    outs = {}
    if "batched" in forms:
        outs["batched"] = lf.backproject_batched(plans, Hs)
    if "plain" in forms:
        outs["plain"] = [lf.backproject_array(p, h) for p, h in zip(plans, Hs)]
    lf.sync_status()
    for i, (s, H) in enumerate(zip(specs, Hs)):
        want = oracle.transpose(H.cpu().numpy(), s.Nx, s.Ny, s.Ks, s.Kt)
        for form, o in outs.items():
            _assert_same_bits(o[i], want, f"{name}[{i}] {form}")
        for form in outs:
            outs[form][i] = None
        Hs[i] = None
        del want
        torch.cuda.empty_cache()


def test_mid_workload_full(lf):
    _full_workload(lf, "mid")


def test_highres_workload_full_fp32(lf):
    _full_workload(lf, "highres")


def test_highres_workload_full_fp16(lf):
    _full_workload(lf, "highres", dtype=torch.float16)


def test_ragged_workload_full(lf):
    _full_workload(lf, "ragged")


def test_autograd_workload_map(lf):
    _full_workload(lf, "autograd")


@pytest.mark.parametrize("path", ["copy", "copy_rotation", "zerocopy"])
def test_host_to_host_pipeline(lf, path, monkeypatch):
    """Pinned host H -> H' -> pinned host: by default aligned byte ranges are
    staged through the device buffers with overlapped copies (here 1 MB ranges,
    so that depths straddle them), the depths in memory order
    (LFBP_HOST_ORDER=rotate: in a rotation that starts at the smallest);
    LFBP_HOST_PATH=zerocopy lets the kernel read and write the mapped host
    buffers itself."""
    if path == "zerocopy":
        monkeypatch.setenv("LFBP_HOST_PATH", "zerocopy")
    else:
        monkeypatch.setenv("LFBP_HOST_CHUNK_MB", "1")
    if path == "copy_rotation":
        monkeypatch.setenv("LFBP_HOST_ORDER", "rotate")
    for name, dtype in (("mid", torch.float32), ("tiny", torch.float16)):
        spec = lfgen.config_specs(name)[0]
        plan = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, dtype)
        H = lfgen.generate(spec, device="cuda").to(dtype).cpu().pin_memory()
        out = lf.backproject_array_host(plan, H)
        torch.cuda.current_stream().synchronize()
        lf.sync_status()
        _assert_same_bits(out, oracle.transpose(H.numpy(), spec.Nx, spec.Ny, spec.Ks, spec.Kt),
                          f"host pipeline {name} ({path})")


@pytest.mark.parametrize("path", ["copy", "zerocopy"])
def test_host_to_host_pageable_and_odd_shapes(lf, path, monkeypatch):
    """Both host paths on pinned and pageable buffers (pageable ones always
    take the staged copies), on shapes with column splits, fp16, an even
    cut-out, and ranges of 1 MB that cut through depths."""
    if path == "zerocopy":
        monkeypatch.setenv("LFBP_HOST_PATH", "zerocopy")
    monkeypatch.setenv("LFBP_HOST_CHUNK_MB", "1")
    for Nx, Ny, Ks, Kt, dtype, mode in ((51, 51, [153], [153], torch.float32, 0),
                                        (9, 13, [27, 3, 1], [39, 13, 5], torch.float16, 0),
                                        (19, 19, [57, 95, 19, 133], [57, 95, 19, 133], torch.float16, 0),
                                        (5, 5, [16, 10], [16, 10], torch.float32, 1)):
        plan = lf.Plan(Nx, Ny, Ks, Kt, dtype, mode=mode)
        Hd = _random_bits(plan.elems, dtype, 15)
        Hn = Hd.cpu().numpy()
        want = (oracle.paper_window(Hn, Nx, Ny, Ks, Kt) if mode else
                oracle.transpose(Hn, Nx, Ny, Ks, Kt))
        for pinned in (True, False):
            H = Hd.cpu().pin_memory() if pinned else Hd.cpu()
            out = lf.backproject_array_host(plan, H)
            torch.cuda.current_stream().synchronize()
            lf.sync_status()
            _assert_same_bits(out, want, f"host {Nx}x{Ny} pinned={pinned} ({path})")


def test_tuner_then_batched(lf, tmp_path, monkeypatch):
    """The autotuner picks a shape from its grid; batched calls stay bit-exact after it."""
    monkeypatch.setenv("LFBP_TUNE_CACHE", str(tmp_path / "tune.txt"))
    shapes = [(5, 5, [15, 25], [15, 25], torch.float32), (19, 19, [57, 95], [57, 95], torch.float16)]
    plans = [lf.Plan(a, b, c, d, t) for a, b, c, d, t in shapes]
    Hs = [_random_bits(p.elems, p.dtype, 40 + i) for i, p in enumerate(plans)]
    tb, cps, st, pairs, form = lf.tune_batched(plans, Hs, reps=1)
    assert tb in (12288, 16384, 24576, 32768, 40960, 49152, 65536)
    assert pairs in (0, 1) and form in (0, 1, 2) and (cps in (1, 2, 3, 4) if form == 0 else cps == 0)
    assert (tmp_path / "tune.txt").read_text().strip()
    for rep in range(2):
        outs = lf.backproject_batched(plans, Hs)
        for p, H, o in zip(plans, Hs, outs):
            _assert_same_bits(o, oracle.transpose(H.cpu().numpy(), p.Nx, p.Ny, p.Ks, p.Kt), "tuned")
    # a second process-level tune reads the cache instead of timing
    assert lf.tune_batched(plans, Hs, reps=1) == (tb, cps, st, pairs, form)
    lf.sync_status()


@pytest.mark.parametrize("form", ["0", "1", "2"])
@pytest.mark.parametrize("pairs", ["1", "0"])
def test_random_bits_batched_pair_consumer_on_off(lf, pairs, form, monkeypatch):
    """The batched form with the pair consumer switched on and off (LFBP_PAIRS)
    and as persistent CTAs, one tile per CTA, or a graph of per-depth grids
    (LFBP_FORM), the autotuner's last two dimensions: the same bits either way."""
    monkeypatch.setenv("LFBP_PAIRS", pairs)
    monkeypatch.setenv("LFBP_FORM", form)
    for Nx, Ny, Ks, Kt in SHAPES:
        for dtype in (torch.float32, torch.float16):
            plan = lf.Plan(Nx, Ny, Ks, Kt, dtype)
            H = _random_bits(plan.elems, dtype, 16)
            _assert_same_bits(lf.backproject_batched([plan], [H])[0],
                              oracle.transpose(H.cpu().numpy(), Nx, Ny, Ks, Kt),
                              f"pairs={pairs} {Nx}x{Ny}")
    lf.sync_status()


def test_ragged_workload_full_tuned(lf):
    """The ragged batch in the launch shape the bench times: the autotuner's pick."""
    specs = lfgen.config_specs("ragged")
    plans = [lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, s.torch_dtype) for s in specs]
    Hs = [lfgen.generate(s, device="cuda").to(s.torch_dtype) for s in specs]
    lf.tune_batched(plans, Hs, reps=1)
    outs = lf.backproject_batched(plans, Hs)
    lf.sync_status()
    for i, (s, H) in enumerate(zip(specs, Hs)):
        want = oracle.transpose(H.cpu().numpy(), s.Nx, s.Ny, s.Ks, s.Kt)
        _assert_same_bits(outs[i], want, f"ragged[{i}] tuned")
        outs[i] = None
        Hs[i] = None
        del want
        torch.cuda.empty_cache()


def test_every_launch_shape_of_the_tuner_grid(lf, monkeypatch):
    """Each launch shape the autotuner may pick maps bit-exactly (mid workload,
    fp32, and its fp16 copy in the same batch): persistent CTAs at every tile
    size x CTAs per SM, and the two one-tile-per-CTA forms at every tile size."""
    spec = lfgen.config_specs("mid")[0]
    H32 = lfgen.generate(spec, device="cuda")
    H16 = H32.half()
    plans = [lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float32),
             lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float16)]
    want = [oracle.transpose(h.cpu().numpy(), spec.Nx, spec.Ny, spec.Ks, spec.Kt) for h in (H32, H16)]
    shapes = [("0", tb, cps) for tb in (12288, 16384, 24576, 32768, 40960, 49152, 65536)
              for cps in (1, 2, 3, 4)]
    shapes += [(form, tb, 0) for form in ("1", "2") for tb in (24576, 32768, 40960, 49152, 65536)]
    for form, tb, cps in shapes:
        monkeypatch.setenv("LFBP_FORM", form)
        monkeypatch.setenv("LFBP_TILE_BYTES", str(tb))
        monkeypatch.setenv("LFBP_CTAS_PER_SM", str(max(cps, 1)))
        outs = lf.backproject_batched(plans, [H32, H16])
        lf.sync_status()
        for o, w in zip(outs, want):
            _assert_same_bits(o, w, f"form {form} tile {tb} cps {cps}")


# Table 1 of the paper (n_s = n_t, n_x, n_y): K not a multiple of N, rows of
# up to 507 elements, cells of up to 95 x 55 positions
TABLE1 = [(89, 11, 11), (177, 11, 11), (287, 11, 11), (507, 11, 11), (91, 15, 15), (121, 15, 15),
          (211, 21, 21), (249, 31, 31), (311, 31, 31), (307, 51, 51), (181, 95, 55)]


@pytest.mark.parametrize("K,Nx,Ny", TABLE1, ids=lambda v: str(v))
def test_table1_shapes_full_size(lf, K, Nx, Ny):
    """Two depths of each Table 1 size (the full per-depth size; the paper's
    arrays repeat it 11 times), fp32 random bits, plain and batched."""
    Ks = [K, K]
    plan = lf.Plan(Nx, Ny, Ks, Ks, torch.float32)
    bits = np.random.default_rng(K * 1000 + Nx).integers(0, 2 ** 32, plan.elems, dtype=np.uint32)
    Hn = bits.view(np.float32)
    H = torch.from_numpy(Hn).cuda()
    want = oracle.transpose(Hn, Nx, Ny, Ks, Ks)
    _assert_same_bits(lf.backproject_batched([plan], [H])[0], want, "batched")
    _assert_same_bits(lf.backproject_array(plan, H), want, "plain")
    lf.sync_status()


EVEN_SHAPES = [  # Nx, Ny, Ks, Kt: the literal Eq. 8 with even n_s / n_t (paper-window mode)
    (3, 1, [4], [1]),
    (3, 3, [6, 4], [4, 9]),
    (5, 3, [14, 15], [15, 6]),
    (1, 1, [2, 8], [6, 3]),
    (19, 19, [76, 57], [76, 58]),
    (95, 55, [96], [110]),
]


def _window_sources(Nx, Ny, Ks, Kt):
    """For every H' entry the 1-based H index the literal loop copies into it
    (0: never written), from the oracle run on an index array."""
    n = sum(Nx * Ny * a * b for a, b in zip(Ks, Kt))
    idx = np.arange(1, n + 1, dtype=np.int64)
    return oracle.paper_window(idx, Nx, Ny, Ks, Kt)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("shape", EVEN_SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_K{s[2][0]}x{s[3][0]}")
def test_even_cutouts_literal_window(lf, shape, dtype):
    """Even cut-outs, literal Eqs. (4)-(9): H' bit for bit against the oracle's
    paper-window evaluation, and the adjoint moves each written entry back to
    its source (zero elsewhere)."""
    Nx, Ny, Ks, Kt = shape
    plan = lf.Plan(Nx, Ny, Ks, Kt, dtype, mode=lf.MAP_PAPER_WINDOW)
    H = _random_bits(plan.elems, dtype, 15)
    Hn = H.cpu().numpy()
    _assert_same_bits(lf.backproject_array(plan, H), oracle.paper_window(Hn, Nx, Ny, Ks, Kt),
                      "literal window")
    src = _window_sources(Nx, Ny, Ks, Kt)
    dHp = _random_bits(plan.elems, dtype, 16)
    d = dHp.cpu().numpy()
    want = np.zeros_like(d)
    w = src > 0
    want[src[w] - 1] = d[w]
    _assert_same_bits(lf.adjoint(plan, dHp), want, "literal window adjoint")
    # the batched form takes even cut-outs too, beside an odd array of the same mode
    odd = lf.Plan(5, 5, [15], [15], dtype, mode=lf.MAP_PAPER_WINDOW)
    H2 = _random_bits(odd.elems, dtype, 17)
    got = lf.backproject_batched([plan, odd], [H, H2])
    _assert_same_bits(got[0], oracle.paper_window(Hn, Nx, Ny, Ks, Kt), "literal window batched")
    _assert_same_bits(got[1], oracle.paper_window(H2.cpu().numpy(), 5, 5, [15], [15]),
                      "paper window batched (odd)")
    lf.sync_status()


def test_highres_even_cutouts_full(lf):
    """The highres workload with every cut-out one pixel larger (even K: the
    literal Eq. 8), fp32, through the batched form at full size: every depth
    bit for bit against the oracle's Eqs. 4-9, and the adjoint on every fourth
    depth (each written entry moved back to its source, zero elsewhere)."""
    spec = lfgen.config_specs("highres")[0]
    Ks = [k + 1 for k in spec.Ks]
    plan = lf.Plan(spec.Nx, spec.Ny, Ks, Ks, torch.float32, mode=lf.MAP_PAPER_WINDOW)
    g = torch.Generator(device="cuda").manual_seed(23)
    H = torch.randint(-2 ** 31, 2 ** 31 - 1, (plan.elems,), generator=g, device="cuda",
                      dtype=torch.int64).to(torch.int32).view(torch.float32)
    Hp = lf.backproject_batched([plan], [H])[0]
    dH = lf.adjoint(plan, Hp)
    lf.sync_status()
    off = [0]
    for k in Ks:
        off.append(off[-1] + spec.Nx * spec.Ny * k * k)
    for z in range(len(Ks)):
        a, b = off[z], off[z + 1]
        Hz = H[a:b].cpu().numpy()
        want = oracle.paper_window(Hz, spec.Nx, spec.Ny, [Ks[z]], [Ks[z]])
        _assert_same_bits(Hp[a:b], want, f"even highres depth {z}")
        if z % 4 == 0 or z == len(Ks) - 1:
            src = oracle.paper_window(np.arange(1, b - a + 1, dtype=np.int32), spec.Nx, spec.Ny,
                                      [Ks[z]], [Ks[z]])
            w = src > 0
            back = np.zeros_like(Hz)
            back[src[w] - 1] = want[w]
            _assert_same_bits(dH[a:b], back, f"even highres adjoint depth {z}")
