"""The C-ABI library loads, exports what include/lfbp.h declares, and
validates its arguments on the host (CPU only: no call here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lfbp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2003_09133_gb300 import _lib
    return _lib.load(build_if_missing=True)


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lfbp_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lfbp_backproject_array" in names and "lfbp_adjoint" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2003_09133_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def _c_kind(decl):
    """'p' (pointer or opaque plan handle), 'i' (int or enum), 's' (size_t),
    'c' (const char*) or '' (void) for one C type or parameter."""
    decl = decl.strip()
    if decl in ("void", ""):
        return ""
    if re.match(r"const\s+char\s*\*", decl):
        return "c"
    if "*" in decl or re.match(r"(const\s+)?lfbp_plan\b", decl):
        return "p"
    if decl.startswith("size_t"):
        return "s"
    if re.match(r"(int|lfbp_dtype|lfbp_mode)\b", decl):
        return "i"
    raise AssertionError(f"unexpected C type in the header: {decl!r}")


def test_binding_signatures_match_the_header():
    """Every argument and return type the binding marshals has the kind the
    header declares (a pointer passed as an int, or a size_t as an int, would
    be truncated on a 64-bit host)."""
    from paper_2003_09133_gb300 import _lib
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"^\s*((?:const\s+)?[a-z_]+\s*\**)\s*(lfbp_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                       text, flags=re.M)
    assert sorted(d[1] for d in decls) == _declared()
    kinds = {ctypes.c_void_p: "p", ctypes.c_int: "i", ctypes.c_size_t: "s",
             ctypes.c_char_p: "c", None: ""}
    for ret, name, params in decls:
        args, res = _lib.SIGNATURES[name]
        want = [_c_kind(a) for a in params.split(",")] if params.strip() != "void" else []
        got = [kinds.get(a, "p" if isinstance(a, type) and issubclass(a, ctypes._Pointer) else "?")
               for a in args]
        assert got == want, (name, got, want)
        assert kinds[res] == _c_kind(ret), (name, res, ret)


def _plan(lib, Nx, Ny, Ks, Kt, dt=0, mode=0):
    h = ctypes.c_void_p()
    n = len(Ks)
    ks = (ctypes.c_int * max(1, n))(*Ks)
    kt = (ctypes.c_int * max(1, n))(*Kt)
    rc = lib.lfbp_plan_create2(ctypes.byref(h), Nx, Ny, n, ctypes.cast(ks, ctypes.c_void_p),
                               ctypes.cast(kt, ctypes.c_void_p), dt, mode)
    return rc, h


@pytest.mark.parametrize("args,code", [
    ((4, 5, [15], [15]), -1),      # even Nx (Sec. 4 requires odd n_x)
    ((5, 6, [15], [15]), -1),      # even Ny
    ((5, 5, [14], [15]), -1),      # even Ks
    ((5, 5, [15], [0]), -1),       # Kt < 1
    ((0, 5, [15], [15]), -1),
    ((1025, 5, [15], [15]), -1),   # beyond the supported cell size
    ((5, 5, [15], [15], 7), -5),   # unknown dtype
    ((5, 5, [15], [15], 0, 3), -9),  # unknown mode
])
def test_plan_validation(lib, args, code):
    rc, h = _plan(lib, *args)
    assert rc == code
    assert not h.value
    assert lib.lfbp_last_error()


def test_plan_sizes_and_offsets(lib):
    Ks, Kt = [15, 5, 25], [9, 3, 27]
    rc, h = _plan(lib, 5, 3, Ks, Kt, 1)
    assert rc == 0
    sizes = [5 * 3 * a * b for a, b in zip(Ks, Kt)]
    assert lib.lfbp_plan_elems(h) == sum(sizes)
    assert lib.lfbp_plan_esize(h) == 2
    acc = 0
    for z in range(3):
        assert lib.lfbp_plan_depth_offset(h, z) == acc
        acc += sizes[z]
    assert lib.lfbp_plan_depth_offset(h, 3) == acc
    lib.lfbp_plan_destroy(h)


def test_empty_plan(lib):
    rc, h = _plan(lib, 5, 5, [], [])
    assert rc == 0 and lib.lfbp_plan_elems(h) == 0
    lib.lfbp_plan_destroy(h)


def test_empty_inputs_return_before_any_cuda_call(lib):
    """An empty plan (no depths) and batches of empty plans succeed with NULL
    buffers on a machine without a GPU: the map entry points return before
    their first CUDA call, so nothing is launched or allocated."""
    rc, h = _plan(lib, 5, 5, [], [])
    assert rc == 0
    assert lib.lfbp_backproject_array(h, None, None, None) == 0
    assert lib.lfbp_adjoint(h, None, None, None) == 0
    assert lib.lfbp_backproject_array_host(h, None, None, None, None, None) == 0
    plans = (ctypes.c_void_p * 3)(h, h, h)
    nul = (ctypes.c_void_p * 3)(None, None, None)
    assert lib.lfbp_backproject_batched(3, plans, nul, nul, None) == 0
    assert lib.lfbp_backproject_batched_noalloc(3, plans, nul, nul, None) == 0
    assert lib.lfbp_backproject_batched(0, None, None, None, None) == 0
    lib.lfbp_plan_destroy(h)


def test_buffer_validation_before_any_launch(lib):
    rc, h = _plan(lib, 5, 5, [15], [15])
    assert rc == 0
    nbytes = 5 * 5 * 15 * 15 * 4
    A, B = 0x10000000, 0x20000000   # never dereferenced: validation fails first
    assert lib.lfbp_backproject_array(None, A, B, None) == -2
    assert lib.lfbp_backproject_array(h, None, B, None) == -2
    assert lib.lfbp_backproject_array(h, A + 4, B, None) == -3
    assert lib.lfbp_backproject_array(h, A, B + 8, None) == -3
    assert lib.lfbp_backproject_array(h, A, A, None) == -4
    assert lib.lfbp_backproject_array(h, A, A + ((nbytes - 16) & ~15), None) == -4
    assert lib.lfbp_adjoint(h, A, A + 16, None) == -4
    assert b"overlap" in lib.lfbp_last_error()
    arr = (ctypes.c_void_p * 1)(h)
    ins = (ctypes.c_void_p * 1)(A)
    outs = (ctypes.c_void_p * 1)(A + 32)
    P = ctypes.c_void_p
    assert lib.lfbp_backproject_batched(1, ctypes.cast(arr, P), ctypes.cast(ins, P),
                                        ctypes.cast(outs, P), None) == -4
    assert lib.lfbp_backproject_batched(65, ctypes.cast(arr, P), ctypes.cast(ins, P),
                                        ctypes.cast(outs, P), None) == -9
    assert lib.lfbp_backproject_batched(0, None, None, None, None) == 0
    lib.lfbp_plan_destroy(h)


def test_rl_step_validation_before_any_launch(lib):
    """Eq. (2) entry points reject bad arguments before touching the GPU."""
    rc, h = _plan(lib, 3, 3, [9], [9])
    assert rc == 0
    W = 12
    img, vol = W * W * 4, W * W * 4
    H, Hp, norm, f, g, out, work = (0x10000000 + i * 0x01000000 for i in range(7))
    assert lib.lfbp_rl_step(h, H, None, norm, f, W, W, g, out, work, None) == -2
    assert lib.lfbp_rl_step_fused(None, H, norm, f, W, W, g, out, work, None) == -2
    assert lib.lfbp_rl_step_fused(h, H, norm, f, 0, W, g, out, work, None) == -1
    assert lib.lfbp_rl_step_fused(h, H, norm, f, W, W, g, out, None, None) == -2
    assert lib.lfbp_rl_step_fused(h, H, norm + 2, f, W, W, g, out, work, None) == -3
    assert lib.lfbp_rl_step_fused(h, H, norm, f, W, W, g, out, out + 64, None) == -4
    assert lib.lfbp_rl_step_fused(h, H, norm, f, W, W, g, g + 4, work, None) == -4
    assert lib.lfbp_rl_step_fused(h, H, norm, f, W, W, g, norm, work, None) == -4
    assert lib.lfbp_rl_normaliser(h, H, None, W, W, norm, norm + 8, None) == -4
    rc, h16 = _plan(lib, 3, 3, [9], [9], 1)
    assert lib.lfbp_rl_step_fused(h16, H, norm, f, W, W, g, out, work, None) == -5
    assert lib.lfbp_backproject_volume_from_h(h16, H, f, W, W, g, None) == -5
    lib.lfbp_plan_destroy(h)
    lib.lfbp_plan_destroy(h16)


def test_python_binding_refuses_without_library(monkeypatch, tmp_path):
    from paper_2003_09133_gb300 import _lib, build
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_injected_plan_failure(lib, monkeypatch):
    """LFBP_FAULT=plan: plan creation fails as an allocation failure would,
    leaves no handle, and the next call without the injection succeeds."""
    monkeypatch.setenv("LFBP_FAULT", "plan")
    rc, h = _plan(lib, 5, 5, [15], [15])
    assert rc == -8 and not h.value
    assert b"injected" in lib.lfbp_last_error()
    monkeypatch.delenv("LFBP_FAULT")
    rc, h = _plan(lib, 5, 5, [15], [15])
    assert rc == 0 and h.value
    lib.lfbp_plan_destroy(h)


def test_gradient_validation_sizes_the_gradient_volume(lib):
    """lfbp_backproject_volume_grad's dL/dg is an Nz x Wx x Wy volume: an output
    starting inside it (or inside f) is an overlap, rejected before any launch.
    (That an output right after it is accepted is checked on the GPU.)"""
    rc, h = _plan(lib, 3, 3, [9, 15], [9, 15])   # 3*3*(81+225) = 2754 elements
    assert rc == 0
    W = 12
    vol = 2 * W * W * 4                          # 1152 bytes: smaller than the plan
    f, dg = 0x10000000, 0x20000000
    assert lib.lfbp_backproject_volume_grad(h, f, dg, W, W, dg + vol - 16, None) == -4
    assert lib.lfbp_backproject_volume_grad(h, f, dg, W, W, f + W * W * 4 - 16, None) == -4
    lib.lfbp_plan_destroy(h)


def test_even_cutouts_need_the_paper_window(lib):
    """Even Ks or Kt: Eq. 8 then defines a partial map, so only the literal
    paper-window mode takes it (every map entry point does); the projectors,
    which need a cut-out centre, reject such a plan before any launch."""
    rc, h = _plan(lib, 5, 3, [14, 15], [15, 6], 0, 0)
    assert rc == -1 and not h.value
    rc, h = _plan(lib, 5, 3, [14, 15], [15, 6], 0, 1)
    assert rc == 0 and h.value
    assert lib.lfbp_plan_elems(h) == 5 * 3 * (14 * 15 + 15 * 6)
    A, B = 0x10000000, 0x20000000   # never dereferenced: validation fails first
    assert lib.lfbp_backproject_volume_from_h(h, A, B, 12, 12, 0x30000000, None) in (-1, -5)
    assert lib.lfbp_rl_normaliser(h, A, None, 12, 12, B, 0x30000000, None) in (-1, -5)
    lib.lfbp_plan_destroy(h)


def test_noalloc_size_check_before_any_cuda_call(lib, monkeypatch):
    """The no-allocation batched entry point counts a batch's tiles and refuses
    one that its fixed work-list array cannot hold before its first CUDA call,
    so the (never dereferenced) buffer addresses below are safe on a machine
    without a GPU.  One depth of 51 x 51 cells with 1001 x 1001 cut-outs needs
    459,459 tiles at the default 32 KiB target but 255,255 with 48 KiB tiles:
    it fits through the larger-tile fallback; two such depths do not.  (Each
    depth adds a few slots for its tile shapes.)"""
    import torch
    if torch.cuda.is_available():
        pytest.skip("fake buffer addresses may only meet a library that has no GPU")
    monkeypatch.delenv("LFBP_TILE_BYTES", raising=False)
    P = ctypes.c_void_p
    A, B = 1 << 40, (1 << 40) + (1 << 39)
    ins = ctypes.cast((P * 1)(A), P)
    outs = ctypes.cast((P * 1)(B), P)
    rc, two = _plan(lib, 51, 51, [1001] * 2, [1001] * 2)
    assert rc == 0
    assert lib.lfbp_backproject_batched_noalloc(1, ctypes.cast((P * 1)(two), P), ins, outs,
                                                None) == -1
    msg = lib.lfbp_last_error().decode()
    need = int(re.search(r"needs (\d+) descriptor slots", msg).group(1))
    assert need >= 510510 and "at most 262144" in msg
    rc, one = _plan(lib, 51, 51, [1001], [1001])
    assert rc == 0
    for tile_bytes in (None, "16384", "65536"):
        if tile_bytes:
            monkeypatch.setenv("LFBP_TILE_BYTES", tile_bytes)
        # past the size check: the next step is the first CUDA call, which
        # fails here for want of a device
        assert lib.lfbp_backproject_batched_noalloc(1, ctypes.cast((P * 1)(one), P), ins, outs,
                                                    None) == -6, tile_bytes
        assert b"cudaGetDevice" in lib.lfbp_last_error()
    lib.lfbp_plan_destroy(one)
    lib.lfbp_plan_destroy(two)


@pytest.mark.parametrize("nparts", [1, 2, 3, 4, 8, 64])
def test_plan_partition_covers_and_balances(lib, nparts):
    """Contiguous depth ranges covering every depth once, each boundary at the
    depth start nearest to its share of the elements (host only)."""
    Ks = [15 * (3 + 2 * (abs(z - 25) // 5)) for z in range(51)]   # the mid workload's cut-outs
    rc, h = _plan(lib, 15, 15, Ks, Ks)
    assert rc == 0
    off = [lib.lfbp_plan_depth_offset(h, z) for z in range(len(Ks) + 1)]
    total = off[-1]
    z0, z1 = ctypes.c_int(), ctypes.c_int()
    prev = 0
    for part in range(nparts):
        assert lib.lfbp_plan_partition(h, nparts, part, ctypes.byref(z0), ctypes.byref(z1)) == 0
        assert z0.value == prev and z1.value >= z0.value
        if part + 1 < nparts:
            target = total * (part + 1) / nparts
            best = min(abs(o - target) for o in off)
            assert abs(off[z1.value] - target) == best
        prev = z1.value
    assert prev == len(Ks)
    assert lib.lfbp_plan_partition(h, 0, 0, ctypes.byref(z0), ctypes.byref(z1)) == -9
    assert lib.lfbp_plan_partition(h, 2, 2, ctypes.byref(z0), ctypes.byref(z1)) == -9
    lib.lfbp_plan_destroy(h)


def test_binding_has_no_cpu_path():
    """The binding refuses host tensors before calling the library: there is no
    CPU fallback for any step of the path."""
    import torch
    import paper_2003_09133_gb300 as lf
    lf.load(build_if_missing=True)
    plan = lf.Plan(3, 3, [9], [9], torch.float32)
    H = torch.zeros(plan.elems)                      # a host tensor
    with pytest.raises(ValueError, match="CUDA"):
        lf.backproject_array(plan, H)
    with pytest.raises(ValueError, match="CUDA"):
        lf.backproject_batched([plan], [H])
    with pytest.raises(ValueError, match="CUDA"):
        lf.adjoint(plan, H)
    f, g = torch.zeros((12, 12)), torch.zeros((1, 12, 12))
    for call in (lambda: lf.backproject_volume_from_h(plan, H, f),
                 lambda: lf.forward_project(plan, H, g),
                 lambda: lf.backproject_volume_grad(plan, f, g)):
        with pytest.raises((ValueError, TypeError)):
            call()
