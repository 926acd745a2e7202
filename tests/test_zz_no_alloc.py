"""The no-allocation batched entry point, called through the C-ABI (needs a GPU).

lfbp_backproject_batched_noalloc serves callers that may not allocate device
memory (for instance a host application that owns all device memory in its
own pool): it keeps the kernel's work list in a fixed array inside the library
instead of allocating one.  These tests compare its output with the oracle's
H' bit for bit (the map moves values, so the two must agree exactly), on two
calls in a row with one list of plans, then on a second list and the first
again.  Its size limit is checked on the CPU (tests/test_abi.py), before any
CUDA call, so no test here hands the library an address that is not a live
allocation.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_2003_09133_gb300 as m
    m.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return m


def _bits(n, dtype, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    if dtype == torch.float32:
        x = torch.randint(-2 ** 31, 2 ** 31 - 1, (n,), generator=g, dtype=torch.int64)
        return x.to(torch.int32).view(torch.float32).cuda()
    x = torch.randint(-2 ** 15, 2 ** 15 - 1, (n,), generator=g, dtype=torch.int32)
    return x.to(torch.int16).view(torch.float16).cuda()


def _noalloc(lf, plans, Hs, outs):
    lib = lf.load()
    P = ctypes.c_void_p
    n = len(plans)
    hp = (P * n)(*[p.handle for p in plans])
    ip = (P * n)(*[h.data_ptr() for h in Hs])
    op = (P * n)(*[o.data_ptr() for o in outs])
    return lib.lfbp_backproject_batched_noalloc(n, ctypes.cast(hp, P), ctypes.cast(ip, P),
                                                ctypes.cast(op, P),
                                                torch.cuda.current_stream().cuda_stream)


def _oracle_bits(plan, H):
    """H' of the oracle (the transpose of Eq. 1's operator) as raw bit patterns."""
    import oracle
    h = H.cpu().numpy()
    want = oracle.transpose(h, plan.Nx, plan.Ny, plan.Ks, plan.Kt)
    return want.view(np.uint32 if h.dtype == np.float32 else np.uint16)


def _bits_of(t):
    a = t.cpu().numpy()
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint16)


def _check_call(lf, plans, seed):
    Hs = [_bits(p.elems, p.dtype, seed + i) for i, p in enumerate(plans)]
    outs = [torch.full_like(h, float("nan")) for h in Hs]
    assert _noalloc(lf, plans, Hs, outs) == 0, lf.load().lfbp_last_error()
    lf.sync_status()
    for p, h, o in zip(plans, Hs, outs):
        assert np.array_equal(_bits_of(o), _oracle_bits(p, h)), f"seed {seed}"


def test_noalloc_matches_the_oracle_over_changing_lists(lf):
    """Two calls in a row with one list of plans, then another list (which
    replaces the array's contents), then the first list again: every output
    equals the oracle's H' bit for bit."""
    shapes = [(5, 5, [15, 25, 15], [15, 25, 15], torch.float32),
              (19, 19, [57, 133], [57, 133], torch.float16),
              (3, 7, [9, 27], [21, 35], torch.float32)]
    plans_x = [lf.Plan(a, b, c, d, t) for a, b, c, d, t in shapes]
    plans_y = [lf.Plan(11, 11, [33, 99], [33, 99], torch.float32)]
    for plans, seed in [(plans_x, 0), (plans_x, 100), (plans_y, 7), (plans_x, 200)]:
        _check_call(lf, plans, seed)


def test_empty_arrays_alone_and_inside_a_batch(lf):
    """Empty inputs: a plan without depths maps to an empty H' through every
    entry point, and an empty array inside a batch leaves the others exact."""
    import oracle
    empty = lf.Plan(5, 5, [], [], torch.float32)
    E = torch.empty(0, dtype=torch.float32, device="cuda")
    assert lf.backproject_array(empty, E).numel() == 0
    assert lf.adjoint(empty, E).numel() == 0
    assert lf.backproject_batched([empty], [E])[0].numel() == 0
    lf.sync_status()
    plan = lf.Plan(5, 3, [15, 9], [9, 21], torch.float32)
    H = _bits(plan.elems, torch.float32, 11)
    want = oracle.transpose(H.cpu().numpy(), 5, 3, [15, 9], [9, 21])
    got = lf.backproject_batched([empty, plan, empty], [E, H, E])
    lf.sync_status()
    assert got[0].numel() == 0 and got[2].numel() == 0
    assert np.array_equal(got[1].cpu().numpy().view(np.uint32), want.view(np.uint32))
    outs = [torch.empty_like(E), torch.full_like(H, float("nan"))]
    assert _noalloc(lf, [empty, plan], [E, H], outs) == 0
    lf.sync_status()
    assert np.array_equal(outs[1].cpu().numpy().view(np.uint32), want.view(np.uint32))
