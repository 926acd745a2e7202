"""The no-allocation batched entry point, called through the C-ABI (needs a GPU).

lfbp_backproject_batched_noalloc serves callers that may not allocate device
memory (for instance a host application that owns all device memory in its
own pool): it keeps the kernel's work list in a fixed array inside the library
instead of allocating one.  These tests compare its output with that of the
ordinary batched entry point, bit for bit (the map moves values, so the two
must agree exactly), on two calls in a row, and check the size limit.  The
file is named so that pytest collects it last.
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


def _same(a, b):
    ia = a.view(torch.int32 if a.dtype == torch.float32 else torch.int16)
    ib = b.view(torch.int32 if b.dtype == torch.float32 else torch.int16)
    return torch.equal(ia, ib)


def test_noalloc_matches_batched_two_calls(lf):
    shapes = [(5, 5, [15, 25, 15], [15, 25, 15], torch.float32),
              (19, 19, [57, 133], [57, 133], torch.float16),
              (3, 7, [9, 27], [21, 35], torch.float32)]
    plans = [lf.Plan(a, b, c, d, t) for a, b, c, d, t in shapes]
    for call in range(2):
        Hs = [_bits(p.elems, p.dtype, 100 * call + i) for i, p in enumerate(plans)]
        ref = lf.backproject_batched(plans, Hs)
        outs = [torch.full_like(h, float("nan")) for h in Hs]
        assert _noalloc(lf, plans, Hs, outs) == 0, lf.load().lfbp_last_error()
        lf.sync_status()
        for r, o in zip(ref, outs):
            assert _same(r, o), f"call {call}"
    # a different list of plans on the next call replaces the array's contents
    plan2 = [lf.Plan(11, 11, [33, 99], [33, 99], torch.float32)]
    H2 = [_bits(plan2[0].elems, torch.float32, 7)]
    out2 = [torch.empty_like(H2[0])]
    assert _noalloc(lf, plan2, H2, out2) == 0
    lf.sync_status()
    assert _same(lf.backproject_batched(plan2, H2)[0], out2[0])


def test_noalloc_rejects_too_many_tiles(lf):
    # ~8.5 G elements of tiles would need far more than 262,144 descriptors;
    # rejected before any work is queued, so the buffers are never touched
    plan = lf.Plan(51, 51, [1001] * 30, [1001] * 30, torch.float32)
    lib = lf.load()
    P = ctypes.c_void_p
    fake_in, fake_out = 1 << 40, (1 << 40) + (1 << 39)
    hp = (P * 1)(plan.handle)
    rc = lib.lfbp_backproject_batched_noalloc(1, ctypes.cast(hp, P),
                                              ctypes.cast((P * 1)(fake_in), P),
                                              ctypes.cast((P * 1)(fake_out), P), None)
    assert rc == -1
    assert b"no-allocation path holds at most 262144" in lib.lfbp_last_error()


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
