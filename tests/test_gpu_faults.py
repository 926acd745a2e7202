"""Failure detection without a GPU fault (needs a GPU).

Every in-kernel wait of the persistent gather is bounded (2 s of wall time);
when one runs out the kernel records LFBP_ERR_TIMEOUT in a device status word,
stops its CTA cleanly and returns, and lfbp_sync_status reports it.  The
injection LFBP_FAULT=stall makes the producers register the bytes of their
copies on the stage barrier without issuing the copies, so the barrier phase
is never completed and every consumer wait runs out -- a wait on a flag
nothing sets, with no bad address, trap or endless loop.  After the timeout
the context stays usable: the next launch without the injection gives the
exact map.  The host-side injections (plan, alloc, graph) fail the calls that
would fail under memory pressure or a driver error and leave nothing behind.
"""
import time

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_2003_09133_gb300 as m
    m.load(build_if_missing=True)
    torch.cuda.set_device(0)
    return m


SHAPE = (5, 5, [15, 25], [15, 25])


def _input(plan, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(plan.elems).astype(np.float32)


def _check_exact(lf, plan, H, Hp):
    want = oracle.transpose(H, *SHAPE)
    got = Hp.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_stalled_waits_time_out_and_the_context_recovers(lf, monkeypatch):
    plan = lf.Plan(*SHAPE, torch.float32)
    H = _input(plan, 31)
    Hd = torch.from_numpy(H).cuda()
    lf.sync_status()  # no status left over from earlier tests
    monkeypatch.setenv("LFBP_FAULT", "stall")
    out = torch.zeros_like(Hd)
    t0 = time.monotonic()
    lf.backproject_batched([plan], [Hd], [out])
    with pytest.raises(lf.LfbpError) as ei:
        lf.sync_status()
    elapsed = time.monotonic() - t0
    assert ei.value.code == -7
    assert 1.5 <= elapsed <= 30.0, elapsed  # the 2 s wait limit, not a hang
    # the status word was cleared by the report
    lf.sync_status()
    monkeypatch.delenv("LFBP_FAULT")
    out2 = lf.backproject_batched([plan], [Hd])[0]
    lf.sync_status()
    _check_exact(lf, plan, H, out2)


def test_injected_allocation_and_graph_failures(lf, monkeypatch):
    for mode, code in (("alloc", -8), ("graph", -6)):
        plan = lf.Plan(*SHAPE, torch.float32)  # a new plan: its batch state is built afresh
        H = _input(plan, 32)
        Hd = torch.from_numpy(H).cuda()
        monkeypatch.setenv("LFBP_FAULT", mode)
        with pytest.raises(lf.LfbpError) as ei:
            lf.backproject_batched([plan], [Hd])
        assert ei.value.code == code and "injected" in str(ei.value)
        monkeypatch.delenv("LFBP_FAULT")
        out = lf.backproject_batched([plan], [Hd])[0]
        lf.sync_status()
        _check_exact(lf, plan, H, out)


def test_injected_plan_failure_through_the_binding(lf, monkeypatch):
    monkeypatch.setenv("LFBP_FAULT", "plan")
    with pytest.raises(lf.LfbpError) as ei:
        lf.Plan(*SHAPE, torch.float32)
    assert ei.value.code == -8


@pytest.mark.parametrize("Ks", [[9, 3], [9, 9, 9]], ids=["one_depth_blocks", "depth_group"])
@pytest.mark.parametrize("pipe", ["1", "0"])
def test_projector_tma_waits_time_out_and_recover(lf, monkeypatch, pipe, Ks):
    """The projectors' TMA-path waits are bounded too.  Under LFBP_FAULT=stall
    their TMA copies register their bytes without being issued, so the waits
    on those copies run out.  The pipelined kernels (producer, consumers,
    pair barriers), the barrier kernels (LFBP_PROJ_PIPE=0) and the grouped
    backprojection (three equal cut-outs) all end with LFBP_ERR_TIMEOUT, and
    the next call without the injection is correct."""
    Nx, Ny, W = 3, 3, 12
    plan = lf.Plan(Nx, Ny, Ks, Ks, torch.float32)
    rng = np.random.default_rng(33)
    H = rng.uniform(0, 1, plan.elems).astype(np.float32)
    f = rng.uniform(0.1, 1, (W, W)).astype(np.float32)
    dg = rng.uniform(-1, 1, (len(Ks), W, W)).astype(np.float32)
    Hd, fd, dgd = (torch.from_numpy(x).cuda() for x in (H, f, dg))
    monkeypatch.setenv("LFBP_PROJ_PIPE", pipe)
    lf.sync_status()
    for call in (lambda: lf.backproject_volume_from_h(plan, Hd, fd),
                 lambda: lf.backproject_volume_grad(plan, fd, dgd)):
        monkeypatch.setenv("LFBP_FAULT", "stall")
        t0 = time.monotonic()
        call()
        with pytest.raises(lf.LfbpError) as ei:
            lf.sync_status()
        assert ei.value.code == -7
        assert time.monotonic() - t0 <= 60.0
        monkeypatch.delenv("LFBP_FAULT")
    Hp = oracle.transpose(H, Nx, Ny, Ks, Ks)
    want = oracle.backproject(Hp, Nx, Ny, Ks, Ks, f)
    got = lf.backproject_volume_from_h(plan, Hd, fd).cpu().numpy()
    lf.sync_status()
    n2 = (np.array([a * a for a in Ks]) * 2.0 ** -23)[:, None, None]
    assert (np.abs(got - want) <= n2 * np.abs(want) + 1e-30).all()
