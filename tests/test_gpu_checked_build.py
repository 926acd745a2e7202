"""The self-checking build (LFBP_CHECK=1 loads liblfbp_check.so, compiled with
-DLFBP_CHECK): every shared-memory load, global store, bulk copy and tail load
of the tile code is bounds- and alignment-checked on the GPU, the first
violation is recorded (the access skipped, no trap) and lfbp_sync_status
reports it.  Here the gather runs through it on tile shapes of every kind
(one-row and multi-row tiles, column splits, fp16, the paper window, the
batched form in each of its three shapes) and must report nothing and still
match the oracle bit for bit.
The library is chosen at load time, so this runs in a child process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch, oracle
import paper_2003_09133_gb300 as lf
lib = lf.load(build_if_missing=True)
assert lib._name.endswith("liblfbp_check.so"), lib._name
torch.cuda.set_device(0)
SHAPES = [(5, 5, [15, 25], [15, 25]), (19, 19, [399, 95], [399, 95]), (51, 51, [153], [153]),
          (95, 55, [181], [181]), (3, 5, [9, 3, 15], [15, 5, 5]), (11, 11, [99, 33], [99, 33]),
          (7, 27, [21, 35], [21, 35]),                       # stripes in bands
          (19, 19, [96, 20], [96, 20]), (5, 3, [14, 15], [15, 6]),  # even cut-outs
          (11, 7, [90, 12], [34, 89])]
for Nx, Ny, Ks, Kt in SHAPES:
    even = any(k % 2 == 0 for k in Ks + Kt)
    for dt in (torch.float32, torch.float16):
        modes = (lf.MAP_PAPER_WINDOW,) if even else (lf.MAP_TRANSPOSE, lf.MAP_PAPER_WINDOW)
        for mode in modes:
            plan = lf.Plan(Nx, Ny, Ks, Kt, dt, mode=mode)
            g = torch.Generator(device="cpu").manual_seed(Nx + len(Ks))
            bits = torch.randint(-2 ** 15, 2 ** 15 - 1, (plan.elems * (2 if dt == torch.float32 else 1),),
                                 generator=g, dtype=torch.int32).to(torch.int16)
            H = bits.view(dt).cuda()
            Hn = H.cpu().numpy()
            want = (oracle.transpose if mode == lf.MAP_TRANSPOSE else oracle.paper_window)(
                Hn, Nx, Ny, Ks, Kt)
            outs = [lf.backproject_array(plan, H), lf.backproject_batched([plan], [H])[0]]
            if mode == lf.MAP_TRANSPOSE:
                outs.append(lf.adjoint(plan, H))  # the map is its own adjoint
            else:
                lf.adjoint(plan, outs[0])  # the windowed adjoint's accesses (values: test_gpu_map)
            for got in outs:
                lf.sync_status()  # raises on a recorded violation
                w = np.uint32 if dt == torch.float32 else np.uint16
                assert np.array_equal(got.cpu().numpy().view(w), want.view(w)), (Nx, Ks, dt, mode)
            lf.sync_status()
print("checked ok")
"""


@pytest.mark.parametrize("form", ["0", "1", "2"])
def test_self_checking_build_reports_nothing(form):
    """Each batched form (persistent CTAs, one tile per CTA, per-depth grids)."""
    env = dict(os.environ, LFBP_CHECK="1", LFBP_FORM=form)
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=1500)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-3000:]
    assert "checked ok" in out.stdout
