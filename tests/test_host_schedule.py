"""The order of copies and maps of the host-to-host path (lfbp_host_sched.h),
checked on the CPU: every chunk goes in once and back once, every depth is
mapped once after all chunks it overlaps have arrived (copies in complete in
issue order), every chunk goes back only after all depths overlapping it are
mapped; and the optional rotation starts and ends on small depths, so that
less has to arrive before the first map and less is left to go back after
the last copy in than in memory order (the default)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import lfgen

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
K_IN, K_MAP, K_OUT = 0, 1, 2


@pytest.fixture(scope="module")
def sched(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("sched") / "libsched.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-Wall", "-Werror", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_2003_09133_gb300", "csrc"), "-o", so,
                           os.path.join(HERE, "host_emu", "host_sched.cpp")])
    lib = ctypes.CDLL(so)
    lib.sched_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_int]
    lib.sched_run.restype = ctypes.c_int

    def run(sizes, chunk, memory_order=False):
        zoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        out = np.zeros(4 * 100000, dtype=np.int32)
        n = lib.sched_run(zoff.ctypes.data, len(sizes), chunk, int(memory_order),
                          out.ctypes.data, 100000)
        assert n >= 0
        return zoff, [tuple(int(v) for v in out[4 * i:4 * i + 4]) for i in range(n)]
    return run


def _chunks(zoff, z, chunk):
    return range(int(zoff[z]) // chunk, (int(zoff[z + 1]) - 1) // chunk + 1)


def _check(zoff, ops, chunk):
    """The schedule's invariants; returns (bytes in before the first map,
    bytes back after the last copy in)."""
    nz = len(zoff) - 1
    total = int(zoff[-1])
    nch = -(-total // chunk)
    in_at, out_at, map_at, pos = {}, {}, {}, {}
    for i, (kind, a, b, wait) in enumerate(ops):
        if kind == K_IN:
            assert a not in in_at and 0 <= a < nch
            in_at[a] = i
            pos[a] = len(pos)
        elif kind == K_OUT:
            assert a not in out_at and a in in_at
            out_at[a] = i
        else:
            assert kind == K_MAP and 0 <= a < b <= nz
            assert wait in pos, "a map waits for a chunk not yet issued"
            for z in range(a, b):
                assert z not in map_at
                map_at[z] = i
                for k in _chunks(zoff, z, chunk):  # arrived by the wait (issue order)
                    assert k in pos and pos[k] <= pos[wait], (z, k, wait)
    assert sorted(in_at) == list(range(nch)) and sorted(out_at) == list(range(nch))
    nonempty = [z for z in range(nz) if zoff[z + 1] > zoff[z]]
    assert sorted(map_at) == nonempty
    for z in nonempty:
        for k in _chunks(zoff, z, chunk):
            assert out_at[k] > map_at[z], (k, z)
    size = lambda k: min(chunk, total - k * chunk)
    first_map = min(map_at.values())
    fill = sum(size(k) for k, i in in_at.items() if i < first_map)
    last_in = max(in_at.values())
    drain = sum(size(k) for k, i in out_at.items() if i > last_in)
    return fill, drain


def _highres_sizes():
    s = lfgen.config_specs("highres")[0]
    return [s.Nx * s.Ny * a * b * 4 for a, b in zip(s.Ks, s.Kt)]


@pytest.mark.parametrize("memory_order", [False, True])
@pytest.mark.parametrize("chunk_mb", [1, 16, 64, 256, 8192])
def test_highres_schedule(sched, memory_order, chunk_mb):
    chunk = chunk_mb << 20
    zoff, ops = sched(_highres_sizes(), chunk, memory_order)
    _check(zoff, ops, chunk)


def test_rotation_shortens_fill_and_drain(sched):
    """The highres workload (41 depths, 12 to 219 MiB, the largest at both ends)
    with 64 MiB chunks: one chunk has to arrive before the first map and three
    go back after the last copy in (the chunk where the rotation started waits
    for the last depth), against four and a bit over three in memory order."""
    chunk = 64 << 20
    sizes = _highres_sizes()
    zoff, ops = sched(sizes, chunk)
    fill, drain = _check(zoff, ops, chunk)
    zoff_m, ops_m = sched(sizes, chunk, True)
    fill_m, drain_m = _check(zoff_m, ops_m, chunk)
    assert fill <= chunk and drain <= 3 * chunk
    assert fill_m >= 4 * chunk and drain_m > 3 * chunk
    first = next(op for op in ops if op[0] == K_MAP)
    assert first[1] <= int(np.argmin(sizes)) < first[2]  # the smallest depth is in the first map


@pytest.mark.parametrize("seed", range(12))
def test_random_depth_sizes(sched, seed):
    """Random depth sizes with empty depths, chunks smaller and larger than the
    depths, in both orders."""
    rng = np.random.default_rng(seed)
    nz = int(rng.integers(1, 40))
    sizes = (rng.integers(1, 5000, nz) * 4).astype(np.int64)
    sizes[rng.random(nz) < 0.2] = 0
    if sizes.sum() == 0:
        sizes[0] = 4
    for chunk in (16, 1024, 4096, 1 << 20):
        for memory_order in (False, True):
            zoff, ops = sched(list(sizes), chunk, memory_order)
            _check(zoff, ops, chunk)


def test_degenerate_inputs(sched):
    assert sched([0, 0], 64)[1] == []          # nothing to move
    zoff, ops = sched([100], 64)               # one depth over two chunks
    assert [op[0] for op in ops] == [K_IN, K_IN, K_MAP, K_OUT, K_OUT]
    for sizes in ([8, 8], [8, 0, 8], [4, 8, 12]):
        for mo in (False, True):
            zoff, ops = sched(sizes, 8, mo)
            _check(zoff, ops, 8)
