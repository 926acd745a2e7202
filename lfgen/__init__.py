"""Seeded synthetic light-field PSF arrays shaped like the paper's workloads.

This module only *makes inputs*.  It holds none of the H -> H' arithmetic
(no index map, no transpose, no projector): both the CUDA path's tests and
the CPU oracle's tests draw their inputs from here, and nothing here depends
on either of them.

Array layout (shared by every consumer): one flat buffer per PSF array,
depth-major and ragged in depth.  Depth z holds ``Nx*Ny*Ks[z]*Kt[z]``
elements in row-major ``[a][b][s][t]`` order, where (a, b) is the source
(voxel) position inside the elementary cell (paper Sec. 2.1, the (x, y)
dimensions of H) and (s, t) the sensor pixel inside the voxel-centred
cut-out (the (s, t) dimensions of H).  Depth z starts at
``sum_{z'<z} Nx*Ny*Ks[z']*Kt[z']``.

Kernel recipe (synthetic stand-in for the wave-optics PSFs of the paper's
Table 1 and for the experimental R29 PSF, neither of which is available):
each (z, a, b) cut-out is an FP64 sum of point-sampled isotropic Gaussian
spots of sigma 0.6 px, centred at ``(c + j*Nx + (a-h_x), c_t + k*Ny + (b-h_y))``
for integer (j, k) with ``j^2 + k^2 <= r_z^2`` (lenslet pitch = N pixels),
with uniform(0.5, 1) amplitudes drawn from ``numpy.random.default_rng(seed)``
as a full (2r+1)^2 block per (z, a, b) in (z, a, b, j, k) order and masked
to the disk.  Each cut-out is normalised to unit sum in FP64, values below
1e-6 become exactly 0, and the result is cast to fp32 (then to fp16 with
round-to-nearest-even where fp16 storage is asked for).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np
import torch

SIGMA_PX = 0.6
ZERO_BELOW = 1e-6

__all__ = [
    "ArraySpec", "config_specs", "generate", "array_elems", "depth_offsets",
    "random_array", "raw_image", "blob_volume", "CONFIG_NAMES",
]


@dataclasses.dataclass(frozen=True)
class ArraySpec:
    """Shape and recipe of one ragged PSF array.

    Nx, Ny: lenslet-cell sizes (odd, paper Sec. 4 requires odd n_x, n_y).
    Ks, Kt: per-depth cut-out sizes in pixels along s and t (odd).
    radius: per-depth spot radius r_z in lenslets.
    dtype: "f32" or "f16" storage.
    seed: numpy seed of the amplitudes.
    """
    Nx: int
    Ny: int
    Ks: tuple
    Kt: tuple
    radius: tuple
    dtype: str
    seed: int
    name: str = ""

    @property
    def Nz(self) -> int:
        return len(self.Ks)

    @property
    def esize(self) -> int:
        return 4 if self.dtype == "f32" else 2

    @property
    def torch_dtype(self):
        return torch.float32 if self.dtype == "f32" else torch.float16


def array_elems(spec: ArraySpec) -> int:
    return int(sum(spec.Nx * spec.Ny * ks * kt for ks, kt in zip(spec.Ks, spec.Kt)))


def depth_offsets(spec: ArraySpec) -> List[int]:
    out, acc = [], 0
    for ks, kt in zip(spec.Ks, spec.Kt):
        out.append(acc)
        acc += spec.Nx * spec.Ny * ks * kt
    return out


def _square(N, Ls, dtype, seed, radius=None, name=""):
    Ks = tuple(int(L * N) for L in Ls)
    if radius is None:
        radius = tuple(int((L - 1) // 2) for L in Ls)
    return ArraySpec(N, N, Ks, Ks, tuple(radius), dtype, seed, name)


CONFIG_NAMES = ("tiny", "mid", "ragged", "highres", "autograd")


def config_specs(name: str) -> List[ArraySpec]:
    """The five synthetic workloads (tiny, mid, ragged, highres, autograd).

    tiny:     N=5, K=15 at three depths z in {-1,0,1}, r_z = 1+|z|, fp32, seed 0.
    mid:      N=15, 51 depths, K_z = 15*min(3+2*floor(|zi-25|/5), 11), fp32, seed 1.
    ragged:   16 arrays, seeds 2..17; per array N from {9..19 odd}, Nz in [11,61],
              per-depth L_z from {3,5,..,15}, K_z = L_z*N; fp16 for even seeds.
    highres:  N=19, 41 depths, L_z = 5+2*floor(2|zi-20|/5) in {5..21} (K up to 399),
              fp32, seed 18 (the fp16 copy is the fp32 array cast to half).
    autograd: N=11, 21 depths, L_z = 3+2*floor(3|zi-10|/10) in {3..9}, fp32, seed 21.
    """
    if name == "tiny":
        return [_square(5, [3, 3, 3], "f32", 0, radius=[2, 1, 2], name="tiny")]
    if name == "mid":
        Ls = [min(3 + 2 * (abs(zi - 25) // 5), 11) for zi in range(51)]
        return [_square(15, Ls, "f32", 1, name="mid")]
    if name == "highres":
        Ls = [5 + 2 * ((2 * abs(zi - 20)) // 5) for zi in range(41)]
        return [_square(19, Ls, "f32", 18, name="highres")]
    if name == "autograd":
        Ls = [3 + 2 * ((3 * abs(zi - 10)) // 10) for zi in range(21)]
        return [_square(11, Ls, "f32", 21, name="autograd")]
    if name == "ragged":
        specs = []
        for seed in range(2, 18):
            rng = np.random.default_rng(seed)
            N = int(rng.choice([9, 11, 13, 15, 17, 19]))
            Nz = int(rng.integers(11, 62))
            Ls = [int(x) for x in rng.choice([3, 5, 7, 9, 11, 13, 15], size=Nz)]
            specs.append(_square(N, Ls, "f16" if seed % 2 == 0 else "f32",
                                 seed, name=f"ragged{seed}"))
        return specs
    raise ValueError(f"unknown workload {name!r}")


def _amplitude_draws(spec: ArraySpec):
    """Yield the per-depth amplitude blocks [Nx][Ny][2r+1][2r+1] (masked to the disk)."""
    rng = np.random.default_rng(spec.seed)
    if spec.name.startswith("ragged"):
        # replay the shape draws so the amplitudes follow them in the same stream
        rng.choice([9, 11, 13, 15, 17, 19])
        nz = int(rng.integers(11, 62))
        rng.choice([3, 5, 7, 9, 11, 13, 15], size=nz)
    for r in spec.radius:
        amp = rng.uniform(0.5, 1.0, size=(spec.Nx, spec.Ny, 2 * r + 1, 2 * r + 1))
        j = np.arange(-r, r + 1)
        disk = (j[:, None] ** 2 + j[None, :] ** 2) <= r * r
        yield amp * disk[None, None]


def _gauss_factor(n_cell: int, K: int, r: int, device) -> torch.Tensor:
    """[n_cell][K][2r+1]: 1-D Gaussian of spot j seen from pixel s, for source a."""
    h = (n_cell - 1) // 2
    c = (K - 1) // 2
    a = torch.arange(n_cell, device=device, dtype=torch.float64)[:, None, None]
    s = torch.arange(K, device=device, dtype=torch.float64)[None, :, None]
    j = torch.arange(-r, r + 1, device=device, dtype=torch.float64)[None, None, :]
    centre = c + j * n_cell + (a - h)
    return torch.exp(-((s - centre) ** 2) / (2.0 * SIGMA_PX * SIGMA_PX))


def generate(spec: ArraySpec, device="cpu") -> torch.Tensor:
    """Return the flat ragged array for ``spec`` on ``device`` in its storage dtype."""
    out = torch.empty(array_elems(spec), dtype=spec.torch_dtype, device=device)
    off = 0
    for z, amp in enumerate(_amplitude_draws(spec)):
        ks, kt, r = spec.Ks[z], spec.Kt[z], spec.radius[z]
        A = torch.from_numpy(amp).to(device)
        Gs = _gauss_factor(spec.Nx, ks, r, device)   # [a][s][j]
        Gt = _gauss_factor(spec.Ny, kt, r, device)   # [b][t][k]
        # kernel[a][b][s][t] = sum_jk Gs[a][s][j] A[a][b][j][k] Gt[b][t][k]
        tmp = torch.einsum("asj,abjk->absk", Gs, A)
        ker = torch.einsum("absk,btk->abst", tmp, Gt)
        ker = ker / ker.sum(dim=(2, 3), keepdim=True)
        ker = torch.where(ker < ZERO_BELOW, torch.zeros_like(ker), ker)
        n = spec.Nx * spec.Ny * ks * kt
        v = ker.reshape(-1).to(torch.float32)
        out[off:off + n] = v.to(spec.torch_dtype)
        off += n
        del tmp, ker, v
    return out


def random_array(Nx, Ny, Ks: Sequence[int], Kt: Sequence[int], dtype="f32", seed=0,
                 device="cpu") -> torch.Tensor:
    """Uniform(-1, 1) values in the same ragged layout (dense, no zeros)."""
    n = int(sum(Nx * Ny * ks * kt for ks, kt in zip(Ks, Kt)))
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.rand(n, generator=g, dtype=torch.float64) * 2.0 - 1.0
    v = v.to(torch.float32)
    if dtype == "f16":
        v = v.half()
    return v.to(device)


def raw_image(n_lenslets: int, N: int, seed: int) -> np.ndarray:
    """Seeded uniform(0,1) raw sensor image of n_lenslets*N pixels per side (FP64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n_lenslets * N, n_lenslets * N))


def blob_volume(W: int, Nz: int, n_blobs: int, seed: int) -> np.ndarray:
    """Seeded volume [Nz][W][W] (FP64) holding a sum of anisotropic Gaussian blobs.

    Blob centres are uniform over the volume, lateral sigma uniform(1, 4) px,
    axial sigma 1 depth plane, amplitude uniform(0.5, 1).
    """
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, W, n_blobs)
    cy = rng.uniform(0, W, n_blobs)
    cz = rng.uniform(0, Nz, n_blobs)
    sl = rng.uniform(1.0, 4.0, n_blobs)
    amp = rng.uniform(0.5, 1.0, n_blobs)
    vol = np.zeros((Nz, W, W))
    x = np.arange(W)
    zz = np.arange(Nz)
    for i in range(n_blobs):
        gx = np.exp(-((x - cx[i]) ** 2) / (2 * sl[i] ** 2))
        gy = np.exp(-((x - cy[i]) ** 2) / (2 * sl[i] ** 2))
        gz = np.exp(-((zz - cz[i]) ** 2) / 2.0)
        vol += amp[i] * gz[:, None, None] * gx[:, None][None] * gy[None, None, :]
    return vol
