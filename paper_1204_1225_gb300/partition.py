"""Image-partitioned migration over several GPUs (one process per GPU).

Every (image point, offset bin) output of Eq. (1) is an independent sum over traces, so the
image can be split across GPUs with no exchange of partial results: rank r migrates the columns
[i0_r, i0_r + nx_r) of the image with every trace (its plan's binning sort drops the traces whose
midpoints lie farther than the aperture from its columns), and the slabs are concatenated along x
(an all-gather, only if every rank needs the whole image).  This is the partition of the image
grid; the paper's MapReduce instead partitions the traces and sums partial images in its reduce
step (Sec. 4), which the image partition makes unnecessary.

This module holds the host logic only: the slab layout, the per-rank survey and the assembly.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

# Slab widths are multiples of this many columns where the image allows it, so that each slab
# is cut along the migration kernel's tile boundaries (16 columns per tile in 3D, 64 in 2D).
SLAB_ALIGN = {3: 16, 2: 64}


def image_slabs(s, world: int) -> List[Tuple[int, int]]:
    """(i0, nx_r) of each rank's slab of image columns: contiguous, disjoint, covering [0, nx),
    as even as the alignment allows (a rank may get an empty slab when nx is small)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    a = SLAB_ALIGN.get(s.dim, 16)
    units = -(-s.nx // a)                       # aligned column groups
    bounds = [min(s.nx, (units * r // world) * a) for r in range(world + 1)]
    bounds[-1] = s.nx
    return [(bounds[r], bounds[r + 1] - bounds[r]) for r in range(world)]


def slab_survey(s, i0: int, nx_r: int):
    """The survey restricted to image columns [i0, i0 + nx_r): the same traces, bins, model and
    sampling, the image origin moved to column i0."""
    return s.replace(ox=s.ox + i0 * s.dx, nx=max(nx_r, 0), name=f"{s.name}-cols{i0}-{i0 + nx_r}")


def assemble(slabs, s) -> np.ndarray:
    """The full image [n_bins, ny, nx, nz] from the slab images in rank order."""
    parts = [np.asarray(p).reshape(s.n_bins, s.ny if s.dim == 3 else 1, -1, s.nz) for p in slabs]
    img = np.concatenate(parts, axis=2)
    if img.shape[2] != s.nx:
        raise ValueError(f"slabs cover {img.shape[2]} columns, the image has {s.nx}")
    return img


def gather_image(slab_image, s, world: int, group=None):
    """All-gather of the ranks' slab images (torch tensors on any device) into the full image on
    every rank: slabs are padded to the widest one for the collective, then trimmed."""
    import torch
    import torch.distributed as dist
    slabs = image_slabs(s, world)
    wmax = max(n for _, n in slabs)
    ny = s.ny if s.dim == 3 else 1
    pad = torch.zeros((s.n_bins, ny, wmax, s.nz), dtype=slab_image.dtype, device=slab_image.device)
    pad[:, :, :slab_image.shape[2]] = slab_image
    out = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(out, pad, group=group)
    return torch.cat([o[:, :, :n] for o, (_, n) in zip(out, slabs)], dim=2)
