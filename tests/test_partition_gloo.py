"""Image-partitioned migration (one process per GPU, no exchange of partial sums), tested on CPU:
the slab layout tiles the image exactly; two gloo ranks each migrate their slab of columns with
the FP64 oracle and all-gather the slabs, and the assembled image equals the one-process image
(with the aperture taper and operator anti-aliasing on: both act per column)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1204_1225_gb300 import partition  # noqa: E402
from paper_1204_1225_gb300 import survey as sv  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("dim,nx,world", [(3, 256, 8), (3, 50, 3), (2, 512, 4), (2, 100, 2), (3, 16, 4)])
def test_slabs_tile_the_image(dim, nx, world):
    s = sv.survey_random(np.random.default_rng(1), dim, 4, nx, 8, 8, 16)
    slabs = partition.image_slabs(s, world)
    assert len(slabs) == world
    assert slabs[0][0] == 0 and sum(n for _, n in slabs) == nx
    for (a, n), (b, _) in zip(slabs, slabs[1:]):
        assert a + n == b and n >= 0
    align = partition.SLAB_ALIGN[dim]
    assert all(i0 % align == 0 for i0, _ in slabs)
    sub = partition.slab_survey(s, *slabs[-1])
    assert sub.nx == slabs[-1][1] and sub.ox == s.ox + slabs[-1][0] * s.dx


def _survey():
    rng = np.random.default_rng(5)
    s = sv.survey_random(rng, 2, 60, 150, 1, 30, 300, vel="linear", weight="obliq", aperture=250.0,
                         n_bins=3, h=10.0, v0=1800.0, k=0.5)
    # with the taper and operator anti-aliasing: both are per (column, trace), so slab-local
    s = s.replace(taper=0.2, aa_spacing=20.0)
    return s, sv.random_traces(s, 3, smooth=5).astype(np.float64)


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, d = _survey()
    i0, n = partition.image_slabs(s, world)[rank]
    mine = oracle.migrate(partition.slab_survey(s, i0, n), d) if n > 0 else \
        np.zeros((s.n_bins, 1, 0, s.nz))
    full = partition.gather_image(torch.as_tensor(mine), s, world)
    if rank == 0:
        q.put(full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_the_one_process_image():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, d = _survey()
    want = oracle.migrate(s, d)
    assert got.shape == want.shape
    assert np.count_nonzero(want) > 0
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert not np.allclose(oracle.migrate(s.replace(aa_spacing=0.0), d), want)   # the weight acts
    # the same assembly in one process
    parts = [oracle.migrate(partition.slab_survey(s, i0, n), d) for i0, n in partition.image_slabs(s, 2)]
    assert np.array_equal(partition.assemble(parts, s), got)
