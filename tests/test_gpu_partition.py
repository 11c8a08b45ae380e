"""Image-partitioned migration through the CUDA library: two processes (gloo for the gather, both on
the one GPU this test has; their kernels never wait on each other) migrate their slabs of image
columns with every trace, and the gathered image matches the FP64 oracle's whole image."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _survey():
    from paper_1204_1225_gb300 import survey as sv
    rng = np.random.default_rng(9)
    s = sv.survey_random(rng, 3, 300, 40, 24, 48, 400, vel="linear", weight="obliq", aperture=180.0,
                         n_bins=3, h=12.5, v0=1700.0, k=0.6)
    return s, sv.random_traces(s, 4, smooth=5)


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1204_1225_gb300 import kirchhoff as kh
    from paper_1204_1225_gb300 import partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s, d = _survey()
    i0, n = partition.image_slabs(s, world)[rank]
    sub = partition.slab_survey(s, i0, n)
    p = kh.Plan(sub)
    img = p.migrate(kh.Headers.of(sub), torch.as_tensor(d, device="cuda"))
    p.sync()
    full = partition.gather_image(img.cpu(), s, world)
    if rank == 0:
        q.put(full.double().numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_slabs_make_the_image():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, d = _survey()
    want = oracle.migrate(s, d)
    assert got.shape == want.shape
    assert np.count_nonzero(want) > want.size // 10
    err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    assert err < 1e-5
