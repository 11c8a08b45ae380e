"""The binding refuses tensors whose dtype, size or device differ from what the library reads
or writes through their pointers, before any library call (a short buffer would otherwise be
read past its end on the GPU).  These checks run on the CPU: the plan object is built
without a device handle, and every refusal happens before the handle is used."""
import numpy as np
import pytest
import torch

from paper_1204_1225_gb300 import kirchhoff as kh
from paper_1204_1225_gb300 import survey as sv


def _survey():
    rng = np.random.default_rng(3)
    return sv.survey_random(rng, 3, 12, 6, 5, 8, 40, vel="linear", n_bins=2, h=12.5, k=0.5)


def _plan(s, trace_dtype=torch.float32):
    p = kh.Plan.__new__(kh.Plan)          # no kirchhoff_create: nothing may reach the library
    p.handle = None
    p.survey, p.trace_dtype, p.nt, p.device = s, trace_dtype, s.nt, 0
    p.image_shape = (s.n_bins, s.ny, s.nx, s.nz)
    return p


def _refused(fn, *words):
    with pytest.raises(ValueError) as ei:
        fn()
    for w in words:
        assert w in str(ei.value), str(ei.value)


def test_migrate_refusals():
    s = _survey()
    p, hdr = _plan(s), kh.Headers.of(s, device="cpu")
    good = torch.zeros(s.ntr, s.nt)
    _refused(lambda: p.migrate(hdr, good.half()), "traces", "float32")
    _refused(lambda: p.migrate(hdr, good.double()), "traces", "float32")     # gradcheck inputs
    _refused(lambda: p.migrate(hdr, good[:-1]), "traces", "elements")
    _refused(lambda: p.migrate(hdr, good, out=torch.zeros(3, 3)), "image", "shape")
    _refused(lambda: p.migrate(hdr, good, out=torch.zeros(p.image_shape, dtype=torch.float16)),
             "image", "float32")
    short = kh.Headers(s.sx[:-1], s.sy[:-1], s.rx[:-1], s.ry[:-1], device="cpu")
    _refused(lambda: p.migrate(short, good), "traces", "elements")
    # right types and sizes, wrong device: still refused before the library is called
    _refused(lambda: p.migrate(hdr, good), "CUDA")
    f16 = _plan(s, torch.float16)
    _refused(lambda: f16.migrate(hdr, good), "traces", "float16")


def test_demigrate_and_gradient_refusals():
    s = _survey()
    p, hdr = _plan(s), kh.Headers.of(s, device="cpu")
    img = torch.zeros(p.image_shape)
    tr = torch.zeros(s.ntr, s.nt)
    _refused(lambda: p.demigrate(hdr, img[:1]), "image", "shape")
    _refused(lambda: p.demigrate(hdr, img, out=torch.zeros(s.ntr, s.nt - 1)), "traces_out")
    _refused(lambda: p.velocity_grad(hdr, img.double(), tr), "image", "float32")
    _refused(lambda: p.velocity_grad(hdr, img, tr.half()), "traces", "float32")
    _refused(lambda: p.velocity_grad(hdr, img, tr, out=torch.zeros(2)), "out_dv0_dk", "float64")
    _refused(lambda: p.count(kh.Headers(s.sx, s.sy, s.rx, s.ry[:3], device="cpu")), "ry")


def test_noalloc_refusals():
    s = _survey()
    d = kh.desc_from(s)
    hdr = kh.Headers.of(s, device="cpu")
    img = torch.zeros(s.n_bins, s.ny, s.nx, s.nz)
    tr = torch.zeros(s.ntr, s.nt)
    _refused(lambda: kh.kirchhoff_migrate_noalloc(d, s.ntr, *hdr.args(), tr.half(), img), "traces")
    _refused(lambda: kh.kirchhoff_migrate_noalloc(d, s.ntr, *hdr.args(), tr, img[:1]), "image")
    _refused(lambda: kh.kirchhoff_migrate_noalloc(d, s.ntr + 1, *hdr.args(), tr, img), "sx")
    _refused(lambda: kh.kirchhoff_migrate_noalloc(d, s.ntr, *hdr.args(), tr, img,
                                                  status=torch.zeros(1)), "status", "int32")


def test_host_entry_point_refusals():
    s = _survey()
    p = _plan(s)
    hdr = kh.Headers.of(s, device="cpu").args()
    tr = torch.zeros(s.ntr, s.nt)
    img = torch.zeros(p.image_shape)
    _refused(lambda: p.migrate_host(hdr, tr.half(), img), "traces", "float32")
    _refused(lambda: p.migrate_host(hdr, tr[:-1], img), "traces", "elements")
    _refused(lambda: p.migrate_host(hdr, tr, img[:1]), "image", "shape")
    _refused(lambda: p.migrate_host(hdr, tr, img.double()), "image", "float32")
    _refused(lambda: p.migrate_host(hdr[:3] + (hdr[3][:2],), tr, img), "ry", "elements")
    _refused(lambda: p.migrate_host(hdr, tr.t(), img), "traces", "contiguous")
    # the device-resident entry point's tensors are refused here (host memory only)
    meta = torch.zeros(s.ntr, s.nt, device="meta")
    _refused(lambda: p.migrate_host(hdr, meta, img), "traces")
