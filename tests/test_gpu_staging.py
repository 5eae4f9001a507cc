"""Transfer arenas (paper_2601_04860_b300.staging.Arena): every named buffer is a
256-byte aligned view of one pinned host tensor and one device tensor, one
copy moves them all, and a one-call step run on arena views gives the step's
result on separate tensors (GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2601_04860_b300 import VoxelFusion, PreparedViews
from paper_2601_04860_b300.staging import Arena
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def test_arena_layout_and_round_trip():
    specs = [("a", (3, 5), torch.float32), ("b", (7,), torch.uint8),
             ("c", (2, 9), torch.int32), ("d", (1,), torch.float16)]
    ar = Arena(specs, "cuda")
    offs = [ar.offsets[n][0] for n, _, _ in specs]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    for (n, shape, dtype), o in zip(specs, offs):
        assert ar.host[n].shape == shape and ar.host[n].dtype == dtype
        assert ar.device[n].data_ptr() - ar.device_bytes.data_ptr() == o
        assert ar.device[n].data_ptr() % 256 == 0
    assert ar.host_bytes.is_pinned()
    g = torch.Generator().manual_seed(5)
    for n, shape, dtype in specs:
        ar.host[n].copy_((torch.rand(shape, generator=g) * 100).to(dtype))
    ref = {n: ar.host[n].clone() for n in ar.host}
    ar.upload()
    torch.cuda.synchronize()
    for n in ar.host:
        assert torch.equal(ar.device[n].cpu(), ref[n]), n
    for n in ar.host:
        ar.host[n].zero_()
    ar.download()
    torch.cuda.synchronize()
    for n in ar.host:
        assert torch.equal(ar.host[n], ref[n]), n
    assert ar.payload_bytes() == sum(t.numel() * t.element_size() for t in ref.values())


def test_step_on_arena_views_equals_step_on_tensors():
    wl = synth.config1()
    d = H.upload(wl)
    prm = H.to_params(oracle.Params())
    fu = VoxelFusion(wl.grid, occ=d["occ"], params=prm)
    score = torch.empty(fu.n_cells, dtype=torch.float32, device="cuda")
    labels = torch.empty(len(d["points"]), dtype=torch.uint8, device="cuda")
    fu.step(PreparedViews(wl.cams, d["depth"], d["mask"], wl.mask_type), occ=d["occ"],
            score=score, xyz=d["points"], labels=labels)
    torch.cuda.synchronize()
    ref = H.state_of(fu, score, labels)

    specs = [("occ", tuple(d["occ"].shape), d["occ"].dtype)]
    specs += [(f"depth{k}", tuple(t.shape), t.dtype) for k, t in enumerate(d["depth"])]
    specs += [(f"mask{k}", tuple(t.shape), t.dtype) for k, t in enumerate(d["mask"])]
    specs.append(("pts", tuple(d["points"].shape), d["points"].dtype))
    ai = Arena(specs, "cuda")
    ao = Arena([("labels", tuple(labels.shape), labels.dtype)], "cuda")
    ai.host["occ"].copy_(d["occ"].cpu())
    for k, t in enumerate(d["depth"]):
        ai.host[f"depth{k}"].copy_(t.cpu())
    for k, t in enumerate(d["mask"]):
        ai.host[f"mask{k}"].copy_(t.cpu())
    ai.host["pts"].copy_(d["points"].cpu())
    ai.upload()
    fu2 = VoxelFusion(wl.grid, occ=ai.device["occ"], params=prm)
    score2 = torch.empty_like(score)
    pv = PreparedViews(wl.cams, [ai.device[f"depth{k}"] for k in range(len(d["depth"]))],
                       [ai.device[f"mask{k}"] for k in range(len(d["mask"]))], wl.mask_type)
    fu2.step(pv, occ=ai.device["occ"], score=score2, xyz=ai.device["pts"],
             labels=ao.device["labels"])
    ao.download()
    torch.cuda.synchronize()
    got = H.state_of(fu2, score2, ao.device["labels"])
    for k in ("active", "W", "Z", "bits", "vmask", "score", "labels"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(ao.host["labels"].numpy(), ref["labels"])
    fu.close()
    fu2.close()
