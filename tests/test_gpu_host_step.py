"""mm_step_host: one whole step on host arrays, its copies overlapped with the
step on a second stream, equals mm_step on device copies of the same arrays
bit for bit (positions, charges, dt), for the integrators and state layouts
it serves, with page-locked and pageable host memory."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _state(torch, ctx, w):
    pos = H.to_dev(torch, w.pos.T)
    mesh = ctx.mm_tessellate(pos, w.box)
    U = ctx.mm_prims_to_charges(mesh, H.to_dev(torch, w.rho), H.to_dev(torch, w.vel.T), H.to_dev(torch, w.pres))
    return pos, U


@pytest.mark.parametrize("cfg", [dict(), dict(entropy=1), dict(integrator=1), dict(precision=1)],
                         ids=["fp64", "entropy", "heun", "mixed"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_step_equals_device_step(cfg, pinned):
    import torch
    from paper_1707_05333_gb300 import binding
    binding.load()
    w = WL.shear_layer(20)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = binding.Context(stream=stream, gamma=5.0 / 3.0, **cfg)
        pos, U = _state(torch, ctx, w)
        if cfg.get("entropy"):
            assert U.shape[0] == 6
        pos_h, U_h = pos.cpu(), U.cpu()
        if pinned:
            pos_h, U_h = pos_h.pin_memory(), U_h.pin_memory()
        dt_h = torch.zeros(1, dtype=torch.float64)
        dt_d = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(3):
            ctx.mm_step(pos, U, w.box, dt_out=dt_d)
            ctx.mm_step_host(pos_h, U_h, w.box, dt_out=dt_h)
            stream.synchronize()
            assert torch.equal(pos_h, pos.cpu()) and torch.equal(U_h, U.cpu())
            assert dt_h.item() == dt_d.item() and dt_h.item() > 0.0
        ctx.close()


def test_host_step_rejects_device_tensors_and_bad_shapes():
    import torch
    from paper_1707_05333_gb300 import binding
    binding.load()
    w = WL.shear_layer(8)
    ctx = binding.Context()
    pos, U = _state(torch, ctx, w)
    with pytest.raises(ValueError):
        ctx.mm_step_host(pos, U.cpu(), w.box)
    with pytest.raises(ValueError):
        ctx.mm_step_host(pos.cpu(), U.cpu()[:4].contiguous(), w.box)
    # the context still steps on the host
    pos_h, U_h = pos.cpu().pin_memory(), U.cpu().pin_memory()
    m0 = U_h[0].sum().item()
    ctx.mm_step_host(pos_h, U_h, w.box)
    assert abs(U_h[0].sum().item() - m0) <= 1e-12 * abs(m0)
    ctx.close()
