"""Host-memory forms of the field calls give the same bits as device buffers.

xlb_init and xlb_macroscopic take device, pageable host or page-locked host
buffers.  Page-locked (mapped) host memory is read and written by the
library's kernels directly; pageable memory goes through a staging copy.  On
the 22 x 18 x 16 D3Q19 cavity all three forms give bit-identical fields after
initialisation and after 30 steps.
"""
import numpy as np
import pytest
import torch

from paper_2311_16080_gb300 import inputs as I
from paper_2311_16080_gb300 import xlb as X

pytestmark = pytest.mark.gpu


def _run(kind, rho0, u0, mask):
    nz, ny, nx = mask.shape
    sim = X.Simulation(19, (nx, ny, nz), 1.6, "bgk", "f32")
    sim.set_mask(mask)
    sim.set_bc(X.XLB_CELL_LID, 1.0, (0.05, 0.0, 0.0))
    if kind == "device":
        r_in, u_in = torch.from_numpy(rho0).cuda(), torch.from_numpy(u0).cuda()
        r_out = torch.empty_like(r_in)
        v_out = torch.empty_like(u_in)
    elif kind == "pinned":
        r_in, u_in = torch.from_numpy(rho0).pin_memory(), torch.from_numpy(u0).pin_memory()
        r_out = torch.empty(rho0.shape, dtype=torch.float32).pin_memory()
        v_out = torch.empty(u0.shape, dtype=torch.float32).pin_memory()
    else:
        r_in, u_in = rho0.copy(), u0.copy()
        r_out = np.empty_like(rho0)
        v_out = np.empty_like(u0)
    sim.init(r_in, u_in)
    res = []
    for steps in (0, 30):
        if steps:
            sim.step(steps)
        X.xlb_macroscopic(sim.ctx, r_out, v_out)
        torch.cuda.synchronize()
        to_np = (lambda t: t.cpu().numpy().copy()) if isinstance(r_out, torch.Tensor) else (lambda a: a.copy())
        res.append((to_np(r_out), to_np(v_out)))
    sim.close()
    return res


def test_pinned_pageable_and_device_fields_agree():
    mask = I.lid_driven_cavity_mask(22, 18, 16)
    rho0, u0 = I.random_flow(mask.shape, 3, seed=21, rho_amp=0.01, u_amp=0.03)
    rho0 = rho0.astype(np.float32)
    u0 = u0.astype(np.float32)
    ref = _run("device", rho0, u0, mask)
    for kind in ("pinned", "pageable"):
        got = _run(kind, rho0, u0, mask)
        for (ra, ua), (rb, ub) in zip(ref, got):
            assert np.array_equal(ra, rb) and np.array_equal(ua, ub), kind
