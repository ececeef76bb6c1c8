"""Host batches through the stages (dg_rk_stage_batch): every item's result
equals the one of dg_set_state, the stages and dg_get_state bitwise (FP64 and
FP32-mixed, with and without the wall model), the context's own state is not
touched, and the FP64 result matches the oracle's stage."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, torch_cuda

pytestmark = pytest.mark.gpu


def _items(U, k):
    return [np.ascontiguousarray(I.perturb(U, rel=1e-3, seed=100 + i)) for i in range(k)]


def _sequential(torch, g, U, nstages, dt):
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    for s in range(nstages):
        g.rk_stage(s, 0.0, dt)
    out = torch.empty_like(Ud)
    g.get_state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("label,wl_name,N,elems,precision,ic", [
    ("tgv_n3_fp64", "tgv_n3_4", 3, (4, 4, 4), dg.FP64, "tgv"),
    ("tgv_n7_mixed", "tgv_n3_4", 7, (3, 2, 2), dg.FP32_MIXED, "tgv"),
    ("channel_n3_fp64", "channel_n5", 3, (4, 4, 2), dg.FP64, "channel"),
])
@pytest.mark.parametrize("nstages", [1, 5])
def test_batch_equals_sequential_stages(ora, label, wl_name, N, elems, precision, ic, nstages):
    torch = torch_cuda()
    wl = I.workload(wl_name, N=N, elems=elems)
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, precision=precision, ic=ic)
    dt = 0.5 * o.dt(U, 0.9)
    items = _items(U, 3)
    ref = [_sequential(torch, g, u, nstages, dt) for u in items]
    # the context's own state before the batch
    mark = torch.from_numpy(U).cuda()
    g.set_state(mark)
    ins = [torch.from_numpy(u).pin_memory().numpy() for u in items]
    outs = [torch.empty(u.shape, dtype=torch.float64).pin_memory().numpy() for u in items]
    g.rk_stage_batch(ins, outs, nstages, 0.0, dt)
    g.check_status()
    for a, b in zip(outs, ref):
        assert np.array_equal(a, b)
    after = torch.empty_like(mark)
    g.get_state(after)
    assert torch.equal(after, mark)
    if precision == dg.FP64 and nstages == 1:
        # one stage from a zero register: U + B_0 dt Ut (the oracle's stage)
        # (the increment U_out - U_in also carries the rounding of U_out: a
        # few units of the state's last place)
        Uo = items[0].copy(); dUo = np.zeros_like(Uo)
        o.rk_stage(Uo, dUo, 0, 0.0, dt)
        a = (outs[0] - items[0]).reshape(5, -1); b = (Uo - items[0]).reshape(5, -1)
        u = np.abs(items[0]).reshape(5, -1).max(axis=1)
        for v in range(5):
            err = np.abs(a[v] - b[v]).max()
            print(label, "batch stage increment", v, err, np.abs(b[v]).max(), u[v])
            assert err <= 1e-12 * np.abs(b[v]).max() + 4 * np.finfo(float).eps * u[v]


def test_batch_pageable_buffers_and_arguments(ora):
    torch = torch_cuda()
    wl = I.workload("tgv_n3_4", N=3, elems=(2, 2, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=1, ic="tgv", extended=False)
    dt = 0.5 * o.dt(U, 0.9)
    items = _items(U, 2)
    outs = [np.empty_like(u) for u in items]
    g.rk_stage_batch(items, outs, 2, 0.0, dt)   # pageable host memory: correct, not overlapped
    for a, u in zip(outs, items):
        assert np.array_equal(a, _sequential(torch, g, u, 2, dt))
    g.rk_stage_batch([], [], 1, 0.0, dt)
    for bad in (0, 6):
        with pytest.raises(dg.DGError) as ei:
            g.rk_stage_batch(items, outs, bad, 0.0, dt)
        assert ei.value.code == -1
