"""Runtime error paths of the C ABI on the GPU: calls before the state is
set, bad stage indices, wrong array sizes, and the device-side failure flag
for a non-finite state (raised by the stage kernel as a flag, read on the
host by dg_check_status; the GPU context stays usable)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _op(torch, **kw):
    spec = I.BoxSpec(2, 2, 2, 2)
    x, w = dg.lgl_nodes(spec.N)
    X = I.node_coordinates(spec, x)
    phys = I.phys_params()
    U = I.perturb(I.taylor_green(X, phys), rel=1e-3)
    return dg.Operator(spec.N, X, I.connectivity(spec), phys, **kw), torch.from_numpy(U).cuda()


def test_state_must_be_set_first():
    torch = torch_cuda()
    op, Ud = _op(torch)
    with pytest.raises(dg.DGError) as ei:
        op.rk_stage(0, 0.0, 1e-3)
    assert ei.value.code == -2
    with pytest.raises(dg.DGError) as ei:
        op.time_derivative(torch.empty_like(Ud))
    assert ei.value.code == -2


def test_bad_stage_and_sizes():
    torch = torch_cuda()
    op, Ud = _op(torch)
    op.set_state(Ud)
    with pytest.raises(dg.DGError) as ei:
        op.rk_stage(5, 0.0, 1e-3)
    assert ei.value.code == -1
    with pytest.raises(ValueError):
        op.time_derivative(torch.empty(10, dtype=torch.float64, device="cuda"), Ud)


@pytest.mark.parametrize("precision", [dg.FP64, dg.FP32_MIXED])
def test_non_finite_state_is_flagged_and_the_context_recovers(precision):
    torch = torch_cuda()
    op, Ud = _op(torch, precision=precision)
    bad = Ud.clone()
    bad[4, 3, 5] = float("nan")
    op.set_state(bad)
    op.rk_stage(0, 0.0, 1e-3)
    with pytest.raises(dg.DGError) as ei:
        op.check_status()
    assert ei.value.code == -5
    # the flag is cleared by the read; a finite state runs cleanly again
    op.set_state(Ud)
    op.rk_steps(0.0, 1e-3, 1)
    op.check_status()
    out = torch.empty_like(Ud)
    op.get_state(out)
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("precision", [dg.FP64, dg.FP32_MIXED])
def test_wall_solve_iteration_cap_flags_no_convergence(precision):
    """SolveWallStress (Sec. 3.2, Algorithms 1-2) under an iteration cap of 1:
    no wall node can bracket its root and take a Newton step within one
    evaluation of the law, so the wall kernel flags non-convergence, which
    dg_check_status reports as DG_ERR_WM_NOCONV (a bounded loop that runs out,
    no wait and no trap).  With the cap restored the same context evaluates
    cleanly again, bitwise like a fresh context."""
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    x, w = dg.lgl_nodes(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    Ud = torch.from_numpy(I.channel_profile(X, wl.phys)).cuda()
    op = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=precision, surf_flux=2, law=1)
    fresh = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=precision, surf_flux=2, law=1)
    op.set_state(Ud)
    op.set_wall_solve_limit(1)
    out = torch.empty_like(Ud)
    op.time_derivative(out)
    with pytest.raises(dg.DGError) as ei:
        op.check_status()
    assert ei.value.code == -6
    op.set_wall_solve_limit(200)
    op.set_state(Ud)  # clears the warm starts left by the capped solve
    op.time_derivative(out)
    op.check_status()
    fresh.set_state(Ud)
    ref = torch.empty_like(Ud)
    fresh.time_derivative(ref)
    fresh.check_status()
    assert torch.equal(out, ref)
    with pytest.raises(dg.DGError) as ei:
        op.set_wall_solve_limit(0)
    assert ei.value.code == -1
    op.close(); fresh.close()
