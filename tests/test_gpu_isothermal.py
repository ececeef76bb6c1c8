"""Isothermal wall-modelled walls on the GPU (the wall heat flux q_w that the
paper's wall-stress coupling imposes at isothermal walls, Sec. 3.1) against
the oracle: FP64 parity 1e-12 in the relative max norm, the FP32-mixed error,
and the adjoint's refusal."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, gpu_ut, parity, parity_per_var, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _phys(factor):
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    phys = dict(wl.phys)
    phys["T_wall"] = factor * phys["p0"] / phys["R"]
    return wl, phys


@pytest.mark.parametrize("factor", [0.9, 1.2])
@pytest.mark.parametrize("law", [1, 0])
def test_isothermal_channel_matches_oracle(ora, factor, law):
    torch = torch_cuda()
    wl, phys = _phys(factor)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, law=law, ic="channel")
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print("isothermal", factor, "law", law, "parity", e, ["%.1e" % x for x in parity_per_var(out, ref)])
    assert e <= TOL, e
    # the heat flux changes the energy equation against the adiabatic walls
    wl2, phys2 = _phys(factor)
    phys2["T_wall"] = 0.0
    o2, g2, _, _ = case(ora, wl.spec, phys2, surf_flux=2, law=law, ic="channel", extended=False)
    ad = gpu_ut(torch, g2, U).reshape(5, -1)
    assert np.abs(out.reshape(5, -1)[4] - ad[4]).max() > 1e-6 * np.abs(ad[4]).max()


def test_isothermal_channel_mixed_and_steps(ora):
    torch = torch_cuda()
    wl, phys = _phys(1.2)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, law=1, ic="channel", precision=dg.FP32_MIXED)
    a = gpu_ut(torch, g, U).reshape(5, -1)
    b = o.time_derivative(U).reshape(5, -1)
    e = [float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5)]
    print("isothermal mixed rel L2", ["%.1e" % x for x in e])
    assert max(e) <= 1e-5, e
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, law=1, ic="channel")
    dt = o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    e = parity(Ug.cpu().numpy() - U, o.rk_steps(U, dt, 2) - U)
    print("isothermal rk steps parity (increment)", e)
    assert e <= TOL, e


def test_adjoint_and_wall_shear_refuse_isothermal_walls(ora):
    torch = torch_cuda()
    wl, phys = _phys(1.1)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, law=1, ic="channel", extended=False)
    Ud = torch.from_numpy(U).cuda()
    with pytest.raises(dg.DGError) as ei:
        g.vjp(torch.ones_like(Ud), torch.empty_like(Ud), U=Ud)
    assert ei.value.code == -8
    with pytest.raises(dg.DGError) as ei:
        g.wall_shear(Ud)
    assert ei.value.code == -8
