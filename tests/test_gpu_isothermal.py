"""Isothermal wall-modelled walls on the GPU (the wall heat flux q_w that the
paper's wall-stress coupling imposes at isothermal walls, Sec. 3.1) against
the oracle: FP64 parity 1e-12 in the relative max norm, the FP32-mixed error,
and the adjoint with the wall heat flux's derivative."""
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


@pytest.mark.parametrize("law,vol", [(1, 0), (0, 0), (1, 2)])
def test_isothermal_adjoint_matches_oracle(ora, law, vol):
    """Dot-product test of the adjoint at isothermal walls against the
    extended oracle's forward-mode derivative (the wall heat flux q_w and the
    Crocco-Busemann transform differentiated with the stress), and the
    (kappa, B) cotangents."""
    torch = torch_cuda()
    wl, phys = _phys(1.15)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, vol_flux=vol, law=law, ic="channel")
    lam = I.random_direction(U.shape, seed=41)
    Ud = torch.from_numpy(U).cuda()
    gU = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.vjp(torch.from_numpy(lam).cuda(), gU, Ud, gth)
    g.check_status()
    gU = gU.cpu().numpy(); th = gth.cpu().numpy()
    d = I.random_direction(U.shape, seed=42) * np.abs(U)
    _, Jd = o.jvp(U, d)
    a = float((lam * Jd).sum()); b = float((gU * d).sum())
    print("isothermal law", law, "vol", vol, "dot", a, b)
    assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()
    for k, (dk, dB) in enumerate(((1.0, 0.0), (0.0, 1.0))):
        _, Jt = o.jvp(U, None, dk, dB)
        ref = float((lam * Jt).sum())
        print("  dtheta", k, ref, th[k])
        assert abs(ref - th[k]) <= 1e-10 * np.abs(lam * Jt).sum()


def test_isothermal_wall_shear_and_rollout_gradient(ora):
    """Mean wall shear at isothermal walls and the gradient of a 10-step
    rollout of it against the oracle's forward-mode derivative."""
    torch = torch_cuda()
    wl, phys = _phys(0.9)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, law=1, ic="channel", extended=False)
    Ud = torch.from_numpy(U).cuda()
    L0 = g.wall_shear(Ud)
    ref = o.wall_shear(U)
    print("isothermal wall shear", L0, ref)
    assert abs(L0 - ref) <= 1e-12 * abs(ref)
    dt = 0.5 * o.dt(U, 0.9)
    gU0 = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = g.rollout_vjp(Ud, 10, dt, gU0, gth)
    g.check_status()
    d = I.random_direction(U.shape, seed=43) * np.abs(U)
    L_ref, dL = o.rollout_jvp(U, d, 0.0, 0.0, 10, dt)
    _, dLk = o.rollout_jvp(U, None, 1.0, 0.0, 10, dt)
    ad = float((gU0.cpu().numpy() * d).sum())
    th = gth.cpu().numpy()
    print("rollout loss", L, L_ref, "dU0", ad, dL, "dkappa", th[0], dLk)
    assert abs(L - L_ref) <= 1e-11 * abs(L_ref)
    assert abs(ad - dL) <= 1e-9 * abs(dL)
    assert abs(th[0] - dLk) <= 1e-9 * abs(dLk)
