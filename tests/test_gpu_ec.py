"""The paper's production scheme on the GPU (Sec. 4): Chandrashekar's
entropy-conserving volume flux, Roe's surface flux with Harten's entropy fix
and Sutherland's viscosity, against the oracle.

FP64 tolerance: relative max-norm 1e-12 per variable, as for the KEP fluxes.
The logarithmic means take a series branch for close arguments and a
logarithm otherwise: the small perturbation (rel 1e-3) keeps every pair on
the series branch, the large one (rel 0.2) sends most pairs to the
logarithm."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, gpu_ut, parity, parity_per_var, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-12
EC = dg.VOL_EC_CHANDRASHEKAR


@pytest.mark.parametrize("label,spec,surf,visc,suth,rel", [
    ("n3_4^3_roe_suth", I.BoxSpec(3, 4, 4, 4), 2, 1, True, 1e-3),
    ("n7_sine_roe_suth", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1), 2, 1, True, 1e-3),
    ("n4_sine_central_euler_rough", I.BoxSpec(4, 3, 2, 2, geometry="sine", amplitude=0.3), 0, 0, False, 0.2),
    ("n5_llf_rough", I.BoxSpec(5, 2, 3, 2, geometry="sine", amplitude=0.2), 1, 1, True, 0.2),
    ("n2_ragged_roe", I.BoxSpec(2, 3, 2, 5), 2, 1, False, 0.05),
    ("n8_roe_suth", I.BoxSpec(8, 2, 1, 2, geometry="sine", amplitude=0.1), 2, 1, True, 1e-3),
])
def test_ec_time_derivative_matches_oracle(ora, label, spec, surf, visc, suth, rel):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0, sutherland=suth)
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, vol_flux=EC, viscous=visc, rel=rel)
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print(label, "parity", e, ["%.1e" % x for x in parity_per_var(out, ref)])
    assert e <= TOL, e


def test_ec_wall_model_channel_sutherland(ora):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    phys = dict(wl.phys)
    phys.update(T_ref=phys["p0"], suth_S=phys["p0"] * 110.4 / 288.15)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, vol_flux=EC, law=1, ic="channel")
    e = parity(gpu_ut(torch, g, U), o.time_derivative(U))
    print("channel EC + Sutherland parity", e)
    assert e <= TOL, e


def test_ec_entropy_conservation_on_device(ora):
    # the device operator itself conserves the total entropy with the
    # entropy-conserving flux at the faces too (inviscid, periodic, curved)
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3)
    spec = I.BoxSpec(4, 3, 3, 2, geometry="sine", amplitude=0.3)
    o, g, X, U = case(ora, spec, phys, surf_flux=0, vol_flux=EC, viscous=0, rel=0.2)
    Ut = gpu_ut(torch, g, U).reshape(5, -1)
    Ur = U.reshape(5, -1)
    gam = phys["gamma"]
    rho = Ur[0]; u = Ur[1:4] / rho
    p = (gam - 1) * (Ur[4] - 0.5 * rho * (u * u).sum(0))
    s = np.log(p) - gam * np.log(rho)
    W = np.concatenate([((gam - s) / (gam - 1) - 0.5 * rho * (u * u).sum(0) / p)[None], rho * u / p,
                        (-rho / p)[None]])
    x, w, D = ora.lgl(spec.N)
    n = spec.N + 1
    wq = (np.tile(w, n * n) * np.tile(np.repeat(w, n), n) * np.repeat(w, n * n))[None, :]
    Ja, J = o.metrics()
    wJ = (wq * J).reshape(-1)
    ds = (wJ * (W * Ut).sum(0)).sum()
    scale = (wJ * np.abs(W * Ut).sum(0)).sum()
    print("device entropy balance", ds / scale)
    assert abs(ds) < 1e-12 * scale


def test_ec_rk_steps_match_oracle(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0, sutherland=True)
    o, g, X, U = case(ora, I.BoxSpec(3, 3, 2, 2, geometry="sine", amplitude=0.2), phys, surf_flux=2,
                      vol_flux=EC)
    dt = o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    Uo = o.rk_steps(U, dt, 2)
    e = parity(Ug.cpu().numpy() - U, Uo - U)
    print("EC rk steps parity (increment)", e)
    assert e <= TOL, e


@pytest.mark.parametrize("label,spec,surf", [
    ("n3_4^3_roe", I.BoxSpec(3, 4, 4, 4), 2),
    ("n7_sine_roe", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1), 2),
])
def test_ec_mixed_error(ora, label, spec, surf):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0, sutherland=True)
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, vol_flux=EC, precision=dg.FP32_MIXED)
    out = gpu_ut(torch, g, U).reshape(5, -1)
    ref = o.time_derivative(U).reshape(5, -1)
    e = [float(np.linalg.norm(out[v] - ref[v]) / np.linalg.norm(ref[v])) for v in range(5)]
    print(label, "EC mixed rel L2", ["%.1e" % x for x in e])
    assert max(e) <= 1e-4, e


def _vjp(torch, g, U, lam):
    Ud = torch.from_numpy(U).cuda()
    gU = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.vjp(torch.from_numpy(np.ascontiguousarray(lam)).cuda(), gU, Ud, gth)
    torch.cuda.synchronize()
    g.check_status()
    return gU.cpu().numpy(), gth.cpu().numpy()


@pytest.mark.parametrize("label,spec,surf,suth,ic", [
    ("n3_sine_roe_suth", I.BoxSpec(3, 3, 2, 2, geometry="sine", amplitude=0.2), 2, True, "tgv_shift"),
    ("n3_llf_const", I.BoxSpec(3, 2, 3, 2), 1, False, "tgv_shift"),
    ("n7_sine_roe_suth", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, True, "tgv_shift"),
    ("n7_sine_roe_suth_sonic", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, True, "tgv_sonic"),
    ("n4_central_euler", I.BoxSpec(4, 2, 2, 3, geometry="sine", amplitude=0.2), 0, False, "tgv_shift"),
])
def test_production_scheme_adjoint_against_oracle_jvp(ora, label, spec, surf, suth, ic):
    """The adjoint of the paper's Sec. 4 scheme (entropy-conserving volume
    flux, Roe + Harten faces, Sutherland's law): dot-product test
    <lam, J d> = <J^T lam, d> with J d the extended oracle's forward-mode
    derivative (the reverse mode of the logarithmic means and of mu(T), k(T))."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=200.0, sutherland=suth)
    visc = 0 if "euler" in label else 1
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, vol_flux=EC, viscous=visc, rel=1e-2, ic=ic)
    lam = I.random_direction(U.shape, seed=3)
    gU, _ = _vjp(torch, g, U, lam)
    for seed in (4, 5):
        d = I.random_direction(U.shape, seed=seed) * np.abs(U)
        _, Jd = o.jvp(U, d)
        a = float((lam * Jd).sum()); b = float((gU * d).sum())
        print(label, "dot", a, b, abs(a - b) / abs(a))
        assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()


@pytest.mark.parametrize("law", [1, 0])
def test_production_scheme_channel_adjoint(ora, law):
    """Wall-modelled channel with the production scheme: state and (kappa, B)
    cotangents against the oracle (the wall viscosity mu(T_w) by Sutherland's
    law in the wall model's derivative), and central finite differences of the
    GPU operator."""
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    phys = dict(wl.phys)
    phys.update(T_ref=phys["p0"], suth_S=phys["p0"] * 110.4 / 288.15)
    o, g, X, U = case(ora, wl.spec, phys, surf_flux=2, vol_flux=EC, law=law, ic="channel")
    lam = I.random_direction(U.shape, seed=6)
    gU, gth = _vjp(torch, g, U, lam)
    d = I.random_direction(U.shape, seed=7) * np.abs(U)
    _, Jd = o.jvp(U, d)
    a = float((lam * Jd).sum()); b = float((gU * d).sum())
    print("EC channel law", law, "dot", a, b)
    assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()
    for k, (dk, dB) in enumerate(((1.0, 0.0), (0.0, 1.0))):
        _, Jt = o.jvp(U, None, dk, dB)
        ref = float((lam * Jt).sum())
        print("  dtheta", k, ref, gth[k])
        assert abs(ref - gth[k]) <= 1e-10 * np.abs(lam * Jt).sum()
    # central finite differences of the GPU operator along d
    eps = 1e-6
    Up = torch.from_numpy(U + eps * d).cuda(); Um = torch.from_numpy(U - eps * d).cuda()
    fa = torch.empty_like(Up); fb = torch.empty_like(Up)
    g.time_derivative(fa, Up); g.time_derivative(fb, Um)
    fd = float((lam * (fa - fb).cpu().numpy()).sum()) / (2 * eps)
    print("  FD", fd, "adjoint", b)
    assert abs(fd - b) <= 1e-6 * abs(b)


def test_adjoint_refuses_kennedy_gruber(ora):
    torch = torch_cuda()
    spec = I.BoxSpec(2, 2, 2, 2)
    o, g, X, U = case(ora, spec, I.phys_params(), surf_flux=2, vol_flux=1)
    Ud = torch.from_numpy(U).cuda()
    with pytest.raises(dg.DGError) as ei:
        g.vjp(torch.ones_like(Ud), torch.empty_like(Ud), U=Ud)
    assert ei.value.code == -8
