"""Inflow and outflow boundaries on the GPU (paper Sec. 4: Dirichlet inflow,
subsonic pressure outflow) against the oracle: FP64 parity 1e-12 in the
relative max norm, free-stream preservation on the device, the FP32-mixed
error, and the adjoint through the exterior states."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import gpu_ut, parity, parity_per_var, tgv_with_offset, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _phys(Ma=0.3, Re=400.0):
    phys = I.phys_params(Ma=Ma, Re=Re)
    g, p0 = phys["gamma"], phys["p0"]
    rho, u, v = 1.02, 0.75, 0.05
    phys.update(U_in=np.array([rho, rho * u, rho * v, 0.0, 1.03 * p0 / (g - 1) + 0.5 * rho * (u * u + v * v)]),
                p_out=0.98 * p0)
    return phys


def _case(ora, spec, phys, surf=2, viscous=1, precision=dg.FP64, extended=True, law=1):
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, surf_flux=surf, viscous=viscous, law=law, extended=extended)
    g = dg.Operator(spec.N, X, nbr, phys, precision=precision, surf_flux=surf, viscous=viscous, law=law)
    U = I.perturb(tgv_with_offset(X, phys, offset=(0.6, 0.05, 0.0)), rel=1e-3)
    return o, g, X, U


CASES = [
    ("n3_box_in_out_periodic_yz", I.BoxSpec(3, 4, 2, 2, geometry="sine", amplitude=0.2, periodic=(False, True, True),
                                            boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))),
    # stretched channel without the interior warp: the wall normals stay
    # normal to the inflow and outflow planes, so every wall-model sample
    # point lies inside the (non-periodic) box
    ("n5_channel_in_out_walls", I.BoxSpec(5, 3, 4, 2, lengths=(6.0, 2.0, 3.0), geometry="channel", amplitude=0.0,
                                          periodic=(False, False, True),
                                          boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))),
    ("n7_outflow_both_ends", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1, periodic=(True, True, False),
                                       boundary=((I.WALL, I.WALL), (I.WALL, I.WALL), (I.OUTFLOW, I.OUTFLOW)))),
]


@pytest.mark.parametrize("label,spec", CASES)
@pytest.mark.parametrize("surf", [1, 2])
def test_inflow_outflow_match_oracle(ora, label, spec, surf):
    torch = torch_cuda()
    o, g, X, U = _case(ora, spec, _phys(), surf=surf)
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print(label, surf, "parity", e, ["%.1e" % x for x in parity_per_var(out, ref)])
    assert e <= TOL, e


def test_free_stream_through_inflow_and_outflow_on_device(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=400.0)
    g0 = phys["gamma"]; p0 = phys["p0"]
    vel = (0.6, 0.2, -0.1)
    U0 = np.array([1.0, *vel, p0 / (g0 - 1) + 0.5 * np.dot(vel, vel)])
    phys.update(U_in=U0, p_out=p0)
    spec = CASES[0][1]
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    g = dg.Operator(spec.N, X, I.connectivity(spec), phys, surf_flux=2)
    shape = X[0].shape
    U = I.conservative(np.ones(shape), vel[0] * np.ones(shape), vel[1] * np.ones(shape), vel[2] * np.ones(shape),
                       p0 * np.ones(shape), g0)
    Ut = gpu_ut(torch, g, U)
    print("free stream max |Ut|", np.abs(Ut).max())
    assert np.abs(Ut).max() < 1e-10


def test_inflow_outflow_mixed_error(ora):
    torch = torch_cuda()
    o, g, X, U = _case(ora, CASES[0][1], _phys(), precision=dg.FP32_MIXED)
    a = gpu_ut(torch, g, U).reshape(5, -1)
    b = o.time_derivative(U).reshape(5, -1)
    e = [float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5)]
    print("inflow/outflow mixed rel L2", ["%.1e" % x for x in e])
    assert max(e) <= 1e-4, e


def test_inflow_outflow_rk_steps_match_oracle(ora):
    torch = torch_cuda()
    o, g, X, U = _case(ora, CASES[1][1], _phys())
    dt = o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    e = parity(Ug.cpu().numpy() - U, o.rk_steps(U, dt, 2) - U)
    print("inflow/outflow rk steps parity (increment)", e)
    assert e <= TOL, e


def _vjp(torch, g, U, lam):
    Ud = torch.from_numpy(U).cuda()
    gU = torch.empty_like(Ud)
    g.vjp(torch.from_numpy(np.ascontiguousarray(lam)).cuda(), gU, U=Ud)
    torch.cuda.synchronize()
    g.check_status()
    return gU.cpu().numpy()


@pytest.mark.parametrize("label,spec", [CASES[0], CASES[2]])
@pytest.mark.parametrize("surf,vol", [(2, 0), (1, 0), (2, 2)])
def test_adjoint_through_inflow_and_outflow(ora, label, spec, surf, vol):
    """Dot-product test <lam, J d> = <J^T lam, d> with J d the extended
    oracle's forward-mode derivative: the inflow state is a constant, the
    outflow state depends on the interior density and momentum (its energy
    p_out / (gamma - 1) + |m|^2 / (2 rho), its temperature p_out / (rho R)
    in the lifting)."""
    torch = torch_cuda()
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    phys = _phys()
    o = ora.Oracle(spec.N, X, nbr, phys, vol_flux=vol, surf_flux=surf, viscous=1, law=1, extended=True)
    g = dg.Operator(spec.N, X, nbr, phys, vol_flux=vol, surf_flux=surf, viscous=1, law=1)
    U = I.perturb(tgv_with_offset(X, phys, offset=(0.6, 0.05, 0.0)), rel=1e-2)
    lam = I.random_direction(U.shape, seed=31)
    gU = _vjp(torch, g, U, lam)
    for seed in (32, 33):
        d = I.random_direction(U.shape, seed=seed) * np.abs(U)
        _, Jd = o.jvp(U, d)
        a = float((lam * Jd).sum()); b = float((gU * d).sum())
        print(label, surf, vol, "dot", a, b, abs(a - b) / abs(a))
        assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()


def test_adjoint_inflow_outflow_finite_differences(ora):
    """The same cotangent against central differences of the GPU operator
    (no oracle in the loop)."""
    torch = torch_cuda()
    o, g, X, U = _case(ora, CASES[1][1], _phys(), extended=False)
    lam = I.random_direction(U.shape, seed=34)
    gU = _vjp(torch, g, U, lam)
    d = I.random_direction(U.shape, seed=35) * np.abs(U)
    eps = 1e-6
    fa = torch.empty((5,) + U.shape[1:], dtype=torch.float64, device="cuda")
    fb = torch.empty_like(fa)
    g.time_derivative(fa, torch.from_numpy(U + eps * d).cuda())
    g.time_derivative(fb, torch.from_numpy(U - eps * d).cuda())
    fd = float((lam * (fa - fb).cpu().numpy()).sum()) / (2 * eps)
    b = float((gU * d).sum())
    print("inflow/outflow FD", fd, "adjoint", b)
    assert abs(fd - b) <= 1e-6 * abs(b)
