"""Pins of the oracle's operator by invariants the discretisation must keep.

* Curl-form metrics satisfy the discrete metric identities and reproduce
  the exact metrics of an affine map.
* Free-stream preservation on deformed meshes (the split-form DGSEM of
  paper Sec. 2.2 / Sec. 4 with curl-form metrics keeps a uniform state).
* Discrete conservation of mass, momentum and energy on periodic meshes.
* Kinetic-energy preservation of the KEP split forms (and of Chandrashekar's
  flux) with a central surface flux at constant pressure.
* Semi-discrete entropy conservation of the split form with Chandrashekar's
  entropy-conserving flux in the volume and at the faces (paper Sec. 4).
* Sutherland's law reduces to constant viscosity at uniform temperature.
Each is a property of the mathematics, not of the code: a dropped metric
term, a wrong sign in the surface correction or a transposed index breaks
one of them."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import oracle_case, quad_weights

EPS = np.finfo(np.float64).eps


def _metric_identity_residual(ora, o):
    x, w, D = ora.lgl(o.N)
    n = o.n
    Ja, J = o.metrics()
    Jr = Ja.reshape(o.K, n, n, n, 3, 3)
    res = (np.einsum("im,ekjmc->ekjic", D, Jr[..., 0, :]) +
           np.einsum("jm,ekmic->ekjic", D, Jr[..., 1, :]) +
           np.einsum("km,emjic->ekjic", D, Jr[..., 2, :]))
    return np.abs(res).max(), np.abs(Ja).max()


@pytest.mark.parametrize("geom", ["sine", "channel"])
@pytest.mark.parametrize("N", [3, 7])
def test_metric_identities(ora, geom, N):
    if geom == "sine":
        spec = I.BoxSpec(N, 3, 3, 3, geometry="sine", amplitude=0.3)
    else:
        spec = I.BoxSpec(N, 4, 4, 2, lengths=(2 * math.pi, 2.0, math.pi), geometry="channel",
                         amplitude=0.05, periodic=(True, False, True))
    o, X, nbr = oracle_case(ora, spec, I.phys_params(), viscous=0)
    r, s = _metric_identity_residual(ora, o)
    x, w, D = ora.lgl(N)
    # roundoff of two chained derivative applications: eps |Ja| |D| n
    assert r < 20 * EPS * s * np.abs(D).max() * (N + 1)


def test_affine_metrics_closed_form(ora):
    spec = I.BoxSpec(3, 2, 3, 4, lengths=(2.0, 3.0, 8.0))
    o, X, nbr = oracle_case(ora, spec, I.phys_params(), viscous=0)
    Ja, J = o.metrics()
    hx, hy, hz = 2.0 / 2 / 2, 3.0 / 3 / 2, 8.0 / 4 / 2  # half element sizes
    ref = np.diag([hy * hz, hx * hz, hx * hy])
    assert np.abs(Ja - ref).max() < 1e-13
    assert np.abs(J - hx * hy * hz).max() < 1e-13


def _freestream_scale(ora, o, U, phys):
    """Roundoff scale of the free-stream residual,
    n * max|D|^2 * max|F| * max|Ja| / min J: the metrics carry roundoff of
    order eps |D| |Ja| and the divergence multiplies it by n |D| |F| / J."""
    x, w, D = ora.lgl(o.N)
    Ja, J = o.metrics()
    rho = U[0]; u = U[1:4] / rho
    p = (phys["gamma"] - 1) * (U[4] - 0.5 * rho * (u * u).sum(0))
    Fmax = np.abs(U[4] + p).max() * np.abs(u).max() + np.abs(p).max()
    return o.n * np.abs(D).max() ** 2 * Fmax * np.abs(Ja).max() / J.min()


@pytest.mark.parametrize("N", [3, 7])
@pytest.mark.parametrize("surf", [1, 2])
@pytest.mark.parametrize("amp", [0.1, 0.8])
def test_free_stream_sine_mesh(ora, N, surf, amp):
    phys = I.phys_params(Ma=0.3)
    spec = I.BoxSpec(N, 3, 2, 2, geometry="sine", amplitude=amp)
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=surf)
    U = I.free_stream(X, phys, velocity=(1.0, -0.5, 0.25))
    Ut = o.time_derivative(U)
    assert np.abs(Ut).max() < 50 * EPS * _freestream_scale(ora, o, U, phys)


@pytest.mark.parametrize("N", [3, 5])
def test_free_stream_channel_mesh(ora, N):
    # wall-parallel uniform flow on the warped channel: slip walls keep it
    phys = I.phys_params()
    spec = I.BoxSpec(N, 4, 4, 2, lengths=(2 * math.pi, 2.0, math.pi), geometry="channel",
                     amplitude=0.05, periodic=(True, False, True))
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=2, viscous=0)
    U = I.free_stream(X, phys, velocity=(1.0, 0.0, 0.5))
    Ut = o.time_derivative(U)
    assert np.abs(Ut).max() < 50 * EPS * _freestream_scale(ora, o, U, phys)


@pytest.mark.parametrize("viscous,surf", [(0, 1), (1, 1), (1, 2), (1, 0)])
def test_discrete_conservation(ora, viscous, surf):
    phys = I.phys_params(Re=100.0)
    spec = I.BoxSpec(3, 3, 3, 2, geometry="sine", amplitude=0.3)
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=surf, viscous=viscous)
    U = I.perturb(I.taylor_green(X, phys), rel=5e-2)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    wJ = quad_weights(ora, o)
    for v in range(5):
        tot = (wJ * Ut[v]).sum()
        mag = (wJ * np.abs(Ut[v])).sum()
        assert abs(tot) <= 1e-13 * mag, (v, tot, mag)


@pytest.mark.parametrize("vol", [0, 1, 2])
def test_kinetic_energy_preservation(ora, vol):
    # constant pressure, random density and velocity, inviscid, central surface flux
    phys = I.phys_params(Ma=0.3)
    spec = I.BoxSpec(4, 3, 2, 2, geometry="sine", amplitude=0.4)
    o, X, nbr = oracle_case(ora, spec, phys, vol_flux=vol, surf_flux=0, viscous=0)
    shape = X[0].shape
    rho = 1.0 + 0.5 * I.uniform(X[0].size, 0, 1, seed=11).reshape(shape)
    vel = I.uniform(3 * X[0].size, -1, 1, seed=12).reshape(3, *shape)
    U = I.conservative(rho, vel[0], vel[1], vel[2], phys["p0"] * np.ones(shape), phys["gamma"])
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    Ur = U.reshape(5, o.K, o.n3)
    u = Ur[1:4] / Ur[0]
    wJ = quad_weights(ora, o)
    dke = (wJ * ((u * Ut[1:4]).sum(0) - 0.5 * (u * u).sum(0) * Ut[0])).sum()
    scale = (wJ * ((np.abs(u * Ut[1:4])).sum(0) + 0.5 * (u * u).sum(0) * np.abs(Ut[0]))).sum()
    assert abs(dke) < 1e-13 * scale, (dke, scale)
    # with dissipation (LLF) the kinetic energy must decrease instead
    o2, _, _ = oracle_case(ora, spec, phys, vol_flux=vol, surf_flux=1, viscous=0)
    Ut2 = o2.time_derivative(U).reshape(5, o.K, o.n3)
    dke2 = (wJ * ((u * Ut2[1:4]).sum(0) - 0.5 * (u * u).sum(0) * Ut2[0])).sum()
    assert dke2 < -1e-6 * scale


def _entropy_variables(U, gamma):
    rho = U[0]; u = U[1:4] / rho
    p = (gamma - 1) * (U[4] - 0.5 * rho * (u * u).sum(0))
    s = np.log(p) - gamma * np.log(rho)
    return np.concatenate([((gamma - s) / (gamma - 1) - 0.5 * rho * (u * u).sum(0) / p)[None],
                           rho * u / p, (-rho / p)[None]])


@pytest.mark.parametrize("N", [3, 4])
def test_entropy_conservation(ora, N):
    # With the entropy-conserving two-point flux in the volume and at the
    # faces, inviscid and periodic, the split-form DGSEM on a curvilinear mesh
    # conserves the total entropy: sum_nodes wJ w(U) . Ut = 0.  With Roe's
    # flux at the faces it must produce entropy decay instead.
    phys = I.phys_params(Ma=0.3)
    spec = I.BoxSpec(N, 3, 2, 2, geometry="sine", amplitude=0.4)
    o, X, nbr = oracle_case(ora, spec, phys, vol_flux=2, surf_flux=0, viscous=0)
    U = I.perturb(I.taylor_green(X, phys), rel=0.2)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    W = _entropy_variables(U.reshape(5, o.K, o.n3), phys["gamma"])
    wJ = quad_weights(ora, o)
    ds = (wJ * (W * Ut).sum(0)).sum()
    scale = (wJ * np.abs(W * Ut).sum(0)).sum()
    assert abs(ds) < 1e-13 * scale, (ds, scale)
    o2, _, _ = oracle_case(ora, spec, phys, vol_flux=2, surf_flux=2, viscous=0)
    Ut2 = o2.time_derivative(U).reshape(5, o.K, o.n3)
    ds2 = (wJ * (W * Ut2).sum(0)).sum()
    assert ds2 < -1e-6 * scale


def test_sutherland_uniform_temperature(ora):
    # at a uniform temperature T0 Sutherland's law is the constant viscosity
    # mu(T0): the whole operator (viscous fluxes, lifting, wall-free periodic
    # mesh) must match the constant-viscosity run with that mu
    phys = I.phys_params(Re=200.0)
    spec = I.BoxSpec(3, 2, 2, 2, geometry="sine", amplitude=0.3)
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    shape = X[0].shape
    rho = 1.0 + 0.3 * I.uniform(X[0].size, 0, 1, seed=21).reshape(shape)
    vel = I.uniform(3 * X[0].size, -1, 1, seed=22).reshape(3, *shape)
    T0 = 1.3
    p = rho * phys["R"] * T0
    U = I.conservative(rho, vel[0], vel[1], vel[2], p, phys["gamma"])
    ps = dict(phys, suth_S=0.4, T_ref=0.9)
    mu0 = ora.viscosity(ps, T0)
    assert mu0 == pytest.approx(phys["mu"] * (T0 / 0.9) ** 1.5 * (0.9 + 0.4) / (T0 + 0.4), rel=1e-14)
    a = ora.Oracle(spec.N, X, nbr, ps, surf_flux=2).time_derivative(U)
    b = ora.Oracle(spec.N, X, nbr, dict(phys, mu=mu0), surf_flux=2).time_derivative(U)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    c = ora.Oracle(spec.N, X, nbr, phys, surf_flux=2).time_derivative(U)
    assert np.abs(a - c).max() > 1e-6 * np.abs(b).max()


def test_energy_balance_with_isothermal_walls(ora):
    # periodic in x and z, isothermal wall-modelled walls in y, no body force:
    # the total energy changes only through the walls, by the inviscid wall
    # flux (slip, mirror state) minus the wall heat flux q_w into the fluid
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    spec = I.BoxSpec(wl.spec.N, wl.spec.nx, wl.spec.ny, wl.spec.nz, lengths=wl.spec.lengths,
                     geometry="channel", amplitude=0.0, periodic=wl.spec.periodic)
    phys = dict(wl.phys)
    phys.update(fx=0.0, fy=0.0, fz=0.0)
    phys["T_wall"] = 1.1 * phys["p0"] / phys["R"]
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, surf_flux=2, viscous=1, law=1)
    U = I.channel_profile(X, phys)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    wJ = quad_weights(ora, o)
    lhs = (wJ * Ut[4]).sum()
    qw = o.wall_heat(U)
    n = spec.N + 1
    s = (spec.lengths[0] / spec.nx / 2) * (spec.lengths[2] / spec.nz / 2)
    Ur = U.reshape(5, o.K, o.n3)
    rhs = 0.0
    slot = 0
    for e in range(o.K):
        for l in range(6):
            if nbr[e, l] != I.WALL:
                continue
            nout = np.array([0.0, -1.0 if l == 2 else 1.0, 0.0])
            for b in range(n):
                for a in range(n):
                    p = [None, None, a + n * n * b, a + n * ((n - 1) + n * b)][l]
                    Um = Ur[:, e, p]
                    mn = Um[1:4] @ nout
                    Ub = Um.copy(); Ub[1:4] = Um[1:4] - 2 * mn * nout
                    F = ora.riemann(phys, 0, 2, Um, Ub, nout)
                    rhs -= w[a] * w[b] * s * (F[4] - qw[slot + a + n * b])
            slot += n * n
    heat = sum(w[a] * w[b] * s * qw[k * n * n + a + n * b] for k in range(len(qw) // (n * n))
               for b in range(n) for a in range(n))
    assert abs(heat) > 1e-6 * abs(lhs) + 1e-12     # the walls do exchange heat
    assert abs(lhs - rhs) <= 1e-11 * (abs(rhs) + abs(heat)), (lhs, rhs, heat)
