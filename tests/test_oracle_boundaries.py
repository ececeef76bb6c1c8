"""Pins of the oracle's inflow and outflow boundaries (paper Sec. 4: the
cascade's supersonic Dirichlet inflow and subsonic pressure outflow).

A boundary face sees an exterior state: the prescribed inflow state, or the
interior density and velocity with the prescribed outflow pressure.  The
inviscid flux is the selected Riemann solver between the interior and that
state, the lifting averages with it, and the viscous flux is the interior one.

* Free-stream preservation: when the exterior states equal a uniform interior
  state, Ut = 0 on a curved mesh (viscous, LLF and Roe).
* Global balance: on an affine mesh the rate of change of the total of every
  conserved variable equals minus the boundary flux, recomputed here from the
  exterior states and the oracle's point Riemann solver."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import quad_weights

EPS = np.finfo(np.float64).eps


def _uniform(X, phys, vel, p):
    shape = X[0].shape
    return I.conservative(np.ones(shape), vel[0] * np.ones(shape), vel[1] * np.ones(shape),
                          vel[2] * np.ones(shape), p * np.ones(shape), phys["gamma"])


def _case(ora, spec, phys, surf=1, viscous=1):
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, surf_flux=surf, viscous=viscous)
    return o, X, nbr


@pytest.mark.parametrize("surf", [1, 2])
@pytest.mark.parametrize("N", [3, 5])
def test_free_stream_with_inflow_outflow(ora, surf, N):
    phys = I.phys_params(Ma=0.3, Re=100.0)
    vel, p = (0.6, 0.2, -0.1), phys["p0"]
    U0 = np.array([1.0, *vel, p / (phys["gamma"] - 1) + 0.5 * np.dot(vel, vel)])
    phys.update(U_in=U0, p_out=p)
    spec = I.BoxSpec(N, 3, 2, 2, geometry="sine", amplitude=0.3, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    o, X, nbr = _case(ora, spec, phys, surf=surf)
    U = _uniform(X, phys, vel, p)
    Ut = o.time_derivative(U)
    x, w, D = ora.lgl(N)
    Ja, J = o.metrics()
    scale = (N + 1) * np.abs(D).max() ** 2 * (p + 1.0) * np.abs(Ja).max() / J.min()
    assert np.abs(Ut).max() < 50 * EPS * scale, np.abs(Ut).max()


def _ghost(U, code, phys, n):
    g = phys["gamma"]
    if code == I.INFLOW:
        return np.asarray(phys["U_in"], dtype=float)
    out = U.copy()
    out[4] = phys["p_out"] / (g - 1) + 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    return out


@pytest.mark.parametrize("surf", [1, 2])
def test_boundary_flux_balance(ora, surf):
    phys = I.phys_params(Ma=0.3)
    g = phys["gamma"]
    phys.update(U_in=np.array([1.05, 0.7, 0.05, 0.0, phys["p0"] * 1.02 / (g - 1) + 0.5 * 0.7 ** 2 / 1.05]),
                p_out=phys["p0"] * 0.98)
    L = (3.0, 2.0, 2.5)
    spec = I.BoxSpec(3, 3, 2, 2, lengths=L, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    o, X, nbr = _case(ora, spec, phys, surf=surf, viscous=0)
    base = _uniform(X, phys, (0.6, 0.0, 0.0), phys["p0"])
    U = I.perturb(base, rel=2e-2)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    wJ = quad_weights(ora, o)
    lhs = (wJ[None] * Ut).sum(axis=(1, 2))
    # boundary fluxes on the x faces of the affine box
    x, w, D = ora.lgl(spec.N)
    n = spec.N + 1
    hy, hz = L[1] / spec.ny / 2, L[2] / spec.nz / 2
    s = hy * hz
    Ur = U.reshape(5, o.K, o.n3)
    rhs = np.zeros(5)
    for e in range(o.K):
        for side, code, i, nx in ((0, I.INFLOW, 0, -1.0), (1, I.OUTFLOW, n - 1, 1.0)):
            if nbr[e, side] != code:
                continue
            for b in range(n):
                for a in range(n):
                    p = i + n * (a + n * b)
                    Um = Ur[:, e, p]
                    nv = np.array([nx, 0.0, 0.0])
                    F = ora.riemann(phys, 0, surf, Um, _ghost(Um, code, phys, nv), nv)
                    rhs -= w[a] * w[b] * s * F
    err = np.abs(lhs - rhs) / (np.abs(rhs).max() + np.abs(lhs).max())
    assert err.max() < 1e-12, (lhs, rhs)
    assert np.abs(rhs).max() > 1e-3  # the boundaries do carry flux


def test_viscous_boundary_flux_is_the_interior_one(ora):
    # u = u0 + a x, rho = 1, p = p0 on an affine box: the lifted gradient is
    # exact, the exterior states equal the interior traces, so the boundary
    # flux is F(U).n - Fv.n with Fv from tau_xx = 4/3 mu a and no heat flux
    phys = I.phys_params(Ma=0.3, Re=50.0)
    g, mu, p0 = phys["gamma"], phys["mu"], phys["p0"]
    L = (3.0, 2.0, 2.5)
    u0, a = 0.4, 0.1
    U_in = np.array([1.0, u0, 0.0, 0.0, p0 / (g - 1) + 0.5 * u0 ** 2])
    phys.update(U_in=U_in, p_out=p0)
    spec = I.BoxSpec(3, 3, 2, 2, lengths=L, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    o, X, nbr = _case(ora, spec, phys, surf=2, viscous=1)
    shape = X[0].shape
    u = u0 + a * X[0]
    U = I.conservative(np.ones(shape), u, np.zeros(shape), np.zeros(shape), p0 * np.ones(shape), g)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    lhs = (quad_weights(ora, o)[None] * Ut).sum(axis=(1, 2))
    x, w, D = ora.lgl(spec.N)
    n = spec.N + 1
    s = (L[1] / spec.ny / 2) * (L[2] / spec.nz / 2)
    tau = 4.0 / 3.0 * mu * a
    Ur = U.reshape(5, o.K, o.n3)
    rhs = np.zeros(5)
    for e in range(o.K):
        for side, code, i, nx in ((0, I.INFLOW, 0, -1.0), (1, I.OUTFLOW, n - 1, 1.0)):
            if nbr[e, side] != code:
                continue
            for b in range(n):
                for aa in range(n):
                    p = i + n * (aa + n * b)
                    Um = Ur[:, e, p]
                    nv = np.array([nx, 0.0, 0.0])
                    F = ora.riemann(phys, 0, 2, Um, _ghost(Um, code, phys, nv), nv)
                    ub = Um[1] / Um[0]
                    Fv = np.array([0.0, tau * nx, 0.0, 0.0, tau * ub * nx])
                    rhs -= w[aa] * w[b] * s * (F - Fv)
    err = np.abs(lhs - rhs) / np.abs(rhs).max()
    assert err.max() < 1e-12, (lhs, rhs)
