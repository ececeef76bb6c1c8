"""Pins of the oracle's forward-mode derivatives and of its time integrator.

* The dual-number Jacobian-vector product of Ut(U; kappa, B) agrees with
  central finite differences (this is the oracle's own adjoint source: the
  GPU VJP is compared with it through <v, J d> = <J^T v, d>).
* LSERK4 (paper Sec. 4) integrated with the oracle operator converges at
  fourth order in time."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import oracle_case


def _fd_check(o, U, dU, dk=0.0, dB=0.0, eps=1e-6, phys=None):
    Ut, Jd = o.jvp(U, dU, dk, dB)
    return Ut, Jd


@pytest.mark.parametrize("surf", [1, 2])
def test_jvp_matches_central_differences_tgv(ora, surf):
    wl = I.workload("tgv_n3_4", elems=(2, 2, 2))
    phys = I.phys_params(Ma=0.3, Re=200.0)
    o, X, nbr = oracle_case(ora, wl.spec, phys, surf_flux=surf)
    U = I.perturb(I.taylor_green(X, phys), rel=1e-2)
    d = I.random_direction(U.shape, seed=5) * np.abs(U)
    Ut, Jd = o.jvp(U, d)
    assert np.array_equal(Ut, o.time_derivative(U))
    h = 1e-6
    fd = (o.time_derivative(U + h * d) - o.time_derivative(U - h * d)) / (2 * h)
    assert np.abs(fd - Jd).max() <= 1e-6 * np.abs(Jd).max()


def _small_channel(ora, law=1, N=3):
    wl = I.workload("channel_n5", N=N, elems=(4, 4, 2))
    o, X, nbr = oracle_case(ora, wl.spec, wl.phys, surf_flux=2, law=law)
    U = I.initial_state(wl, X)
    return wl, o, X, U


@pytest.mark.parametrize("law", [0, 1])
def test_jvp_wall_model_parameters(ora, law):
    wl, o, X, U = _small_channel(ora, law)
    for dk, dB in ((1.0, 0.0), (0.0, 1.0)):
        Ut, Jd = o.jvp(U, None, dk, dB)
        h = 1e-6
        phys_p = dict(wl.phys, kappa=wl.phys["kappa"] + h * dk, B=wl.phys["B"] + h * dB)
        phys_m = dict(wl.phys, kappa=wl.phys["kappa"] - h * dk, B=wl.phys["B"] - h * dB)
        op, _, _ = oracle_case(ora, wl.spec, phys_p, surf_flux=2, law=law)
        om, _, _ = oracle_case(ora, wl.spec, phys_m, surf_flux=2, law=law)
        fd = (op.time_derivative(U) - om.time_derivative(U)) / (2 * h)
        assert np.abs(Jd).max() > 0
        assert np.abs(fd - Jd).max() <= 1e-6 * np.abs(Jd).max()


def test_jvp_wall_model_state(ora):
    wl, o, X, U = _small_channel(ora)
    d = I.random_direction(U.shape, seed=9) * np.abs(U)
    Ut, Jd = o.jvp(U, d)
    h = 1e-6
    fd = (o.time_derivative(U + h * d) - o.time_derivative(U - h * d)) / (2 * h)
    assert np.abs(fd - Jd).max() <= 1e-6 * np.abs(Jd).max()


def test_rollout_loss_derivative(ora):
    wl, o, X, U = _small_channel(ora)
    dt = 0.5 * o.dt(U, 0.9)
    nsteps = 3
    L0, dL = o.rollout_jvp(U, None, 1.0, 0.0, nsteps, dt)
    h = 1e-6
    op, _, _ = oracle_case(ora, wl.spec, dict(wl.phys, kappa=wl.phys["kappa"] + h), surf_flux=2)
    om, _, _ = oracle_case(ora, wl.spec, dict(wl.phys, kappa=wl.phys["kappa"] - h), surf_flux=2)
    Lp = op.wall_shear(op.rk_steps(U, dt, nsteps))
    Lm = om.wall_shear(om.rk_steps(U, dt, nsteps))
    assert abs(L0 - o.wall_shear(o.rk_steps(U, dt, nsteps))) <= 1e-14 * abs(L0)
    assert abs((Lp - Lm) / (2 * h) - dL) <= 1e-6 * abs(dL)


def test_lserk4_temporal_order(ora):
    wl = I.workload("tgv_n3_4", elems=(2, 2, 2))
    phys = I.phys_params(Ma=0.3, Re=400.0)
    o, X, nbr = oracle_case(ora, wl.spec, phys, surf_flux=1)
    U0 = I.perturb(I.taylor_green(X, phys))
    dt0 = o.dt(U0, 0.9)
    T = 8 * dt0
    sols = [o.rk_steps(U0, T / m, m) for m in (8, 16, 32, 64)]
    e = [np.abs(sols[i] - sols[i + 1]).max() for i in range(3)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert rates[-1] > 3.7, (e, rates)


def test_jvp_inflow_outflow_and_isothermal(ora):
    """The forward-mode derivative through the inflow and outflow exterior
    states and through an isothermal wall's heat flux (the GPU adjoint's
    source at those faces) against central differences."""
    phys = I.phys_params(Ma=0.3, Re=400.0)
    g, p0 = phys["gamma"], phys["p0"]
    rho, u, v = 1.02, 0.75, 0.05
    phys.update(U_in=np.array([rho, rho * u, rho * v, 0.0, 1.03 * p0 / (g - 1) + 0.5 * rho * (u * u + v * v)]),
                p_out=0.98 * p0)
    spec = I.BoxSpec(3, 3, 2, 2, geometry="sine", amplitude=0.2, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    o, X, nbr = oracle_case(ora, spec, phys, vol_flux=2, surf_flux=2)
    U = I.perturb(I.taylor_green(X, phys), rel=1e-2)
    U[1] += 0.6 * U[0]
    d = I.random_direction(U.shape, seed=11) * np.abs(U)
    Ut, Jd = o.jvp(U, d)
    h = 1e-6
    fd = (o.time_derivative(U + h * d) - o.time_derivative(U - h * d)) / (2 * h)
    assert np.abs(fd - Jd).max() <= 1e-6 * np.abs(Jd).max()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    phys = dict(wl.phys, T_wall=1.15 * wl.phys["p0"] / wl.phys["R"])
    o, X, nbr = oracle_case(ora, wl.spec, phys, surf_flux=2)
    U = I.initial_state(wl, X)
    d = I.random_direction(U.shape, seed=12) * np.abs(U)
    Ut, Jd = o.jvp(U, d)
    fd = (o.time_derivative(U + h * d) - o.time_derivative(U - h * d)) / (2 * h)
    assert np.abs(fd - Jd).max() <= 1e-6 * np.abs(Jd).max()
    _, Jk = o.jvp(U, None, 1.0, 0.0)
    op, _, _ = oracle_case(ora, wl.spec, dict(phys, kappa=phys["kappa"] + h), surf_flux=2)
    om, _, _ = oracle_case(ora, wl.spec, dict(phys, kappa=phys["kappa"] - h), surf_flux=2)
    fd = (op.time_derivative(U) - om.time_derivative(U)) / (2 * h)
    assert np.abs(fd - Jk).max() <= 1e-6 * np.abs(Jk).max()
