"""The oracle's BR1 lifting and viscous divergence against a closed form
(paper Sec. 2.2: the viscous fluxes of the DGSEM from the BR1-lifted
gradients, with the arithmetic-mean interface states W* = (W- + W+) / 2).

A periodic box of two elements along x (one along y and z, each its own
neighbour there) holds a state at rest with unit density and a temperature
that is constant in each element, T_A and T_B.  In element A the lifted
temperature gradient vanishes except at its two x faces, where BR1's surface
correction (T* - T_A) n_x (2 / h) / w_0 gives -g at the left face and +g at
the right one, g = (T_B - T_A) / (h w_0) (h the element length, w_0 the
end-point LGL weight).  The viscous energy flux k dT/dx then has equal values
on both sides of each face, so the surface term of the divergence vanishes
and only the volume derivative of the flux remains:

    Ut_E(i) = (2 / h) k sum_m D_im G_m = 2 k (T_B - T_A) (D_iN - D_i0) / (h^2 w_0).

At rest the inviscid energy flux is zero (central surface flux).  A wrong
interface average, surface weight, sign or viscous face average changes the
result at O(1)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import oracle_case


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_br1_piecewise_constant_temperature(ora, N):
    phys = I.phys_params(Ma=0.3, Re=50.0)
    Lx = 3.0
    spec = I.BoxSpec(N, 2, 1, 1, lengths=(Lx, 1.0, 1.5))
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=0, viscous=1)
    n = N + 1
    T = {0: 1.3, 1: 0.8}
    shape = X[0].shape  # [K, n^3]
    Tn = np.stack([np.full(shape[1], T[e]) for e in range(2)])
    U = I.conservative(np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape), phys["R"] * Tn,
                       phys["gamma"])
    Ut = o.time_derivative(U).reshape(5, 2, n, n, n)  # [v][e][k][j][i]
    x, w, D = ora.lgl(N)
    h = Lx / 2
    cp = phys["gamma"] * phys["R"] / (phys["gamma"] - 1.0)
    kc = phys["mu"] * cp / phys["Pr"]
    for e, other in ((0, 1), (1, 0)):
        ref = 2.0 * kc * (T[other] - T[e]) * (D[:, N] - D[:, 0]) / (h * h * w[0])
        got = Ut[4, e]
        assert np.allclose(got, np.broadcast_to(ref, got.shape), rtol=1e-12, atol=1e-12 * np.abs(ref).max()), \
            (e, got[0, 0], ref)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_br1_piecewise_constant_shear(ora, N):
    """The same box with uniform density and pressure, at rest along x and
    with a tangential velocity v constant in each element (v_A, v_B): the
    lifted dv/dx is the surface correction alone (-g, +g at the two x faces
    of element A, g = (v_B - v_A) / (h w_0)), so tau_xy = mu dv/dx, the
    divergence of u vanishes and the inviscid fluxes are constant.  In
    element A
      Ut_{rho v}(i) = (2 / h) mu g (D_iN - D_i0),
      Ut_E(i) = (2 / h) mu g [v_A (D_iN - D_i0) + (v_B - v_A)(d_iN + d_i0) / (2 w_0)],
    the last term from the viscous work v tau_xy, whose face average differs
    from each side's value by mu g (v_B - v_A) / 2."""
    phys = I.phys_params(Ma=0.3, Re=50.0)
    Lx = 2.5
    spec = I.BoxSpec(N, 2, 1, 1, lengths=(Lx, 1.2, 0.9))
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=0, viscous=1)
    n = N + 1
    V = {0: 0.4, 1: -0.3}
    shape = X[0].shape
    vn = np.stack([np.full(shape[1], V[e]) for e in range(2)])
    U = I.conservative(np.ones(shape), np.zeros(shape), vn, np.zeros(shape), np.ones(shape), phys["gamma"])
    Ut = o.time_derivative(U).reshape(5, 2, n, n, n)
    x, w, D = ora.lgl(N)
    h = Lx / 2
    mu = phys["mu"]
    ends = np.zeros(n); ends[0] = ends[N] = 1.0
    for e, other in ((0, 1), (1, 0)):
        g = (V[other] - V[e]) / (h * w[0])
        ref_m = 2.0 / h * mu * g * (D[:, N] - D[:, 0])
        ref_e = 2.0 / h * mu * g * (V[e] * (D[:, N] - D[:, 0]) + (V[other] - V[e]) * ends / (2 * w[0]))
        # (the uniform pressure's inviscid fluxes cancel to rounding, which
        # the derivative amplifies: about 1e-12 of the viscous terms here)
        for row, ref in ((2, ref_m), (4, ref_e)):
            got = Ut[row, e]
            assert np.allclose(got, np.broadcast_to(ref, got.shape), rtol=1e-10,
                               atol=1e-10 * np.abs(ref).max()), (e, row, got[0, 0], ref)
        for row in (0, 1, 3):
            assert np.abs(Ut[row, e]).max() <= 1e-10 * np.abs(ref_m).max(), (e, row)
