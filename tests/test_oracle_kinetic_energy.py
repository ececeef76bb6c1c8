"""Pin of the oracle's kinetic-energy diagnostic (the Taylor-Green quantity
KE = (1/|Omega|) sum_nodes w_i w_j w_k J rho |u|^2 / 2).

The unperturbed Taylor-Green state (rho = 1, u = sin x cos y cos z,
v = -cos x sin y cos z, w = 0) has the exact mean kinetic energy 1/8 on
[0, 2 pi]^3.  On affine meshes of 4 elements per direction the composite
Gauss-Lobatto quadrature integrates it exactly for every N >= 2 (the element
boundaries at multiples of pi/2 make the quadrature errors of the cos 2x,
cos 2y, cos 2z terms cancel by symmetry); on the curved sine mesh it
converges to 1/8 at least at the quadrature's order 2N.  A missing factor
1/2, a missing Jacobian or a wrong normalisation by the volume fails."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import oracle_case


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_taylor_green_kinetic_energy_exact(ora, N):
    phys = I.phys_params()
    o, X, nbr = oracle_case(ora, I.BoxSpec(N, 4, 4, 4), phys)
    assert abs(o.kinetic_energy(I.taylor_green(X, phys)) - 0.125) <= 1e-13  # summation roundoff


@pytest.mark.parametrize("N", [2, 3, 4])
def test_taylor_green_kinetic_energy_converges_on_curved_mesh(ora, N):
    phys = I.phys_params()
    errs = []
    for ne in (2, 4, 8):
        o, X, nbr = oracle_case(ora, I.BoxSpec(N, ne, ne, ne, geometry="sine", amplitude=0.1), phys)
        errs.append(abs(o.kinetic_energy(I.taylor_green(X, phys)) - 0.125))
    rates = [math.log2(errs[i] / max(errs[i + 1], 1e-300)) for i in range(2)]
    print("N", N, errs, rates)
    assert errs[0] > 1e-6  # the coarse curved mesh is not exact
    assert errs[-1] <= 1e-8
    assert min(rates) >= 2 * N


def test_kinetic_energy_of_a_uniform_flow(ora):
    """rho = 2, u = (1, 0.5, 0.25) on a curved mesh: KE = rho |u|^2 / 2 exactly
    (the quadrature integrates a constant exactly; the weights w J sum to the
    volume)."""
    phys = I.phys_params()
    o, X, nbr = oracle_case(ora, I.BoxSpec(3, 3, 2, 2, geometry="sine", amplitude=0.2), phys)
    U = I.free_stream(X, phys, velocity=(1.0, 0.5, 0.25), rho=2.0)
    assert abs(o.kinetic_energy(U) - 2.0 * (1 + 0.25 + 0.0625) / 2) <= 1e-14
