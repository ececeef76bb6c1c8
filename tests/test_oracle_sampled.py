"""The sampled oracle of the full-size parity tests: the oracle on the
sub-mesh of some elements and their two rings of face neighbours gives
bitwise the time derivative that the oracle on the whole mesh gives on those
elements (the result depends only on the element, its neighbours and their
neighbours, and on nothing of the element numbering)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import SampledOracle, oracle_case


@pytest.mark.parametrize("surf,viscous", [(2, 1), (1, 0)])
def test_sampled_oracle_equals_whole_mesh(ora, surf, viscous):
    phys = I.phys_params(Ma=0.3, Re=800.0)
    spec = I.BoxSpec(3, 5, 4, 6, geometry="sine", amplitude=0.2)
    o, X, nbr = oracle_case(ora, spec, phys, surf_flux=surf, viscous=viscous)
    U = I.perturb(I.taylor_green(X, phys), rel=1e-2)
    sel = np.array([0, 7, 33, 119], dtype=np.int64)
    ref = o.time_derivative(U)[:, sel]
    so = SampledOracle(ora, spec.N, X, nbr, phys, sel, extended=False, surf_flux=surf, viscous=viscous)
    assert len(so.ids) < spec.K
    got = so.time_derivative_on_sample(U)
    assert np.array_equal(got, ref)
