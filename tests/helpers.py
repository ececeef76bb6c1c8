"""Small shared helpers for the tests (no method arithmetic)."""
import numpy as np

from paper_2606_18927_gb300 import inputs as I


def oracle_case(ora, spec, phys, vol_flux=0, surf_flux=1, viscous=1, law=1):
    """Mesh nodes from the oracle's own LGL nodes, plus the oracle instance."""
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, vol_flux=vol_flux, surf_flux=surf_flux, viscous=viscous, law=law)
    return o, X, nbr


def quad_weights(ora, o):
    """w_i w_j w_k J per node, shape [K, n^3]."""
    x, w, D = ora.lgl(o.N)
    n = o.n
    wi = np.tile(w, n * n)
    wj = np.tile(np.repeat(w, n), n)
    wk = np.repeat(w, n * n)
    Ja, J = o.metrics()
    return (wi * wj * wk)[None, :] * J


def rel_max_err(a, b):
    """max over variables of max|a_v - b_v| / max|b_v| (the parity norm)."""
    a = a.reshape(5, -1); b = b.reshape(5, -1)
    return float(max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5)))
