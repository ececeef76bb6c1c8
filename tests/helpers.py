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


OUTFLOW = -3


def submesh(nbr, sel, rings=2):
    """Elements of sel and `rings` rings of face neighbours: (global ids,
    local connectivity with the faces leaving the set marked as outflow
    boundaries, local ids of sel in the order of sel)."""
    keep = set(int(e) for e in sel)
    front = set(keep)
    for _ in range(rings):
        nxt = set()
        for e in front:
            for q in nbr[e]:
                if q >= 0 and int(q) not in keep:
                    nxt.add(int(q))
        keep |= nxt
        front = nxt
    ids = np.array(sorted(keep), dtype=np.int64)
    g2l = {int(e): k for k, e in enumerate(ids)}
    loc = np.array([[g2l.get(int(q), OUTFLOW) if q >= 0 else int(q) for q in nbr[e]] for e in ids],
                   dtype=np.int32)
    return ids, loc, np.array([g2l[int(e)] for e in sel], dtype=np.int32)


class SampledOracle:
    """The oracle's time derivative on sampled elements of a mesh too large to
    evaluate whole.  The oracle runs on the sub-mesh of the samples and the two
    rings of face neighbours their time derivative depends on (lifted
    gradients of ring 1, primitives of ring 2), with its subset evaluation
    restricted to the samples; faces leaving the sub-mesh become outflow
    boundaries, which only ring 2 touches (its lifting and time derivative are
    not evaluated).  Periodic meshes without walls only."""

    def __init__(self, ora, N, X, nbr, phys, sel, extended=True, **opts):
        self.n3 = (N + 1) ** 3
        self.K = X.size // (3 * self.n3)
        self.ids, loc, self.lsel = submesh(nbr, sel)
        Xs = np.ascontiguousarray(X.reshape(3, self.K, -1)[:, self.ids])
        self.o = ora.Oracle(N, Xs, loc, phys, extended=extended, subset=self.lsel, **opts)

    def time_derivative_on_sample(self, U):
        """Ut of the sampled elements, [5][len(sel)][n^3]."""
        Us = np.ascontiguousarray(U.reshape(5, self.K, -1)[:, self.ids])
        return self.o.time_derivative(Us)[:, self.lsel]


def bump_wall(X, A=0.15):
    """Bottom wall y = A s(x) s(z), s(t) = sin^2(t - pi/2) on pi/2 < t < 3 pi/2
    and 0 elsewhere (continuous with its slope; the mesh lines x, z = pi/2,
    3 pi/2 bound the curved part), blended linearly to the flat top wall
    y = 2.  A sample point is located in the mesh as it is, without periodic
    images, so the elements at the periodic boundaries are kept affine (their
    discrete normals are exactly +-y and no sample leaves through them)."""
    x, y, z = X

    def s(t):
        return np.where((t > np.pi / 2) & (t < 1.5 * np.pi), np.sin(t - np.pi / 2) ** 2, 0.0)

    return np.ascontiguousarray(np.stack([x, y + A * s(x) * s(z) * (1 - y / 2), z]))
