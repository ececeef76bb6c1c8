"""Pins of the oracle's wall-model sampling points (reading of Sec. 3.1-3.2:
the model samples the solution at distance h_wm from the wall; located on
the element maps at set-up).

For every wall-face node x_w the oracle stores a sample element and reference
coordinates, and the Lagrange weights of those coordinates.  Checked here
with the test's own evaluation of the degree-N element maps:
* the stored point maps to x_w - h_wm n_out, h_wm from the wall along the
  inward normal.  On the channel the walls are the planes y = 0 and y = 2
  (the warp vanishes there), so the inward normal is +-y exactly, independent
  of the oracle's metrics; on a curved wall the normal is the unit vector of
  the oracle's metric row at the node, which must point into the element and
  agree in direction with the cross product of the face's tangent vectors
  (to the mapping's truncation error);
* the reference coordinates lie in [-1, 1] (to 1e-8), and the element is
  the first of the wall element's column that contains the point (the wall
  element, then its neighbours away from the wall), else the lowest-index
  element that does (checked by the test's own Newton on the element maps);
* the stored weights reproduce every polynomial of degree N at the sample
  (Lagrange interpolation is exact there), and the mapped point itself.
A sample taken along +n, at the wall node, or with wrong weights fails."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import bump_wall

WALL = -1


def _lagrange(xi, r):
    """Lagrange basis of the nodes xi at r (product form)."""
    n = len(xi)
    out = np.ones(n)
    for i in range(n):
        for m in range(n):
            if m != i:
                out[i] *= (r - xi[m]) / (xi[i] - xi[m])
    return out


def _dlagrange(xi, r):
    """Derivatives of the Lagrange basis of the nodes xi at r."""
    n = len(xi)
    out = np.zeros(n)
    for i in range(n):
        for q in range(n):
            if q == i:
                continue
            t = 1.0 / (xi[i] - xi[q])
            for m in range(n):
                if m != i and m != q:
                    t *= (r - xi[m]) / (xi[i] - xi[m])
            out[i] += t
    return out


def _locate(X, e, xi, xs):
    """Reference coordinates of xs in element e (Newton on the test's own
    evaluation of the element map), or None if Newton fails."""
    n = len(xi)
    Xe = np.stack([X[c].reshape(-1, n, n, n)[e] for c in range(3)])  # [c][k][j][i]
    r = np.zeros(3)
    for _ in range(60):
        L = [_lagrange(xi, r[d]) for d in range(3)]
        dL = [_dlagrange(xi, r[d]) for d in range(3)]
        x = np.einsum("ckji,k,j,i->c", Xe, L[2], L[1], L[0])
        Jm = np.stack([np.einsum("ckji,k,j,i->c", Xe, L[2], L[1], dL[0]),
                       np.einsum("ckji,k,j,i->c", Xe, L[2], dL[1], L[0]),
                       np.einsum("ckji,k,j,i->c", Xe, dL[2], L[1], L[0])], axis=1)
        dr = np.linalg.solve(Jm, xs - x)
        r = np.clip(r + dr, -3.0, 3.0)
        if np.abs(dr).max() < 1e-15:
            break
    return r


def _contains(X, e, xi, xs):
    return np.abs(_locate(X, e, xi, xs)).max() <= 1.0 + 1e-8


def _face_node(N, l, a, b):
    n = N + 1
    i, j, k = [(0, a, b), (N, a, b), (a, 0, b), (a, N, b), (a, b, 0), (a, b, N)][l]
    return i + n * (j + n * k)


def _wall_nodes(nbr, N):
    """(element, face, a, b) of every wall slot, in the oracle's slot order
    (elements ascending, faces ascending, b outer, a inner)."""
    n = N + 1
    out = []
    for e in range(len(nbr)):
        for l in range(6):
            if nbr[e][l] == WALL:
                for b in range(n):
                    for a in range(n):
                        out.append((e, l, a, b))
    return out


def _map(X, e, xi, ref):
    n = len(xi)
    L = [_lagrange(xi, ref[d]) for d in range(3)]
    w = np.einsum("k,j,i->kji", L[2], L[1], L[0]).reshape(-1)
    return np.array([float((X[c].reshape(-1, n ** 3)[e] * w).sum()) for c in range(3)])


def _column(nbr, e, l, layers=4):
    col = [e]
    c = e
    for _ in range(layers - 1):
        c = nbr[c][l ^ 1]
        if c < 0:
            break
        col.append(int(c))
    return col


def _check(ora, spec, phys, flat_walls, deform=None):
    x0, w0, D0 = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x0)
    if deform is not None:
        X = deform(X)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, surf_flux=2)
    N = spec.N
    n = N + 1
    xi, w, D = ora.lgl(N)
    el, ref = o.wall_samples()
    lw = o.wall_weights()
    nodes = _wall_nodes(nbr, N)
    assert len(nodes) == len(el) > 0
    Ja, J = o.metrics()
    hwm = phys["hwm"]
    rng = np.random.default_rng(5)
    coef = rng.uniform(-1, 1, size=(n, n, n))  # a polynomial of degree N per direction
    for s, (e, l, a, b) in enumerate(nodes):
        p = _face_node(N, l, a, b)
        xw = np.array([X[c].reshape(-1, n ** 3)[e, p] for c in range(3)])
        xs = _map(X, el[s], xi, ref[s])
        d = xs - xw
        assert abs(np.linalg.norm(d) - hwm) <= 1e-12
        if flat_walls or xw[1] > 1.0:  # (the bump's top wall is flat too)
            inward = np.array([0.0, 1.0 if xw[1] < 1.0 else -1.0, 0.0])
        else:
            row = Ja[e, p, l // 2]
            nout = (1.0 if l & 1 else -1.0) * row / np.linalg.norm(row)
            inward = -nout
            # independent direction: tangents of the polynomial face map
            node_ijk = [p % n, (p // n) % n, p // (n * n)]
            dirs = [dd for dd in range(3) if dd != l // 2]
            tang = []
            for dd in dirs:
                t = np.zeros(3)
                for m in range(n):
                    q = list(node_ijk); q[dd] = m
                    qi = q[0] + n * (q[1] + n * q[2])
                    t += D[node_ijk[dd], m] * np.array([X[c].reshape(-1, n ** 3)[e, qi] for c in range(3)])
                tang.append(t)
            cr = np.cross(tang[0], tang[1])
            cr /= np.linalg.norm(cr)
            # the curl-form metric and the cross product of the interpolated
            # tangents differ at the mapping's truncation error (a few per
            # cent at N = 3 where the bump starts): a direction check
            assert abs(float(cr @ inward)) >= 0.98
            centre = np.array([X[c].reshape(-1, n ** 3)[e].mean() for c in range(3)])
            assert float(inward @ (centre - xw)) > 0.0
        assert np.abs(d - hwm * inward).max() <= 1e-12
        assert np.abs(ref[s]).max() <= 1.0 + 1e-8
        # the element rule: the first element of the wall element's column
        # that contains the point, else the lowest-index one that does
        col = _column(nbr, e, l)
        first = next((c for c in col if _contains(X, c, xi, xw + hwm * inward)), None)
        if first is not None:
            assert el[s] == first
        else:
            assert not any(_contains(X, c, xi, xw + hwm * inward) for c in range(el[s]))
        # stored weights: the test's own Lagrange basis at the same point,
        # exact reproduction of a degree-N polynomial, and the mapped point
        for dd in range(3):
            assert np.abs(lw[s, dd] - _lagrange(xi, ref[s][dd])).max() <= 1e-13
        Kg, Jg, Ig = np.meshgrid(xi, xi, xi, indexing="ij")
        poly_nodes = np.polynomial.polynomial.polyval3d(Ig, Jg, Kg, coef)  # [k][j][i]
        val = np.einsum("k,j,i,kji->", lw[s, 2], lw[s, 1], lw[s, 0], poly_nodes)
        exact = np.polynomial.polynomial.polyval3d(ref[s][0], ref[s][1], ref[s][2], coef)
        assert abs(val - exact) <= 1e-12 * max(1.0, abs(exact))
        xr = [np.einsum("k,j,i,kji->", lw[s, 2], lw[s, 1], lw[s, 0],
                        X[c].reshape(-1, n, n, n)[el[s]]) for c in range(3)]
        assert np.abs(np.array(xr) - xw - hwm * inward).max() <= 1e-12
    return el, nodes


@pytest.mark.parametrize("N", [3, 5])
def test_channel_wall_samples(ora, N):
    wl = I.workload("channel_n5", N=N, elems=(4, 4, 2))
    _check(ora, wl.spec, wl.phys, flat_walls=True)


@pytest.mark.parametrize("N", [3, 4])
def test_curved_wall_samples(ora, N):
    phys = I.phys_params(Ma=0.3, Re=800.0, hwm=0.3)
    spec = I.BoxSpec(N, 4, 3, 4, lengths=(2 * np.pi, 2.0, 2 * np.pi), periodic=(True, False, True))
    el, nodes = _check(ora, spec, phys, flat_walls=False, deform=bump_wall)
    # the tilted normals carry some samples out of their wall element
    moved = sum(1 for s, (e, l, a, b) in enumerate(nodes) if el[s] != e)
    print("samples outside their wall element:", moved, "of", len(nodes))
    assert moved > 0
