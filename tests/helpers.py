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


# ---------------------------------------------------------------------------
# General conforming meshes: elements whose local frames are rotated against
# the structured box, and their connectivity (neighbour element, neighbour
# face, orientation code) found by matching face nodes geometrically.
# ---------------------------------------------------------------------------
def proper_rotations():
    """The 24 proper rotations of the index cube as (perm, flips): new local
    axis d runs along old axis perm[d], reversed where flips[d]."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        sgn = np.linalg.det(np.eye(3)[list(perm)])
        for flips in itertools.product((0, 1), repeat=3):
            if sgn * (-1) ** sum(flips) > 0:
                out.append((perm, flips))
    return out


def rotate_elements(X, N, rots):
    """X[V][K][n^3] (coordinates, or any nodal field) with element e's nodes
    renumbered by rots[e] (None: kept)."""
    n = N + 1
    V, K = X.shape[0], X.shape[1]
    Xn = X.reshape(V, K, n, n, n).copy()  # [c][e][k][j][i]
    r = np.arange(n)
    for e, rot in enumerate(rots):
        if rot is None:
            continue
        perm, flips = rot
        new = np.empty((V, n, n, n))
        for kk in range(n):
            for jj in range(n):
                for ii in range(n):
                    rn = (ii, jj, kk)
                    old = [0, 0, 0]
                    for d in range(3):
                        old[perm[d]] = N - rn[d] if flips[d] else rn[d]
                    new[:, kk, jj, ii] = Xn[:, e, old[2], old[1], old[0]]
        Xn[:, e] = new
    return np.ascontiguousarray(Xn.reshape(V, K, n ** 3))


def face_node_indices(N, l):
    """Volume node index of face-local node (a, b) of local face l, as [b][a]."""
    n = N + 1
    idx = np.empty((n, n), dtype=np.int64)
    for b in range(n):
        for a in range(n):
            i, j, k = [(0, a, b), (N, a, b), (a, 0, b), (a, N, b), (a, b, 0), (a, b, N)][l]
            idx[b, a] = i + n * (j + n * k)
    return idx


def orient_map(o, N, a, b):
    s, t = (b, a) if o & 1 else (a, b)
    return (N - s if o & 2 else s), (N - t if o & 4 else t)


def conforming_connectivity(X, N, lengths, periodic, boundary=-1, tol=1e-9):
    """(nbr, nbr_face, orient) [K, 6] of a conforming hexahedral mesh, from
    coincidence of face nodes up to a periodic translation; unmatched faces
    get the boundary code."""
    n = N + 1
    K = X.shape[1]
    Xe = X.reshape(3, K, n ** 3)
    L = np.array(lengths, dtype=float)
    faces = {}
    cent = {}
    for e in range(K):
        for l in range(6):
            pts = Xe[:, e, face_node_indices(N, l).reshape(-1)]  # [3][n^2]
            c = pts.mean(axis=1)
            for d in range(3):
                if periodic[d]:
                    c[d] = c[d] % L[d]
                    if abs(c[d] - L[d]) < 1e-7:
                        c[d] = 0.0
            key = tuple(np.round(c, 6))
            faces.setdefault(key, []).append((e, l))
            cent[(e, l)] = pts
    nbr = np.full((K, 6), boundary, dtype=np.int32)
    nface = np.zeros((K, 6), dtype=np.int32)
    orient = np.zeros((K, 6), dtype=np.int32)
    for key, lst in faces.items():
        if len(lst) == 1:
            continue
        assert len(lst) == 2, (key, lst)
        (e, l), (e2, l2) = lst
        A = cent[(e, l)].reshape(3, n, n)   # [c][b][a]
        B = cent[(e2, l2)].reshape(3, n, n)
        found = None
        for o in range(8):
            ok = True
            shift = None
            for b in range(n):
                for a in range(n):
                    a2, b2 = orient_map(o, N, a, b)
                    dvec = B[:, b2, a2] - A[:, b, a]
                    if shift is None:
                        shift = dvec
                    elif np.abs(dvec - shift).max() > tol * max(1.0, L.max()):
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                found = o
                break
        assert found is not None, (e, l, e2, l2)
        inv = (1 | (((found >> 2) & 1) << 1) | (((found >> 1) & 1) << 2)) if found & 1 else found
        nbr[e, l], nface[e, l], orient[e, l] = e2, l2, found
        nbr[e2, l2], nface[e2, l2], orient[e2, l2] = e, l, inv
    return nbr, nface, orient


def rotated_mesh(spec, x, seed=3, frac=0.5):
    """The structured mesh of spec with a seeded random half of its elements'
    local frames rotated: (X, nbr, nbr_face, orient, rots)."""
    X0 = I.node_coordinates(spec, x)
    K = spec.K
    rng = np.random.default_rng(seed)
    rot_all = proper_rotations()
    rots = [rot_all[rng.integers(1, len(rot_all))] if rng.random() < frac else None for _ in range(K)]
    X = rotate_elements(X0, spec.N, rots)
    nbr, nface, orient = conforming_connectivity(X, spec.N, spec.lengths, spec.periodic)
    return X, nbr, nface, orient, rots


def unrotate_field(F, N, rots):
    """A nodal field [v][K][n^3] on the rotated mesh renumbered back to the
    structured elements' node order."""
    n = N + 1
    V, K = F.shape[0], F.shape[1]
    Fn = F.reshape(V, K, n, n, n)
    out = Fn.copy()
    for e, rot in enumerate(rots):
        if rot is None:
            continue
        perm, flips = rot
        for kk in range(n):
            for jj in range(n):
                for ii in range(n):
                    rn = (ii, jj, kk)
                    old = [0, 0, 0]
                    for d in range(3):
                        old[perm[d]] = N - rn[d] if flips[d] else rn[d]
                    out[:, e, old[2], old[1], old[0]] = Fn[:, e, kk, jj, ii]
    return out.reshape(V, K, n ** 3)
