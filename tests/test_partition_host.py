"""Host logic of the partitioned meshes (paper Sec. 2.1: space-filling-curve
subdomains): the partition, the local meshes and the pairing of their halo
faces.  The library's host functions run without a GPU."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, halo, inputs as I


def _mesh(N=2, e=(4, 3, 5), periodic=(True, True, True), geometry="affine", boundary=None):
    kw = {} if boundary is None else {"boundary": boundary}
    spec = I.BoxSpec(N, *e, geometry=geometry, amplitude=0.2 if geometry == "sine" else 0.0,
                     periodic=periodic, **kw)
    x, w = dg.lgl_nodes(N)
    return spec, I.node_coordinates(spec, x), I.connectivity(spec)


FACE_NODE = {
    0: lambda n, a, b: n * (a + n * b),
    1: lambda n, a, b: (n - 1) + n * (a + n * b),
    2: lambda n, a, b: a + n * n * b,
    3: lambda n, a, b: a + n * ((n - 1) + n * b),
    4: lambda n, a, b: a + n * b,
    5: lambda n, a, b: a + n * (b + n * (n - 1)),
}


@pytest.mark.parametrize("P", [1, 2, 3, 7, 60])
def test_partition_sizes_and_determinism(P):
    spec, X, nbr = _mesh()
    part = dg.partition_sfc(spec.N, X, P)
    counts = np.bincount(part, minlength=P)
    assert counts.sum() == spec.K and counts.min() >= spec.K // P and counts.max() <= -(-spec.K // P)
    assert np.array_equal(part, dg.partition_sfc(spec.N, X, P))


def test_partition_is_compact():
    # along the Morton curve 8 parts of an 8^3 box are its octants: 768 cut
    # element faces (counted from both sides), fewer than the 1024 of eight
    # slabs and far fewer than a random assignment
    spec, X, nbr = _mesh(e=(8, 8, 8))
    P = 8
    part = dg.partition_sfc(spec.N, X, P)
    cut = lambda p: sum(1 for e in range(spec.K) for l in range(6) if nbr[e, l] >= 0 and p[nbr[e, l]] != p[e])
    assert cut(part) == 768
    rng = np.random.default_rng(3)
    assert cut(part) < 0.35 * cut(rng.permutation(np.arange(spec.K) % P))


@pytest.mark.parametrize("P", [2, 3, 5])
@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, False)])
def test_local_meshes_and_halo_pairing(P, periodic):
    spec, X, nbr = _mesh(periodic=periodic)
    part = dg.partition_sfc(spec.N, X, P)
    locs = [dg.partition_local(nbr, part, r) for r in range(P)]
    # every element on exactly one rank, in ascending global order
    allg = np.concatenate([loc[0] for loc in locs])
    assert np.array_equal(np.sort(allg), np.arange(spec.K))
    for r, (l2g, nbl, _, _, hl) in enumerate(locs):
        assert np.all(np.diff(l2g) > 0) and np.all(part[l2g] == r)
        g2l = {g: i for i, g in enumerate(l2g)}
        for i, g in enumerate(l2g):
            for l in range(6):
                gn = nbr[g, l]
                if gn < 0:
                    assert nbl[i, l] == gn
                elif part[gn] == r:
                    assert nbl[i, l] == g2l[gn]
                else:
                    h = dg.DG_BC_HALO_BASE - nbl[i, l]
                    assert tuple(hl[h]) == (part[gn], i, l, l % 2)
        # the blocks shared with a peer line up face by face
        for q, (a, b) in halo.peer_blocks(hl).items():
            l2q, _, _, _, hq = locs[q]
            qa, qb = halo.peer_blocks(hq)[r]
            assert b - a == qb - qa
            for k in range(b - a):
                _, e, l, m = hl[a + k]
                _, eq, lq, mq = hq[qa + k]
                assert lq == l ^ 1 and m + mq == 1
                assert nbr[l2g[e], l] == l2q[eq]


def test_halo_codes_are_negative_and_distinct():
    spec, X, nbr = _mesh()
    part = dg.partition_sfc(spec.N, X, 4)
    l2g, nbl, _, _, hl = dg.partition_local(nbr, part, 1)
    codes = nbl[nbl <= dg.DG_BC_HALO_BASE]
    assert len(codes) == len(hl) and len(set(codes.tolist())) == len(codes)
