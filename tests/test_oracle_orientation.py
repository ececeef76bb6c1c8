"""Pins of the oracle on general conforming meshes (neighbour face and
orientation code per element face): a periodic box whose elements have
randomly rotated local frames (every proper rotation of the index cube
occurs), with the connectivity found by matching face nodes geometrically.

* The operator does not depend on the elements' local frames: Ut on the
  rotated mesh, renumbered back, equals Ut on the structured mesh (same
  nodes, same state) to roundoff.  A face paired with the wrong neighbour
  face, a node order read without its orientation, or a normal taken from the
  wrong side breaks this at O(1).
* Free-stream preservation and discrete conservation hold on it.
* The wall model's column search crosses rotated elements (channel).
* Inconsistent connectivity is rejected."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from helpers import oracle_case, quad_weights, rotate_elements, rotated_mesh, unrotate_field


def _rel(a, b):
    a = a.reshape(5, -1); b = b.reshape(5, -1)
    return max(float(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max()) for v in range(5))


@pytest.mark.parametrize("N,surf,visc", [(3, 2, 1), (4, 1, 0), (2, 0, 1)])
def test_rotated_frames_give_the_structured_operator(ora, N, surf, visc):
    phys = I.phys_params(Ma=0.3, Re=800.0)
    spec = I.BoxSpec(N, 3, 3, 3, geometry="sine", amplitude=0.2)
    x, w, D = ora.lgl(N)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x)
    assert (ori != 0).sum() > 20 and (nf != (np.arange(6)[None, :] ^ 1)).sum() > 20
    o = ora.Oracle(N, X, nbr, phys, surf_flux=surf, viscous=visc, nbr_face=nf, orient=ori, extended=True)
    o0, X0, nbr0 = oracle_case(ora, spec, phys, surf_flux=surf, viscous=visc)
    o0 = ora.Oracle(N, X0, nbr0, phys, surf_flux=surf, viscous=visc, extended=True)
    U0 = I.perturb(I.taylor_green(X0, phys), rel=1e-2)
    Ut = o.time_derivative(rotate_elements(U0, N, rots))
    e = _rel(unrotate_field(Ut, N, rots), o0.time_derivative(U0))
    print("rotated vs structured", e)
    assert e <= 1e-13


def test_free_stream_and_conservation_on_rotated_mesh(ora):
    phys = I.phys_params(Ma=0.3, Re=800.0)
    spec = I.BoxSpec(3, 3, 3, 3, geometry="sine", amplitude=0.2)
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=5)
    o = ora.Oracle(3, X, nbr, phys, surf_flux=2, nbr_face=nf, orient=ori, extended=True)
    Uf = I.free_stream(X, phys)
    assert np.abs(o.time_derivative(Uf)).max() * (2 * np.pi / 3) / phys["p0"] <= 1e-13
    U = I.perturb(I.taylor_green(X, phys), rel=5e-2)
    Ut = o.time_derivative(U).reshape(5, o.K, o.n3)
    wJ = quad_weights(ora, o)
    for v in range(5):
        assert abs((wJ * Ut[v]).sum()) <= 1e-13 * (wJ * np.abs(Ut[v])).sum()


@pytest.mark.parametrize("law", [1, 0])
def test_wall_model_across_rotated_elements(ora, law):
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(wl.spec, x, seed=8, frac=0.6)
    o = ora.Oracle(3, X, nbr, wl.phys, surf_flux=2, law=law, nbr_face=nf, orient=ori, extended=True)
    X0 = I.node_coordinates(wl.spec, x)
    o0 = ora.Oracle(3, X0, I.connectivity(wl.spec), wl.phys, surf_flux=2, law=law, extended=True)
    U0 = I.channel_profile(X0, wl.phys)
    Ut = o.time_derivative(rotate_elements(U0, 3, rots))
    e = _rel(unrotate_field(Ut, 3, rots), o0.time_derivative(U0))
    print("channel rotated vs structured", e)
    assert e <= 1e-12


def test_inconsistent_connectivity_is_rejected(ora):
    phys = I.phys_params()
    spec = I.BoxSpec(2, 2, 2, 2, geometry="sine", amplitude=0.1)
    x, w, D = ora.lgl(2)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=2)
    ora.Oracle(2, X, nbr, phys, nbr_face=nf, orient=ori)  # consistent: accepted
    e, l = np.argwhere(nbr >= 0)[0]
    bad = ori.copy(); bad[e, l] ^= 2                     # the neighbour no longer lists the inverse
    with pytest.raises(ValueError):
        ora.Oracle(2, X, nbr, phys, nbr_face=nf, orient=bad)
    bad = ori.copy(); e2, l2 = nbr[e, l], nf[e, l]
    bad[e, l] ^= 6; bad[e2, l2] = ((1 | (((bad[e, l] >> 2) & 1) << 1) | (((bad[e, l] >> 1) & 1) << 2))
                                   if bad[e, l] & 1 else bad[e, l])  # reciprocal but the nodes do not meet
    with pytest.raises(ValueError):
        ora.Oracle(2, X, nbr, phys, nbr_face=nf, orient=bad)
