"""Argument and mesh validation of dg_init_mesh (host side: it rejects a bad
mesh before touching the device, so these run without a GPU)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I

ARG, MESH = -1, -3


def _mesh(N=2, e=(2, 2, 2), **kw):
    spec = I.BoxSpec(N, *e, **kw)
    x, w = dg.lgl_nodes(N)
    return spec, I.node_coordinates(spec, x), I.connectivity(spec)


def _init(N, X, nbr, phys=None, **opts):
    with pytest.raises(dg.DGError) as ei:
        dg.Operator(N, X, nbr, phys or I.phys_params(), stream=0, **opts)
    return ei.value.code, str(ei.value)


def test_bad_degree_and_options():
    spec, X, nbr = _mesh()
    assert _init(9, X, nbr)[0] == ARG
    assert _init(spec.N, X, nbr, precision=7)[0] == ARG
    assert _init(spec.N, X, nbr, vol_flux=3)[0] == ARG
    assert _init(spec.N, X, nbr, surf_flux=5)[0] == ARG


def test_neighbour_out_of_range_and_not_reciprocal():
    spec, X, nbr = _mesh()
    bad = nbr.copy(); bad[0, 1] = spec.K + 3
    assert _init(spec.N, X, bad)[0] == MESH
    bad = nbr.copy(); bad[0, 1] = -7          # neither a boundary code nor a halo code
    assert _init(spec.N, X, bad)[0] == MESH
    bad = nbr.copy(); bad[0, 1], bad[0, 3] = bad[0, 3], bad[0, 1]
    code, msg = _init(spec.N, X, bad)
    assert code == MESH


def test_faces_that_do_not_match():
    spec, X, nbr = _mesh()
    Xb = X.copy()
    Xb[0, 1, :] += 0.05 * np.arange(Xb.shape[2])   # distort element 1 only
    assert _init(spec.N, Xb, nbr)[0] == MESH


def test_inverted_element():
    spec, X, nbr = _mesh(periodic=(False, False, False))
    Xb = X.copy()
    n = spec.N + 1
    # mirror element 0 in x: its Jacobian turns negative
    Xb[0, 0, :] = -Xb[0, 0, :]
    assert _init(spec.N, Xb, nbr)[0] == MESH


def test_wall_faces_need_a_sampling_distance():
    spec, X, nbr = _mesh(periodic=(True, False, True))
    phys = I.phys_params(); phys["hwm"] = 0.0
    assert _init(spec.N, X, nbr, phys)[0] == ARG


def test_sutherland_needs_a_reference_temperature():
    spec, X, nbr = _mesh()
    phys = I.phys_params(); phys.update(suth_S=0.4, T_ref=0.0)
    assert _init(spec.N, X, nbr, phys)[0] == ARG


def test_reference_density_must_not_be_negative():
    spec, X, nbr = _mesh()
    phys = I.phys_params(); phys["rho_ref"] = -1.0
    assert _init(spec.N, X, nbr, phys, precision=dg.FP32_MIXED)[0] == ARG


def test_inflow_and_outflow_states_must_be_physical():
    spec, X, nbr = _mesh(periodic=(False, True, True),
                         boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    phys = I.phys_params(); phys.update(U_in=np.array([-1.0, 0, 0, 0, 1.0]), p_out=1.0)
    assert _init(spec.N, X, nbr, phys)[0] == ARG
    phys.update(U_in=np.array([1.0, 0.5, 0, 0, 10.0]), p_out=0.0)
    assert _init(spec.N, X, nbr, phys)[0] == ARG


def test_halo_codes_must_be_dense():
    spec, X, nbr = _mesh(e=(4, 2, 2))
    part = dg.partition_sfc(spec.N, X, 2)
    l2g, nbl, _, _, hl = dg.partition_local(nbr, part, 0)
    Xl = X[:, l2g, :]
    bad = nbl.copy()
    bad[bad == dg.DG_BC_HALO_BASE] = dg.DG_BC_HALO_BASE - 1000   # halo index beyond n_halo
    assert _init(spec.N, Xl, bad)[0] == MESH


def test_face_orientation_must_be_consistent():
    """A neighbour face or orientation code that the neighbour does not list
    back, or under which the face nodes do not coincide, is rejected."""
    spec, X, nbr = _mesh()
    nf = np.tile(np.arange(6, dtype=np.int32) ^ 1, (spec.K, 1))
    ori = np.zeros((spec.K, 6), dtype=np.int32)
    bad = ori.copy(); bad[0, 1] = 9                   # not a code
    assert _init(spec.N, X, nbr, nbr_face=nf, orient=bad)[0] == MESH
    bad = ori.copy(); bad[0, 1] = 2                   # the neighbour lists 0
    assert _init(spec.N, X, nbr, nbr_face=nf, orient=bad)[0] == MESH
    bad = ori.copy(); bad[0, 1] = 2; bad[nbr[0, 1], 0] = 2   # reciprocal, nodes do not meet
    assert _init(spec.N, X, nbr, nbr_face=nf, orient=bad)[0] == MESH
    badf = nf.copy(); badf[0, 1] = 3                  # wrong neighbour face
    assert _init(spec.N, X, nbr, nbr_face=badf, orient=ori)[0] == MESH


def test_batch_call_refuses_a_null_context():
    import ctypes
    from paper_2606_18927_gb300 import dg
    L = dg.lib()
    assert L.dg_rk_stage_batch(None, 1, None, None, 1, 0.0, 1e-3) == -1
