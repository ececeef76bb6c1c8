"""dg_time_derivative_noalloc: the operator evaluation that allocates nothing.

Host programs that manage all device memory through their own allocator
(the paper's Fortran core allocates and copies every GPU array itself,
Sec. 2.1) cannot let a library call cudaMalloc when it computes.  This entry
point takes its inter-kernel scratch from a static device array instead of
the context's buffers.  Its results must equal those of dg_time_derivative,
call after call (the array keeps the previous call's contents).  This file
is collected last so that a failing run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _rel(a, b):
    a = a.reshape(5, -1); b = b.reshape(5, -1)
    return max(float(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max()) for v in range(5))


def _noalloc(op, U, out):
    return dg.lib().dg_time_derivative_noalloc(op.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("name,N,elems", [("tgv_n3_4", 3, (4, 4, 4)), ("channel_n5", 3, (4, 4, 2))])
def test_noalloc_matches_time_derivative(name, N, elems):
    torch = _cuda()
    wl = I.workload(name, N=N, elems=elems)
    x, w = dg.lgl_nodes(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U1 = I.initial_state(wl, X)
    U2 = I.perturb(U1, rel=1e-2, seed=77)
    op = dg.Operator(wl.spec.N, X, nbr, wl.phys, vol_flux=wl.vol_flux, surf_flux=wl.surf_flux,
                     viscous=wl.viscous, law=wl.law)
    for U in (U1, U2):  # two calls in a row, different states
        Ud = torch.from_numpy(U).cuda()
        ref = torch.empty_like(Ud)
        op.time_derivative(ref, Ud)
        out = torch.full_like(Ud, float("nan"))
        rc = _noalloc(op, Ud, out)
        assert rc == 0, dg.lib().dg_last_error(op.h).decode()
        torch.cuda.synchronize()
        op.check_status()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL
    op.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    torch = _cuda()
    wl = I.workload("tgv_n7_32", elems=(12, 12, 12))  # 884,736 DOF: above the static limit
    x, w = dg.lgl_nodes(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    op = dg.Operator(wl.spec.N, X, I.connectivity(wl.spec), wl.phys, surf_flux=wl.surf_flux)
    Ud = torch.zeros(op.numel, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(Ud)
    rc = _noalloc(op, Ud, out)
    assert rc == -1
    assert b"static limit" in dg.lib().dg_last_error(op.h)
    op.close()
