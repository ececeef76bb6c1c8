"""dg_time_derivative_noalloc: the operator evaluation that allocates nothing.

Host programs that manage all device memory through their own allocator
(the paper's Fortran core allocates and copies every GPU array itself,
Sec. 2.1) cannot let a library call cudaMalloc when it computes.  This entry
point takes its inter-kernel scratch from a static device array instead of
the context's buffers.  Its results must equal those of dg_time_derivative,
call after call (the array keeps the previous call's contents), and match the
extended-precision oracle like every other evaluation (relative max norm
1e-12 in FP64, relative L2 1e-5 in the FP32-mixed form).  This file is
collected last so that a failing run has already run every other test.
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


def _l2(a, b):
    a = a.reshape(5, -1); b = b.reshape(5, -1)
    return max(float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5))


@pytest.mark.parametrize("name,N,elems,precision", [
    ("tgv_n3_4", 3, (4, 4, 4), dg.FP64),
    ("channel_n5", 3, (4, 4, 2), dg.FP64),
    ("tgv_n7_32", 7, (3, 2, 3), dg.FP64),
    ("tgv_n3_4", 3, (4, 4, 4), dg.FP32_MIXED),
    ("tgv_n7_32", 7, (3, 2, 3), dg.FP32_MIXED),
    ("channel_n5", 5, (4, 4, 2), dg.FP32_MIXED),
])
def test_noalloc_matches_time_derivative(ora, name, N, elems, precision):
    torch = _cuda()
    wl = I.workload(name, N=N, elems=elems)
    x, w, D = ora.lgl(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U1 = I.initial_state(wl, X)
    U2 = I.perturb(U1, rel=1e-2, seed=77)
    op = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=precision, vol_flux=wl.vol_flux,
                     surf_flux=wl.surf_flux, viscous=wl.viscous, law=wl.law)
    o = ora.Oracle(wl.spec.N, X, nbr, wl.phys, vol_flux=wl.vol_flux, surf_flux=wl.surf_flux,
                   viscous=wl.viscous, law=wl.law, extended=True)
    for U in (U1, U2):  # two calls in a row, different states
        Ud = torch.from_numpy(U).cuda()
        ref = torch.empty_like(Ud)
        op.time_derivative(ref, Ud)
        out = torch.full_like(Ud, float("nan"))
        rc = _noalloc(op, Ud, out)
        assert rc == 0, dg.lib().dg_last_error(op.h).decode()
        torch.cuda.synchronize()
        op.check_status()
        got = out.cpu().numpy()
        assert _rel(got, ref.cpu().numpy()) <= TOL
        Uo = o.time_derivative(U)
        if precision == dg.FP64:
            e = _rel(got, Uo)
            print(name, N, "noalloc vs oracle", e)
            assert e <= TOL
        else:
            e = _l2(got, Uo)
            print(name, N, "noalloc (FP32-mixed) vs oracle, rel L2", e)
            assert e <= 1e-5
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
