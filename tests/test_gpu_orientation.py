"""The CUDA path on general conforming meshes: elements with rotated local
frames, joined face to face with neighbour faces and orientation codes
(dg_mesh_desc.nbr_face / orient).  Parity with the extended-precision oracle
on the same mesh (relative max norm 1e-12 in FP64, relative L2 1e-5 in the
FP32-mixed form), the wall model across rotated elements, partitioned
contexts on such a mesh, and the adjoint."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, halo, inputs as I
from gpu_helpers import gpu_ut, parity, tgv_with_offset, torch_cuda
from helpers import rotate_elements, rotated_mesh

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel_l2(a, b):
    a = a.reshape(5, -1); b = b.reshape(5, -1)
    return max(float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5))


@pytest.mark.parametrize("N,elems,surf,visc", [(3, (3, 3, 3), 2, 1), (7, (2, 3, 2), 2, 1), (4, (3, 2, 3), 1, 0),
                                               (5, (2, 2, 3), 0, 1)])
def test_rotated_mesh_matches_oracle(ora, N, elems, surf, visc):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(N, *elems, geometry="sine", amplitude=0.15)
    x, w, D = ora.lgl(N)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=N)
    o = ora.Oracle(N, X, nbr, phys, surf_flux=surf, viscous=visc, nbr_face=nf, orient=ori, extended=True)
    g = dg.Operator(N, X, nbr, phys, surf_flux=surf, viscous=visc, nbr_face=nf, orient=ori)
    U = rotate_elements(I.perturb(I.taylor_green(I.node_coordinates(spec, x), phys), rel=1e-3), N, rots)
    ref = o.time_derivative(U)
    e = parity(gpu_ut(torch, g, U), ref)
    print("rotated N", N, "parity", e)
    assert e <= TOL
    # one LSERK4 step through the fused stage kernel
    dt = 0.5 * o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 1)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    # the increment agrees to the tolerance of its size plus the rounding of
    # the state it is added to (with the central flux the density increment
    # is small against the density)
    Uo = o.rk_steps(U, dt, 1)
    dif = np.abs(Ug.cpu().numpy() - Uo).reshape(5, -1)
    inc = np.abs(Uo - U).reshape(5, -1)
    bound = TOL * inc.max(axis=1, keepdims=True) + 2 * np.spacing(np.abs(Uo).reshape(5, -1))
    print("  step increment parity", parity(Ug.cpu().numpy() - U, Uo - U))
    assert np.all(dif <= bound)
    # FP32-mixed form on the same mesh
    gm = dg.Operator(N, X, nbr, phys, precision=dg.FP32_MIXED, surf_flux=surf, viscous=visc, nbr_face=nf,
                     orient=ori)
    em = _rel_l2(gpu_ut(torch, gm, U), ref)
    print("  mixed rel L2", em)
    assert em <= (1e-5 if surf != 0 else 3e-5)  # (central flux: see test_gpu_mixed)
    g.close(); gm.close()


def test_rotated_channel_wall_model_matches_oracle(ora):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(wl.spec, x, seed=8, frac=0.6)
    o = ora.Oracle(3, X, nbr, wl.phys, surf_flux=2, law=1, nbr_face=nf, orient=ori, extended=True)
    g = dg.Operator(3, X, nbr, wl.phys, surf_flux=2, law=1, nbr_face=nf, orient=ori)
    U = rotate_elements(I.channel_profile(I.node_coordinates(wl.spec, x), wl.phys), 3, rots)
    e = parity(gpu_ut(torch, g, U), o.time_derivative(U))
    print("rotated channel parity", e)
    assert e <= TOL


@pytest.mark.parametrize("P", [2, 3])
def test_rotated_mesh_partitioned(ora, P):
    """Ranks of a space-filling-curve partition of the rotated mesh: halo
    traces cross in the master's face-node order; bitwise equal to the
    single-domain context, and equal to the oracle."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(3, 4, 3, 3, geometry="sine", amplitude=0.15)
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=11)
    U = I.perturb(tgv_with_offset(X, phys, offset=(0.3, 0.1, 0.05)), rel=1e-3)
    Ud = torch.from_numpy(U).cuda()
    g = dg.Operator(3, X, nbr, phys, surf_flux=2, nbr_face=nf, orient=ori)
    dt = g.time_step(0.9, Ud)
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    ref = torch.empty_like(Ud)
    g.get_state(ref)
    ranks = halo.LocalRanks(3, X, nbr, phys, P, nbr_face=nf, orient=ori, surf_flux=2)
    assert sum(len(h) for h in ranks.halo) > 0
    ranks.set_state(Ud)
    ranks.steps(0.0, dt, 2)
    out = torch.empty_like(Ud)
    ranks.get_state(out)
    ranks.check_status()
    ut = torch.empty_like(Ud)
    ranks.time_derivative(ut, Ud)
    torch.cuda.synchronize()
    ranks.close(); g.close()
    assert torch.equal(out, ref)
    o = ora.Oracle(3, X, nbr, phys, surf_flux=2, nbr_face=nf, orient=ori, extended=True)
    assert parity(ut.cpu().numpy(), o.time_derivative(U)) <= TOL
    assert parity(out.cpu().numpy() - U, o.rk_steps(U, dt, 2) - U) <= TOL


def test_rotated_mesh_adjoint(ora):
    """Dot-product test of dg_vjp on the rotated mesh against the oracle's
    forward-mode derivative."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=200.0)
    spec = I.BoxSpec(3, 3, 2, 2, geometry="sine", amplitude=0.2)
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=4)
    o = ora.Oracle(3, X, nbr, phys, surf_flux=2, nbr_face=nf, orient=ori, extended=True)
    g = dg.Operator(3, X, nbr, phys, surf_flux=2, nbr_face=nf, orient=ori)
    U = I.perturb(tgv_with_offset(X, phys), rel=1e-2)
    lam = I.random_direction(U.shape, seed=3)
    Ud = torch.from_numpy(U).cuda()
    gU = torch.empty_like(Ud)
    g.vjp(torch.from_numpy(lam).cuda(), gU, Ud)
    torch.cuda.synchronize()
    g.check_status()
    d = I.random_direction(U.shape, seed=4) * np.abs(U)
    _, Jd = o.jvp(U, d)
    a = float((lam * Jd).sum()); b = float((gU.cpu().numpy() * d).sum())
    print("rotated adjoint dot", a, b)
    assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()
