"""Parity of the sm_103a FP64 operator with the CPU oracle (paper Sec. 2.2 /
Sec. 4 split-form DGSEM, Sec. 3 wall model), element by element on the same
seeded inputs, through the C ABI.

Tolerance: relative max-norm 1e-12 per variable (normalised by max|Ut_v| of
the oracle), the FP64 parity target of the operator."""
import math

import numpy as np
import pytest

from paper_2606_18927_gb300 import inputs as I
from gpu_helpers import case, gpu_ut, parity, parity_per_var, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("label,spec,surf,vol,visc", [
    ("tgv_n3_4^3_llf", I.BoxSpec(3, 4, 4, 4), 1, 0, 1),
    ("n2_ragged_sine_roe", I.BoxSpec(2, 3, 2, 5, geometry="sine", amplitude=0.3), 2, 0, 1),
    ("n4_central_kg", I.BoxSpec(4, 2, 3, 2, geometry="sine", amplitude=0.2), 0, 1, 1),
    ("n5_roe_euler", I.BoxSpec(5, 2, 2, 3, geometry="sine", amplitude=0.2), 2, 0, 0),
    ("n7_roe_sine", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1), 2, 0, 1),
    # N = 7 without viscous terms (primitives formed by the face and volume
    # kernels themselves) and with the Kennedy-Gruber flux
    ("n7_llf_kg_euler", I.BoxSpec(7, 2, 3, 2, geometry="sine", amplitude=0.1), 1, 1, 0),
    ("n7_central_kg", I.BoxSpec(7, 3, 2, 2, geometry="sine", amplitude=0.1), 0, 1, 1),
    ("n1_llf", I.BoxSpec(1, 3, 3, 3), 1, 0, 1),
    ("n6_llf_periodic_self", I.BoxSpec(6, 1, 2, 1), 1, 0, 1),
    ("n8_roe", I.BoxSpec(8, 2, 1, 2, geometry="sine", amplitude=0.1), 2, 0, 1),
])
def test_time_derivative_matches_oracle(ora, label, spec, surf, vol, visc):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, vol_flux=vol, viscous=visc)
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print(label, "parity", e, ["%.1e" % x for x in parity_per_var(out, ref)])
    assert e <= TOL, e


@pytest.mark.parametrize("law", [1, 0])
def test_wall_model_channel_matches_oracle(ora, law):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=law, ic="channel")
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print("channel law", law, "parity", e)
    assert e <= TOL, e


def test_channel_full_size_matches_oracle(ora):
    """16 x 8 x 8 elements, N = 5 (221,184 DOF), Reichardt wall model."""
    torch = torch_cuda()
    wl = I.workload("channel_n5")
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=1, ic="channel")
    e = parity(gpu_ut(torch, g, U), o.time_derivative(U))
    print("channel full parity", e)
    assert e <= TOL, e


def test_rk_step_matches_oracle(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(3, 4, 4, 4)
    o, g, X, U = case(ora, spec, phys, surf_flux=1)
    dt = o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_state(Ud)
    nsteps = 2
    g.rk_steps(0.0, dt, nsteps)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    Uo = o.rk_steps(U, dt, nsteps)
    # compare the change of the state over the steps
    e = parity(Ug.cpu().numpy() - U, Uo - U)
    print("rk steps parity (increment)", e)
    assert e <= TOL, e


def test_single_stage_dU(ora):
    """Three LSERK4 stages: the register dU (the stage increment before it is
    added to the O(1..200) state) agrees to the FP64 tolerance; U agrees to
    that tolerance of its increment plus one rounding of U itself."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(4, 3, 2, 2, geometry="sine", amplitude=0.2)
    o, g, X, U = case(ora, spec, phys, surf_flux=2)
    dt = 1e-3
    g.set_state(torch.from_numpy(U).cuda())
    Uo = U.copy(); dUo = np.zeros_like(U)
    for s in range(3):
        g.rk_stage(s, 0.0, dt)
        o.rk_stage(Uo, dUo, s, 0.0, dt)
    Ug = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    dUg = torch.empty_like(Ug)
    g.get_state(Ug)
    g.get_rk_register(dUg)
    g.check_status()
    e = parity(dUg.cpu().numpy(), dUo)
    print("stage register parity", e)
    assert e <= TOL, e
    dif = np.abs(Ug.cpu().numpy() - Uo).reshape(5, -1)
    inc = np.abs(Uo - U).reshape(5, -1)
    bound = TOL * inc.max(axis=1, keepdims=True) + 2 * np.spacing(np.abs(Uo).reshape(5, -1))
    assert np.all(dif <= bound)


def test_host_pointer_path(ora):
    """dg_time_derivative with host arrays (upload, operator, download)."""
    torch = torch_cuda()
    phys = I.phys_params()
    o, g, X, U = case(ora, I.BoxSpec(3, 2, 2, 2), phys)
    Ut = np.zeros_like(U)
    g.time_derivative(Ut, U)
    assert parity(Ut, o.time_derivative(U)) <= TOL


def _euler_flux_max(U, gamma):
    """max over nodes, directions and variables of |F_d(U)| (Euler flux)."""
    r = U[0]
    vel = U[1:4] / r
    p = (gamma - 1.0) * (U[4] - 0.5 * r * (vel ** 2).sum(axis=0))
    m = 0.0
    for d in range(3):
        F = [U[1 + d], U[1] * vel[d], U[2] * vel[d], U[3] * vel[d], (U[4] + p) * vel[d]]
        F[1 + d] = F[1 + d] + p
        m = max(m, max(float(np.abs(f).max()) for f in F))
    return m


@pytest.mark.parametrize("N,ne", [(3, 8), (5, 4), (7, 3)])
def test_free_stream_and_conservation_on_device(ora, N, ne):
    """Free-stream preservation on a curved periodic mesh, scaled as
    max|Ut| h / max|F| <= 1e-13 (h the element size, F the Euler flux), for
    the device operator and the extended-precision oracle; then discrete
    conservation of the device operator on a perturbed Taylor-Green state:
    |sum_nodes w J Ut_v| <= 1e-13 sum_nodes w J |Ut_v| per variable."""
    from helpers import quad_weights
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3)
    spec = I.BoxSpec(N, ne, ne, ne, geometry="sine", amplitude=0.1)
    o, g, X, U = case(ora, spec, phys, surf_flux=2, ic="free")
    Ut = gpu_ut(torch, g, U)
    ref = o.time_derivative(U)
    h = 2.0 * math.pi / ne
    Fm = _euler_flux_max(U, phys["gamma"])
    sg = float(np.abs(Ut).max()) * h / Fm
    so = float(np.abs(ref).max()) * h / Fm
    print("free stream N", N, "scaled residual gpu", sg, "oracle", so)
    assert sg <= 1e-13 and so <= 1e-13
    o2, g2, X2, U2 = case(ora, spec, phys, surf_flux=2, ic="tgv", rel=5e-2)
    Ut2 = gpu_ut(torch, g2, U2).reshape(5, -1)
    wJ = quad_weights(ora, o2).reshape(-1)
    for v in range(5):
        tot = abs(float((wJ * Ut2[v]).sum()))
        scale = float((wJ * np.abs(Ut2[v])).sum())
        print("  conservation var", v, tot / scale)
        assert tot <= 1e-13 * scale


@pytest.mark.parametrize("label,spec", [
    ("n3_roe_sonic", I.BoxSpec(3, 4, 3, 2)),
    ("n7_roe_sonic_sine", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1)),
])
def test_roe_entropy_fix_states_match_oracle(ora, label, spec):
    """Roe's flux with Harten's entropy fix (Sec. 4) on a state whose mean
    flow runs at the speed of sound along x: on part of the xi faces
    |u_n - c| < c / 10, where the fix replaces the acoustic eigenvalue."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=1600.0)
    o, g, X, U = case(ora, spec, phys, surf_flux=2, ic="tgv_sonic")
    n = spec.N + 1
    Un = U.reshape(5, spec.K, n, n, n)  # [v][e][k][j][i]
    face = Un[..., [0, spec.N]]          # the xi faces (i = 0, N)
    r = face[0]
    u = face[1] / r
    p = (phys["gamma"] - 1.0) * (face[4] - 0.5 * (face[1] ** 2 + face[2] ** 2 + face[3] ** 2) / r)
    c = np.sqrt(phys["gamma"] * p / r)
    inside = int((np.abs(u - c) < 0.1 * c).sum())
    assert inside > 0
    ref = o.time_derivative(U)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print(label, "xi-face nodes inside the fix", inside, "of", r.size, "parity", e)
    assert e <= TOL, e


def test_time_step_and_kinetic_energy(ora):
    """CFL time step (reading R9) and the volume-averaged kinetic energy on
    the GPU against the oracle's definitions."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    o, g, X, U = case(ora, I.BoxSpec(4, 3, 2, 2, geometry="sine", amplitude=0.2), phys, surf_flux=2)
    Ud = torch.from_numpy(U).cuda()
    dt = g.time_step(0.9, Ud)
    ke = g.kinetic_energy(Ud)
    assert abs(dt - o.dt(U, 0.9)) <= 1e-13 * dt
    assert abs(ke - o.kinetic_energy(U)) <= 1e-13 * ke


def test_graph_replay_equals_stream_launches(ora):
    """A CUDA-graph replay of whole LSERK4 steps gives bitwise the state of
    the same steps launched kernel by kernel."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    o, g, X, U = case(ora, I.BoxSpec(3, 4, 4, 4), phys, surf_flux=1)
    Ud = torch.from_numpy(U).cuda()
    dt = g.time_step(0.9, Ud)
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 3)
    a = torch.empty_like(Ud)
    g.get_state(a)
    g.set_state(Ud)
    g.rk_steps_graph(0.0, dt, 3)
    b = torch.empty_like(Ud)
    g.get_state(b)
    g.check_status()
    assert torch.equal(a, b)


def test_wall_side_stream_and_graph_on_channel(ora):
    """Wall-modelled channel: the wall-model kernel on its side stream gives
    bitwise the result of the in-line launch, also when whole steps are
    replayed from a CUDA graph (the fork and join are captured), and the
    step still matches the oracle."""
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(4, 4, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=1, ic="channel")
    Ud = torch.from_numpy(U).cuda()
    dt = g.time_step(0.9, Ud)
    out = []
    for overlap, graph in ((False, False), (True, False), (True, True)):
        g.set_overlap(overlap)
        g.set_state(Ud)
        (g.rk_steps_graph if graph else g.rk_steps)(0.0, dt, 2)
        r = torch.empty_like(Ud)
        g.get_state(r)
        g.check_status()
        out.append(r)
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])
    e = parity(out[1].cpu().numpy() - U, o.rk_steps(U, dt, 2) - U)
    print("channel side-stream steps parity (increment)", e)
    assert e <= TOL, e
    # per-kernel timing sees the wall kernel on its stream
    g.set_overlap(True)
    g.profile_enable(True)
    g.rk_stage(0, 0.0, dt)
    prof = g.profile_read()
    g.profile_enable(False)
    assert prof["wall"][1] == 1 and prof["wall"][0] > 0.0


@pytest.mark.parametrize("N", [3, 5])
def test_curved_wall_model_matches_oracle(ora, N):
    """Wall model on a curved wall (a bump of the lower wall): the sample
    points leave their wall elements at some nodes, so the CUDA path's host
    geometry must locate them in the same elements and at the same reference
    coordinates as the oracle (Sec. 3.2; reading R10)."""
    from helpers import bump_wall
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.2, Re=2000.0, force=(0.01, 0.0, 0.0), hwm=0.3)
    spec = I.BoxSpec(N, 4, 3, 4, lengths=(2 * math.pi, 2.0, 2 * math.pi), periodic=(True, False, True))
    x, w, D = ora.lgl(N)
    X = bump_wall(I.node_coordinates(spec, x))
    nbr = I.connectivity(spec)
    from paper_2606_18927_gb300 import dg
    o = ora.Oracle(N, X, nbr, phys, surf_flux=2, law=1, extended=True)
    g = dg.Operator(N, X, nbr, phys, surf_flux=2, law=1)
    U = I.channel_profile(X, phys)
    e = parity(gpu_ut(torch, g, U), o.time_derivative(U))
    print("curved wall N", N, "parity", e)
    assert e <= TOL, e
