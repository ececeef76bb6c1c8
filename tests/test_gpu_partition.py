"""Partitioned meshes on one GPU: the ranks of a space-filling-curve
partition (paper Sec. 2.1) as contexts in one process, their halo exchanges
done by device copies between the phases.  Every stage must reproduce the
unpartitioned context bitwise; the time derivative likewise.  The assembled
partitioned results are also compared with the extended-precision oracle
directly (relative max norm 1e-12 in FP64, relative L2 1e-5 in the
FP32-mixed form)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, halo, inputs as I
from gpu_helpers import parity, tgv_with_offset, torch_cuda

TOL = 1e-12


def _oracle_check(ora, spec, X, nbr, phys, U, ut, state, dt, nsteps, opts, law=1):
    """Partitioned Ut and state increment over nsteps against the oracle."""
    o = ora.Oracle(spec.N, X, nbr, phys, vol_flux=opts.get("vol_flux", 0), surf_flux=opts.get("surf_flux", 1),
                   viscous=opts.get("viscous", 1), law=law, extended=True)
    ref_ut = o.time_derivative(U)
    ref_inc = o.rk_steps(U, dt, nsteps) - U
    got_ut = ut.cpu().numpy(); got_inc = state.cpu().numpy() - U
    if opts.get("precision", dg.FP64) == dg.FP64:
        e1 = parity(got_ut, ref_ut); e2 = parity(got_inc, ref_inc)
        print("  vs oracle: Ut", e1, "state increment", e2)
        assert e1 <= TOL and e2 <= TOL
    else:
        a = got_ut.reshape(5, -1); b = ref_ut.reshape(5, -1)
        l2 = max(float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(5))
        print("  vs oracle (mixed): Ut rel L2", l2)
        assert l2 <= 1e-5

pytestmark = pytest.mark.gpu


def _setup(spec, phys, **opts):
    x, w = dg.lgl_nodes(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    U = I.perturb(tgv_with_offset(X, phys, offset=(0.3, 0.1, 0.05)), rel=1e-3)
    return X, nbr, U


def _compare(torch, spec, phys, P, nsteps=2, ora=None, **opts):
    X, nbr, U = _setup(spec, phys)
    Ud = torch.from_numpy(U).cuda()
    g = dg.Operator(spec.N, X, nbr, phys, **opts)
    dt = g.time_step(0.9, Ud)
    g.set_state(Ud)
    g.rk_steps(0.0, dt, nsteps)
    ref = torch.empty_like(Ud)
    g.get_state(ref)
    g.check_status()
    ranks = halo.LocalRanks(spec.N, X, nbr, phys, P, **opts)
    ranks.set_state(Ud)
    ranks.steps(0.0, dt, nsteps)
    out = torch.empty_like(Ud)
    ranks.get_state(out)
    ranks.check_status()
    # time derivative through the phases
    ut_ref = torch.empty_like(Ud)
    g.time_derivative(ut_ref, Ud)
    ut = torch.empty_like(Ud)
    ranks.time_derivative(ut, Ud)
    torch.cuda.synchronize()
    nh = [len(h) for h in ranks.halo]
    ranks.close(); g.close()
    if ora is not None:
        _oracle_check(ora, spec, X, nbr, phys, U, ut, out, dt, nsteps, opts)
    return ref, out, ut_ref, ut, nh


@pytest.mark.parametrize("P", [2, 3, 5])
def test_partitioned_tgv_bitwise(ora, P):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(3, 4, 4, 3, geometry="sine", amplitude=0.2)
    ref, out, ut_ref, ut, nh = _compare(torch, spec, phys, P, ora=ora, surf_flux=2)
    print("TGV P", P, "halo faces", nh)
    assert min(nh) > 0
    assert torch.equal(out, ref)
    assert torch.equal(ut, ut_ref)


def test_partitioned_tgv_n7_bitwise(ora):
    # N = 7 runs the even/odd lifting contractions, the once-formed
    # half-distance pairs and the swizzled shared-memory layout of the volume
    # kernel; the halo faces take the FP64 primitives the lifting kernel keeps
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(7, 4, 2, 2, geometry="sine", amplitude=0.1)
    ref, out, ut_ref, ut, nh = _compare(torch, spec, phys, 3, ora=ora, surf_flux=2)
    assert min(nh) > 0
    assert torch.equal(out, ref)
    assert torch.equal(ut, ut_ref)


@pytest.mark.parametrize("P", [2, 5])
def test_partitioned_tgv_mixed(ora, P):
    # the FP32 flux arithmetic of a halo face runs in another kernel than that
    # of an interior face, where the compiler may contract it differently:
    # agreement to FP32 rounding of the fluxes, not bitwise
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(3, 4, 4, 3, geometry="sine", amplitude=0.2)
    X, nbr, U = _setup(spec, phys)
    U0 = torch.from_numpy(U).cuda()
    ref, out, ut_ref, ut, nh = _compare(torch, spec, phys, P, ora=ora, precision=dg.FP32_MIXED, surf_flux=2)
    e_state = float((out - ref).abs().max() / (ref - U0).abs().max())
    e_ut = max(float((ut[v] - ut_ref[v]).abs().max() / ut_ref[v].abs().max()) for v in range(5))
    print("mixed P", P, "state increment diff", e_state, "Ut diff", e_ut, "bitwise", torch.equal(out, ref))
    assert e_state <= 1e-5 and e_ut <= 1e-5


def test_partitioned_production_scheme_with_inflow_outflow_bitwise(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=400.0, sutherland=True)
    g0, p0 = phys["gamma"], phys["p0"]
    phys.update(U_in=np.array([1.0, 0.5, 0.0, 0.0, p0 / (g0 - 1) + 0.125]), p_out=0.99 * p0)
    spec = I.BoxSpec(4, 5, 2, 3, geometry="sine", amplitude=0.1, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    ref, out, ut_ref, ut, nh = _compare(torch, spec, phys, 3, ora=ora, vol_flux=dg.VOL_EC_CHANDRASHEKAR, surf_flux=2)
    assert torch.equal(out, ref) and torch.equal(ut, ut_ref)


@pytest.mark.parametrize("P", [2, 4])
def test_partitioned_wall_modelled_channel_bitwise(ora, P):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(8, 4, 4))
    X, nbr, U = _setup(wl.spec, wl.phys)
    U = I.channel_profile(X, wl.phys)
    Ud = torch.from_numpy(U).cuda()
    g = dg.Operator(wl.spec.N, X, nbr, wl.phys, surf_flux=2, law=1)
    dt = g.time_step(0.9, Ud)
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    ref = torch.empty_like(Ud)
    g.get_state(ref)
    ranks = halo.LocalRanks(wl.spec.N, X, nbr, wl.phys, P, surf_flux=2, law=1)
    ranks.set_state(Ud)
    ranks.steps(0.0, dt, 2)
    out = torch.empty_like(Ud)
    ranks.get_state(out)
    ranks.check_status()
    assert torch.equal(out, ref)
    ut = torch.empty_like(Ud)
    ranks.time_derivative(ut, Ud)
    torch.cuda.synchronize()
    ranks.close(); g.close()
    _oracle_check(ora, wl.spec, X, nbr, wl.phys, U, ut, out, dt, 2, dict(surf_flux=2), law=1)


def test_fused_calls_refuse_partitioned_contexts():
    torch = torch_cuda()
    phys = I.phys_params()
    spec = I.BoxSpec(2, 4, 2, 2)
    X, nbr, U = _setup(spec, phys)
    ranks = halo.LocalRanks(spec.N, X, nbr, phys, 2)
    op = ranks.ops[0]
    Ul = torch.from_numpy(halo.local_state(U, ranks.l2g[0])).cuda()
    op.set_state(Ul)
    with pytest.raises(dg.DGError) as ei:
        op.rk_stage(0, 0.0, 1e-3)
    assert ei.value.code == -1
    with pytest.raises(dg.DGError) as ei:
        op.vjp(torch.ones_like(Ul), torch.empty_like(Ul), U=Ul)
    assert ei.value.code in (-1, -8)


def _vjp_compare(torch, ora, spec, phys, P, X=None, nbr=None, U=None, nbr_face=None, orient=None, law=1, **opts):
    """The partitioned adjoint (four phases, three exchanges) against dg_vjp
    on the unpartitioned mesh, and a dot product against the extended
    oracle's forward-mode derivative."""
    if X is None:
        X, nbr, U = _setup(spec, phys)
    Ud = torch.from_numpy(U).cuda()
    lam = torch.from_numpy(I.random_direction(U.shape, seed=51)).cuda()
    g = dg.Operator(spec.N, X, nbr, phys, nbr_face=nbr_face, orient=orient, law=law, **opts)
    ref = torch.empty_like(Ud)
    th_ref = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.vjp(lam, ref, Ud, th_ref)
    g.check_status()
    ranks = halo.LocalRanks(spec.N, X, nbr, phys, P, nbr_face=nbr_face, orient=orient, law=law, **opts)
    assert sum(len(h) for h in ranks.halo) > 0
    out = torch.empty_like(Ud)
    th = torch.zeros(2, dtype=torch.float64, device="cuda")
    ranks.vjp(lam, out, Ud, th)
    ranks.check_status()
    torch.cuda.synchronize()
    a = out.cpu().numpy(); b = ref.cpu().numpy()
    e = parity(a, b)
    print("  partitioned VJP vs unpartitioned", e, "gtheta", th.cpu().numpy(), th_ref.cpu().numpy())
    assert e <= 1e-13
    thr = th_ref.cpu().numpy()
    assert np.all(np.abs(th.cpu().numpy() - thr) <= 1e-12 * np.abs(thr).max() + 1e-300)
    o = ora.Oracle(spec.N, X, nbr, phys, vol_flux=opts.get("vol_flux", 0), surf_flux=opts.get("surf_flux", 1),
                   viscous=opts.get("viscous", 1), law=law, extended=True, nbr_face=nbr_face, orient=orient)
    d = I.random_direction(U.shape, seed=52) * np.abs(U)
    _, Jd = o.jvp(U, d)
    lm = lam.cpu().numpy()
    x = float((lm * Jd).sum()); y = float((a * d).sum())
    print("  dot", x, y)
    assert abs(x - y) <= 1e-11 * np.abs(lm * Jd).sum()
    ranks.close(); g.close()


@pytest.mark.parametrize("P", [2, 3])
def test_partitioned_adjoint_taylor_green(ora, P):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=200.0)
    _vjp_compare(torch, ora, I.BoxSpec(3, 4, 3, 2, geometry="sine", amplitude=0.2), phys, P, surf_flux=2)


def test_partitioned_adjoint_production_scheme_with_boundaries(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=400.0, sutherland=True)
    g0, p0 = phys["gamma"], phys["p0"]
    phys.update(U_in=np.array([1.0, 0.5, 0.0, 0.0, p0 / (g0 - 1) + 0.125]), p_out=0.99 * p0)
    spec = I.BoxSpec(4, 5, 2, 3, geometry="sine", amplitude=0.1, periodic=(False, True, True),
                     boundary=((I.INFLOW, I.OUTFLOW), (I.WALL, I.WALL), (I.WALL, I.WALL)))
    _vjp_compare(torch, ora, spec, phys, 3, vol_flux=dg.VOL_EC_CHANDRASHEKAR, surf_flux=2)


@pytest.mark.parametrize("P", [2, 4])
def test_partitioned_adjoint_wall_modelled_channel(ora, P):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=3, elems=(8, 4, 4))
    X, nbr, _ = _setup(wl.spec, wl.phys)
    U = I.channel_profile(X, wl.phys)
    _vjp_compare(torch, ora, wl.spec, wl.phys, P, X=X, nbr=nbr, U=U, surf_flux=2)


def test_partitioned_adjoint_refusals():
    torch = torch_cuda()
    phys = I.phys_params()
    spec = I.BoxSpec(2, 4, 2, 2)
    X, nbr, U = _setup(spec, phys)
    ranks = halo.LocalRanks(spec.N, X, nbr, phys, 2)
    op = ranks.ops[0]
    Ul = torch.from_numpy(halo.local_state(U, ranks.l2g[0])).cuda()
    for bad in (0, 5):
        with pytest.raises(dg.DGError) as ei:
            op.vjp_phase(bad, torch.ones_like(Ul), torch.empty_like(Ul), Ul)
        assert ei.value.code == -1
    g = dg.Operator(spec.N, X, nbr, phys)
    Ud = torch.from_numpy(U).cuda()
    with pytest.raises(dg.DGError) as ei:
        g.vjp_phase(2, torch.ones_like(Ud), torch.empty_like(Ud), Ud)
    assert ei.value.code == -1
    ranks.close(); g.close()


@pytest.mark.parametrize("P", [2, 3])
def test_partitioned_adjoint_rotated_mesh(ora, P):
    """General conforming connectivity: the cotangent traces cross in the
    master's face-node order like the state traces."""
    from helpers import rotated_mesh
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    spec = I.BoxSpec(3, 4, 3, 3, geometry="sine", amplitude=0.15)
    x, w, D = ora.lgl(3)
    X, nbr, nf, ori, rots = rotated_mesh(spec, x, seed=11)
    U = I.perturb(tgv_with_offset(X, phys, offset=(0.3, 0.1, 0.05)), rel=1e-3)
    _vjp_compare(torch, ora, spec, phys, P, X=X, nbr=nbr, U=U, nbr_face=nf, orient=ori, surf_flux=2)
