"""The hand-written adjoint (dg_vjp) against the oracle and finite differences.

* dot-product tests <lam, J d> = <J^T lam, d>: J d is the extended-precision
  oracle's exact forward-mode (dual number) derivative of Ut;
* the wall-law constants: <lam, dUt/dkappa> and <lam, dUt/dB> from the oracle;
* on tiny meshes, J^T lam element by element, J assembled column by column
  from the oracle's JVPs;
* central finite differences of the GPU operator itself (relative 1e-6)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, torch_cuda

pytestmark = pytest.mark.gpu


def _vjp(torch, g, U, lam):
    Ud = torch.from_numpy(U).cuda()
    ld = torch.from_numpy(np.ascontiguousarray(lam)).cuda()
    gU = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.vjp(ld, gU, Ud, gth)
    torch.cuda.synchronize()
    g.check_status()
    return gU.cpu().numpy(), gth.cpu().numpy()


# states with a uniform velocity offset keep |u_n| in the Riemann dissipation
# away from its kink at 0
CASES = [
    ("tgv_n3_llf", I.BoxSpec(3, 3, 2, 2), 1, 1, "tgv_shift"),
    ("sine_n4_roe", I.BoxSpec(4, 2, 2, 3, geometry="sine", amplitude=0.2), 2, 1, "tgv_shift"),
    ("sine_n5_central_euler", I.BoxSpec(5, 2, 2, 2, geometry="sine", amplitude=0.2), 0, 0, "tgv_shift"),
    ("sine_n4_roe_sonic", I.BoxSpec(4, 3, 2, 2, geometry="sine", amplitude=0.2), 2, 1, "tgv_sonic"),
    ("tgv_n3_llf_sonic", I.BoxSpec(3, 3, 2, 2), 1, 1, "tgv_sonic"),
    # N = 7: the adjoint element kernel's even/odd contractions and its warp
    # layout (the path of the benchmarked VJP), curved, viscous, Roe; the
    # sonic state puts part of the xi faces inside Harten's entropy fix
    ("sine_n7_roe", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, 1, "tgv_shift"),
    ("sine_n7_roe_sonic", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, 1, "tgv_sonic"),
    ("sine_n7_llf_ragged", I.BoxSpec(7, 3, 1, 2, geometry="sine", amplitude=0.1), 1, 1, "tgv_shift"),
]


@pytest.mark.parametrize("label,spec,surf,visc,ic", CASES)
def test_dot_product_against_oracle_jvp(ora, label, spec, surf, visc, ic):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=200.0)
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, viscous=visc, rel=1e-2, ic=ic)
    lam = I.random_direction(U.shape, seed=3)
    gU, _ = _vjp(torch, g, U, lam)
    for seed in (4, 5):
        d = I.random_direction(U.shape, seed=seed) * np.abs(U)
        _, Jd = o.jvp(U, d)
        a = float((lam * Jd).sum()); b = float((gU * d).sum())
        print(label, "dot", a, b, abs(a - b) / abs(a))
        assert abs(a - b) <= 1e-11 * (np.abs(lam * Jd).sum())


@pytest.mark.parametrize("N,law", [(3, 1), (3, 0), (5, 1), (5, 0)])
def test_channel_state_and_parameters(ora, N, law):
    # N = 5 is the degree of the wall-modelled channel workload
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=N, elems=(4, 4, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=law, ic="channel")
    lam = I.random_direction(U.shape, seed=6)
    gU, gth = _vjp(torch, g, U, lam)
    d = I.random_direction(U.shape, seed=7) * np.abs(U)
    _, Jd = o.jvp(U, d)
    a = float((lam * Jd).sum()); b = float((gU * d).sum())
    print("channel N", N, "law", law, "dot", a, b)
    assert abs(a - b) <= 1e-11 * np.abs(lam * Jd).sum()
    for k, (dk, dB) in enumerate(((1.0, 0.0), (0.0, 1.0))):
        _, Jt = o.jvp(U, None, dk, dB)
        ref = float((lam * Jt).sum())
        print("  dtheta", k, ref, gth[k])
        assert abs(ref - gth[k]) <= 1e-10 * np.abs(lam * Jt).sum()


@pytest.mark.parametrize("label,spec,ic,law", [
    ("tiny_sine_n2", I.BoxSpec(2, 2, 2, 2, geometry="sine", amplitude=0.2), "tgv_shift", 1),
    ("tiny_channel_n2", I.BoxSpec(2, 2, 2, 1, lengths=(2 * np.pi, 2.0, np.pi), geometry="channel",
                                  amplitude=0.05, periodic=(True, False, True)), "channel", 0),
])
def test_full_transpose_on_tiny_mesh(ora, label, spec, ic, law):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.2, Re=500.0, force=(0.01, 0.0, 0.0))
    # J is assembled from ~1000 JVPs of the FP64 oracle (the extended build is
    # software quad precision on aarch64); on these states the two agree to
    # ~1e-15 relative
    o, g, X, U = case(ora, spec, phys, surf_flux=2, law=law, ic=ic, rel=1e-2, extended=False)
    lam = I.random_direction(U.shape, seed=8)
    gU, _ = _vjp(torch, g, U, lam)
    ref = np.zeros(U.size)
    flat = U.reshape(-1)
    for k in range(U.size):
        e = np.zeros(U.size); e[k] = 1.0
        _, col = o.jvp(U, e.reshape(U.shape))
        ref[k] = float((lam.reshape(-1) * col.reshape(-1)).sum())
    err = np.abs(gU.reshape(-1) - ref).max() / np.abs(ref).max()
    print(label, "J^T lam max rel", err)
    assert err <= 1e-10


@pytest.mark.parametrize("N", [3, 5])
def test_finite_differences_of_the_gpu_operator(ora, N):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=N, elems=(4, 4, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=1, ic="channel")
    lam = I.random_direction(U.shape, seed=10)
    gU, gth = _vjp(torch, g, U, lam)
    d = I.random_direction(U.shape, seed=11) * np.abs(U)
    eps = 1e-6
    Up = torch.from_numpy(U + eps * d).cuda(); Um = torch.from_numpy(U - eps * d).cuda()
    a = torch.empty_like(Up); b = torch.empty_like(Up)
    g.time_derivative(a, Up); g.time_derivative(b, Um)
    fd = float((lam * (a - b).cpu().numpy()).sum()) / (2 * eps)
    ad = float((gU * d).sum())
    print("FD", fd, "adjoint", ad)
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    # wall-law constants by finite differences of the GPU operator
    x, w, D = ora.lgl(wl.spec.N)
    for k, key in enumerate(("kappa", "B")):
        vals = []
        for sgn in (1, -1):
            ph = dict(wl.phys); ph[key] = ph[key] + sgn * eps
            gp = dg.Operator(wl.spec.N, X, I.connectivity(wl.spec), ph, surf_flux=2, law=1)
            out = torch.empty_like(Up)
            gp.time_derivative(out, torch.from_numpy(U).cuda())
            vals.append(out.cpu().numpy())
            gp.close()
        fdt = float((lam * (vals[0] - vals[1])).sum()) / (2 * eps)
        print("FD", key, fdt, gth[k])
        assert abs(fdt - gth[k]) <= 1e-6 * abs(gth[k])


def test_full_transpose_at_n7_one_element(ora):
    """N = 7 on one periodic curved element (each face its own neighbour):
    J^T lam against J assembled from the oracle's 2560 JVP columns, so that
    every entry of the even/odd adjoint element kernel is checked, not only
    its action on random directions."""
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.3, Re=200.0)
    spec = I.BoxSpec(7, 1, 1, 1, geometry="sine", amplitude=0.2)
    o, g, X, U = case(ora, spec, phys, surf_flux=2, ic="tgv_shift", rel=1e-2, extended=False)
    lam = I.random_direction(U.shape, seed=12)
    gU, _ = _vjp(torch, g, U, lam)
    ref = np.zeros(U.size)
    for k in range(U.size):
        e = np.zeros(U.size); e[k] = 1.0
        _, col = o.jvp(U, e.reshape(U.shape))
        ref[k] = float((lam.reshape(-1) * col.reshape(-1)).sum())
    err = np.abs(gU.reshape(-1) - ref).max() / np.abs(ref).max()
    print("n7 one element J^T lam max rel", err)
    assert err <= 1e-10
