"""Rollout adjoint of the wall-modelled channel (LSERK4 with per-step
checkpoints, dg_rollout_vjp) and the torch.autograd bindings.

Loss: mean wall shear of the final state (quadrature-weighted tau_w t_x over
both walls).  References: the oracle's forward-mode derivative through the
same rollout (dual numbers through every stage, the implicit function theorem
in the wall model), and central finite differences of the GPU forward."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, torch_cuda

pytestmark = pytest.mark.gpu
NSTEPS = 20


def _setup(ora, law=1, extended=False, N=3, elems=(4, 4, 2)):
    wl = I.workload("channel_n5", N=N, elems=elems)
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=law, ic="channel", extended=extended)
    dt = 0.5 * o.dt(U, 0.9)
    return wl, o, g, X, U, dt


def test_wall_shear_loss_matches_oracle(ora):
    torch = torch_cuda()
    wl, o, g, X, U, dt = _setup(ora, extended=True)
    L = g.wall_shear(torch.from_numpy(U).cuda())
    ref = o.wall_shear(U)
    print("loss", L, ref)
    assert abs(L - ref) <= 1e-12 * abs(ref)


# (16, 8, 8) at N = 5 is the full wall-modelled channel workload (221,184 DOF)
@pytest.mark.parametrize("N,elems,law", [(3, (4, 4, 2), 1), (3, (4, 4, 2), 0), (5, (4, 4, 2), 0),
                                         (5, (16, 8, 8), 1)])
def test_rollout_gradient_matches_oracle_derivative(ora, N, elems, law):
    torch = torch_cuda()
    wl, o, g, X, U, dt = _setup(ora, law, N=N, elems=elems)
    Ud = torch.from_numpy(U).cuda()
    gU0 = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = g.rollout_vjp(Ud, NSTEPS, dt, gU0, gth)
    g.check_status()
    d = I.random_direction(U.shape, seed=21) * np.abs(U)
    L_ref, dL = o.rollout_jvp(U, d, 0.0, 0.0, NSTEPS, dt)
    _, dLk = o.rollout_jvp(U, None, 1.0, 0.0, NSTEPS, dt)
    _, dLB = o.rollout_jvp(U, None, 0.0, 1.0, NSTEPS, dt)
    ad = float((gU0.cpu().numpy() * d).sum())
    th = gth.cpu().numpy()
    print("N", N, elems, "law", law, "loss", L, L_ref, "dU0", ad, dL, "dkappa", th[0], dLk, "dB", th[1], dLB)
    assert abs(L - L_ref) <= 1e-11 * abs(L_ref)
    assert abs(ad - dL) <= 1e-9 * abs(dL)
    assert abs(th[0] - dLk) <= 1e-9 * abs(dLk)
    assert abs(th[1] - dLB) <= 1e-9 * abs(dLB)


@pytest.mark.parametrize("N", [3, 5])
def test_rollout_gradient_finite_differences(ora, N):
    torch = torch_cuda()
    wl, o, g, X, U, dt = _setup(ora, N=N)
    Ud = torch.from_numpy(U).cuda()
    gU0 = torch.empty_like(Ud)
    gth = torch.zeros(2, dtype=torch.float64, device="cuda")
    g.rollout_vjp(Ud, NSTEPS, dt, gU0, gth)
    th = gth.cpu().numpy()

    def loss(Uinit, kappa, B):
        g.set_params(kappa, B)
        g.set_state(torch.from_numpy(Uinit).cuda())
        g.rk_steps(0.0, dt, NSTEPS)
        val = g.wall_shear()
        g.set_params(wl.phys["kappa"], wl.phys["B"])
        return val

    k0, B0 = wl.phys["kappa"], wl.phys["B"]
    eps = 1e-6
    fd_k = (loss(U, k0 + eps, B0) - loss(U, k0 - eps, B0)) / (2 * eps)
    fd_B = (loss(U, k0, B0 + eps) - loss(U, k0, B0 - eps)) / (2 * eps)
    # the state step is relative to |U| (E ~ 180): a smaller step keeps the
    # central difference's truncation error below the tolerance
    d = I.random_direction(U.shape, seed=22) * np.abs(U)
    eu = 1e-8
    fd_U = (loss(U + eu * d, k0, B0) - loss(U - eu * d, k0, B0)) / (2 * eu)
    ad_U = float((gU0.cpu().numpy() * d).sum())
    print("FD kappa", fd_k, th[0], "B", fd_B, th[1], "U0", fd_U, ad_U)
    assert abs(fd_k - th[0]) <= 1e-6 * abs(th[0])
    assert abs(fd_B - th[1]) <= 1e-6 * abs(th[1])
    assert abs(fd_U - ad_U) <= 1e-6 * abs(ad_U)


def test_autograd_bindings(ora):
    torch = torch_cuda()
    wl, o, g, X, U, dt = _setup(ora)
    U0 = torch.from_numpy(U).cuda().requires_grad_(True)
    lam = torch.from_numpy(I.random_direction(U.shape, seed=23)).cuda()
    Ut = dg.dg_operator(U0, g)
    (Ut * lam).sum().backward()
    gU = torch.empty_like(lam)
    g.vjp(lam, gU, U0.detach())
    assert torch.equal(U0.grad, gU)
    theta = torch.tensor([wl.phys["kappa"], wl.phys["B"]], dtype=torch.float64, requires_grad=True)
    U1 = torch.from_numpy(U).cuda().requires_grad_(True)
    L = dg.wall_shear_rollout(U1, theta, g, 3, dt)
    L.backward()
    assert theta.grad is not None and U1.grad is not None
    assert torch.isfinite(U1.grad).all() and bool(torch.isfinite(theta.grad).all())
