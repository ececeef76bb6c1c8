"""Shared set-up of the GPU parity tests (no method arithmetic)."""
import numpy as np

from paper_2606_18927_gb300 import dg, inputs as I


def torch_cuda():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def case(ora, spec, phys, surf_flux=1, vol_flux=0, viscous=1, law=1, precision=0, ic="tgv", rel=1e-3,
         extended=True):
    """Oracle and GPU operator on the same mesh nodes (the oracle's LGL
    nodes) and the same seeded state.  The oracle is evaluated in extended
    precision by default: the FP64 oracle's own rounding error (momentum Ut
    is a small difference of O(p0) fluxes at Mach 0.1) exceeds the FP64
    parity tolerance."""
    x, w, D = ora.lgl(spec.N)
    X = I.node_coordinates(spec, x)
    nbr = I.connectivity(spec)
    o = ora.Oracle(spec.N, X, nbr, phys, vol_flux=vol_flux, surf_flux=surf_flux, viscous=viscous, law=law,
                   extended=extended)
    g = dg.Operator(spec.N, X, nbr, phys, precision=precision, vol_flux=vol_flux, surf_flux=surf_flux,
                    viscous=viscous, law=law)
    if ic == "tgv":
        U = I.perturb(I.taylor_green(X, phys), rel=rel)
    elif ic == "tgv_shift":
        U = I.perturb(tgv_with_offset(X, phys), rel=rel)
    elif ic == "tgv_sonic":
        # mean flow at the speed of sound along x: |u_n - c| < c / 10 on part
        # of the xi faces, where Harten's entropy fix replaces |u_n - c|
        c0 = np.sqrt(phys["gamma"] * phys["p0"])
        U = I.perturb(tgv_with_offset(X, phys, offset=(c0, 0.4, 0.3)), rel=rel)
    elif ic == "channel":
        U = I.channel_profile(X, phys)
    else:
        U = I.free_stream(X, phys)
    return o, g, X, U


def tgv_with_offset(X, phys, offset=(0.7, 0.4, 0.3)):
    """Taylor-Green state plus a uniform velocity: the normal velocity stays
    away from 0 on the faces, where |u_n| in the Riemann dissipation has a
    kink (derivative tests need a differentiable point)."""
    U = I.taylor_green(X, phys)
    rho = U[0]
    u = U[1] / rho + offset[0]; v = U[2] / rho + offset[1]; w = U[3] / rho + offset[2]
    q0 = (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    p = (phys["gamma"] - 1.0) * (U[4] - 0.5 * q0)
    return I.conservative(rho, u, v, w, p, phys["gamma"])


def gpu_ut(torch, g, U):
    Ud = torch.from_numpy(U).cuda()
    Ut = torch.empty_like(Ud)
    g.time_derivative(Ut, Ud)
    torch.cuda.synchronize()
    g.check_status()
    return Ut.cpu().numpy()


def parity_per_var(a, ref):
    a = a.reshape(5, -1); ref = ref.reshape(5, -1)
    return [float(np.abs(a[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300)) for v in range(5)]


def parity(a, ref):
    """max over variables of max|a_v - ref_v| / max|ref_v|."""
    a = a.reshape(5, -1); ref = ref.reshape(5, -1)
    return max(float(np.abs(a[v] - ref[v]).max() / max(np.abs(ref[v]).max(), 1e-300)) for v in range(5))
