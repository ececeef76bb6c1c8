"""The double-float lifting kernel (FP64 viscous form at odd N, the
library's default there, dg_set_lifting_arithmetic(1)) against the
extended-precision oracle and against the FP64 lifting kernel (mode 0): FP64
parity bound 1e-12 in the relative max norm per variable, on the cases of the
FP64 parity suite at N = 7 (curved meshes, Roe with sonic states, walls with
the wall model, inflow / outflow, the entropy-conserving flux with
Sutherland's law) and on the full-size benchmark case (sampled elements)."""
import numpy as np
import pytest

from paper_2606_18927_gb300 import dg, inputs as I
from gpu_helpers import case, gpu_ut, parity, parity_per_var, torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.mark.parametrize("label,spec,surf,vol,ic,ma,suth", [
    ("n7_roe_sine", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1), 2, 0, "tgv", 0.1, False),
    ("n7_roe_affine_3x2x2", I.BoxSpec(7, 3, 2, 2), 2, 0, "tgv_shift", 0.1, False),
    ("n7_roe_sonic", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, 0, "tgv_sonic", 0.3, False),
    ("n7_llf_ma03", I.BoxSpec(7, 2, 3, 2, geometry="sine", amplitude=0.1), 1, 0, "tgv", 0.3, False),
    ("n7_ec_suth", I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.2), 2, 2, "tgv_shift", 0.3, True),
    # the other odd degrees (natural node slots)
    ("n5_roe_sine", I.BoxSpec(5, 3, 2, 2, geometry="sine", amplitude=0.2), 2, 0, "tgv_shift", 0.1, False),
    ("n3_llf_4x3x2", I.BoxSpec(3, 4, 3, 2, geometry="sine", amplitude=0.2), 1, 0, "tgv", 0.3, False),
    ("n1_roe", I.BoxSpec(1, 4, 4, 3), 2, 0, "tgv_shift", 0.1, False),
])
def test_double_float_lifting_matches_oracle(ora, label, spec, surf, vol, ic, ma, suth):
    torch = torch_cuda()
    phys = I.phys_params(Ma=ma, Re=1600.0 if not suth else 200.0, sutherland=suth)
    o, g, X, U = case(ora, spec, phys, surf_flux=surf, vol_flux=vol, ic=ic)
    ref = o.time_derivative(U)
    g.set_lifting_arithmetic(0)
    f64 = gpu_ut(torch, g, U)
    g.set_lifting_arithmetic(1)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print(label, "double-float lifting parity", e, ["%.1e" % x for x in parity_per_var(out, ref)],
          "FP64 lifting", parity(f64, ref), "between them", parity(out, f64))
    assert e <= TOL, e
    assert not np.array_equal(out, f64)  # the other kernel ran


@pytest.mark.parametrize("N", [5, 7])
def test_double_float_lifting_walls_and_boundaries(ora, N):
    torch = torch_cuda()
    wl = I.workload("channel_n5", N=N, elems=(4, 2, 2))
    o, g, X, U = case(ora, wl.spec, wl.phys, surf_flux=2, law=1, ic="channel")
    ref = o.time_derivative(U)
    g.set_lifting_arithmetic(1)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print("channel N=%d double-float lifting parity" % N, e)
    assert e <= TOL, e
    phys = I.phys_params(Ma=0.3, Re=400.0)
    g0, p0 = phys["gamma"], phys["p0"]
    rho, u, v = 1.02, 0.75, 0.05
    phys.update(U_in=np.array([rho, rho * u, rho * v, 0.0, 1.03 * p0 / (g0 - 1) + 0.5 * rho * (u * u + v * v)]),
                p_out=0.98 * p0)
    spec = I.BoxSpec(N, 2, 2, 2, geometry="sine", amplitude=0.1, periodic=(True, True, False),
                     boundary=((I.WALL, I.WALL), (I.WALL, I.WALL), (I.INFLOW, I.OUTFLOW)))
    o, g, X, U = case(ora, spec, phys, surf_flux=2, ic="tgv_shift")
    ref = o.time_derivative(U)
    g.set_lifting_arithmetic(1)
    out = gpu_ut(torch, g, U)
    e = parity(out, ref)
    print("inflow/outflow N=%d double-float lifting parity" % N, e)
    assert e <= TOL, e


def test_double_float_lifting_stages_and_mode_switch(ora):
    torch = torch_cuda()
    phys = I.phys_params(Ma=0.1, Re=1600.0)
    o, g, X, U = case(ora, I.BoxSpec(7, 2, 2, 2, geometry="sine", amplitude=0.1), phys, surf_flux=2)
    dt = o.dt(U, 0.9)
    Ud = torch.from_numpy(U).cuda()
    g.set_lifting_arithmetic(1)
    g.set_state(Ud)
    g.rk_steps(0.0, dt, 2)
    Ug = torch.empty_like(Ud)
    g.get_state(Ug)
    g.check_status()
    e = parity(Ug.cpu().numpy() - U, o.rk_steps(U, dt, 2) - U)
    print("double-float lifting, two steps (increment)", e)
    assert e <= TOL, e
    with pytest.raises(dg.DGError) as ei:
        g.set_lifting_arithmetic(2)
    assert ei.value.code == -1
