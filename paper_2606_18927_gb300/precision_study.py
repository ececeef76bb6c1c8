"""FP64 and FP32-mixed Taylor-Green runs side by side.

Advances the N = 7, 32^3 Taylor-Green vortex (Ma 0.1, Re 1600, seeded
perturbation) with LSERK4 at CFL 0.9 in both precision forms from the same
state, records the volume-averaged kinetic energy KE(t) and its dissipation
rate -dKE/dt every `every` steps, and reports how far the FP32-mixed
trajectory drifts from the FP64 one (relative error of KE and of the
dissipation rate, relative L2 of the state).  The first Ut of both forms is
also compared.

    python -m paper_2606_18927_gb300.precision_study --steps 2000 --out study.json
"""
import argparse
import json
import time

import numpy as np


def run(steps=2000, every=10, elems=None, cfl=0.9, out=None):
    import torch
    from . import dg, inputs as I

    wl = I.workload("tgv_n7_32", elems=elems)
    x, _ = dg.lgl_nodes(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U0 = torch.from_numpy(I.initial_state(wl, X)).cuda()
    ops = {}
    for name, prec in (("fp64", dg.FP64), ("fp32_mixed", dg.FP32_MIXED)):
        ops[name] = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=prec, vol_flux=wl.vol_flux,
                                surf_flux=wl.surf_flux, viscous=wl.viscous)
        ops[name].set_state(U0)
    dt = ops["fp64"].time_step(cfl)
    ut = {k: torch.empty_like(U0) for k in ops}
    for k, op in ops.items():
        op.time_derivative(ut[k], U0)
    a, b = ut["fp32_mixed"].view(5, -1), ut["fp64"].view(5, -1)
    ut_err = [float(torch.linalg.norm(a[v] - b[v]) / torch.linalg.norm(b[v])) for v in range(5)]
    rec = {k: {"t": [], "ke": [], "seconds": 0.0} for k in ops}
    for k, op in ops.items():
        t0 = time.perf_counter()
        t = 0.0
        rec[k]["t"].append(t); rec[k]["ke"].append(op.kinetic_energy())
        for it in range(steps):
            op.rk_steps(t, dt, 1)
            t += dt
            if (it + 1) % every == 0:
                rec[k]["t"].append(t); rec[k]["ke"].append(op.kinetic_energy())
        torch.cuda.synchronize()
        op.check_status()
        rec[k]["seconds"] = time.perf_counter() - t0
    tt = np.array(rec["fp64"]["t"])
    ke64, ke32 = np.array(rec["fp64"]["ke"]), np.array(rec["fp32_mixed"]["ke"])
    eps64, eps32 = -np.gradient(ke64, tt), -np.gradient(ke32, tt)
    Uf = {k: torch.empty_like(U0) for k in ops}
    for k, op in ops.items():
        op.get_state(Uf[k])
    dU = (Uf["fp32_mixed"] - Uf["fp64"]).view(5, -1)
    state_err = [float(torch.linalg.norm(dU[v]) / torch.linalg.norm(Uf["fp64"].view(5, -1)[v])) for v in range(5)]
    result = {
        "workload": wl.name, "N": wl.spec.N, "elements": [wl.spec.nx, wl.spec.ny, wl.spec.nz],
        "steps": steps, "dt": dt, "t_end": float(tt[-1]),
        "ut0_rel_l2_mixed_vs_fp64": ut_err,
        "ke_rel_err_max": float(np.max(np.abs(ke32 - ke64) / np.abs(ke64))),
        "dissipation_rel_err_max": float(np.max(np.abs(eps32 - eps64)) / np.max(np.abs(eps64))),
        "state_rel_l2_end": state_err,
        "seconds": {k: rec[k]["seconds"] for k in rec},
        "t": tt.tolist(), "ke_fp64": ke64.tolist(), "ke_fp32_mixed": ke32.tolist(),
        "dissipation_fp64": eps64.tolist(), "dissipation_fp32_mixed": eps32.tolist(),
    }
    for op in ops.values():
        op.close()
    if out:
        with open(out, "w") as f:
            json.dump(result, f)
    return result


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--elems", type=int, nargs=3, default=None)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    r = run(args.steps, args.every, tuple(args.elems) if args.elems else None, out=args.out)
    short = {k: v for k, v in r.items() if not isinstance(v, list) or len(v) <= 5}
    print(json.dumps(short))


if __name__ == "__main__":
    main()
