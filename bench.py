"""Throughput of the GB300 DGSEM operator: DOF-stage updates/s and PID.

One step = one LSERK4 stage (lifting, face fluxes incl. Riemann solver,
split-form volume integral, surface integral, 1/J scaling and the fused RK
register update) of the whole mesh.  Default workload: Taylor-Green vortex,
N = 7, 32^3 affine periodic elements (16.8M DOF), KEP (Pirozzoli) volume
flux, Roe surface flux, BR1 lifting, FP64 (paper Sec. 2.3 measures the PID of
the N = 7 split-form DGSEM; Eq. for PID: wall time / (DOF * stages)).

Launch: python bench.py [--gpus N --steps K --warmup W] [--precision fp64|fp32]
        [--impl ours|reference]
Under torchrun every rank runs an independent replica of the workload on its
own GPU (the single-GPU operator has no collective); value = DOF-stage
updates of all ranks / max time over ranks ("scaling": "weak").

--impl reference times the plain FP64 CPU oracle (the reference arm) on the
host cores on a bounded sample of the same workload (N = 7, 8^3 elements).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-stage updates/s (PID ns/DOF) at N=7"
UNIT = "DOF-stage/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe of a GB300 SM: 2 DFMA per clock per SM (1 instruction/clock per
# 16 lanes); 152 SMs at the 2070 MHz maximum clock: 152 * 2 * 2 * 2.07e9.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_BYTES = 129e6  # GB300 L2 (nominal)
# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu
# capture of the same kernel build on a 16^3-element case, scaled to the
# launch size by the DOF count (traffic is proportional to the DOF count).
NCU_TRAFFIC_PER_DOF = {("k_volume", "fp64", 7): (830.92e6 + 157.87e6) / 2097152,
                       ("k_volume", "fp32", 7): (308.59e6 + 204.15e6) / 2097152}
# algorithmic HBM bytes per DOF of the FP32-mixed volume kernel (stage form):
# U read 40 and written 40, dU read and written 80, FP32 primitives and the
# velocity's low parts read 36 and written 36, Ja + 1/J 40, R_v 16, surface
# fluxes 3 n^2 / n^3 x 5 x 4 B x 2 sides
MIXED_VOLUME_BYTES_PER_DOF = lambda N: 40 + 40 + 80 + 36 + 36 + 40 + 16 + 3.0 / (N + 1) * 5 * 4 * 2


def algorithmic_flops_per_dof(N, kernel, viscous=True, surf="roe", stored_prims=None, pair_sums=None):
    """Algorithmic FP64 flops per DOF and operator evaluation (FMA = 2).

    Counted on the formulas of the operator, independent of how a kernel
    schedules them (each unordered two-point pair once, as the split form
    with a symmetric flux allows).  The primitive recovery is counted where it
    runs: in the FP64 viscous form (stored_prims, the default there) once per
    node in the lifting window, which stores them for the face and volume
    kernels.  The FP64 volume kernel at N = 7 reads each pair's metric sum,
    stored with the mesh (pair_sums, the default there): those 3 additions
    are not counted."""
    n = N + 1
    if stored_prims is None:
        stored_prims = viscous
    if pair_sums is None:
        pair_sums = N == 7
    if kernel == "volume":
        pairs = 3 * N / 2.0                     # unordered pairs per node, 3 directions
        pair = 6 + (0 if pair_sums else 3) + 5 + 1 + 9 + 1 + 20  # averages, metric sum, u.a, m, F_m, F_E, 2 x 5 FMA
        prim = 1 if stored_prims else 13        # 4 p' (stored) | 1/rho, u, |u|^2, p, h
        surf_int = (6.0 / n) * 5 * 2            # face nodes per DOF x 5 FMA
        return pairs * pair + prim + (4 if viscous else 0) + surf_int + 5 + 20
    if kernel == "lift":
        if not viscous:
            return 0.0
        # the event window holds k_prim64 (the primitives of each node, 13,
        # read by the lifting kernel at the node and at the neighbours' face
        # nodes) and k_lift.  12 line contractions of the gradient and 12 of
        # the weak divergence per node; with an even node count in their
        # even/odd form (D is centro-antisymmetric): n/2 FMA, one addition
        # forming the half-sums, one combining the halves, instead of n FMA;
        # the divergence adds the three directions (8).  With the metric
        # products Ja / J and (Ja Ja^T) / J stored: velocity gradients 9 x 5,
        # the projected temperature gradient 3 x 5, the stress tensor 17, the
        # contravariant momentum fluxes 9 x 5 and energy fluxes 3 x 7
        contr = 12 * (n + 2) if n % 2 == 0 else 24 * n
        return 13 + contr + (6.0 / n) * 24 + 45 + 15 + 17 + 45 + 21 + contr + (8 if n % 2 == 0 else 0)
    if kernel == "face":
        # (both sides' primitives 26 unless stored) + two-point flux 25 + dissipation + viscous average + scaling
        per_node = (0 if stored_prims else 26) + 25 + (80 if surf == "roe" else 12) + 8 + 10
        return (3.0 / n) * per_node
    return 0.0


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def build_case(wl_name, precision, lgl, elems=None):
    from paper_2606_18927_gb300 import inputs as I
    wl = I.workload(wl_name, elems=elems)
    x, _ = lgl(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U = I.initial_state(wl, X)
    return wl, X, nbr, U


def cpu_reference_run(steps, warmup, sample_elems=8, budget_s=None):
    """Oracle timing on the host cores: RK stages on an N = 7, sample^3
    element TGV box (same per-DOF work as the 32^3 workload)."""
    import oracle
    from paper_2606_18927_gb300 import inputs as I
    wl = I.workload("tgv_n7_32", elems=(sample_elems,) * 3)
    x, w, D = oracle.lgl(wl.spec.N)
    X = I.node_coordinates(wl.spec, x)
    nbr = I.connectivity(wl.spec)
    U = I.initial_state(wl, X)
    o = oracle.Oracle(wl.spec.N, X, nbr, wl.phys, vol_flux=wl.vol_flux, surf_flux=wl.surf_flux)
    cores = oracle.max_threads()
    dt = o.dt(U, 0.9)
    dU = np.zeros_like(U)
    Uc = U.copy()
    for s in range(warmup):
        o.rk_stage(Uc, dU, s % 5, 0.0, dt)
    t0 = time.perf_counter()
    done = 0
    for s in range(steps):
        o.rk_stage(Uc, dU, s % 5, 0.0, dt)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    dofs = wl.spec.dofs
    return {"value": dofs * done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "N=7 TGV on %d^3 elements (%d DOF), %d RK stages, Roe/KEP/BR1, FP64, %d OpenMP threads"
                      % (sample_elems, dofs, done, cores),
            "seconds": el, "stages": done, "dofs": dofs}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r = cpu_reference_run(args.steps, args.warmup, budget_s=None)
    ms = 1e3 * r["seconds"] / r["stages"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": r["stages"],
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tgv_n7 (CPU oracle sample: N=7, 8^3 elements)", "N": 7,
                   "elements": [8, 8, 8], "dofs": r["dofs"], "surf_flux": "roe", "vol_flux": "kep_pirozzoli",
                   "pid_ns": 1e9 / r["value"]},
        "impl": "reference",
        "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def max_over_ranks(value, dist=None, device=None):
    """Maximum of a per-rank float over all ranks (the slowest rank's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(dofs_per_rank, steps, world, max_ms):
    """Whole-job DOF-stage updates per second: every rank advances its own
    replica, so the job processes world * dofs * steps in the slowest rank's
    time."""
    return world * dofs_per_rank * steps / (max_ms * 1e-3)


def measure_variants(args, wl, X, nbr, U, op64, stream, dt):
    """FP32-mixed form on the same workload (throughput and its Ut error
    against the FP64 path), and the time of one FP64 VJP."""
    import torch
    from paper_2606_18927_gb300 import dg
    out = {}
    Ud = torch.from_numpy(U).cuda()
    ref = torch.empty_like(Ud)
    op64.time_derivative(ref, Ud)
    # VJP of the operator (FP64, hand-written adjoint)
    lam = torch.ones_like(Ud)
    gU = torch.empty_like(Ud)
    free0 = torch.cuda.mem_get_info()[0]
    op64.vjp(lam, gU, Ud)
    torch.cuda.synchronize()
    vjp_scratch = free0 - torch.cuda.mem_get_info()[0]
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        op64.vjp(lam, gU, Ud)
    e1.record(stream)
    torch.cuda.synchronize()
    out["vjp_fp64"] = {"ms_per_call": e0.elapsed_time(e1) / 3, "scratch_gb": vjp_scratch / 1e9}
    if wl.spec.periodic[1] is False or not all(wl.spec.periodic):
        # wall-modelled channel: 20-step rollout VJP of the mean wall shear
        gth = torch.zeros(2, dtype=torch.float64, device="cuda")
        op64.rollout_vjp(Ud, 2, dt, gU, gth)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        e0.record(stream)
        loss = op64.rollout_vjp(Ud, 20, dt, gU, gth)
        e1.record(stream)
        torch.cuda.synchronize()
        out["rollout_vjp_20_steps"] = {"ms": e0.elapsed_time(e1), "loss": loss,
                                       "dloss_dkappa": float(gth[0]), "dloss_dB": float(gth[1]),
                                       "checkpoint_gb": (free1 - torch.cuda.mem_get_info()[0]) / 1e9}
    if wl.spec.periodic[1] is False or not all(wl.spec.periodic):
        # the same stages with the wall-model kernel in line on one stream
        # (the timed run has it on its own high-priority stream beside the
        # lifting and the faces)
        op64.set_state(Ud)
        op64.set_overlap(False)
        op64.profile_enable(True)
        e0.record(stream)
        for s in range(args.steps):
            op64.rk_stage(s % 5, 0.0, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = op64.profile_read()
        op64.profile_enable(False)
        op64.set_overlap(True)
        ms = e0.elapsed_time(e1) / args.steps
        out["fp64_wall_in_line"] = {"ms_per_step": ms, "value": wl.spec.dofs / (ms * 1e-3), "unit": UNIT,
                                        "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None)
                                                                  for k, v in prof.items()}}
    # whole LSERK4 steps replayed from a CUDA graph (launch overhead removed)
    op64.set_state(Ud)
    op64.rk_steps_graph(0.0, dt, 1)
    torch.cuda.synchronize()
    nst = max(1, args.steps // 5)
    e0.record(stream)
    op64.rk_steps_graph(0.0, dt, nst)
    e1.record(stream)
    torch.cuda.synchronize()
    out["fp64_graph_replay"] = {"ms_per_stage": e0.elapsed_time(e1) / (5 * nst), "steps": nst}
    if wl.spec.N == 7 and wl.viscous:
        # the same stages with the FP64 lifting kernel instead of the
        # double-float one (the other lifting arithmetic of the FP64 form)
        other = 0 if args.lifting == "df" else 1
        op64.set_lifting_arithmetic(other)
        op64.set_state(Ud)
        for s in range(3):
            op64.rk_stage(s, 0.0, dt)
        op64.profile_enable(True)
        e0.record(stream)
        for s in range(args.steps):
            op64.rk_stage(s % 5, 0.0, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = op64.profile_read()
        op64.profile_enable(False)
        op64.set_lifting_arithmetic(1 - other)
        ms = e0.elapsed_time(e1) / args.steps
        out["fp64_lifting_" + ("fp64" if other == 0 else "df")] = {
            "ms_per_step": ms, "value": wl.spec.dofs / (ms * 1e-3), "unit": UNIT,
            "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}}
    # FP32-mixed form
    free2 = torch.cuda.mem_get_info()[0]
    opm = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=dg.FP32_MIXED, vol_flux=wl.vol_flux,
                      surf_flux=wl.surf_flux, viscous=wl.viscous, law=wl.law, stream=stream)
    mixed_footprint = free2 - torch.cuda.mem_get_info()[0]
    utm = torch.empty_like(Ud)
    opm.time_derivative(utm, Ud)
    a = utm.view(5, -1); b = ref.view(5, -1)
    dn = [float(torch.linalg.norm(a[v] - b[v])) for v in range(5)]
    bn = [float(torch.linalg.norm(b[v])) for v in range(5)]
    rel = [dn[v] / bn[v] for v in range(5)]
    # (the whole vector's norm from the rows' norms)
    rel_all = (sum(x * x for x in dn) / sum(x * x for x in bn)) ** 0.5
    opm.set_state(Ud)
    for s in range(args.warmup):
        opm.rk_stage(s % 5, 0.0, dt)
    torch.cuda.synchronize()
    opm.profile_enable(True)
    e0.record(stream)
    for s in range(args.steps):
        opm.rk_stage(s % 5, 0.0, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    prof = opm.profile_read()
    opm.profile_enable(False)
    opm.check_status()
    dofs = wl.spec.dofs
    kms = {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}
    hbm = load_peaks().get("hbm_gbs", 6800.0)
    vol_gbs = MIXED_VOLUME_BYTES_PER_DOF(wl.spec.N) * dofs / (kms["volume"] * 1e-3) / 1e9 if kms["volume"] else None
    out["fp32_mixed"] = {"value": dofs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "pid_ns": ms * 1e6 / dofs,
                         "ut_rel_l2_vs_fp64_per_var": rel, "ut_rel_l2_vs_fp64": rel_all,
                         "dtype": "f32 fluxes, f64 state / RK / pressure recovery",
                         "footprint_gb": mixed_footprint / 1e9, "kernels_ms_per_launch": kms,
                         "volume_roofline": {"bound": "hbm", "achieved": vol_gbs, "peak": hbm, "unit": "GB/s",
                                             "frac": vol_gbs / hbm if vol_gbs else None,
                                             "bytes_per_dof": MIXED_VOLUME_BYTES_PER_DOF(wl.spec.N)}}
    opm.close()
    # the production scheme of Sec. 4: entropy-conserving volume flux, Roe +
    # Harten at the faces, Sutherland viscosity (same mesh and state)
    phys_ec = dict(wl.phys)
    phys_ec.update(T_ref=phys_ec["p0"], suth_S=phys_ec["p0"] * 110.4 / 288.15)
    for name, prec in (("fp64_ec_roe_sutherland", dg.FP64), ("fp32_mixed_ec_roe_sutherland", dg.FP32_MIXED)):
        ope = dg.Operator(wl.spec.N, X, nbr, phys_ec, precision=prec, vol_flux=dg.VOL_EC_CHANDRASHEKAR,
                          surf_flux=dg.SURF_ROE, viscous=wl.viscous, law=wl.law, stream=stream)
        ope.set_state(Ud)
        for s in range(args.warmup):
            ope.rk_stage(s % 5, 0.0, dt)
        torch.cuda.synchronize()
        ope.profile_enable(True)
        e0.record(stream)
        for s in range(args.steps):
            ope.rk_stage(s % 5, 0.0, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        prof = ope.profile_read()
        ope.profile_enable(False)
        ope.check_status()
        out[name] = {"value": dofs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "pid_ns": ms * 1e6 / dofs,
                     "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}}
        ope.close()
    del utm, ref, gU, lam
    return out


def run_ours(args):
    import torch
    from paper_2606_18927_gb300 import dg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    precision = dg.FP32_MIXED if args.precision == "fp32" else dg.FP64
    wl, X, nbr, U = build_case(args.workload, precision, dg.lgl_nodes,
                               elems=tuple(args.elems) if args.elems else None)
    stream = torch.cuda.current_stream()
    Ud = torch.from_numpy(U).cuda()
    torch.cuda.synchronize()
    # device memory of the operator context alone (mesh, metrics, U, dU, scratch)
    free0 = torch.cuda.mem_get_info()[0]
    op = dg.Operator(wl.spec.N, X, nbr, wl.phys, precision=precision, vol_flux=wl.vol_flux,
                     surf_flux=wl.surf_flux, viscous=wl.viscous, law=wl.law, stream=stream)
    if wl.spec.N == 7 and wl.viscous and precision == dg.FP64:
        op.set_lifting_arithmetic(1 if args.lifting == "df" else 0)
    op.set_state(Ud)
    footprint = free0 - torch.cuda.mem_get_info()[0]
    dofs = wl.spec.dofs
    # explicit time step from the CFL rule (CFL 0.9, paper Sec. 4)
    dt = op.time_step(0.9)
    for s in range(args.warmup):
        op.rk_stage(s % 5, 0.0, dt)
    torch.cuda.synchronize()
    op.check_status()

    # ---- timed region: K stages on device-resident data
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        op.rk_stage(s % 5, 0.0, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    # the same K stages again with the per-kernel events on, for the breakdown and
    # the roofline (the events add a record per launch, so the headline loop above
    # runs without them)
    op.profile_enable(True)
    e0.record(stream)
    for s in range(args.steps):
        op.rk_stage(s % 5, 0.0, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_profiled = e0.elapsed_time(e1)
    prof = op.profile_read()
    op.profile_enable(False)
    clk = clocks.stop()
    op.check_status()
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    value = job_throughput(dofs, args.steps, world, ms_total)

    # ---- end to end through the public API with host buffers: every step
    # copies its input state in from page-locked host memory and its result
    # out (dg_rk_stage_batch: the copies of the neighbouring steps overlap
    # the computation of the current one)
    Uh = torch.from_numpy(U).pin_memory()
    outs = [torch.empty_like(Uh).pin_memory() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 20))
    op.rk_stage_batch([Uh.numpy()] * 2, [o.numpy() for o in outs], 1, 0.0, dt)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    op.rk_stage_batch([Uh.numpy()] * e2e_steps, [outs[s % 2].numpy() for s in range(e2e_steps)], 1, 0.0, dt)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = job_throughput(dofs, e2e_steps, world, e2e_s * 1e3)
    nbytes = U.nbytes

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    variants = {}
    if world == 1 and precision == dg.FP64 and not args.no_variants:
        variants = measure_variants(args, wl, X, nbr, U, op, stream, dt)

    # ---- roofline of the dominant kernel
    kernels = {}
    for k, (ms, cnt) in prof.items():
        if cnt:
            flops = algorithmic_flops_per_dof(wl.spec.N, k, bool(wl.viscous), "roe" if wl.surf_flux == 2 else "llf",
                                              stored_prims=bool(wl.viscous) and precision == dg.FP64)
            avg = ms / cnt
            kernels[k] = {"ms_per_launch": avg, "launches": cnt, "share": ms / max(ms_profiled, 1e-30),
                          "flops_per_dof": flops,
                          "achieved_tflops": flops * dofs / (avg * 1e-3) / 1e12 if flops else None}
    # the dominant kernel among those with a flop model (the wall-model kernel,
    # whose work depends on its Newton iterations, runs beside them on a side
    # stream and its event time stretches with the overlap)
    modelled = [k for k in kernels if kernels[k]["flops_per_dof"]] or list(kernels)
    dom = max(modelled, key=lambda k: kernels[k]["ms_per_launch"] * kernels[k]["launches"])
    peaks = load_peaks()
    if precision == dg.FP64:
        achieved = kernels[dom]["achieved_tflops"]
        tpd = NCU_TRAFFIC_PER_DOF.get(("k_" + dom, "fp64", wl.spec.N))
        roof = {"bound": "alu", "kernel": "k_" + dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": tpd * dofs if tpd else None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 pipe)"}
    else:
        # the mixed form's dominant kernel is the volume kernel, against HBM
        hbm = peaks.get("hbm_gbs", 6800.0)
        vol = kernels.get("volume")
        ach = (MIXED_VOLUME_BYTES_PER_DOF(wl.spec.N) * dofs / (vol["ms_per_launch"] * 1e-3) / 1e9) if vol else None
        tpd = NCU_TRAFFIC_PER_DOF.get(("k_volume", "fp32", wl.spec.N))
        roof = {"bound": "hbm", "kernel": "k_volume", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm if ach else None, "traffic": tpd * dofs if tpd else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    # (the FP64 viscous form's lift window holds two launches, k_prim64 and k_lift)
    launches_per_step = sum(2 if (k == "lift" and precision == dg.FP64) else 1 for k in kernels)
    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        r = cpu_reference_run(10 ** 6, 1, sample_elems=8, budget_s=args.cpu_seconds)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == dg.FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.spec.N, "elements": [wl.spec.nx, wl.spec.ny, wl.spec.nz],
                   "dofs": dofs, "precision": args.precision, "vol_flux": "kep_pirozzoli",
                   "surf_flux": {0: "central", 1: "llf", 2: "roe"}[wl.surf_flux], "lifting": "br1",
                   "lifting_arithmetic": ("double-float (FP32 pipe, error-free transformations)"
                                          if wl.spec.N == 7 and wl.viscous and precision == dg.FP64
                                          and args.lifting == "df" else "fp64"),
                   "pid_ns": 1e9 / (value / world), "l2": ("inputs larger than L2 (U alone %.0f MB)" % (nbytes / 1e6) if nbytes > L2_BYTES
                          else "inputs smaller than L2 (U %.0f MB), no flush: a small parity-size case, "
                               "not a headline workload" % (nbytes / 1e6)),
                   "footprint_gb": footprint / 1e9, "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": e2e_steps, "api": "dg_rk_stage_batch (copies overlapped, 2 device slots)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "variants": variants,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--workload", default="tgv_n7_32")
    ap.add_argument("--elems", type=int, nargs=3, default=None,
                    help="element counts of a smaller case of the same workload (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lifting", choices=["fp64", "df"], default="df",
                    help="arithmetic of the FP64 form's lifting kernel at N = 7 (df: double-float, the "
                         "library's default there; fp64: the FP64 kernel)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32-mixed and VJP measurements appended to the line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
