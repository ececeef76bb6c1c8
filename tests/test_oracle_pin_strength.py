"""Strength of the oracle's pins: each test here plants one plausible
mistake in a copy of the oracle's source (a sign, a factor, a missing
absolute value or average, a transposed index), builds that copy with the
oracle's own compiler flags, and requires that at least one pin rejects it.

* Roe solver (paper Sec. 4: Roe with Harten's entropy fix): the pins of
  `test_oracle_fluxes` (Roe's property on supersonic states, the single-wave
  dissipations on subsonic states, the fixed wave speed inside Harten's band).
* The operator (Sec. 2.2: split-form DGSEM, BR1 lifting, viscous fluxes):
  the invariants (metric identities, free stream, conservation, kinetic
  energy), the point-flux symmetry, the manufactured-solution convergence
  and the BR1 closed forms (temperature and shear), run on the planted copy
  in place of the oracle's library.
* The models (Sec. 3 wall model, Sec. 4 entropy-conserving flux, Sutherland's
  law, LSERK4, the inflow / outflow and isothermal-wall boundaries): their
  pins (Tadmor's condition, the air table, the LSERK4 order conditions, the
  Van Driest chain and the isothermal wall's limits, free stream through the
  boundaries and the energy balance).
* The geometry, the basis and the derivatives (LGL weights and derivative
  matrix, the curl-form metrics, the face normals, the Lagrange basis of the
  wall samples, the dual numbers of the forward-mode derivative, the
  implicit-function-theorem derivative of the wall-law solve, the LSERK4
  register update): the basis closed forms and exactness, the metric
  identities and affine metrics, free stream and conservation (also through
  inflow / outflow faces), the rotated element frames, the wall-sample
  geometry, the JVPs against central differences (state, wall-law
  constants, a rollout's loss) and the temporal order of LSERK4.
* General conforming meshes (the face node maps of the orientation codes):
  rotated element frames against the structured mesh, free stream,
  conservation and the wall model across rotated elements, and the
  rejection of inconsistent connectivity (built in both arithmetics, since
  those pins run the extended build).

The unchanged source built the same way must pass all of them (the
controls)."""
import concurrent.futures as cf
import contextlib
import ctypes
import hashlib
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_basis as basis
import test_oracle_boundaries as bnd
import test_oracle_derivatives as deriv
import test_oracle_fluxes as fluxes
import test_oracle_invariants as inv
import test_oracle_lifting as lifting
import test_oracle_mms as mms_tests
import test_oracle_orientation as orient
import test_oracle_wall_samples as wsamp
from test_oracle_fluxes import (check_roe_acoustic_wave, check_roe_entropy_fix, check_roe_linear_wave,
                                check_roe_supersonic, test_consistency_and_symmetry)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dgsem_oracle.cpp")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")

# (name, text in the Roe solver, planted replacement)
MUTANTS = [
    ("entropy_and_shear_waves_not_upwinded",
     "T l1 = fabs(un - ct), l2 = fabs(un), l5 = fabs(un + ct);",
     "T l1 = fabs(un - ct), l2 = un, l5 = fabs(un + ct);"),
    ("acoustic_strength_sign",
     "T a1 = (dp - rt * ct * dun) / (2.0 * c2);",
     "T a1 = (dp + rt * ct * dun) / (2.0 * c2);"),
    ("entropy_strength_sign",
     "T a2 = drho - dp / c2;",
     "T a2 = drho + dp / c2;"),
    ("shear_tangential_projection_sign",
     "for (int c = 0; c < 3; ++c) Dd[1 + c] += l2 * rt * (du[c] - dun * nh[c]);",
     "for (int c = 0; c < 3; ++c) Dd[1 + c] += l2 * rt * (du[c] + dun * nh[c]);"),
    ("entropy_wave_energy_factor",
     "Dd[4] += l2 * a2 * 0.5 * q2;",
     "Dd[4] += l2 * a2 * q2;"),
    ("right_acoustic_eigenvector_sign",
     "for (int c = 0; c < 3; ++c) Dd[1 + c] += l5 * a5 * (ut[c] + ct * nh[c]);",
     "for (int c = 0; c < 3; ++c) Dd[1 + c] += l5 * a5 * (ut[c] - ct * nh[c]);"),
    ("left_acoustic_enthalpy_sign",
     "Dd[4] = l1 * a1 * (Ht - ct * un);",
     "Dd[4] = l1 * a1 * (Ht + ct * un);"),
    ("roe_average_weights_swapped",
     "T Ht = (sL * L.h + sR * R.h) / (sL + sR);",
     "T Ht = (sR * L.h + sL * R.h) / (sL + sR);"),
    ("harten_band_width",
     "T delta = 0.1 * ct;",
     "T delta = 0.2 * ct;"),
    ("harten_fixed_speed_factor",
     "if (val(l5) < val(delta)) l5 = (l5 * l5 + delta * delta) / (2.0 * delta);",
     "if (val(l5) < val(delta)) l5 = (l5 * l5 + delta * delta) / delta;"),
]


def _build(text, extended=False):
    os.makedirs(OUT, exist_ok=True)
    tag = hashlib.sha1(text.encode()).hexdigest()[:16] + ("_ext" if extended else "")
    lib = os.path.join(OUT, "libora_%s.so" % tag)
    if not os.path.exists(lib):
        src = os.path.join(OUT, "ora_%s.cpp" % tag)
        with open(src, "w") as f:
            f.write(text)
        tmp = lib + ".tmp%d" % os.getpid()
        defines = ["-DORA_REAL=long double"] if extended else []
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared"] +
                              defines + [src, "-o", tmp])
        os.replace(tmp, lib)
    return lib


@pytest.fixture(scope="module")
def libs():
    with open(SRC) as f:
        base = f.read()
    texts = {"control": base}
    for name, old, new in MUTANTS:
        assert base.count(old) == 1, name
        texts[name] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        paths = dict(zip(texts, ex.map(_build, texts.values())))
    return paths


def _riemann_of(path):
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    L.ora_riemann.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]

    def riemann(phys, vol_kind, kind, UL, UR, nh):
        pa = np.ascontiguousarray(oracle.phys_array(phys), dtype=np.float64)
        UL = np.ascontiguousarray(UL, dtype=np.float64)
        UR = np.ascontiguousarray(UR, dtype=np.float64)
        nh = np.ascontiguousarray(nh, dtype=np.float64)
        F = np.zeros(5)
        L.ora_riemann(pa.ctypes.data_as(dp), int(vol_kind), int(kind), UL.ctypes.data_as(dp),
                      UR.ctypes.data_as(dp), nh.ctypes.data_as(dp), F.ctypes.data_as(dp))
        return F
    return riemann


CHECKS = [
    ("supersonic +", lambda r: check_roe_supersonic(r, 1.0)),
    ("supersonic -", lambda r: check_roe_supersonic(r, -1.0)),
    ("contact", lambda r: check_roe_linear_wave(r, "contact")),
    ("shear", lambda r: check_roe_linear_wave(r, "shear")),
    ("acoustic -", lambda r: check_roe_acoustic_wave(r, -1.0)),
    ("acoustic +", lambda r: check_roe_acoustic_wave(r, 1.0)),
    ("entropy fix -", lambda r: check_roe_entropy_fix(r, -1.0)),
    ("entropy fix +", lambda r: check_roe_entropy_fix(r, 1.0)),
]


def _failing(riemann):
    failed = []
    for name, chk in CHECKS:
        try:
            chk(riemann)
        except AssertionError:
            failed.append(name)
    return failed


def test_control_passes_every_pin(libs):
    assert _failing(_riemann_of(libs["control"])) == []


@pytest.mark.parametrize("mutant", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(libs, mutant):
    failed = _failing(_riemann_of(libs[mutant]))
    print(mutant, "rejected by", failed)
    assert failed, mutant


# ---------------------------------------------------------------------------
# the operator
# ---------------------------------------------------------------------------
OPERATOR_MUTANTS = [
    ("pirozzoli_enthalpy_one_sided",
     "T h = 0.5 * (L.h + R.h);",
     "T h = L.h;"),
    ("pirozzoli_pressure_sign",
     "for (int c = 0; c < 3; ++c) F[1 + c] = rho * ua * u[c] + p * a[c];",
     "for (int c = 0; c < 3; ++c) F[1 + c] = rho * ua * u[c] - p * a[c];"),
    ("volume_metric_not_averaged",
     "for (int c = 0; c < 3; ++c) abar[c] = 0.5 * (jao[dir * 3 + c] + jam[dir * 3 + c]);",
     "for (int c = 0; c < 3; ++c) abar[c] = jao[dir * 3 + c];"),
    ("volume_factor_two_dropped",
     "for (int v = 0; v < 5; ++v) V[v] += 2.0 * Dim * F[v];",
     "for (int v = 0; v < 5; ++v) V[v] += Dim * F[v];"),
    ("viscous_volume_term_sign",
     "V[v] -= Dim * W.G[",
     "V[v] += Dim * W.G["),
    ("br1_average_one_sided",
     "T Ws = 0.5 * (Wo[w] + Wn[w]);",
     "T Ws = Wn[w];"),
    ("lifting_surface_weight_inverted",
     "(Ws - Wo[w]) * ns[d] * invJ / wperp;",
     "(Ws - Wo[w]) * ns[d] * invJ * wperp;"),
    ("stress_transposed_index",
     "tau[i][j] = mu * (g[j][i] + g[i][j]);",
     "tau[i][j] = mu * (g[j][i] + g[j][i]);"),
    ("stress_bulk_factor",
     "if (i == j) tau[i][j] -= (2.0 / 3.0) * mu * div;",
     "if (i == j) tau[i][j] -= (1.0 / 3.0) * mu * div;"),
    ("heat_flux_sign",
     "+ kcond * g[d][3];",
     "- kcond * g[d][3];"),
    ("face_viscous_flux_one_sided",
     "for (int v = 0; v < 5; ++v) Fv[v] = 0.5 * (Fa[v] + Fb[v]);",
     "for (int v = 0; v < 5; ++v) Fv[v] = Fa[v];"),
]


@pytest.fixture(scope="module")
def operator_libs():
    with open(SRC) as f:
        base = f.read()
    texts = {"control": base}
    for name, old, new in OPERATOR_MUTANTS:
        assert base.count(old) == 1, name
        texts[name] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        paths = dict(zip(texts, ex.map(_build, texts.values())))
    return paths


@pytest.fixture(scope="module")
def mms_sources():
    return mms_tests._mms_source(), mms_tests._mms_source(mu=0.0)


@contextlib.contextmanager
def _oracle_with(path):
    """The oracle module with its FP64 library replaced by the build at path."""
    saved = oracle._libs.get(False)
    oracle._libs[False] = oracle.bind(path)
    try:
        yield oracle
    finally:
        if saved is None:
            oracle._libs.pop(False, None)
        else:
            oracle._libs[False] = saved


def _operator_checks(sources):
    ns, euler = sources
    return [
        ("point-flux symmetry", lambda o: [test_consistency_and_symmetry(o, v, k) for v in (0, 1) for k in (0, 2)]),
        ("metric identities", lambda o: inv.test_metric_identities(o, "sine", 3)),
        ("free stream", lambda o: inv.test_free_stream_sine_mesh(o, 3, 2, 0.8)),
        ("conservation", lambda o: [inv.test_discrete_conservation(o, vs, sf) for vs, sf in ((0, 1), (1, 2))]),
        ("kinetic energy", lambda o: inv.test_kinetic_energy_preservation(o, 0)),
        ("MMS Euler N=3", lambda o: mms_tests.test_manufactured_solution_convergence_euler(o, euler, 3)),
        ("MMS Navier-Stokes N=3", lambda o: mms_tests.test_manufactured_solution_convergence(o, ns, 3)),
        ("BR1 closed form N=3", lambda o: lifting.test_br1_piecewise_constant_temperature(o, 3)),
        ("BR1 shear closed form N=3", lambda o: lifting.test_br1_piecewise_constant_shear(o, 3)),
    ]


def _operator_failing(path, sources):
    failed = []
    with _oracle_with(path) as o:
        for name, chk in _operator_checks(sources):
            try:
                chk(o)
            except AssertionError:
                failed.append(name)
    return failed


def test_operator_control_passes_every_pin(operator_libs, mms_sources):
    assert _operator_failing(operator_libs["control"], mms_sources) == []


@pytest.mark.parametrize("mutant", [m[0] for m in OPERATOR_MUTANTS])
def test_planted_operator_mistake_is_caught(operator_libs, mms_sources, mutant):
    failed = _operator_failing(operator_libs[mutant], mms_sources)
    print(mutant, "rejected by", failed)
    assert failed, mutant


# ---------------------------------------------------------------------------
# the models: entropy-conserving flux, Sutherland, LSERK4, wall model, boundaries
# ---------------------------------------------------------------------------
MODEL_MUTANTS = [
    ("sutherland_ratio_inverted",
     "return P.mu * x * sqrt(x) * (P.T_ref + P.suth_S) / (Tt + P.suth_S);",
     "return P.mu * x * sqrt(x) * (Tt + P.suth_S) / (P.T_ref + P.suth_S);"),
    ("logmean_wrong_denominator",
     "return d / log1p(d / b);",
     "return d / log1p(d / (a + b));"),
    ("ec_energy_factor_two_dropped",
     "F[4] = F[0] * (1.0 / (2.0 * (gamma - 1.0) * b_ln) - 0.5 * u2) + u[0] * F[1] + u[1] * F[2] + u[2] * F[3];",
     "F[4] = F[0] * (1.0 / ((gamma - 1.0) * b_ln) - 0.5 * u2) + u[0] * F[1] + u[1] * F[2] + u[2] * F[3];"),
    ("ec_pressure_arithmetic_mean",
     "T pt = 0.5 * (L.rho + R.rho) / (bL + bR);",
     "T pt = 0.5 * (L.p + R.p);"),
    ("lserk4_coefficient_digit",
     "5161836677717.0 / 13612068292357.0,",
     "5161836677717.0 / 13612068292367.0,"),
    ("wall_heat_flux_sign",
     "if (P.T_wall > 0.0) *qw = -(cp / P.Pr) * tw * (Taw - Tw) / umag;",
     "if (P.T_wall > 0.0) *qw = (cp / P.Pr) * tw * (Taw - Tw) / umag;"),
    ("van_driest_transform_dropped",
     "uvd = asin(a * umag) / a;",
     "uvd = umag;"),
    ("recovery_temperature_factor",
     "T Taw = s.T_ + r * u2 / (2.0 * cp);",
     "T Taw = s.T_ + r * u2 / cp;"),
    ("wall_density_temperature_ratio_inverted",
     "T rhow = s.rho * s.T_ / Tw;",
     "T rhow = s.rho * Tw / s.T_;"),
    ("reichardt_friction_velocity",
     "if (law == LAW_REICHARDT) ut = exp(tT) * nu / h;",
     "if (law == LAW_REICHARDT) ut = exp(tT) * h / nu;"),
    ("outflow_energy_factor",
     "Ub[4] = P.p_out / (P.gamma - 1.0) + 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];",
     "Ub[4] = P.p_out / P.gamma + 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];"),
    ("llf_minimum_speed",
     "T lam = val(lamL) >= val(lamR) ? lamL : lamR;",
     "T lam = val(lamL) >= val(lamR) ? lamR : lamL;"),
    ("kennedy_gruber_pressure_work_dropped",
     "F[4] = rho * ua * e + p * ua;",
     "F[4] = rho * ua * e;"),
    ("slip_wall_mirror_factor",
     "for (int c = 0; c < 3; ++c) Ub[1 + c] = U[1 + c] - 2.0 * mn * nh[c];",
     "for (int c = 0; c < 3; ++c) Ub[1 + c] = U[1 + c] - mn * nh[c];"),
    ("wall_sample_outward",
     "xs[c] = M.X[(size_t)c * K * n3 + (size_t)e * n3 + p] - hwm * nout;",
     "xs[c] = M.X[(size_t)c * K * n3 + (size_t)e * n3 + p] + hwm * nout;"),
]


@pytest.fixture(scope="module")
def model_libs():
    with open(SRC) as f:
        base = f.read()
    texts = {"control": base}
    for name, old, new in MODEL_MUTANTS:
        assert base.count(old) == 1, name
        texts[name] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        paths = dict(zip(texts, ex.map(_build, texts.values())))
    return paths


MODEL_CHECKS = [
    ("Tadmor condition", lambda o: [fluxes.test_chandrashekar_entropy_conservation(o, c) for c in (False, True)]),
    ("EC kinetic-energy form", lambda o: fluxes.test_chandrashekar_kinetic_energy_form(o)),
    ("entropy conservation", lambda o: inv.test_entropy_conservation(o, 3)),
    ("Sutherland air table", lambda o: fluxes.test_sutherland_air_table(o)),
    ("LSERK4 order conditions", lambda o: basis.test_lserk4_order_conditions(o)),
    ("Spalding as printed", lambda o: fluxes.test_spalding_as_printed(o)),
    ("Reichardt limits", lambda o: fluxes.test_reichardt_limits(o)),
    ("wall law solve", lambda o: [fluxes.test_wall_law_solve(o, law) for law in (0, 1)]),
    ("Van Driest chain", lambda o: [fluxes.test_wall_flux_van_driest_chain(o, law, Ma)
                                    for law in (0, 1) for Ma in (0.1, 0.8)]),
    ("isothermal wall model", lambda o: [fluxes.test_isothermal_wall_model(o, law, 0.8) for law in (0, 1)]),
    ("isothermal at recovery temperature", lambda o: fluxes.test_isothermal_wall_at_recovery_temperature_is_adiabatic(o)),
    ("isothermal conduction limit", lambda o: fluxes.test_isothermal_wall_laminar_conduction_limit(o)),
    ("free stream through inflow / outflow", lambda o: bnd.test_free_stream_with_inflow_outflow(o, 2, 3)),
    ("boundary flux balance", lambda o: bnd.test_boundary_flux_balance(o, 2)),
    ("energy balance, isothermal walls", lambda o: inv.test_energy_balance_with_isothermal_walls(o)),
    ("LLF dissipation bounds", lambda o: fluxes.test_llf_dissipation_bounds(o)),
    ("point-flux consistency", lambda o: [test_consistency_and_symmetry(o, v, k) for v in (0, 1, 2) for k in (0, 1, 2)]),
    ("free stream, walled channel", lambda o: inv.test_free_stream_channel_mesh(o, 3)),
    ("wall samples", lambda o: wsamp.test_channel_wall_samples(o, 3)),
]


def _model_failing(path):
    failed = []
    with _oracle_with(path) as o:
        for name, chk in MODEL_CHECKS:
            try:
                chk(o)
            except (AssertionError, RuntimeError, ValueError):
                failed.append(name)
    return failed


def test_model_control_passes_every_pin(model_libs):
    assert _model_failing(model_libs["control"]) == []


@pytest.mark.parametrize("mutant", [m[0] for m in MODEL_MUTANTS])
def test_planted_model_mistake_is_caught(model_libs, mutant):
    failed = _model_failing(model_libs[mutant])
    print(mutant, "rejected by", failed)
    assert failed, mutant


# ---------------------------------------------------------------------------
# geometry, basis, derivatives
# ---------------------------------------------------------------------------
GEOMETRY_MUTANTS = [
    ("lgl_weight_power",
     "w[i] = 2.0 / (N * (N + 1.0) * P * P);",
     "w[i] = 2.0 / (N * (N + 1.0) * P);"),
    ("derivative_matrix_barycentric_ratio",
     "D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);",
     "D[i * n + j] = (lam[i] / lam[j]) / (x[i] - x[j]);"),
    ("curl_metric_component_sign",
     "ja[1 * 3 + nn] = -(dv[0][2] - dv[2][0]);",
     "ja[1 * 3 + nn] = (dv[0][2] - dv[2][0]);"),
    ("face_normal_orientation_dropped",
     "for (int c = 0; c < 3; ++c) nh[c] = face_sign(ml) * ja[c] / ss;",
     "for (int c = 0; c < 3; ++c) nh[c] = ja[c] / ss;"),
    ("lagrange_basis_denominator",
     "real f = (s - x[k]) / (x[j] - x[k]);",
     "real f = (s - x[k]) / (x[j] + x[k]);"),
    ("dual_sqrt_derivative",
     "inline Dual sqrt(Dual a) { real s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }",
     "inline Dual sqrt(Dual a) { real s = std::sqrt(a.v); return Dual(s, a.d / s); }"),
    ("dual_quotient_rule_sign",
     "return Dual(r, (a.d - r * b.d) / b.v);",
     "return Dual(r, (a.d + r * b.d) / b.v);"),
    ("implicit_function_theorem_sign",
     "tT = T(t) - (FT - T(val(FT))) / Ft_t;",
     "tT = T(t) + (FT - T(val(FT))) / Ft_t;"),
    ("lserk4_register_update_order",
     "dU[x] = RK_A[s] * dU[x] + dt * Ut[x];",
     "dU[x] = RK_B[s] * dU[x] + dt * Ut[x];"),
]


@pytest.fixture(scope="module")
def geometry_libs():
    with open(SRC) as f:
        base = f.read()
    texts = {"control": base}
    for name, old, new in GEOMETRY_MUTANTS:
        assert base.count(old) == 1, name
        texts[name] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        paths = dict(zip(texts, ex.map(_build, texts.values())))
    return paths


GEOMETRY_CHECKS = [
    ("LGL closed forms", lambda o: basis.test_lgl_closed_forms(o, 3)),
    ("quadrature and derivative exactness", lambda o: basis.test_lgl_quadrature_and_derivative_exactness(o, 5)),
    ("summation by parts", lambda o: basis.test_summation_by_parts(o, 3)),
    ("metric identities", lambda o: inv.test_metric_identities(o, "sine", 3)),
    ("affine metrics", lambda o: inv.test_affine_metrics_closed_form(o)),
    ("free stream", lambda o: inv.test_free_stream_sine_mesh(o, 3, 2, 0.8)),
    ("conservation", lambda o: inv.test_discrete_conservation(o, 1, 2)),
    ("wall samples", lambda o: wsamp.test_channel_wall_samples(o, 3)),
    ("JVP vs central differences", lambda o: deriv.test_jvp_matches_central_differences_tgv(o, 2)),
    ("free stream through inflow / outflow", lambda o: bnd.test_free_stream_with_inflow_outflow(o, 2, 3)),
    ("rotated element frames", lambda o: orient.test_free_stream_and_conservation_on_rotated_mesh(o)),
    ("JVP of the wall-law constants", lambda o: deriv.test_jvp_wall_model_parameters(o, 1)),
    ("rollout loss derivative", lambda o: deriv.test_rollout_loss_derivative(o)),
    ("LSERK4 temporal order", lambda o: deriv.test_lserk4_temporal_order(o)),
]


def _geometry_failing(path):
    failed = []
    with _oracle_with(path) as o:
        for name, chk in GEOMETRY_CHECKS:
            try:
                chk(o)
            except (AssertionError, ValueError, RuntimeError):
                failed.append(name)
    return failed


def test_geometry_control_passes_every_pin(geometry_libs):
    assert _geometry_failing(geometry_libs["control"]) == []


@pytest.mark.parametrize("mutant", [m[0] for m in GEOMETRY_MUTANTS])
def test_planted_geometry_mistake_is_caught(geometry_libs, mutant):
    failed = _geometry_failing(geometry_libs[mutant])
    print(mutant, "rejected by", failed)
    assert failed, mutant


# ---------------------------------------------------------------------------
# general conforming meshes: face maps and orientations (their pins compare
# rotated meshes with the structured one in the extended build, so the
# planted copies are built in both arithmetics)
# ---------------------------------------------------------------------------
ORIENTATION_MUTANTS = [
    ("orientation_flip_bits_swapped",
     "const int a2 = (o & 2) ? M.N - s : s, b2 = (o & 4) ? M.N - t : t;",
     "const int a2 = (o & 4) ? M.N - s : s, b2 = (o & 2) ? M.N - t : t;"),
    ("orientation_transpose_inverted",
     "const int s = (o & 1) ? b : a, t = (o & 1) ? a : b;",
     "const int s = (o & 1) ? a : b, t = (o & 1) ? b : a;"),
    ("orientation_inverse_identity",
     "return (o & 1) ? (1 | (((o >> 2) & 1) << 1) | (((o >> 1) & 1) << 2)) : o;",
     "return o;"),
]


@pytest.fixture(scope="module")
def orientation_libs():
    with open(SRC) as f:
        base = f.read()
    texts = {"control": base}
    for name, old, new in ORIENTATION_MUTANTS:
        assert base.count(old) == 1, name
        texts[name] = base.replace(old, new)
    jobs = [(name, text, ext) for name, text in texts.items() for ext in (False, True)]
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        built = list(ex.map(lambda j: _build(j[1], j[2]), jobs))
    paths = {}
    for (name, _, ext), path in zip(jobs, built):
        paths.setdefault(name, {})[ext] = path
    return paths


@contextlib.contextmanager
def _oracle_with_both(paths):
    """The oracle module with both of its libraries replaced."""
    saved = dict(oracle._libs)
    oracle._libs[False] = oracle.bind(paths[False])
    oracle._libs[True] = oracle.bind(paths[True])
    try:
        yield oracle
    finally:
        oracle._libs.clear()
        oracle._libs.update(saved)


ORIENTATION_CHECKS = [
    ("rotated frames give the structured operator",
     lambda o: orient.test_rotated_frames_give_the_structured_operator(o, 3, 2, 1)),
    ("free stream and conservation, rotated mesh", lambda o: orient.test_free_stream_and_conservation_on_rotated_mesh(o)),
    ("wall model across rotated elements", lambda o: orient.test_wall_model_across_rotated_elements(o, 1)),
    ("inconsistent connectivity rejected", lambda o: orient.test_inconsistent_connectivity_is_rejected(o)),
]


def _orientation_failing(paths):
    failed = []
    with _oracle_with_both(paths) as o:
        for name, chk in ORIENTATION_CHECKS:
            try:
                chk(o)
            except (AssertionError, ValueError, RuntimeError):
                failed.append(name)
    return failed


def test_orientation_control_passes_every_pin(orientation_libs):
    assert _orientation_failing(orientation_libs["control"]) == []


@pytest.mark.parametrize("mutant", [m[0] for m in ORIENTATION_MUTANTS])
def test_planted_orientation_mistake_is_caught(orientation_libs, mutant):
    failed = _orientation_failing(orientation_libs[mutant])
    print(mutant, "rejected by", failed)
    assert failed, mutant
