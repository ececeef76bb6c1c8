"""Strength of the Roe-flux pins: each test here plants one plausible
mistake in a copy of the oracle's Roe solver (a sign, a factor, a missing
absolute value, swapped Roe-average weights; paper Sec. 4: Roe solver with
Harten's entropy fix), builds that copy with the oracle's own compiler
flags, and requires that at least one of the pins of `test_oracle_fluxes`
(Roe's property on supersonic states, the single-wave dissipations on
subsonic states) rejects it.  The unchanged source built the same way must
pass all of them (the control)."""
import concurrent.futures as cf
import ctypes
import hashlib
import os
import subprocess

import numpy as np
import pytest

import oracle
from test_oracle_fluxes import check_roe_acoustic_wave, check_roe_linear_wave, check_roe_supersonic

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
]


def _build(text):
    os.makedirs(OUT, exist_ok=True)
    tag = hashlib.sha1(text.encode()).hexdigest()[:16]
    lib = os.path.join(OUT, "libora_%s.so" % tag)
    if not os.path.exists(lib):
        src = os.path.join(OUT, "ora_%s.cpp" % tag)
        with open(src, "w") as f:
            f.write(text)
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               src, "-o", tmp])
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
