"""ctypes front end of the plain FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``dgsem_oracle.cpp``: the
textbook strong-form split DGSEM for the compressible Navier-Stokes equations
(paper Sec. 2.2 and Sec. 4), the equilibrium wall model (Sec. 3.2,
Algorithms 1-2) and the LSERK4 update (Sec. 4), written out loop by loop.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_libs = {}

PHYS_KEYS = ("gamma", "R", "mu", "Pr", "fx", "fy", "fz", "kappa", "B", "hwm", "suth_S", "T_ref",
             "U_in0", "U_in1", "U_in2", "U_in3", "U_in4", "p_out", "T_wall")
PHYS_DEFAULTS = {"suth_S": 0.0, "T_ref": 1.0, "U_in0": 1.0, "U_in4": 1.0, "p_out": 1.0}


def lib(extended=False):
    """The FP64 oracle library, or its extended-precision build."""
    if extended not in _libs:
        _libs[extended] = bind(_build.build(extended=extended))
    return _libs[extended]


def bind(path):
    """The oracle's C interface from the shared library at path (its own
    builds; the pin-strength tests also load copies built with a planted
    mistake)."""
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    vp = ctypes.c_void_p
    L.ora_viscosity.argtypes = [dp, ctypes.c_double]
    L.ora_viscosity.restype = ctypes.c_double
    L.ora_lgl.argtypes = [ctypes.c_int, dp, dp, dp]
    L.ora_lserk4.argtypes = [dp, dp, dp]
    L.ora_set_threads.argtypes = [ctypes.c_int]
    L.ora_max_threads.restype = ctypes.c_int
    L.ora_create.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ip, ip, dp, ip, ctypes.c_char_p, ctypes.c_int]
    L.ora_create.restype = vp
    L.ora_create_subset.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ip, ip, dp, ip, ctypes.c_int, ip,
                                    ctypes.c_char_p, ctypes.c_int]
    L.ora_create_subset.restype = vp
    L.ora_destroy.argtypes = [vp]
    L.ora_get_metrics.argtypes = [vp, dp, dp]
    L.ora_num_wall.argtypes = [vp]
    L.ora_get_wall_samples.argtypes = [vp, ip, dp]
    L.ora_get_wall_weights.argtypes = [vp, dp]
    L.ora_time_derivative.argtypes = [vp, dp, ctypes.c_double, dp]
    L.ora_wall_heat.argtypes = [vp, dp, dp]
    L.ora_jvp.argtypes = [vp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
    L.ora_rk_stage.argtypes = [vp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.ora_rk_steps.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.ora_dt.argtypes = [vp, dp, ctypes.c_double, dp]
    L.ora_wall_shear.argtypes = [vp, dp, dp]
    L.ora_rollout_jvp.argtypes = [vp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_double, dp, dp]
    L.ora_kinetic_energy.argtypes = [vp, dp, dp]
    L.ora_solve_utau.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, dp]
    L.ora_law_value.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.ora_law_value.restype = ctypes.c_double
    L.ora_wall_flux.argtypes = [dp, ctypes.c_int, dp, dp, dp, dp, dp]
    L.ora_riemann.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    L.ora_real_digits.restype = ctypes.c_int
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lgl(N):
    """LGL nodes, weights and derivative matrix D[i, j] = l_j'(x_i)."""
    x = np.zeros(N + 1); w = np.zeros(N + 1); D = np.zeros((N + 1, N + 1))
    if lib().ora_lgl(N, _p(x), _p(w), _p(D)) != 0:
        raise ValueError("bad N")
    return x, w, D


def lserk4():
    A = np.zeros(5); B = np.zeros(5); c = np.zeros(5)
    lib().ora_lserk4(_p(A), _p(B), _p(c))
    return A, B, c


def set_threads(n):
    lib().ora_set_threads(int(n))


def max_threads():
    return lib().ora_max_threads()


def phys_array(phys):
    """Parameter vector of the C interface; the inflow state comes from
    phys["U_in"] (5 conservative values)."""
    d = dict(phys)
    if "U_in" in d:
        for v in range(5):
            d["U_in%d" % v] = float(d["U_in"][v])
    return np.array([float(d.get(k, PHYS_DEFAULTS.get(k, 0.0))) for k in PHYS_KEYS], dtype=np.float64)


class Oracle:
    """One mesh + parameter set.  U arrays are SoA [5][K][n^3] float64.

    extended=True evaluates everything (geometry included) in long double and
    rounds the results to double: the parity reference.  subset: element
    indices; Ut is then evaluated on those elements only (the rest of the
    output is 0), which lets the oracle sample meshes too large to evaluate
    whole.  nbr_face, orient: [K, 6] neighbour faces and orientation codes of
    a general conforming mesh (None: the structured default)."""

    def __init__(self, N, X, nbr, phys, vol_flux=0, surf_flux=1, viscous=1, law=1, extended=False, subset=None,
                 nbr_face=None, orient=None):
        self.L = lib(extended)
        self.extended = extended
        self.N = int(N)
        self.n = self.N + 1
        self.n3 = self.n ** 3
        X = _f64(X)
        self.K = X.size // (3 * self.n3)
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        nf = None if nbr_face is None else np.ascontiguousarray(nbr_face, dtype=np.int32)
        ori = None if orient is None else np.ascontiguousarray(orient, dtype=np.int32)
        pnf = None if nf is None else _ip(nf)
        por = None if ori is None else _ip(ori)
        self._phys = phys_array(phys)
        opts = np.array([vol_flux, surf_flux, viscous, law], dtype=np.int32)
        err = ctypes.create_string_buffer(512)
        if subset is None:
            self.h = self.L.ora_create(self.N, self.K, _p(X), _ip(nbr), pnf, por, _p(self._phys), _ip(opts), err,
                                       512)
        else:
            sel = np.ascontiguousarray(subset, dtype=np.int32)
            self.h = self.L.ora_create_subset(self.N, self.K, _p(X), _ip(nbr), pnf, por, _p(self._phys),
                                              _ip(opts), int(sel.size), _ip(sel), err, 512)
        if not self.h:
            raise ValueError("oracle mesh rejected: " + err.value.decode())
        self.shape = (5, self.K, self.n3)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.ora_destroy(h)
            self.h = None

    def metrics(self):
        Ja = np.zeros((self.K, self.n3, 3, 3)); J = np.zeros((self.K, self.n3))
        self.L.ora_get_metrics(self.h, _p(Ja), _p(J))
        return Ja, J

    def wall_samples(self):
        nw = self.L.ora_num_wall(self.h)
        el = np.zeros(nw, dtype=np.int32); ref = np.zeros((nw, 3))
        self.L.ora_get_wall_samples(self.h, _ip(el), _p(ref))
        return el, ref

    def wall_weights(self):
        """Lagrange weights of the wall samples, [n_wall][3][n]."""
        nw = self.L.ora_num_wall(self.h)
        out = np.zeros((nw, 3, self.n))
        self.L.ora_get_wall_weights(self.h, _p(out))
        return out

    def time_derivative(self, U, t=0.0):
        U = _f64(U); Ut = np.zeros_like(U)
        st = self.L.ora_time_derivative(self.h, _p(U), float(t), _p(Ut))
        if st != 0:
            raise RuntimeError("oracle wall model did not converge")
        return Ut

    def wall_heat(self, U):
        """Wall heat flux q_w into the fluid per wall slot (face-major, n^2 per face)."""
        U = _f64(U)
        out = np.zeros(self.L.ora_num_wall(self.h))
        st = self.L.ora_wall_heat(self.h, _p(U), _p(out))
        if st != 0:
            raise RuntimeError("oracle wall model did not converge")
        return out

    def jvp(self, U, dU=None, dkappa=0.0, dB=0.0, t=0.0):
        U = _f64(U); Ut = np.zeros_like(U); dUt = np.zeros_like(U)
        dptr = None
        if dU is not None:
            dU = _f64(dU); dptr = _p(dU)
        st = self.L.ora_jvp(self.h, _p(U), dptr, float(dkappa), float(dB), float(t), _p(Ut), _p(dUt))
        if st != 0:
            raise RuntimeError("oracle wall model did not converge")
        return Ut, dUt

    def rk_stage(self, U, dU, s, t, dt):
        """In-place LSERK4 stage on float64 arrays U, dU."""
        assert U.dtype == np.float64 and U.flags.c_contiguous
        assert dU.dtype == np.float64 and dU.flags.c_contiguous
        return self.L.ora_rk_stage(self.h, _p(U), _p(dU), int(s), float(t), float(dt))

    def rk_steps(self, U, dt, nsteps, t0=0.0):
        U = _f64(U).copy()
        self.L.ora_rk_steps(self.h, _p(U), float(t0), float(dt), int(nsteps))
        return U

    def dt(self, U, cfl=0.9):
        U = _f64(U); out = np.zeros(1)
        self.L.ora_dt(self.h, _p(U), float(cfl), _p(out))
        return float(out[0])

    def wall_shear(self, U):
        U = _f64(U); out = np.zeros(1)
        st = self.L.ora_wall_shear(self.h, _p(U), _p(out))
        if st != 0:
            raise RuntimeError("oracle wall model did not converge")
        return float(out[0])

    def rollout_jvp(self, U0, dU0, dkappa, dB, nsteps, dt):
        U0 = _f64(U0)
        loss = np.zeros(1); dl = np.zeros(1)
        dptr = None
        if dU0 is not None:
            dU0 = _f64(dU0); dptr = _p(dU0)
        st = self.L.ora_rollout_jvp(self.h, _p(U0), dptr, float(dkappa), float(dB), int(nsteps),
                                   float(dt), _p(loss), _p(dl))
        if st != 0:
            raise RuntimeError("oracle wall model did not converge")
        return float(loss[0]), float(dl[0])

    def kinetic_energy(self, U):
        U = _f64(U); out = np.zeros(1)
        self.L.ora_kinetic_energy(self.h, _p(U), _p(out))
        return float(out[0])


def solve_utau(law, u, h, nu, kappa, B):
    out = np.zeros(1)
    it = lib().ora_solve_utau(int(law), float(u), float(h), float(nu), float(kappa), float(B), _p(out))
    return float(out[0]), it


def law_value(law, x, kappa, B):
    return lib().ora_law_value(int(law), float(x), float(kappa), float(B))


def wall_flux(phys, law, U5, nout, heat=False):
    """(momentum flux, wall shear vector, status[, wall heat flux q_w])."""
    pa = phys_array(phys)
    U5 = _f64(U5); nout = _f64(nout)
    fm = np.zeros(3); tau = np.zeros(3); qw = np.zeros(1)
    st = lib().ora_wall_flux(_p(pa), int(law), _p(U5), _p(nout), _p(fm), _p(tau), _p(qw))
    return (fm, tau, st, float(qw[0])) if heat else (fm, tau, st)


def viscosity(phys, T):
    return lib().ora_viscosity(_p(phys_array(phys)), float(T))


def riemann(phys, vol_kind, kind, UL, UR, nh):
    pa = phys_array(phys)
    UL = _f64(UL); UR = _f64(UR); nh = _f64(nh); F = np.zeros(5)
    lib().ora_riemann(_p(pa), int(vol_kind), int(kind), _p(UL), _p(UR), _p(nh), _p(F))
    return F
