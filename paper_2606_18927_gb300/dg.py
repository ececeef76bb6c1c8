"""Python binding of libdg_gb300.so (the C ABI declared in include/dg.h).

Argument marshalling only: every step of the operator runs in the library's
sm_103a kernels.  Device arrays are torch CUDA tensors (float64, contiguous,
SoA layout [5][K][n^3]); the stream is torch's current stream unless one is
given.  There is no CPU fallback: if the library cannot be loaded or a call
fails, an exception is raised.
"""
import ctypes
import os
import re

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(_HERE, "..", "include", "dg.h")

FP64, FP32_MIXED = 0, 1
VOL_KEP_PIROZZOLI, VOL_KEP_KENNEDY_GRUBER, VOL_EC_CHANDRASHEKAR = 0, 1, 2
DG_BC_WALL, DG_BC_INFLOW, DG_BC_OUTFLOW, DG_BC_HALO_BASE = -1, -2, -3, -16
SURF_CENTRAL, SURF_LLF, SURF_ROE = 0, 1, 2
LAW_SPALDING, LAW_REICHARDT = 0, 1

ERRORS = {
    -1: "DG_ERR_ARG", -2: "DG_ERR_NOT_INIT", -3: "DG_ERR_MESH", -4: "DG_ERR_CUDA",
    -5: "DG_ERR_NONFINITE", -6: "DG_ERR_WM_NOCONV", -7: "DG_ERR_DEVICE_BOUNDS",
    -8: "DG_ERR_NOT_IMPLEMENTED", -9: "DG_ERR_OOM",
}


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class _MeshDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int),
                ("X", ctypes.POINTER(ctypes.c_double)), ("nbr", ctypes.POINTER(ctypes.c_int)),
                ("nbr_face", ctypes.POINTER(ctypes.c_int)), ("orient", ctypes.POINTER(ctypes.c_int))]


class _Phys(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("R", ctypes.c_double), ("mu", ctypes.c_double),
                ("Pr", ctypes.c_double), ("force", ctypes.c_double * 3), ("kappa", ctypes.c_double),
                ("B", ctypes.c_double), ("hwm", ctypes.c_double), ("law", ctypes.c_int),
                ("p_ref", ctypes.c_double), ("suth_S", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("U_in", ctypes.c_double * 5), ("p_out", ctypes.c_double), ("T_wall", ctypes.c_double),
                ("rho_ref", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("vol_flux", ctypes.c_int), ("surf_flux", ctypes.c_int),
                ("viscous", ctypes.c_int)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) the shared library."""
    global _lib
    if _lib is not None:
        return _lib
    # DG_LIBRARY_VARIANT=debug: the bounds-checking build (index checks in the kernels)
    path = _build.build(variant=os.environ.get("DG_LIBRARY_VARIANT", "release"))
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    sig = {
        "dg_lgl_nodes": (c_int, [c_int, dp, dp]),
        "dg_init_mesh": (c_int, [ctypes.POINTER(vp), ctypes.POINTER(_MeshDesc), ctypes.POINTER(_Phys),
                                 ctypes.POINTER(_Options), vp]),
        "dg_destroy": (c_int, [vp]),
        "dg_last_error": (ctypes.c_char_p, [vp]),
        "dg_set_stream": (c_int, [vp, vp]),
        "dg_sizes": (c_int, [vp, ip, ip, ctypes.POINTER(ctypes.c_longlong)]),
        "dg_set_state": (c_int, [vp, vp, c_int]),
        "dg_get_state": (c_int, [vp, vp, c_int]),
        "dg_time_derivative": (c_int, [vp, vp, vp, c_double, c_int]),
        "dg_rk_stage": (c_int, [vp, c_int, c_double, c_double]),
        "dg_rk_steps": (c_int, [vp, c_double, c_double, c_int]),
        "dg_rk_steps_graph": (c_int, [vp, c_double, c_double, c_int]),
        "dg_rk_stage_batch": (c_int, [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int, c_double,
                                      c_double]),
        "dg_check_status": (c_int, [vp]),
        "dg_get_rk_register": (c_int, [vp, vp, c_int]),
        "dg_set_rk_register": (c_int, [vp, vp, c_int]),
        "dg_get_metrics": (c_int, [vp, dp, dp]),
        "dg_time_derivative_noalloc": (c_int, [vp, vp, vp]),
        "dg_vjp": (c_int, [vp, vp, vp, vp, vp]),
        "dg_vjp_phase": (c_int, [vp, c_int, vp, vp, vp, vp]),
        "dg_set_params": (c_int, [vp, c_double, c_double]),
        "dg_set_wall_solve_limit": (c_int, [vp, c_int]),
        "dg_set_lifting_arithmetic": (c_int, [vp, c_int]),
        "dg_wall_shear": (c_int, [vp, vp, dp]),
        "dg_kinetic_energy": (c_int, [vp, vp, dp]),
        "dg_time_step": (c_int, [vp, vp, c_double, dp]),
        "dg_convert_fp32": (c_int, [ctypes.c_longlong, vp, vp, vp, vp, vp]),
        "dg_rollout_vjp": (c_int, [vp, vp, c_int, c_double, dp, vp, vp]),
        "dg_profile_enable": (c_int, [vp, c_int]),
        "dg_set_overlap": (c_int, [vp, c_int]),
        "dg_profile_read": (c_int, [vp, dp, ip]),
        "dg_partition_sfc": (c_int, [c_int, c_int, dp, c_int, ip]),
        "dg_partition_local": (c_int, [c_int, ip, ip, ip, ip, c_int, ip, ip, ip, ip, ip, ip, ip]),
        "dg_halo_buffers": (c_int, [vp, ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp)]),
        "dg_halo_geometry": (c_int, [vp, dp]),
        "dg_halo_set_geometry": (c_int, [vp, dp]),
        "dg_stage_phase": (c_int, [vp, c_int, c_int, c_double, c_double]),
        "dg_time_derivative_phase": (c_int, [vp, c_int, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions():
    """Names of every function declared in include/dg.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*(dg_[a-z0-9_]+)\s*\(", txt, re.M)))


def lgl_nodes(N):
    x = np.zeros(N + 1); w = np.zeros(N + 1)
    rc = lib().dg_lgl_nodes(N, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise DGError(rc, lib().dg_last_error(None).decode())
    return x, w


def convert_fp32(d, g):
    """The FP32-mixed kernels' conversions (dg_convert_fp32) on CUDA tensors:
    d (float64) -> (f, rem) float32, g (float32) -> float64."""
    assert d.is_cuda and d.dtype.is_floating_point and d.element_size() == 8 and d.is_contiguous()
    assert g.is_cuda and g.element_size() == 4 and g.is_contiguous() and g.numel() == d.numel()
    import torch
    f = torch.empty(d.shape, dtype=torch.float32, device=d.device)
    rem = torch.empty_like(f)
    gd = torch.empty(d.shape, dtype=torch.float64, device=d.device)
    rc = lib().dg_convert_fp32(d.numel(), ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                               ctypes.c_void_p(rem.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                               ctypes.c_void_p(gd.data_ptr()))
    if rc != 0:
        raise DGError(rc, "dg_convert_fp32 failed")
    return f, rem, gd


def _ptr(t):
    """Device or host address of a tensor / array, and whether it is on the device."""
    if isinstance(t, np.ndarray):
        assert t.dtype == np.float64 and t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data), 0
    assert t.dtype.is_floating_point and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0


class _DeviceView:
    """A device array described through __cuda_array_interface__, so that
    torch.as_tensor views library-owned device memory without copying."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def partition_sfc(N, X, nranks):
    """Rank of every element along the Morton curve of the centroids (dg_partition_sfc)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n3 = (N + 1) ** 3
    K = X.size // (3 * n3)
    part = np.zeros(K, dtype=np.int32)
    rc = lib().dg_partition_sfc(int(N), int(K), X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nranks),
                                part.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise DGError(rc, "dg_partition_sfc failed")
    return part


def partition_local(nbr, part, rank, nbr_face=None, orient=None):
    """(l2g, nbr_local, nbr_face_local, orient_local, halo[n_halo, 4]) of one
    rank (dg_partition_local)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    K = part.size
    ip = ctypes.POINTER(ctypes.c_int)
    nf = None if nbr_face is None else np.ascontiguousarray(nbr_face, dtype=np.int32)
    ori = None if orient is None else np.ascontiguousarray(orient, dtype=np.int32)
    pnf = None if nf is None else nf.ctypes.data_as(ip)
    por = None if ori is None else ori.ctypes.data_as(ip)
    Kl, nh = ctypes.c_int(), ctypes.c_int()
    L = lib()
    rc = L.dg_partition_local(K, nbr.ctypes.data_as(ip), pnf, por, part.ctypes.data_as(ip), int(rank),
                              ctypes.byref(Kl), None, None, None, None, ctypes.byref(nh), None)
    if rc != 0:
        raise DGError(rc, "dg_partition_local failed")
    l2g = np.zeros(Kl.value, dtype=np.int32)
    nbl = np.zeros((Kl.value, 6), dtype=np.int32)
    nfl = np.zeros((Kl.value, 6), dtype=np.int32)
    orl = np.zeros((Kl.value, 6), dtype=np.int32)
    halo = np.zeros((max(nh.value, 1), 4), dtype=np.int32)
    rc = L.dg_partition_local(K, nbr.ctypes.data_as(ip), pnf, por, part.ctypes.data_as(ip), int(rank),
                              ctypes.byref(Kl), l2g.ctypes.data_as(ip), nbl.ctypes.data_as(ip),
                              nfl.ctypes.data_as(ip), orl.ctypes.data_as(ip), ctypes.byref(nh),
                              halo.ctypes.data_as(ip))
    if rc != 0:
        raise DGError(rc, "dg_partition_local failed")
    return l2g, nbl, nfl, orl, halo[: nh.value]


def _stream_handle(stream):
    """cudaStream_t of a torch stream (None: torch's current stream; 0: the
    legacy default stream, which needs no torch CUDA state)."""
    if isinstance(stream, int) and stream == 0:
        return ctypes.c_void_p(0)
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Operator:
    """Ut = DG_Operator(U) and LSERK4 stages on one mesh (one GPU)."""

    def __init__(self, N, X, nbr, phys, precision=FP64, vol_flux=VOL_KEP_PIROZZOLI, surf_flux=SURF_LLF,
                 viscous=1, law=LAW_REICHARDT, stream=None, nbr_face=None, orient=None):
        """nbr_face, orient: [K, 6] neighbour faces and orientation codes of a
        general conforming mesh (None: the structured default)."""
        L = lib()
        self.N = int(N)
        self.n3 = (self.N + 1) ** 3
        X = np.ascontiguousarray(X, dtype=np.float64)
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.K = X.size // (3 * self.n3)
        ip = ctypes.POINTER(ctypes.c_int)
        nf = None if nbr_face is None else np.ascontiguousarray(nbr_face, dtype=np.int32)
        ori = None if orient is None else np.ascontiguousarray(orient, dtype=np.int32)
        md = _MeshDesc(self.N, self.K, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nbr.ctypes.data_as(ip),
                       None if nf is None else nf.ctypes.data_as(ip), None if ori is None else ori.ctypes.data_as(ip))
        ph = _Phys(phys["gamma"], phys["R"], phys["mu"], phys["Pr"],
                   (ctypes.c_double * 3)(phys.get("fx", 0.0), phys.get("fy", 0.0), phys.get("fz", 0.0)),
                   phys.get("kappa", 0.41), phys.get("B", 5.2), phys.get("hwm", 0.1), int(law),
                   phys.get("p_ref", phys.get("p0", 0.0)), phys.get("suth_S", 0.0), phys.get("T_ref", 1.0),
                   (ctypes.c_double * 5)(*[float(x) for x in phys.get("U_in", (1.0, 0.0, 0.0, 0.0, 1.0))]),
                   float(phys.get("p_out", 1.0)), float(phys.get("T_wall", 0.0)),
                   float(phys.get("rho_ref", 1.0)))
        op = _Options(int(precision), int(vol_flux), int(surf_flux), int(viscous))
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        rc = L.dg_init_mesh(ctypes.byref(h), ctypes.byref(md), ctypes.byref(ph), ctypes.byref(op), self._stream)
        if rc != 0:
            raise DGError(rc, L.dg_last_error(None).decode())
        self.h = h
        self.shape = (5, self.K, self.n3)
        self.numel = 5 * self.K * self.n3
        self.dofs = self.K * self.n3
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            lib().dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise DGError(rc, lib().dg_last_error(self.h).decode())

    def set_stream(self, stream):
        self._stream = _stream_handle(stream)
        self._check(lib().dg_set_stream(self.h, self._stream))

    def set_state(self, U):
        p, dev = _ptr(U)
        count = U.numel() if hasattr(U, "numel") else U.size
        if count != self.numel:
            raise ValueError("state has %d values, expected %d" % (count, self.numel))
        self._check(lib().dg_set_state(self.h, p, dev))

    def get_state(self, out):
        if (out.numel() if hasattr(out, "numel") else out.size) != self.numel:
            raise ValueError("array has the wrong size for this mesh")
        p, dev = _ptr(out)
        self._check(lib().dg_get_state(self.h, p, dev))
        return out

    def get_rk_register(self, out):
        if (out.numel() if hasattr(out, "numel") else out.size) != self.numel:
            raise ValueError("array has the wrong size for this mesh")
        p, dev = _ptr(out)
        self._check(lib().dg_get_rk_register(self.h, p, dev))
        return out

    def set_rk_register(self, dU):
        if (dU.numel() if hasattr(dU, "numel") else dU.size) != self.numel:
            raise ValueError("array has the wrong size for this mesh")
        p, dev = _ptr(dU)
        self._check(lib().dg_set_rk_register(self.h, p, dev))

    def time_derivative(self, Ut, U=None, t=0.0):
        """Ut <- DG_Operator(U) (U None: the context's state).  Ut and U are
        both device tensors or both host arrays."""
        po, dev = _ptr(Ut)
        pu = None
        for a in (Ut, U):
            if a is not None and (a.numel() if hasattr(a, "numel") else a.size) != self.numel:
                raise ValueError("array has the wrong size for this mesh")
        if U is not None:
            pu, devu = _ptr(U)
            if devu != dev:
                raise ValueError("U and Ut must both be on the device or both on the host")
        self._check(lib().dg_time_derivative(self.h, pu, po, float(t), dev))
        return Ut

    def vjp(self, lam, gU, U=None, gtheta=None):
        """gU <- (dUt/dU)^T lam; gtheta (device tensor of 2) <- (dUt/d(kappa, B))^T lam."""
        for a in (lam, gU, U):
            if a is not None and a.numel() != self.numel:
                raise ValueError("array has the wrong size for this mesh")
        pl, _ = _ptr(lam)
        pg, _ = _ptr(gU)
        pu = _ptr(U)[0] if U is not None else None
        pt = _ptr(gtheta)[0] if gtheta is not None else None
        self._check(lib().dg_vjp(self.h, pu, pl, pg, pt))
        return gU

    def vjp_phase(self, phase, lam, gU, U=None, gtheta=None):
        """One phase (1-4) of the adjoint of a partitioned context (dg_vjp_phase)."""
        for a in (lam, gU, U):
            if a is not None and a.numel() != self.numel:
                raise ValueError("array has the wrong size for this mesh")
        pu = _ptr(U)[0] if U is not None else None
        pt = _ptr(gtheta)[0] if gtheta is not None else None
        self._check(lib().dg_vjp_phase(self.h, int(phase), pu, _ptr(lam)[0], _ptr(gU)[0], pt))
        return gU

    def set_params(self, kappa, B):
        self._check(lib().dg_set_params(self.h, float(kappa), float(B)))

    def set_lifting_arithmetic(self, mode):
        """0: FP64 lifting kernel; 1: double-float lifting (FP64 viscous form, odd N; the default)."""
        self._check(lib().dg_set_lifting_arithmetic(self.h, int(mode)))

    def set_wall_solve_limit(self, max_iter):
        """Iteration cap of the wall model's law-of-the-wall solve (default 200)."""
        self._check(lib().dg_set_wall_solve_limit(self.h, int(max_iter)))

    def time_step(self, cfl=0.9, U=None):
        out = ctypes.c_double(0.0)
        pu = _ptr(U)[0] if U is not None else None
        self._check(lib().dg_time_step(self.h, pu, float(cfl), ctypes.byref(out)))
        return out.value

    def kinetic_energy(self, U=None):
        out = ctypes.c_double(0.0)
        pu = _ptr(U)[0] if U is not None else None
        self._check(lib().dg_kinetic_energy(self.h, pu, ctypes.byref(out)))
        return out.value

    def wall_shear(self, U=None):
        out = ctypes.c_double(0.0)
        pu = _ptr(U)[0] if U is not None else None
        self._check(lib().dg_wall_shear(self.h, pu, ctypes.byref(out)))
        return out.value

    def rollout_vjp(self, U0, nsteps, dt, gU0, gtheta=None):
        """Loss (mean wall shear after nsteps steps) and its gradients, see dg.h."""
        out = ctypes.c_double(0.0)
        pt = _ptr(gtheta)[0] if gtheta is not None else None
        self._check(lib().dg_rollout_vjp(self.h, _ptr(U0)[0], int(nsteps), float(dt), ctypes.byref(out),
                                         _ptr(gU0)[0], pt))
        return out.value

    def rk_stage(self, s, t, dt):
        self._check(lib().dg_rk_stage(self.h, int(s), float(t), float(dt)))

    def rk_steps(self, t, dt, nsteps):
        self._check(lib().dg_rk_steps(self.h, float(t), float(dt), int(nsteps)))

    def rk_steps_graph(self, t, dt, nsteps):
        """LSERK4 steps replayed from a CUDA graph of one step."""
        self._check(lib().dg_rk_steps_graph(self.h, float(t), float(dt), int(nsteps)))

    def rk_stage_batch(self, U_in, U_out, nstages, t, dt):
        """Independent host states through stages 0 .. nstages-1 of a step,
        host copies overlapped with the computation (dg_rk_stage_batch).
        U_in, U_out: sequences of C-contiguous float64 host arrays (or CPU
        tensors) of the state's shape, page-locked for the overlap."""
        if len(U_in) != len(U_out):
            raise ValueError("rk_stage_batch: as many outputs as inputs")
        n5 = 5 * self.K * self.n3
        for a in list(U_in) + list(U_out):
            p, dev = _ptr(a)
            if dev or (a.size if isinstance(a, np.ndarray) else a.numel()) != n5:
                raise ValueError("rk_stage_batch: host arrays of the state's size")
        ins = (ctypes.c_void_p * max(1, len(U_in)))(*[_ptr(a)[0].value for a in U_in])
        outs = (ctypes.c_void_p * max(1, len(U_out)))(*[_ptr(a)[0].value for a in U_out])
        self._check(lib().dg_rk_stage_batch(self.h, len(U_in), ins, outs, int(nstages), float(t), float(dt)))

    def check_status(self):
        self._check(lib().dg_check_status(self.h))

    # -- partitioned meshes (see halo.py) ---------------------------------
    def halo_buffers(self):
        """Device views (torch) of the halo buffers: send_U, recv_U
        [n_halo, 5, n2] float64 and send_G, recv_G [n_halo, 4, n2] in the flux
        type.  Empty dict for an unpartitioned context."""
        import torch
        nh = ctypes.c_int()
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        self._check(lib().dg_halo_buffers(self.h, ctypes.byref(nh), *[ctypes.byref(q) for q in ptrs]))
        if nh.value == 0:
            return {}
        n2 = (self.N + 1) ** 2
        gdt = "<f4" if self.precision == FP32_MIXED else "<f8"
        out = {}
        for name, q, rows, dt in (("send_U", ptrs[0], 5, "<f8"), ("recv_U", ptrs[1], 5, "<f8"),
                                  ("send_G", ptrs[2], 4, gdt), ("recv_G", ptrs[3], 4, gdt)):
            out[name] = torch.as_tensor(_DeviceView(q.value, (nh.value, rows, n2), dt), device="cuda")
        return out

    def halo_geometry(self):
        nh = ctypes.c_int()
        self._check(lib().dg_halo_buffers(self.h, ctypes.byref(nh), None, None, None, None))
        out = np.zeros((nh.value, 4, (self.N + 1) ** 2))
        self._check(lib().dg_halo_geometry(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def set_halo_geometry(self, fgeo):
        fgeo = np.ascontiguousarray(fgeo, dtype=np.float64)
        self._check(lib().dg_halo_set_geometry(self.h, fgeo.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def stage_phase(self, phase, s, t, dt):
        self._check(lib().dg_stage_phase(self.h, int(phase), int(s), float(t), float(dt)))

    def time_derivative_phase(self, phase, Ut, U=None):
        pu = _ptr(U)[0] if U is not None else None
        self._check(lib().dg_time_derivative_phase(self.h, int(phase), pu, _ptr(Ut)[0]))

    def set_overlap(self, on=True):
        """Wall-model kernel on its own high-priority stream (default), or in line."""
        self._check(lib().dg_set_overlap(self.h, 1 if on else 0))

    def profile_enable(self, on=True):
        self._check(lib().dg_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel: (total ms, launches)} since the last read (lift, face, wall, volume)."""
        ms = np.zeros(4); cnt = np.zeros(4, dtype=np.int32)
        self._check(lib().dg_profile_read(self.h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(("lift", "face", "wall", "volume"))}

    def metrics(self):
        Ja = np.zeros((self.K, self.n3, 3, 3)); J = np.zeros((self.K, self.n3))
        self._check(lib().dg_get_metrics(self.h, Ja.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         J.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return Ja, J


# ---------------------------------------------------------------------------
# torch.autograd bindings (the backward passes call the library's adjoint)
# ---------------------------------------------------------------------------
def _autograd():
    import torch

    class DGOperatorFunction(torch.autograd.Function):
        """Ut = DG_Operator(U) with its hand-written VJP as backward."""

        @staticmethod
        def forward(ctx, U, op):
            Ut = torch.empty_like(U)
            op.time_derivative(Ut, U.contiguous())
            ctx.save_for_backward(U)
            ctx.op = op
            return Ut

        @staticmethod
        def backward(ctx, g):
            (U,) = ctx.saved_tensors
            gU = torch.empty_like(U)
            ctx.op.vjp(g.contiguous(), gU, U.contiguous())
            return gU, None

    class WallShearRollout(torch.autograd.Function):
        """Mean wall shear after nsteps LSERK4 steps from U0, differentiable in
        U0 and theta = (kappa, B); the gradients come from dg_rollout_vjp
        (per-step checkpoints, reverse sweep) computed during forward."""

        @staticmethod
        def forward(ctx, U0, theta, op, nsteps, dt):
            th = theta.detach().double().cpu()
            op.set_params(float(th[0]), float(th[1]))
            gU0 = torch.empty_like(U0)
            gth = torch.zeros(2, dtype=torch.float64, device=U0.device)
            loss = op.rollout_vjp(U0.contiguous(), nsteps, dt, gU0, gth)
            ctx.save_for_backward(gU0, gth)
            ctx.theta_device, ctx.theta_dtype = theta.device, theta.dtype
            return torch.tensor(loss, dtype=torch.float64, device=U0.device)

        @staticmethod
        def backward(ctx, g):
            gU0, gth = ctx.saved_tensors
            g = g.to(gU0.device)
            return g * gU0, (g * gth).to(ctx.theta_device, ctx.theta_dtype), None, None, None

    return DGOperatorFunction, WallShearRollout


def dg_operator(U, op):
    """Differentiable Ut = DG_Operator(U) for torch CUDA float64 tensors."""
    return _autograd()[0].apply(U, op)


def wall_shear_rollout(U0, theta, op, nsteps, dt):
    """Differentiable mean wall shear after nsteps LSERK4 steps."""
    return _autograd()[1].apply(U0, theta, op, nsteps, dt)
