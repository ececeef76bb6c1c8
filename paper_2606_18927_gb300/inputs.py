"""Seeded synthetic inputs shared by the CUDA path, its tests and the bench.

This module holds no arithmetic of the DG method itself: it lays out
structured hexahedral meshes from reference node positions supplied by the
caller (each side of a comparison passes its own Gauss-Lobatto nodes), maps
them through the analytic geometries of the workloads, and evaluates the
initial conditions at given node coordinates.  Random numbers come from
splitmix64 (Steele, Lea, Flood 2014), counter-based, so every consumer sees
the same stream.

Workloads (paper Sec. 2.2 and 2.3 time the solver on a free-stream /
uniform periodic box; Sec. 3.3 validates the wall model on a turbulent
channel; all sizes below are the synthetic stand-ins for those):
  * Taylor-Green vortex on [0, 2 pi]^3, affine or sine-deformed;
  * wall-modelled channel 2 pi x 2 x pi, tanh wall-normal stretching and a
    sinusoidal interior warp;
  * uniform free-stream state (the paper's scaling test case).
"""
from dataclasses import dataclass, field
import math

import numpy as np

SEED = 20261202
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(count, seed=SEED, offset=0):
    """Outputs offset .. offset+count-1 of the splitmix64 stream as uint64."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(count, lo, hi, seed=SEED, offset=0):
    """Uniform doubles in [lo, hi) from the top 53 bits of splitmix64."""
    z = splitmix64(count, seed, offset)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


# ---------------------------------------------------------------------------
# Meshes
# ---------------------------------------------------------------------------
WALL = -1     # neighbour code of a wall-modelled slip wall
INFLOW = -2   # Dirichlet inflow (prescribed exterior state)
OUTFLOW = -3  # subsonic pressure outflow (prescribed exterior pressure)


@dataclass
class BoxSpec:
    """Structured nx x ny x nz element box mapped by an analytic geometry.

    geometry: 'affine' | 'sine' (x += a sin(y) sin(z), cyclic) |
              'channel' (tanh stretching in y + sinusoidal warp) |
              'wavy' (periodic sine warp on [0, L]^3 used for convergence)
    periodic: per-axis flags; non-periodic axes end in the boundary codes of
    `boundary` ((lo, hi) per axis), wall-modelled walls by default.
    """
    N: int
    nx: int
    ny: int
    nz: int
    lengths: tuple = (2 * math.pi, 2 * math.pi, 2 * math.pi)
    geometry: str = "affine"
    amplitude: float = 0.0
    stretch: float = 1.5
    periodic: tuple = (True, True, True)
    boundary: tuple = ((WALL, WALL), (WALL, WALL), (WALL, WALL))

    @property
    def K(self):
        return self.nx * self.ny * self.nz

    @property
    def n3(self):
        return (self.N + 1) ** 3

    @property
    def dofs(self):
        return self.K * self.n3


def connectivity(spec: BoxSpec):
    """nbr[K, 6] for lexicographic elements e = ex + nx (ey + ny ez).

    Local faces: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z.  A neighbour shares
    the opposite local face with identical face-node ordering; non-periodic
    box ends carry the spec's boundary codes (walls, -1, by default)."""
    nx, ny, nz = spec.nx, spec.ny, spec.nz
    e = np.arange(spec.K)
    ex = e % nx; ey = (e // nx) % ny; ez = e // (nx * ny)
    dims = (nx, ny, nz)
    coords = [ex, ey, ez]
    nbr = np.zeros((spec.K, 6), dtype=np.int32)
    for axis in range(3):
        for side, step in ((0, -1), (1, 1)):
            c = [a.copy() for a in coords]
            c[axis] = c[axis] + step
            out = (c[axis] < 0) | (c[axis] >= dims[axis])
            if spec.periodic[axis]:
                c[axis] %= dims[axis]
                e = c[0] + nx * (c[1] + ny * c[2])
            else:
                e = np.where(out, spec.boundary[axis][side], (c[0] % nx) + nx * ((c[1] % ny) + ny * (c[2] % nz)))
            nbr[:, 2 * axis + side] = e
    return nbr


def _unit_coords(spec: BoxSpec, xi):
    """Computational coordinates s in [0, 1]^3 of every node, shape [3][K][n^3]."""
    xi = np.asarray(xi, dtype=np.float64)
    n = xi.size
    K = spec.K
    e = np.arange(K)
    ex = e % spec.nx; ey = (e // spec.nx) % spec.ny; ez = e // (spec.nx * spec.ny)
    t = (xi + 1.0) * 0.5
    i = np.arange(n ** 3) % n
    j = (np.arange(n ** 3) // n) % n
    k = np.arange(n ** 3) // (n * n)
    sx = (ex[:, None] + t[i][None, :]) / spec.nx
    sy = (ey[:, None] + t[j][None, :]) / spec.ny
    sz = (ez[:, None] + t[k][None, :]) / spec.nz
    return sx, sy, sz


def _quantize(w, spec):
    """Round a displacement to a multiple of the ulp of the largest domain
    coordinate, so that (period + w) and w differ by exactly the period."""
    q = 2.0 ** (math.frexp(max(spec.lengths) + abs(spec.amplitude) + 1.0)[1] - 53)
    return np.round(w / q) * q


def node_coordinates(spec: BoxSpec, xi):
    """Physical node coordinates X[3][K][n^3] of the mapped box.

    xi are the caller's reference nodes on [-1, 1] (Gauss-Lobatto).  The
    warps are evaluated on the unit coordinate wrapped into [0, 1) along
    periodic axes and quantised to the ulp of the domain length, so the two
    periodic images of a face are exact translations of each other."""
    sx, sy, sz = _unit_coords(spec, xi)
    Lx, Ly, Lz = spec.lengths
    a = spec.amplitude
    wrap = [np.where(c >= 1.0, c - 1.0, c) if per else c
            for c, per in zip((sx, sy, sz), spec.periodic)]
    if spec.geometry == "affine":
        X = (Lx * sx, Ly * sy, Lz * sz)
    elif spec.geometry == "sine":
        # x' = x + a sin(y) sin(z), cyclic over the axes
        xw, yw, zw = Lx * wrap[0], Ly * wrap[1], Lz * wrap[2]
        X = (Lx * sx + _quantize(a * np.sin(yw) * np.sin(zw), spec),
             Ly * sy + _quantize(a * np.sin(zw) * np.sin(xw), spec),
             Lz * sz + _quantize(a * np.sin(xw) * np.sin(yw), spec))
    elif spec.geometry == "channel":
        # y = 1 + tanh(beta (2 eta - 1)) / tanh(beta) on [0, 2], then every
        # coordinate += a sin(x) sin(pi y / 2) sin(2 z)
        beta = spec.stretch
        y = 0.5 * Ly * (1.0 + np.tanh(beta * (2.0 * sy - 1.0)) / math.tanh(beta))
        wv = _quantize(a * np.sin(Lx * wrap[0]) * np.sin(math.pi * y / Ly) * np.sin(2.0 * Lz * wrap[2]), spec)
        X = (Lx * sx + wv, y + wv, Lz * sz + wv)
    elif spec.geometry == "wavy":
        # periodic warp on [0, L]^3: x += a sin(2 pi y / L) sin(2 pi z / L), cyclic
        tp = 2 * math.pi
        X = (Lx * sx + _quantize(a * np.sin(tp * wrap[1]) * np.sin(tp * wrap[2]), spec),
             Ly * sy + _quantize(a * np.sin(tp * wrap[2]) * np.sin(tp * wrap[0]), spec),
             Lz * sz + _quantize(a * np.sin(tp * wrap[0]) * np.sin(tp * wrap[1]), spec))
    else:
        raise ValueError("unknown geometry " + spec.geometry)
    return np.ascontiguousarray(np.stack(X))


# ---------------------------------------------------------------------------
# Physical parameters and initial conditions
# ---------------------------------------------------------------------------
def phys_params(Ma=0.1, Re=1600.0, Pr=0.72, gamma=1.4, force=(0.0, 0.0, 0.0),
                kappa=0.41, B=5.2, hwm=0.1, inviscid=False, sutherland=False):
    """Non-dimensional parameters: rho0 = U0 = L = R = 1, mu = 1/Re.

    sutherland: viscosity by Sutherland's law for air, mu = 1/Re at the
    reference temperature T_ref = p0 / (rho0 R) (taken as 288.15 K) and
    S = 110.4 K in the same scale."""
    p0 = 1.0 / (gamma * Ma * Ma)
    d = dict(gamma=gamma, R=1.0, mu=0.0 if inviscid else 1.0 / Re, Pr=Pr,
             fx=force[0], fy=force[1], fz=force[2], kappa=kappa, B=B, hwm=hwm,
             Ma=Ma, p0=p0, rho_ref=1.0)
    if sutherland:
        d.update(T_ref=p0, suth_S=p0 * 110.4 / 288.15)
    return d


def conservative(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, E]))


def taylor_green(X, phys):
    """Taylor-Green vortex: u = sin x cos y cos z, v = -cos x sin y cos z,
    w = 0, rho = 1, p = p0 + (cos 2x + cos 2y)(cos 2z + 2) / 16."""
    x, y, z = X
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    p = phys["p0"] + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return conservative(np.ones_like(x), u, v, w, p, phys["gamma"])


def free_stream(X, phys, velocity=(1.0, 0.5, 0.25), rho=1.0):
    one = np.ones_like(X[0])
    return conservative(rho * one, velocity[0] * one, velocity[1] * one, velocity[2] * one,
                        phys["p0"] * one, phys["gamma"])


def channel_profile(X, phys, Ub=1.0, noise=0.05, seed=SEED):
    """Laminar channel profile u = 1.5 Ub (1 - (y - 1)^2), rho = 1, p = p0,
    plus seeded uniform +-noise*Ub on all three velocity components."""
    x, y, z = X
    shape = x.shape
    cnt = x.size
    r = uniform(3 * cnt, -noise * Ub, noise * Ub, seed=seed, offset=7 * cnt).reshape(3, *shape)
    u = 1.5 * Ub * (1.0 - (y - 1.0) ** 2) + r[0]
    v = r[1]
    w = r[2]
    return conservative(np.ones_like(x), u, v, w, phys["p0"] * np.ones_like(x), phys["gamma"])


def perturb(U, rel=1e-3, seed=SEED):
    """Multiplicative perturbation U <- U (1 + eps), eps ~ U(-rel, rel) i.i.d.
    per variable and node, in memory order of U."""
    eps = uniform(U.size, -rel, rel, seed=seed).reshape(U.shape)
    return np.ascontiguousarray(U * (1.0 + eps))


def random_direction(shape, seed, offset=0):
    return uniform(int(np.prod(shape)), -1.0, 1.0, seed=seed, offset=offset).reshape(shape)


def dean_body_force(Re_b):
    """Body force f = u_tau^2 / delta with Dean's correlation
    C_f = 0.073 Re_m^(-1/4), Re_m = 2 Re_b (delta = Ub = rho = 1)."""
    cf = 0.073 * (2.0 * Re_b) ** -0.25
    return 0.5 * cf


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    spec: BoxSpec
    phys: dict
    ic: str
    vol_flux: int = 0      # 0 KEP Pirozzoli, 1 KEP Kennedy-Gruber
    surf_flux: int = 1     # 0 central, 1 LLF, 2 Roe + Harten
    law: int = 1           # 0 Spalding, 1 Reichardt
    viscous: int = 1
    extra: dict = field(default_factory=dict)


def workload(name, N=None, elems=None):
    """Named workloads.  N / elems override the polynomial degree / element
    counts (used to build small cases of the same structure)."""
    two_pi = 2 * math.pi
    if name == "tgv_n3_4":          # N=3, 4^3 affine periodic, LLF
        N = 3 if N is None else N
        e = elems or (4, 4, 4)
        return Workload(name, BoxSpec(N, *e), phys_params(0.1, 1600.0), "tgv", surf_flux=1)
    if name == "tgv_n7_32":         # N=7, 32^3 affine periodic, Roe
        N = 7 if N is None else N
        e = elems or (32, 32, 32)
        return Workload(name, BoxSpec(N, *e), phys_params(0.1, 1600.0), "tgv", surf_flux=2)
    if name == "channel_n5":        # 16x8x8, N=5, wall model (Reichardt)
        N = 5 if N is None else N
        e = elems or (16, 8, 8)
        Re_b = 20000.0
        f = dean_body_force(Re_b)
        spec = BoxSpec(N, *e, lengths=(two_pi, 2.0, math.pi), geometry="channel", amplitude=0.05,
                       stretch=1.5, periodic=(True, False, True))
        return Workload(name, spec, phys_params(0.1, Re_b, force=(f, 0.0, 0.0), kappa=0.41, B=5.2, hwm=0.1),
                        "channel", surf_flux=2, law=1)
    if name == "tgv_sine_n7_48":    # 48^3, N=7, x + 0.1 sin(y) sin(z), Ma 0.3
        N = 7 if N is None else N
        e = elems or (48, 48, 48)
        spec = BoxSpec(N, *e, geometry="sine", amplitude=0.1)
        return Workload(name, spec, phys_params(0.3, 1600.0), "tgv", surf_flux=2)
    raise ValueError("unknown workload " + name)


def initial_state(wl: Workload, X, perturbation=True):
    if wl.ic == "tgv":
        U = taylor_green(X, wl.phys)
    elif wl.ic == "channel":
        U = channel_profile(X, wl.phys)
    elif wl.ic == "free":
        U = free_stream(X, wl.phys)
    else:
        raise ValueError(wl.ic)
    if perturbation and wl.ic != "channel":
        U = perturb(U)
    return U
