// kernels.cuh -- sm_103a kernels of the DGSEM operator.
//
// One operator evaluation (paper Sec. 2.2 / Sec. 4: split-form DGSEM on LGL
// nodes; Sec. 3: equilibrium wall model) launches:
//   k_prim64    FP64 viscous form: the primitives (rho, u, v, w, p', h, T) of
//               the input state, stored for the three kernels below;
//   k_lift      one CTA per element: primitives (FP64: read from k_prim64's
//               array), BR1 lifting of grad(u,v,w,T), viscous
//               flux, its weak-form volume divergence R_v, and the element's
//               own outward viscous flux at its six faces (FP64, N = 7: line
//               contractions in even/odd form, LineEO);
//   k_face      one thread per interior face node: Riemann flux (central /
//               LLF / Roe with Harten's entropy fix) plus the BR1 average of
//               the viscous flux (FP64: also the halo faces of a partitioned
//               mesh);
//   k_bc        inflow / outflow face nodes (exterior-state Riemann flux);
//   k_halo_face FP32: faces shared with another rank of a partitioned mesh;
//   k_wall      wall face nodes: mirror state and the wall-stress model (may
//               run on a side stream beside k_lift and k_face);
//   k_volume    one CTA per element: two-point flux differencing (KEP or
//               entropy-conserving) with the split-form matrix DVS = 2D - B/w
//               (zero corners), the surface integral, 1/J scaling, body force,
//               and either Ut or the LSERK4 register update of U and dU (N = 7:
//               swizzled shared-memory node slots, vslot; FP64: each pair at
//               distance n/2 formed once).
// R is the arithmetic type of the fluxes and their sums (double, or float in
// the mixed form); the state U, dU, the pressure recovery and the RK update
// are always double.  The FP32 form also keeps per-stage FP32 primitives
// relative to a reference state (k_prim32 / the stage epilogue) and, with the
// Pirozzoli flux, sums flux differences (flux_delta) instead of fluxes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <type_traits>

namespace dg {

enum { ST_NONFINITE = 1, ST_WM_NOCONV = 2, ST_BOUNDS = 4 };

// Index checks of the bounds-checking build (DG_DEBUG_BOUNDS): an index
// gathered through the mesh tables that lies outside [0, n) sets the status
// flag that dg_check_status reports as DG_ERR_DEVICE_BOUNDS and is replaced by
// 0, so that the access stays inside the array; nothing traps.  The ordinary
// build compiles the checks away.
__device__ __forceinline__ int chk_idx(int i, int n, int* status) {
#ifdef DG_DEBUG_BOUNDS
  if (i < 0 || i >= n) {
    if (status) atomicOr(status, ST_BOUNDS);
    return 0;
  }
#else
  (void)n; (void)status;
#endif
  return i;
}

struct PhysDev {
  double gamma, gm1, R, mu, Pr, cp, kcond, rcp_R;
  double rgm1;    // 1 / (gamma - 1)
  double cp_Pr;   // cp / Pr: conductivity per unit viscosity
  double suth_S;  // Sutherland constant (> 0: mu(T) = suth_C T^(3/2) / (T + S))
  double suth_C;  // mu_ref (T_ref + S) / T_ref^(3/2)
  double p_ref;   // constant removed from p in the momentum fluxes
  double rho_ref, h_ref;  // FP32-mixed form: reference density and enthalpy removed from its FP32 primitives
  double ec_q[5];  // 2 (gamma - 1)^-1 times the t^k coefficients of Q(t) = 2 s / sinh 2s (entropy-conserving flux)
  double f[3];
  double kappa, B, hwm;
  int law, vol_flux, surf_flux, viscous;
  int sutherland, has_force;  // suth_S > 0; f != 0
  int fs_diff;                // FP32 Pirozzoli form: surface fluxes stored per side as F* - F(U_side)
  double U_in[5], p_out;      // inflow state (conservative) and outflow pressure
  double T_wall;              // isothermal wall temperature (<= 0: adiabatic walls)
  int wm_maxit;               // iteration cap of the law-of-the-wall solve (bracket growth + Newton)
  int lift_df;                // FP64 viscous form at odd N: lifting in double-float arithmetic (k_lift_df)
  // FP32 copies of the constants the FP32 kernels use (a double-to-float
  // conversion is an FP64-pipe instruction)
  struct {
    float p_ref, rcp_R, rgm1, gamma, mu, kcond, cp_Pr, suth_C, suth_S, rho_ref, h_ref;
    float g_gm1, h_p, h_r;  // gamma / (gamma - 1); p_ref (rho_ref = 0) or 0; p_ref / rho_ref or 0
    float T_lift;           // rho_ref > 0: p_ref / (rho_ref R), else 0
    float ec_q[5];
  } f32c;
};

// a PhysDev constant in the flux type R
template <typename R>
__device__ __forceinline__ R cR(double d, float f) {
  if constexpr (std::is_same<R, float>::value) {
    (void)d;
    return f;
  } else {
    (void)f;
    return (R)d;
  }
}

// device-side views of the context's arrays
template <typename R>
struct MeshDev {
  int K, F, n_interior, n_wall, n_bc;  // faces: interior, walls, inflow / outflow, then halo
  int n_halo;                          // halo faces of a partitioned mesh (the last n_halo faces)
  const double* halo_U;                // [n_halo][5][n2] remote traces of the state
  const R* halo_G;                     // [n_halo][4][n2] remote outward viscous fluxes
  const R* Ja;           // [9][K*n3] (dir*3+comp)
  const R* invJ;         // [K*n3]
  const double* fgeo;    // [4][F*n2]
  const int* nbr;        // [K*6]
  const int* elem_face;  // [K*6]
  const int4* faces;     // [F]
  const int* ws_elem;    // [n_wall*n2]
  const double* ws_lag;  // [n_wall*n2*3*n]
  float* W32;            // FP32-mixed form: [6][K*n3] primitives of the input state (null in FP64)
  double* W64;           // FP64 viscous form: [7][K*n3] primitives (rho, u, v, w, p - p_ref, h, T) of the
                         // input state, stored by k_prim64, read by k_lift, k_face and k_volume (null: formed
                         // per use)
  const double* JaJ;     // FP64 viscous form: [9][K*n3] Ja / J (dir*3+comp)
  const double* Mj;      // FP64 viscous form: [6][K*n3] (Ja Ja^T) / J (00, 11, 22, 01, 02, 12)
  // double-float lifting: Ja, Ja / J and (Ja Ja^T) / J as (hi, lo) float pairs
  // [24][K*n3], and the lifted primitives (u, v, w, T - T_ref) [4][K*n3]
  // written by k_prim64 (null unless that lifting is selected)
  const float2* lift_M2;
  float2* lift_W2;
  // FP64 volume kernel at N = 7: the metric sums a_i + a_m of every pair it
  // evaluates (pair_main / pair_half below), fixed with the mesh
  const double* pairA;
  double* wm_t;          // [n_wall*n2] last wall-law solution per wall node (warm start; may be null)
  int* status;           // device status flags (index checks of the bounds-checking build)
};

template <int N>
struct Tables {
  double D[(N + 1) * (N + 1)];
  double DVS8[(N + 1) * (N + 1)];   // (2D - B/w) / 8
  double Dvisc[(N + 1) * (N + 1)];  // (w_m / w_i) D_mi
  double iw[N + 1];                 // 1 / w
  float D32[(N + 1) * (N + 1)];     // D and Dvisc rounded to FP32 (kernel-parameter
  float Dvisc32[(N + 1) * (N + 1)]; // operands of the FP32 line contractions) and
  float D32lo[(N + 1) * (N + 1)];   // their rounding remainders (the double-float
  float Dvisc32lo[(N + 1) * (N + 1)];  // lifting's coefficients hi + lo), and the
  // even/odd tables of D and Dvisc (LineEO::coef) as hi + lo
  float Deo32[(N + 1) * ((N + 1) / 2)], Deo32lo[(N + 1) * ((N + 1) / 2)];
  float Dveo32[(N + 1) * ((N + 1) / 2)], Dveo32lo[(N + 1) * ((N + 1) / 2)];
};

// Node slot in shared memory of the FP32 lifting kernel at N = 7 (node index
// i + 8 j + 64 k): bank bits (i0^j0^k0, i1^j1^k1, i2^j2^k2, i1^j0, i0^i1^j1),
// row (j2, k).  A bijection of the 512 nodes under which the 32 lanes of a
// warp hit 32 distinct banks when they hold one node each (consecutive
// nodes) and when each holds a line along xi, eta or zeta (consecutive line
// indices, the same position on the line): checked on the host.
__device__ __forceinline__ int lift_slot8(int node) {
  const int i = node & 7, j = (node >> 3) & 7, k = node >> 6;
  const int bank = ((i ^ j ^ k) & 7) | ((((i >> 1) ^ j) & 1) << 3) | (((i ^ (i >> 1) ^ (j >> 1)) & 1) << 4);
  return bank | (((j >> 2) | (k << 1)) << 5);
}

template <int N>
__device__ __forceinline__ int fnode(int l, int a, int b) {
  constexpr int n = N + 1;
  switch (l) {
    case 0: return n * (a + n * b);
    case 1: return N + n * (a + n * b);
    case 2: return a + n * n * b;
    case 3: return a + n * (N + n * b);
    case 4: return a + n * b;
    default: return a + n * (b + n * N);
  }
}

// Face-local index a' + n b' of the node of the other side's face that
// coincides with node ab = a + n b of this side's face, for the orientation
// code o (dg.h): (s, t) = (o & 1) ? (b, a) : (a, b), a' = (o & 2) ? N - s : s,
// b' = (o & 4) ? N - t : t.
template <int N>
__device__ __forceinline__ int omap_ab(int o, int ab) {
  constexpr int n = N + 1;
  const int a = ab % n, b = ab / n;
  const int s = (o & 1) ? b : a, t = (o & 1) ? a : b;
  return ((o & 2) ? N - s : s) + n * ((o & 4) ? N - t : t);
}

__device__ __forceinline__ int orient_inv(int o) {
  return (o & 1) ? (1 | (((o >> 2) & 1) << 1) | (((o >> 1) & 1) << 2)) : o;
}

// Encodings of the face tables (built by the host geometry):
//   faces[f] = (master element, master face, slave element, slave face
//     | 8 o) for interior faces, o the orientation from the master's face
//     nodes to the slave's; halo faces: (local element, local face, halo
//     index, master | 8 o_own), o_own from the local face's nodes to the
//     master's (0 when the local element is the master);
//   elem_face[e * 6 + l] = 16 f + 2 o_own + side (side 1: the slave).
// The face arrays (surface fluxes, normals, halo traces) are indexed in the
// master's face-node order.
template <int N>
struct NbrNode {
  int e;     // neighbour element
  int l;     // its local face
  int ab;    // face-local index of the coinciding node on that face
};

template <int N, typename M>
__device__ __forceinline__ NbrNode<N> neighbour_node(const M& m, int e, int l, int ab) {
  const int code = m.elem_face[e * 6 + l];
  const int4 fc = m.faces[chk_idx(code >> 4, m.F, m.status)];
  if (code & 1) return NbrNode<N>{chk_idx(fc.x, m.K, m.status), fc.y, omap_ab<N>((code >> 1) & 7, ab)};
  return NbrNode<N>{chk_idx(fc.z, m.K, m.status), fc.w & 7, omap_ab<N>(fc.w >> 3, ab)};
}

// (1/x for x > 0: rcp_t, defined after the FP64 <-> FP32 conversions below)
template <typename R>
__device__ __forceinline__ R rcp_t(R x);

// Dynamic viscosity at temperature T: constant mu, or Sutherland's law
// mu_ref (T / T_ref)^(3/2) (T_ref + S) / (T + S) (the paper's Sec. 4 gas model).
template <typename R>
__device__ __forceinline__ R sutherland(const PhysDev& ph, R T) {
  return cR<R>(ph.suth_C, ph.f32c.suth_C) * T * sqrt(T) / (T + cR<R>(ph.suth_S, ph.f32c.suth_S));
}

// Logarithmic mean L(a, b) = (a - b) / ln(a / b) of two positive numbers,
// needed by the entropy-conserving flux, written through s = a + b and
// u = ((a - b) / (a + b))^2.  With f = (a - b) / (a + b), ln(a / b) =
// 2 artanh(f) = 2 f (1 + u/3 + u^2/5 + u^3/7 + ...), so
//   L = (s / 2) g(u),  g = f / artanh(f) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
//   1 / L = (2 / s) P(u),  P = artanh(f) / f = 1 + u/3 + u^2/5 + u^3/7 + ...
// Truncated after u^3 the series are exact to rounding for u below LOGMEAN_CUT
// (next terms 0.03 u^4 and u^4 / 9); above it the logarithm is evaluated.
template <typename R>
struct LogMeanCut;
template <>
struct LogMeanCut<double> { static constexpr double v = 1e-4; };
template <>
struct LogMeanCut<float> { static constexpr float v = 1e-2f; };

template <typename R>
__device__ __forceinline__ R logmean_g(R u) {  // f / artanh(f)
  return R(1) - u * (R(1.0 / 3.0) + u * (R(4.0 / 45.0) + u * R(44.0 / 945.0)));
}
template <typename R>
__device__ __forceinline__ R logmean_P(R u) {  // artanh(f) / f
  return R(1) + u * (R(1.0 / 3.0) + u * (R(1.0 / 5.0) + u * R(1.0 / 7.0)));
}

// ln(a / b) / (2 f) for the slow branch: artanh(f) / f from the logarithm
template <typename R>
__device__ __forceinline__ R logmean_P_slow(R a, R b) {
  const R d = a - b;
  return log1p(d / b) * (a + b) / (R(2) * d);
}

// The volume kernel evaluates the same means without a division per pair,
// through t = (a - b)^2 / (4 a b) = sinh^2(l / 2), l = ln(a / b), formed from
// per-node reciprocals.  With s = asinh(sqrt(t)):
//   L = ((a + b) / 2) G(t),        G = tanh(s) / s
//   1 / L = ((1/a + 1/b) / 2) Q(t), Q = 2 s / sinh(2 s)
//   1 / (a + b) = ((1/a + 1/b) / 4) / (1 + t)
// Series through t^4 (the t^5 terms are below 0.4 t^5):
//   G = 1 - t/3 + 11t^2/45 - 191t^3/945 + 2497t^4/14175,
//   Q = 1 - 2t/3 + 8t^2/15 - 16t^3/35 + 128t^4/315 (the volume kernel takes it
//   times 2 / (gamma - 1) from PhysDev::ec_q), 1 / (1 + t) = 1 - t + t^2 - t^3 + t^4.
template <typename R>
__device__ __forceinline__ R logmean_G(R t) {
  return R(1) + t * (R(-1.0 / 3.0) + t * (R(11.0 / 45.0) + t * (R(-191.0 / 945.0) + t * R(2497.0 / 14175.0))));
}

// exterior state of an inflow (code -2: the prescribed state) or outflow
// (code -3: interior density and velocity, prescribed pressure) face node
__device__ __forceinline__ void ghost_state(const PhysDev& ph, int code, const double U[5], double Ub[5]) {
  if (code == -2) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Ub[v] = ph.U_in[v];
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) Ub[v] = U[v];
    Ub[4] = fma(ph.p_out, ph.rgm1, 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0]);
  }
}

__device__ __forceinline__ bool finite_bits(double x) {
  const unsigned hi = (unsigned)(__double_as_longlong(x) >> 32);
  return (hi & 0x7ff00000u) != 0x7ff00000u;
}

// Conversions between FP64 and FP32 built from the bit patterns with integer
// operations.  On GB300 the conversion instructions issue to the FP64 pipe
// (2 lanes per clock and SM, a 64th of the FP32 rate); the FP32-mixed
// kernels convert some twenty values per node and stage.
//
// f2d_bits: the exact widening of a float (FP32 subnormals give signed zero;
// infinities and NaN stay so).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned x = __float_as_uint(f);
  const unsigned e = (x >> 23) & 0xffu;
  const unsigned s = x & 0x80000000u;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;  // 1023 - 127
  const unsigned hi = e == 0u ? s : (s | (ed << 20) | ((x >> 3) & 0xfffffu));
  const unsigned lo = e == 0u ? 0u : (x << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// d2f_bits: rounding to the nearest float, ties to even, for results in the
// FP32 normal range (smaller magnitudes give signed zero, larger ones
// infinity; NaN stays NaN).  With rem, also the rounding remainder d - f as
// a float, to 2^-46 |d| (the remainder's 29 bits are kept to 23; zero where
// 2^-46 |d| falls below the FP32 normal range).
__device__ __forceinline__ float d2f_bits(double d, float* rem = nullptr) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned s = hi & 0x80000000u;
  const int ed = (int)((hi >> 20) & 0x7ffu);
  const int e = ed - 896;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the 23 bits kept
  const unsigned r = lo & 0x1fffffffu;                        // the 29 bits dropped
  const unsigned up = (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
  unsigned bits = ((unsigned)e << 23 | m) + up;  // a carry moves into the exponent
  bits = e <= 0 ? 0u : bits;
  bits = e >= 255 ? 0x7f800000u : bits;
  bits = (ed == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : bits;
  if (rem) {
    // d - f = (r - up 2^29) 2^(E - 52), E = ed - 1023; |r - up 2^29| <= 2^28,
    // taken to 23 bits (>> 6) and converted exactly by the 1.5 2^23 shift
    const int q = ((int)r - (int)(up << 29)) >> 6;
    const float qf = __int_as_float(0x4B400000 + q) - 12582912.0f;
    const int pe = ed - 1023 - 46 + 127;  // biased exponent of 2^(E - 46)
    const float rm = (pe >= 1 && ed != 0x7ff) ? qf * __int_as_float(pe << 23) : 0.0f;
    *rem = __uint_as_float(__float_as_uint(rm) ^ s);  // the sign of d
  }
  return __uint_as_float(s | bits);
}

// 1/x for x > 0 in double (in the FP32 normal range): the FP32 reciprocal of
// x rounded to FP32, refined by two Newton steps (relative error ~1e-7 ->
// 1e-14 -> below 1 ulp), 4 FP64 FMAs instead of the IEEE division sequence
// (GB300 issues 2 FP64 operations per clock per SM); the conversions are
// built from the bit patterns (the same values as the conversion
// instructions, without their FP64-pipe slots).
__device__ __forceinline__ double rcp_pos(double x) {
  double r = f2d_bits(__frcp_rn(d2f_bits(x)));
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

template <>
__device__ __forceinline__ double rcp_t<double>(double x) { return rcp_pos(x); }
template <>
__device__ __forceinline__ float rcp_t<float>(float x) { return __frcp_rn(x); }

// sqrt(x) for x > 0 in the FP32 normal range: s = x r with r the FP32
// reciprocal square root of x rounded to FP32 (relative error d ~ 2^-22),
// then two Newton steps s <- s + (x - s^2) r / 2, each taking the relative
// error e to about -d e - e^2 / 2 (d -> 1.5 d^2 ~ 1e-13 -> ~1e-20, below
// the final rounding): 5 FP64 operations
__device__ __forceinline__ double sqrt_pos(double x) {
  const float rf = rsqrtf(d2f_bits(x));
  const double r = f2d_bits(rf), hr = f2d_bits(0.5f * rf);
  double s = x * r;
  s = fma(fma(-s, s, x), hr, s);
  s = fma(fma(-s, s, x), hr, s);
  return s;
}

template <typename R>
__device__ __forceinline__ R sqrt_t(R x);
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt_pos(x); }
template <>
__device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }

// Primitive state in the flux type.  p is recovered in double from the
// double state (p = (gamma-1)(E - rho |u|^2 / 2) cancels at low Mach number)
// and stored as p - p_ref (the momentum fluxes see only the deviation from
// the constant reference pressure; a constant pressure contributes nothing to
// the element residual by the discrete metric identities).  h = (E + p)/rho
// uses the full pressure.
template <typename R>
struct Prim {
  R rho, u, v, w, p, h;
};

template <typename R>
__device__ __forceinline__ Prim<R> primitive(const double U0, const double U1, const double U2,
                                             const double U3, const double U4, const PhysDev& ph) {
  Prim<R> q;
  const double ir = rcp_pos(U0);
  const double u = U1 * ir, v = U2 * ir, w = U3 * ir;
  const double p = ph.gm1 * (U4 - 0.5 * (U1 * u + U2 * v + U3 * w));
  q.rho = (R)U0; q.u = (R)u; q.v = (R)v; q.w = (R)w; q.p = (R)(p - ph.p_ref);
  q.h = (R)((U4 + p) * ir);
  return q;
}

// Mixed form: everything in FP32 except the pressure recovery, whose
// cancellation E - rho |u|^2 / 2 is taken in FP64 (two FP64 operations).
// (Forming the velocity in FP64 and rounding it once lowers the Ut error by
// only ~4 % and costs 40 % of the mixed path's time: not done.)
template <>
__device__ __forceinline__ Prim<float> primitive<float>(const double U0, const double U1, const double U2,
                                                        const double U3, const double U4, const PhysDev& ph) {
  Prim<float> q;
  const float rho = (float)U0, ir = 1.0f / rho;
  const float m1 = (float)U1, m2 = (float)U2, m3 = (float)U3;
  q.rho = rho; q.u = m1 * ir; q.v = m2 * ir; q.w = m3 * ir;
  const float ke = 0.5f * (m1 * q.u + m2 * q.v + m3 * q.w);
  const double pr = fma(ph.gm1, U4 - (double)ke, -ph.p_ref);  // p - p_ref
  q.p = (float)pr;
  q.h = ((float)U4 + q.p + ph.f32c.p_ref) * ir;
  return q;
}

// FP32-mixed storage form: (rho - rho_ref, u, v, w, p - p_ref, h - h_ref), the
// shifted density and pressure formed in FP64 before rounding, so that the
// difference of two nodes' values carries the rounding of their deviations
// from the reference state.  The shifted enthalpy follows from those two in
// FP32 (ideal gas, E = p / (gamma - 1) + rho |u|^2 / 2):
//   h - h_ref = (gamma / (gamma - 1) (p' - (p_ref / rho_ref) rho') + rho |u|^2 / 2) / rho
// (rho_ref = 0: h = (gamma / (gamma - 1) (p' + p_ref) + rho |u|^2 / 2) / rho)
//
// With lo given, the velocity is also returned as an unevaluated sum of two
// floats, u = q.u + lo->u to about 1e-12 relative (q.u itself carries a few
// FP32 roundings: of m, of 1 / rho and of the product).  The flux-difference
// form takes the velocity differences of two nodes from these pairs: rounded
// to FP32, the velocity (O(1) at any Mach number) put an error of eps32 |u|
// into every difference, the largest input error of the form (about 1.6e-5
// of the Ut of the 48^3 curved box at Mach 0.3).  The low parts come from
// the FP32 residual m - u rho, formed with FMAs:
//   r = (m_hi - u rho_ref) - u rho' + m_lo,  lo = r / rho,
// where m_lo = m - m_hi is the rounding of the conversion to FP32 (the
// remainder that d2f_bits returns from the dropped bits).
struct Lo3 {
  float u, v, w;
};

__device__ __forceinline__ Prim<float> prim32_shifted(const double U0, const double U1, const double U2,
                                                      const double U3, const double U4, const PhysDev& ph,
                                                      Lo3* lo = nullptr) {
  Prim<float> q;
  const double rd = U0 - ph.rho_ref;
  q.rho = d2f_bits(rd);
  const float ir = 1.0f / (ph.f32c.rho_ref + q.rho);
  float ml1, ml2, ml3;  // the roundings m - (float)m
  const float m1 = d2f_bits(U1, &ml1), m2 = d2f_bits(U2, &ml2), m3 = d2f_bits(U3, &ml3);
  q.u = m1 * ir; q.v = m2 * ir; q.w = m3 * ir;
  const float ke = 0.5f * (m1 * q.u + m2 * q.v + m3 * q.w);
  const double pr = fma(ph.gm1, U4 - f2d_bits(ke), -ph.p_ref);  // p - p_ref
  q.p = d2f_bits(pr);
  q.h = fmaf(ph.f32c.g_gm1, q.p + ph.f32c.h_p - ph.f32c.h_r * q.rho, ke) * ir;
  if (lo) {
    // (the rounding of rho - rho_ref, relative eps32 of a small deviation,
    // changes u by a relative 1e-10 or so: left out)
    auto low = [&](float ml, float mh, float uh) {
      float r = fmaf(-uh, ph.f32c.rho_ref, mh);
      r = fmaf(-uh, q.rho, r);
      return (r + ml) * ir;
    };
    lo->u = low(ml1, m1, q.u);
    lo->v = low(ml2, m2, q.v);
    lo->w = low(ml3, m3, q.w);
  }
  return q;
}

// full values from the storage form
__device__ __forceinline__ Prim<float> unshift32(Prim<float> q, const PhysDev& ph) {
  q.rho += ph.f32c.rho_ref;
  q.h += ph.f32c.h_ref;
  return q;
}

// FP64 primitives and the temperature T = p / (rho R) (from the unshifted p).
// Not inlined: one compiled body serves k_prim64, which stores them for the
// lifting, face and volume kernels, and the kernels that form them for a
// remote trace (or, without the stored array, per use); all then agree
// bitwise whatever the surrounding code lets the compiler contract.
static __device__ __noinline__ Prim<double> primitive_T(const double U0, const double U1, const double U2,
                                                 const double U3, const double U4, const PhysDev& ph, double& T) {
  Prim<double> q;
  const double ir = rcp_pos(U0);
  const double u = U1 * ir, v = U2 * ir, w = U3 * ir;
  const double p = ph.gm1 * (U4 - 0.5 * (U1 * u + U2 * v + U3 * w));
  q.rho = U0; q.u = u; q.v = v; q.w = w; q.p = p - ph.p_ref;
  const double pir = p * ir;  // p / rho: h = E / rho + p / rho, T = (p / rho) / R
  q.h = fma(U4, ir, pir);
  T = pir * ph.rcp_R;
  return q;
}

__device__ __forceinline__ Prim<double> load_prim64(const double* __restrict__ W, size_t S, size_t g) {
  return Prim<double>{W[g], W[S + g], W[2 * S + g], W[3 * S + g], W[4 * S + g], W[5 * S + g]};
}

__device__ __forceinline__ void store_prim64(double* __restrict__ W, size_t S, size_t g, const Prim<double>& q,
                                             double T) {
  W[g] = q.rho; W[S + g] = q.u; W[2 * S + g] = q.v; W[3 * S + g] = q.w;
  W[4 * S + g] = q.p; W[5 * S + g] = q.h; W[6 * S + g] = T;
}

// the primitives of the input state, stored for the operator's kernels (FP64
// viscous form); run before the lifting kernel whenever they are stale
// (W2: the double-float lifting's (u, v, w, T - T_ref) as (hi, lo) float
// pairs, or null)
static __global__ void k_prim64(long long S, const double* __restrict__ U, const PhysDev ph, double* __restrict__ W,
                                float2* __restrict__ W2) {
  const double Tref = ph.rho_ref > 0.0 ? ph.p_ref * ph.rcp_R / ph.rho_ref : 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < S; g += (long long)gridDim.x * blockDim.x) {
    double T;
    const Prim<double> q = primitive_T(U[g], U[S + g], U[2 * S + g], U[3 * S + g], U[4 * S + g], ph, T);
    store_prim64(W, (size_t)S, (size_t)g, q, T);
    if (W2) {
      const double x[4] = {q.u, q.v, q.w, T - Tref};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float lo;
        const float hi = d2f_bits(x[v], &lo);
        W2[v * S + g] = make_float2(hi, lo);
      }
    }
  }
}

// x -> (hi, lo) float pairs, both rounded to nearest (hi + lo = x to 2^-48;
// the double-float kernels' metric arrays, split once)
static __global__ void k_split_pairs(long long n, const double* __restrict__ x, float2* __restrict__ y) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const float hi = __double2float_rn(x[g]);
    y[g] = make_float2(hi, __double2float_rn(x[g] - (double)hi));
  }
}

template <typename R>
__device__ __forceinline__ void velocity_temperature(const double U0, const double U1, const double U2,
                                                     const double U3, const double U4, const PhysDev& ph,
                                                     R& u, R& v, R& w, R& T) {
  const double ir = rcp_pos(U0);
  const double ud = U1 * ir, vd = U2 * ir, wd = U3 * ir;
  const double pr = ph.gm1 * (U4 - 0.5 * U0 * (ud * ud + vd * vd + wd * wd));
  u = (R)ud; v = (R)vd; w = (R)wd; T = (R)(pr * ph.rcp_R * ir);
}

template <>
__device__ __forceinline__ void velocity_temperature<float>(const double U0, const double U1, const double U2,
                                                            const double U3, const double U4,
                                                            const PhysDev& ph, float& u, float& v, float& w,
                                                            float& T) {
  const Prim<float> q = primitive<float>(U0, U1, U2, U3, U4, ph);
  u = q.u; v = q.v; w = q.w;
  T = (q.p + ph.f32c.p_ref) * ph.f32c.rcp_R / q.rho;
}

// FP32 lifting: the velocity and the temperature relative to T_lift =
// p_ref / (rho_ref R), the temperature of the storage form's reference state:
//   T - T_lift = (p' rho_ref - p_ref rho') / (rho rho_ref R)
// from the shifted density and pressure of the storage form.  Rounded to FP32
// the temperature itself (O(p_ref / rho_ref): 7.9 at Mach 0.3, 71 at Mach 0.1)
// would put an error eps32 T into every node's value, which the heat flux,
// the derivative of the lifted gradient, amplifies by (N^2 / h)^2; the
// deviation carries the rounding of the deviation only.  (rho_ref = 0: T.)
__device__ __forceinline__ void velocity_temperature32s(const Prim<float>& q, const PhysDev& ph, float& u, float& v,
                                                        float& w, float& Tp) {
  u = q.u; v = q.v; w = q.w;
  if (ph.f32c.rho_ref > 0.0f) {
    const float rho = ph.f32c.rho_ref + q.rho;
    Tp = fmaf(-ph.f32c.h_r, q.rho, q.p) * ph.f32c.rcp_R / rho;  // h_r = p_ref / rho_ref
  } else {
    Tp = (q.p + ph.f32c.p_ref) * ph.f32c.rcp_R / q.rho;
  }
}

// the same from an FP64 state (traces of halo and boundary faces)
__device__ __forceinline__ void velocity_temperature32s_of(const double U0, const double U1, const double U2,
                                                           const double U3, const double U4, const PhysDev& ph,
                                                           float& u, float& v, float& w, float& Tp) {
  const double ir = 1.0 / U0;
  const double ud = U1 * ir, vd = U2 * ir, wd = U3 * ir;
  const double pr = ph.gm1 * (U4 - 0.5 * U0 * (ud * ud + vd * vd + wd * wd));
  u = (float)ud; v = (float)vd; w = (float)wd;
  Tp = (float)(pr * ph.rcp_R * ir - (double)ph.f32c.T_lift);
}

// Entropy-conserving two-point flux of Chandrashekar (the paper's Sec. 4
// volume flux) along a (a need not be unit), with beta = rho / (2 p):
//   F_rho = ln-mean(rho) {u}.a,  F_m = p~ a + {u} F_rho,
//   F_E = F_rho (1 / (2 (gamma - 1) ln-mean(beta)) - {|u|^2} / 2) + {u} . F_m,
//   p~ = {rho} / (2 {beta}).
// The momentum flux carries p~ - p_ref = (bA p'A + bB p'B) / (bA + bB)
// (p' = p - p_ref), the same value without the O(p_ref) cancellation.
template <typename R>
__device__ __forceinline__ void twopoint_ec(const Prim<R>& A, const Prim<R>& B, R a0, R a1, R a2, R F[5],
                                            const PhysDev& ph) {
  const R pref = cR<R>(ph.p_ref, ph.f32c.p_ref);
  const R bA = A.rho * rcp_t<R>(R(2) * (A.p + pref)), bB = B.rho * rcp_t<R>(R(2) * (B.p + pref));
  const R sr = A.rho + B.rho, dr = A.rho - B.rho, sb = bA + bB, db = bA - bB;
  const R rr = rcp_t<R>(sr), rb = rcp_t<R>(sb);
  const R ur = (dr * rr) * (dr * rr), ub = (db * rb) * (db * rb);
  const R rho_ln = ur < LogMeanCut<R>::v ? R(0.5) * sr * logmean_g<R>(ur) : dr / log1p(dr / B.rho);
  const R Pb = ub < LogMeanCut<R>::v ? logmean_P<R>(ub) : logmean_P_slow<R>(bA, bB);
  const R u = R(0.5) * (A.u + B.u), v = R(0.5) * (A.v + B.v), w = R(0.5) * (A.w + B.w);
  const R ua = u * a0 + v * a1 + w * a2;
  const R pt = (bA * A.p + bB * B.p) * rb;  // p~ - p_ref
  const R f0 = rho_ln * ua;
  F[0] = f0;
  F[1] = f0 * u + pt * a0;
  F[2] = f0 * v + pt * a1;
  F[3] = f0 * w + pt * a2;
  const R k2 = R(0.25) * (A.u * A.u + A.v * A.v + A.w * A.w + B.u * B.u + B.v * B.v + B.w * B.w);
  // 1 / (2 (gamma - 1) beta_ln) = rb P / (gamma - 1)
  F[4] = f0 * (rb * Pb * cR<R>(ph.rgm1, ph.f32c.rgm1) + (u * u + v * v + w * w) - k2) + (pt + pref) * ua;
}

__device__ __forceinline__ void velocity_temperature32(const Prim<float>& q, const PhysDev& ph, float& u, float& v,
                                                       float& w, float& T) {
  u = q.u; v = q.v; w = q.w;
  T = (q.p + ph.f32c.p_ref) * ph.f32c.rcp_R / q.rho;
}

// Two-point KEP flux F#(L, R) . a (a need not be unit); kind 2 is the
// entropy-conserving flux above (FP64 and FP32 only: the adjoint covers the
// KEP fluxes).
template <typename R>
__device__ __forceinline__ void twopoint(int kind, const Prim<R>& A, const Prim<R>& B, R a0, R a1, R a2,
                                         R F[5], const PhysDev& ph) {
  if constexpr (std::is_same<R, double>::value || std::is_same<R, float>::value) {
    if (kind == 2) {
      twopoint_ec<R>(A, B, a0, a1, a2, F, ph);
      return;
    }
  }
  const R pref = cR<R>(ph.p_ref, ph.f32c.p_ref);
  if (kind == 0) {
    // Pirozzoli from the sums S = x_A + x_B ({x} = S / 2), the powers of two
    // applied once: m = {rho}{u}.a = Sr (Su.a) / 4, F_k = m {u_k} + {p} a_k =
    // (m / 2) Su_k + (Sp / 2) a_k, F_4 = m {h} = (m / 2) Sh
    const R Sr = A.rho + B.rho, Su = A.u + B.u, Sv = A.v + B.v, Sw = A.w + B.w, Sp = A.p + B.p;
    const R m4 = Sr * (Su * a0 + Sv * a1 + Sw * a2);
    const R m8 = R(0.125) * m4, hp = R(0.5) * Sp;
    F[0] = R(0.25) * m4;
    F[1] = m8 * Su + hp * a0;
    F[2] = m8 * Sv + hp * a1;
    F[3] = m8 * Sw + hp * a2;
    F[4] = m8 * (A.h + B.h);
    return;
  }
  const R rho = R(0.5) * (A.rho + B.rho);
  const R u = R(0.5) * (A.u + B.u), v = R(0.5) * (A.v + B.v), w = R(0.5) * (A.w + B.w);
  const R p = R(0.5) * (A.p + B.p);
  const R ua = u * a0 + v * a1 + w * a2;
  const R m = rho * ua;
  F[0] = m;
  F[1] = m * u + p * a0;
  F[2] = m * v + p * a1;
  F[3] = m * w + p * a2;
  {  // Kennedy-Gruber: {rho}{u.a}{e} + {p}{u.a}, e = E / rho = h - p / rho (full p)
    const R pA = A.p + pref, pB = B.p + pref;
    const R eA = A.h - pA / A.rho, eB = B.h - pB / B.rho;
    F[4] = m * (R(0.5) * (eA + eB)) + (p + pref) * ua;
  }
}

// Numerical inviscid flux along the unit normal (nx, ny, nz), side A = master;
// dU = U_B - U_A (conservative) for the Lax-Friedrichs dissipation.
// subtracts the dissipation of the selected Riemann solver from F (drho: the
// density jump B - A when the caller has it more accurately than the values)
template <typename R>
__device__ __forceinline__ void riemann_dissipation(const PhysDev& ph, const Prim<R>& A, const Prim<R>& B,
                                                    const R dU[5], R nx, R ny, R nz, R F[5],
                                                    const R* drho = nullptr, const R* dvel = nullptr) {
  const R pref = cR<R>(ph.p_ref, ph.f32c.p_ref);
  const R g = cR<R>(ph.gamma, ph.f32c.gamma);
  if (ph.surf_flux == 1) {  // local Lax-Friedrichs (sound speed from the full pressure)
    const R cA = sqrt_t<R>(g * (A.p + pref) * rcp_t<R>(A.rho)), cB = sqrt_t<R>(g * (B.p + pref) * rcp_t<R>(B.rho));
    const R lA = fabs(A.u * nx + A.v * ny + A.w * nz) + cA;
    const R lB = fabs(B.u * nx + B.v * ny + B.w * nz) + cB;
    const R lam = R(0.5) * (lA >= lB ? lA : lB);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] -= lam * dU[v];
  } else if (ph.surf_flux == 2) {  // Roe with Harten's entropy fix on the acoustic waves
    // (reciprocals by rcp_t: in FP64 a Newton-refined estimate, the FP64
    // pipe being the bound; the correctly rounded reciprocal in FP32)
    const R sA = sqrt_t<R>(A.rho), sB = sqrt_t<R>(B.rho);
    const R is = rcp_t<R>(sA + sB);
    const R rt = sA * sB;
    // (the FP32 difference form passes the velocity jump from the velocities'
    // high and low parts: from the rounded velocities it would carry an error
    // eps32 |u| that the acoustic waves multiply by rho c)
    const R du = dvel ? dvel[0] : B.u - A.u, dv = dvel ? dvel[1] : B.v - A.v, dw = dvel ? dvel[2] : B.w - A.w;
    // Roe averages (sqrt(rho_A) x_A + sqrt(rho_B) x_B) / (sqrt(rho_A) + sqrt(rho_B))
    // as x_A + f (x_B - x_A), f = sqrt(rho_B) / (sqrt(rho_A) + sqrt(rho_B))
    const R f = sB * is;
    const R u = fma(f, du, A.u), v = fma(f, dv, A.v), w = fma(f, dw, A.w);
    const R H = fma(f, B.h - A.h, A.h);
    const R q2 = u * u + v * v + w * w;
    const R c2 = (g - R(1)) * (H - R(0.5) * q2);
    const R c = sqrt_t<R>(c2);
    const R un = u * nx + v * ny + w * nz;
    const R dr = drho ? *drho : B.rho - A.rho, dp = B.p - A.p;
    const R dun = du * nx + dv * ny + dw * nz;
    const R i2c2 = R(0.5) * rcp_t<R>(c2);
    const R a1 = (dp - rt * c * dun) * i2c2;
    const R a2 = dr - R(2) * dp * i2c2;
    const R a5 = (dp + rt * c * dun) * i2c2;
    R l1 = fabs(un - c), l2 = fabs(un), l5 = fabs(un + c);
    const R del = R(0.1) * c;
    if (l1 < del) l1 = (l1 * l1 + del * del) / (R(2) * del);
    if (l5 < del) l5 = (l5 * l5 + del * del) / (R(2) * del);
    const R w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5, ws = l2 * rt;
    const R dut = du - dun * nx, dvt = dv - dun * ny, dwt = dw - dun * nz;
    // sum of the waves' |lambda| alpha r: with the acoustic pair's sum and
    // difference, w1 (u - c n) + w2 u + w5 (u + c n) = u D0 + n c (w5 - w1)
    const R sw = w1 + w5, cdw = c * (w5 - w1);
    const R D0 = sw + w2;
    const R D1 = u * D0 + nx * cdw + ws * dut;
    const R D2 = v * D0 + ny * cdw + ws * dvt;
    const R D3 = w * D0 + nz * cdw + ws * dwt;
    // (u . du - un dun = u . (du - dun n))
    const R D4 = H * sw + un * cdw + w2 * (R(0.5) * q2) + ws * (u * dut + v * dvt + w * dwt);
    F[0] -= R(0.5) * D0; F[1] -= R(0.5) * D1; F[2] -= R(0.5) * D2;
    F[3] -= R(0.5) * D3; F[4] -= R(0.5) * D4;
  }
}

template <typename R>
__device__ __forceinline__ void riemann_d(const PhysDev& ph, const Prim<R>& A, const Prim<R>& B, const R dU[5],
                                          R nx, R ny, R nz, R F[5]) {
  twopoint<R>(ph.vol_flux, A, B, nx, ny, nz, F, ph);
  riemann_dissipation<R>(ph, A, B, dU, nx, ny, nz, F);
}

// FP32-mixed form with the Pirozzoli flux: two-point flux differences
//   G(i -> m) = F#(U_i, U_m; {a}) - F(U_i) . a_i
// formed from the differences of the two nodes' primitives (x_m = x_i + dx,
// {x} = x_i + dx / 2), so that their FP32 rounding error scales with the
// difference, not with the flux itself:
//   {u}.{a} - u_i.a_i = du/2 . {a} + u_i . da/2
//   G_rho = rho_i ({u}.{a} - u_i.a_i) + drho/2 ({u}.{a})
//   G_m   = G_rho {u} + rho_i (u_i.a_i) du/2 + dp/2 {a} + p_i da/2   (p = p - p_ref)
//   G_E   = G_rho {h} + rho_i (u_i.a_i) dh/2
// The split-form volume term is sum_m DVS_im G(i -> m) (the F(U_i) part sums to
// the boundary rows' -B/w F(U_i), which the surface term carries in the same
// difference form, F* - F(U_i)).
//
// G holds the part F(U_i) . da / 2, whose sum over a node's pairs is
// F(U_i) . sum_dir sum_m DVS_im (a_m - a_i) / 2 = F(U_i) . sum_dir sum_m D_im a_m:
// zero by the discrete metric identities of the curl-form metrics.  With the
// metrics rounded to FP32 the identities hold only to eps32 |a|, and that part
// then leaves an error eps32 |F(U_i)| N^2 / h in Ut, which the flux
// differences do not remove (the free-stream error of the rounded metrics;
// the largest error of the form on curved meshes, in the mass and energy rows
// where no p_ref shift makes F(U_i) small).  So G' = G - F(U_i) . da / 2 is
// summed instead, i.e. the identity is applied exactly:
//   G'_rho = rho_i du/2 . {a} + drho/2 ({u}.{a})
//   G'_m   = G'_rho {u} + rho_i (u_i . da/2) du/2 + rho_i (u_i.a_i) du/2 + dp/2 {a}
//   G'_E   = G'_rho {h} + rho_i (u_i . da/2) dh/2 + rho_i (u_i.a_i) dh/2
// (at faces da = 0 and G' = G).
struct NodeF {
  float rho, u, v, w, p, h;
  float ul, vl, wl;  // low parts of the velocity (u = u + ul, see prim32_shifted)
};

// i, m in the storage form of the FP32 primitives (rho, h shifted by
// rho_ref, h_ref): the differences come from the shifted values, the full
// density and enthalpy of node i are rebuilt where they multiply
__device__ __forceinline__ void flux_delta(const NodeF& i, const NodeF& m, float ai0, float ai1, float ai2, float da0,
                                           float da1, float da2, float rho_ref, float h_ref, float G[5]) {
  const float du = (m.u - i.u) + (m.ul - i.ul), dv = (m.v - i.v) + (m.vl - i.vl), dw = (m.w - i.w) + (m.wl - i.wl);
  const float dr = m.rho - i.rho, dp = m.p - i.p, dh = m.h - i.h;
  const float ri = rho_ref + i.rho;
  const float ab0 = fmaf(0.5f, da0, ai0), ab1 = fmaf(0.5f, da1, ai1), ab2 = fmaf(0.5f, da2, ai2);
  const float uia = i.u * ai0 + i.v * ai1 + i.w * ai2;          // u_i . a_i
  const float uida = 0.5f * (i.u * da0 + i.v * da1 + i.w * da2);  // u_i . da / 2
  const float dua = 0.5f * (du * ab0 + dv * ab1 + dw * ab2);      // du/2 . {a}
  const float g0 = ri * dua + 0.5f * dr * (uia + uida + dua);
  const float ruia = ri * (uia + uida);  // rho_i (u_i.a_i + u_i . da/2)
  G[0] = g0;
  G[1] = g0 * fmaf(0.5f, du, i.u) + 0.5f * (ruia * du + dp * ab0);
  G[2] = g0 * fmaf(0.5f, dv, i.v) + 0.5f * (ruia * dv + dp * ab1);
  G[3] = g0 * fmaf(0.5f, dw, i.w) + 0.5f * (ruia * dw + dp * ab2);
  G[4] = g0 * (h_ref + fmaf(0.5f, dh, i.h)) + 0.5f * ruia * dh;
}

// both orientations of a pair, G(i -> m) into Gi and G(m -> i) into Gm: the
// differences change sign between them and {a} does not, so they are formed
// once
__device__ __forceinline__ void flux_delta_pair(const NodeF& i, const NodeF& m, float ai0, float ai1, float ai2,
                                                float am0, float am1, float am2, float rho_ref, float h_ref,
                                                float Gi[5], float Gm[5]) {
  const float du = (m.u - i.u) + (m.ul - i.ul), dv = (m.v - i.v) + (m.vl - i.vl), dw = (m.w - i.w) + (m.wl - i.wl);
  const float dr = m.rho - i.rho, dp = m.p - i.p, dh = m.h - i.h;
  const float da0 = am0 - ai0, da1 = am1 - ai1, da2 = am2 - ai2;
  const float ab0 = fmaf(0.5f, da0, ai0), ab1 = fmaf(0.5f, da1, ai1), ab2 = fmaf(0.5f, da2, ai2);
  const float dua = 0.5f * (du * ab0 + dv * ab1 + dw * ab2);  // du/2 . {a}
  {
    const float ri = rho_ref + i.rho;
    const float uia = i.u * ai0 + i.v * ai1 + i.w * ai2;
    const float uida = 0.5f * (i.u * da0 + i.v * da1 + i.w * da2);
    const float g0 = ri * dua + 0.5f * dr * (uia + uida + dua);
    const float ruia = ri * (uia + uida);
    Gi[0] = g0;
    Gi[1] = g0 * fmaf(0.5f, du, i.u) + 0.5f * (ruia * du + dp * ab0);
    Gi[2] = g0 * fmaf(0.5f, dv, i.v) + 0.5f * (ruia * dv + dp * ab1);
    Gi[3] = g0 * fmaf(0.5f, dw, i.w) + 0.5f * (ruia * dw + dp * ab2);
    Gi[4] = g0 * (h_ref + fmaf(0.5f, dh, i.h)) + 0.5f * ruia * dh;
  }
  {
    // (with du -> -du, drho -> -drho, ..., da -> -da)
    const float rm = rho_ref + m.rho;
    const float uma = m.u * am0 + m.v * am1 + m.w * am2;
    const float umda = -0.5f * (m.u * da0 + m.v * da1 + m.w * da2);
    const float g0 = -(rm * dua + 0.5f * dr * (uma + umda - dua));
    const float ruma = rm * (uma + umda);
    Gm[0] = g0;
    Gm[1] = g0 * fmaf(-0.5f, du, m.u) - 0.5f * (ruma * du + dp * ab0);
    Gm[2] = g0 * fmaf(-0.5f, dv, m.v) - 0.5f * (ruma * dv + dp * ab1);
    Gm[3] = g0 * fmaf(-0.5f, dw, m.w) - 0.5f * (ruma * dw + dp * ab2);
    Gm[4] = g0 * (h_ref + fmaf(-0.5f, dh, m.h)) - 0.5f * ruma * dh;
  }
}

__device__ __forceinline__ NodeF nodef(const Prim<float>& q, const Lo3& l) {
  return NodeF{q.rho, q.u, q.v, q.w, q.p, q.h, l.u, l.v, l.w};
}

// face flux differences for both sides: D_A = F* - F(U_A).n, D_B = F* - F(U_B).n;
// A, B in the storage form (the dissipation takes the full values and the
// density jump of the shifted ones)
__device__ __forceinline__ void face_flux_delta(const PhysDev& ph, const Prim<float>& A, const Prim<float>& B,
                                                const Lo3& la, const Lo3& lb, const float dU[5], float nx, float ny,
                                                float nz, float DA[5], float DB[5]) {
  float Z[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  const float drho = B.rho - A.rho;
  const float dvel[3] = {(B.u - A.u) + (lb.u - la.u), (B.v - A.v) + (lb.v - la.v), (B.w - A.w) + (lb.w - la.w)};
  riemann_dissipation<float>(ph, unshift32(A, ph), unshift32(B, ph), dU, nx, ny, nz, Z, &drho, dvel);
  const float rr = ph.f32c.rho_ref, hr = ph.f32c.h_ref;
  flux_delta_pair(nodef(A, la), nodef(B, lb), nx, ny, nz, nx, ny, nz, rr, hr, DA, DB);
#pragma unroll
  for (int v = 0; v < 5; ++v) { DA[v] += Z[v]; DB[v] += Z[v]; }
}

// FP32 difference form: writes the master's (and, with both, the slave's)
// F* s - F(U_side).(n s) minus the viscous flux vis_w (gA - gB) (gB null: gA)
// into out (master) and out + 5 n2 (slave)
__device__ __forceinline__ void store_face_delta(const PhysDev& ph, const Prim<float>& A, const Prim<float>& B,
                                                 const Lo3& la, const Lo3& lb, const float dU[5], float nx, float ny,
                                                 float nz, float s, const float* gA, const float* gB, float vis_w,
                                                 float* out, int n2, bool both) {
  float DA[5], DB[5];
  face_flux_delta(ph, A, B, la, lb, dU, nx, ny, nz, DA, DB);
  out[0] = DA[0] * s;
  if (both) out[5 * n2] = DB[0] * s;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float vis = ph.viscous ? vis_w * (gB ? gA[v * n2] - gB[v * n2] : gA[v * n2]) : 0.f;
    out[(v + 1) * n2] = DA[v + 1] * s - vis;
    if (both) out[(v + 6) * n2] = DB[v + 1] * s - vis;
  }
}

template <typename R, typename S>
__device__ __forceinline__ void riemann(const PhysDev& ph, const Prim<R>& A, const S UA[5],
                                        const Prim<R>& B, const S UB[5], R nx, R ny, R nz, R F[5]) {
  R dU[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) dU[v] = (R)(UB[v] - UA[v]);
  riemann_d<R>(ph, A, B, dU, nx, ny, nz, F);
}

// ---------------------------------------------------------------------------
// FP32-mixed form: the FP32 primitives (rho, u, v, w, p - p_ref, h) of every
// node and the low parts of its velocity, W[9][K n^3] (rows 6-8: see
// prim32_shifted), formed once per stage from the FP64 state (by k_prim32,
// or by the previous stage's volume epilogue from the updated state) and read
// by the lifting, face and volume kernels.  The FP64 work of the primitive
// recovery (and of the double-to-float conversions) is then done once per node
// and stage instead of once per use.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_prim32(float* __restrict__ W, size_t S, size_t g, const Prim<float>& q,
                                             const Lo3& l) {
  W[g] = q.rho; W[S + g] = q.u; W[2 * S + g] = q.v; W[3 * S + g] = q.w; W[4 * S + g] = q.p; W[5 * S + g] = q.h;
  W[6 * S + g] = l.u; W[7 * S + g] = l.v; W[8 * S + g] = l.w;
}

__device__ __forceinline__ Lo3 load_lo32(const float* __restrict__ W, size_t S, size_t g) {
  return Lo3{W[6 * S + g], W[7 * S + g], W[8 * S + g]};
}

// storage form (rho - rho_ref, u, v, w, p - p_ref, h - h_ref)
__device__ __forceinline__ Prim<float> load_prim32(const float* __restrict__ W, size_t S, size_t g) {
  Prim<float> q;
  q.rho = W[g]; q.u = W[S + g]; q.v = W[2 * S + g]; q.w = W[3 * S + g]; q.p = W[4 * S + g]; q.h = W[5 * S + g];
  return q;
}

// full values (rho, u, v, w, p - p_ref, h)
__device__ __forceinline__ Prim<float> load_prim32_full(const float* __restrict__ W, size_t S, size_t g,
                                                        const PhysDev& ph) {
  return unshift32(load_prim32(W, S, g), ph);
}

// the primitives a boundary or halo face kernel forms from a conservative
// trace: FP64 directly; FP32 in the storage form (*st, for the flux-difference
// form) with the full values rebuilt from it
template <typename R>
__device__ __forceinline__ Prim<R> trace_prims(const double Ut[5], const PhysDev& ph, Prim<R>* st, Lo3* lo) {
  if constexpr (std::is_same<R, float>::value) {
    *st = prim32_shifted(Ut[0], Ut[1], Ut[2], Ut[3], Ut[4], ph, ph.fs_diff ? lo : nullptr);
    if (!ph.fs_diff) *lo = Lo3{0.f, 0.f, 0.f};
    return unshift32(*st, ph);
  } else {
    return primitive<R>(Ut[0], Ut[1], Ut[2], Ut[3], Ut[4], ph);
  }
}

static __global__ void k_prim32(long long S, const double* __restrict__ U, const PhysDev ph, float* __restrict__ W) {
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < S; x += (long long)gridDim.x * blockDim.x) {
    Lo3 l;
    const Prim<float> q = prim32_shifted(U[x], U[S + x], U[2 * S + x], U[3 * S + x], U[4 * S + x], ph, &l);
    store_prim32(W, (size_t)S, (size_t)x, q, l);
  }
}

// ---------------------------------------------------------------------------
// Wall model (paper Sec. 3.2, Algorithms 1-2), always in double.
// ---------------------------------------------------------------------------
// law L(w) and w L'(w) / L(w) for w = y+ (Reichardt, L = u+) or w = u+
// (Spalding, L = y+).  cst is the law's constant part: C = B - ln(kappa) /
// kappa (Reichardt) or e^(-kappa B) (Spalding), see law_const.
__device__ __forceinline__ double law_const(int law, double kap, double B) {
  return law == 1 ? B - log(kap) / kap : exp(-kap * B);
}

__device__ __forceinline__ void law_eval_c(int law, double w, double kap, double cst, double* L, double* wdL) {
  if (law == 1) {
    const double C = cst;
    const double e1 = exp(-w / 11.0), e2 = exp(-0.33 * w);
    const double Lv = log1p(kap * w) / kap + C * (1.0 - e1 - (w / 11.0) * e2);
    const double dL = 1.0 / (1.0 + kap * w) + C * (e1 / 11.0 - e2 / 11.0 + 0.33 * (w / 11.0) * e2);
    *L = Lv; *wdL = w * dL;
  } else {
    const double ku = kap * w;
    const double eb = cst, ek = exp(ku);
    const double t3 = ku * ku * ku / 6.0;
    const double Lv = w + eb * (ek - 1.0 - ku - 0.5 * ku * ku - t3 - 0.25 * ku * t3);
    const double dL = 1.0 + eb * kap * (ek - 1.0 - ku - 0.5 * ku * ku - t3);
    *L = Lv; *wdL = w * dL;
  }
}

__device__ __forceinline__ void law_eval(int law, double w, double kap, double B, double* L, double* wdL) {
  law_eval_c(law, w, kap, law_const(law, kap, B), L, wdL);
}

// Solve t + ln L(e^t) = ln Re_h (Re_h = h u / nu = u+ y+): bracket by growing
// steps from the laminar estimate t = ln(Re_h)/2, then Newton with bisection
// whenever a step would leave the bracket.  Returns u_tau (and *ok).  F is
// increasing in t; its value at the starting point is evaluated once.
static __device__ double solve_utau(int law, double u, double h, double nu, double kap, double B, int maxit,
                                    bool* ok) {
  *ok = true;
  if (!(u > 0.0)) return 0.0;
  const double lnRe = log(h * u / nu);
  const double cst = law_const(law, kap, B);
  auto F = [&](double t, double* dF) {
    const double w = exp(t);
    double L, wdL;
    law_eval_c(law, w, kap, cst, &L, &wdL);
    *dF = 1.0 + wdL / L;
    return t + log(L) - lnRe;
  };
  double dF;
  const double t0 = 0.5 * lnRe;
  const double F0 = F(t0, &dF);
  double lo = t0, hi = t0, st = 1.0;
  int it = 0;
  double Flo = F0;
  while (!(Flo < 0.0) && it < maxit) { lo -= st; st *= 2.0; ++it; Flo = F(lo, &dF); }
  st = 1.0;
  double Fhi = F0;
  while (!(Fhi > 0.0) && it < maxit) { hi += st; st *= 2.0; ++it; Fhi = F(hi, &dF); }
  double t = t0;
  if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
  bool done = false;
  for (; it < maxit; ++it) {
    const double Ft = F(t, &dF);
    if (Ft == 0.0) { done = true; break; }
    if (Ft < 0.0) lo = t; else hi = t;
    double nt = t - Ft / dF;
    const bool newton = (nt >= lo && nt <= hi);
    if (!newton) nt = 0.5 * (lo + hi);
    const double step = fabs(nt - t);
    t = nt;
    const double sc = fmax(1.0, fabs(t));
    if ((newton && step <= 1e-12 * sc) || hi - lo <= 2e-15 * sc) { done = true; break; }
  }
  *ok = done;
  return law == 1 ? exp(t) * nu / h : u / exp(t);
}

// Warm-started solve: up to four Newton steps from t_prev (the node's solution
// at its previous evaluation, NaN if none), stopping by the same rule as the
// bracketed solve; if they do not converge, the bracketed solve from scratch.
// *t_out receives the converged t.  The state changes little between stages, so
// one or two evaluations of F usually suffice instead of about eight.
static __device__ double solve_utau_warm(int law, double u, double h, double nu, double kap, double B, int maxit,
                                         double t_prev, double* t_out, bool* ok) {
  *ok = true;
  if (!(u > 0.0)) { *t_out = t_prev; return 0.0; }
  if (t_prev == t_prev && fabs(t_prev) < 1e3) {
    const double lnRe = log(h * u / nu);
    const double cst = law_const(law, kap, B);
    double t = t_prev;
    for (int k = 0; k < 4 && k < maxit; ++k) {
      const double w = exp(t);
      double L, wdL;
      law_eval_c(law, w, kap, cst, &L, &wdL);
      const double Ft = t + log(L) - lnRe;
      const double dF = 1.0 + wdL / L;
      if (Ft == 0.0) { *t_out = t; return law == 1 ? exp(t) * nu / h : u / exp(t); }
      const double nt = t - Ft / dF;
      if (!(nt == nt) || !(dF > 0.0)) break;
      const double step = fabs(nt - t);
      t = nt;
      if (step <= 1e-12 * fmax(1.0, fabs(t))) { *t_out = t; return law == 1 ? exp(t) * nu / h : u / exp(t); }
    }
  }
  const double ut = solve_utau(law, u, h, nu, kap, B, maxit, ok);
  *t_out = law == 1 ? log(ut * h / nu) : log(u / ut);
  return ut;
}

// FP32 form of the wall model for the FP32-mixed kernels: the same steps in
// FP32 arithmetic, with the Newton stopping tolerances scaled to FP32
// rounding (a step below 1e-6 of max(1, |t|), or a bracket below 4e-7 of it).
__device__ __forceinline__ void law_eval_cf(int law, float w, float kap, float cst, float* L, float* wdL) {
  if (law == 1) {
    const float C = cst;
    const float e1 = expf(-w / 11.0f), e2 = expf(-0.33f * w);
    const float Lv = log1pf(kap * w) / kap + C * (1.0f - e1 - (w / 11.0f) * e2);
    const float dL = 1.0f / (1.0f + kap * w) + C * (e1 / 11.0f - e2 / 11.0f + 0.33f * (w / 11.0f) * e2);
    *L = Lv; *wdL = w * dL;
  } else {
    const float ku = kap * w;
    const float eb = cst, ek = expf(ku);
    const float t3 = ku * ku * ku / 6.0f;
    const float Lv = w + eb * (ek - 1.0f - ku - 0.5f * ku * ku - t3 - 0.25f * ku * t3);
    const float dL = 1.0f + eb * kap * (ek - 1.0f - ku - 0.5f * ku * ku - t3);
    *L = Lv; *wdL = w * dL;
  }
}

static __device__ float solve_utau_f(int law, float u, float h, float nu, float kap, float B, int maxit, bool* ok) {
  *ok = true;
  if (!(u > 0.0f)) return 0.0f;
  const float lnRe = logf(h * u / nu);
  const float cst = law == 1 ? B - logf(kap) / kap : expf(-kap * B);
  auto F = [&](float t, float* dF) {
    const float w = expf(t);
    float L, wdL;
    law_eval_cf(law, w, kap, cst, &L, &wdL);
    *dF = 1.0f + wdL / L;
    return t + logf(L) - lnRe;
  };
  float dF;
  const float t0 = 0.5f * lnRe;
  const float F0 = F(t0, &dF);
  float lo = t0, hi = t0, st = 1.0f;
  int it = 0;
  float Flo = F0;
  while (!(Flo < 0.0f) && it < maxit) { lo -= st; st *= 2.0f; ++it; Flo = F(lo, &dF); }
  st = 1.0f;
  float Fhi = F0;
  while (!(Fhi > 0.0f) && it < maxit) { hi += st; st *= 2.0f; ++it; Fhi = F(hi, &dF); }
  float t = t0;
  if (!(t > lo && t < hi)) t = 0.5f * (lo + hi);
  bool done = false;
  for (; it < maxit; ++it) {
    const float Ft = F(t, &dF);
    if (Ft == 0.0f) { done = true; break; }
    if (Ft < 0.0f) lo = t; else hi = t;
    float nt = t - Ft / dF;
    const bool newton = (nt >= lo && nt <= hi);
    if (!newton) nt = 0.5f * (lo + hi);
    const float step = fabsf(nt - t);
    t = nt;
    const float sc = fmaxf(1.0f, fabsf(t));
    if ((newton && step <= 1e-6f * sc) || hi - lo <= 4e-7f * sc) { done = true; break; }
  }
  *ok = done;
  return law == 1 ? expf(t) * nu / h : u / expf(t);
}

// wall_stress below in FP32, from the sample's primitives
static __device__ void wall_stress_f(const PhysDev& ph, float rho, float u, float v, float w, float T, float nx,
                                     float ny, float nz, float tau[3], float* qw, bool* ok) {
  const float un = u * nx + v * ny + w * nz;
  const float ux = u - un * nx, uy = v - un * ny, uz = w - un * nz;
  const float u2 = ux * ux + uy * uy + uz * uz;
  tau[0] = tau[1] = tau[2] = 0.0f;
  *qw = 0.0f;
  *ok = true;
  if (!(u2 > 0.0f)) return;
  const float cp = (float)ph.cp, Pr = (float)ph.Pr;
  const float um = sqrtf(u2);
  const float r = cbrtf(Pr);
  const float Taw = T + r * u2 / (2.0f * cp);
  float Tw, uvd;
  if (ph.T_wall > 0.0) {
    Tw = (float)ph.T_wall;
    const float b = (Taw - Tw) / (Tw * um);
    const float a2 = r / (2.0f * cp * Tw);
    const float a = sqrtf(a2);
    const float q = sqrtf(b * b + 4.0f * a2);
    uvd = (asinf((2.0f * a2 * um - b) / q) + asinf(b / q)) / a;
  } else {
    Tw = Taw;
    const float a = sqrtf(r / (2.0f * cp * Tw));
    uvd = asinf(a * um) / a;
  }
  const float rhow = rho * T / Tw;
  const float muw = ph.sutherland ? sutherland<float>(ph, Tw) : ph.f32c.mu;
  const float ut = solve_utau_f(ph.law, uvd, (float)ph.hwm, muw / rhow, (float)ph.kappa, (float)ph.B, ph.wm_maxit, ok);
  const float tw = rhow * ut * ut / um;
  tau[0] = tw * ux; tau[1] = tw * uy; tau[2] = tw * uz;
  if (ph.T_wall > 0.0) *qw = -(cp / Pr) * (rhow * ut * ut) * (Taw - Tw) / um;
}

// Wall shear stress (and, at an isothermal wall, the heat flux into the fluid)
// from the sample state.  Adiabatic wall: Van Driest transform with the wall at
// the recovery temperature (Crocco-Busemann: T_w = T + r u^2 / (2 cp), rho_w =
// rho T / T_w, u_VD = asin(a u) / a with a = sqrt(r / (2 cp T_w)), r = Pr^(1/3)).
// Isothermal wall (ph.T_wall > 0): the Crocco-Busemann relation T(u) = T_w +
// (T_aw - T_w) u / u_s - r u^2 / (2 cp) in the transform,
//   u_VD = [asin((2 a^2 u_s - b) / q) + asin(b / q)] / a,
//   b = (T_aw - T_w) / (T_w u_s), a^2 = r / (2 cp T_w), q = sqrt(b^2 + 4 a^2),
// and q_w = -(cp / Pr) tau_w (T_aw - T_w) / u_s.  Then the law of the wall for
// u_tau, tau_w = rho_w u_tau^2 along the sample's wall-parallel velocity.
static __device__ void wall_stress(const PhysDev& ph, const double Us[5], double nx, double ny, double nz,
                            double tau[3], double* qw, bool* ok, double* t_warm = nullptr) {
  const double rho = Us[0], ir = 1.0 / rho;
  const double u = Us[1] * ir, v = Us[2] * ir, w = Us[3] * ir;
  const double p = ph.gm1 * (Us[4] - 0.5 * rho * (u * u + v * v + w * w));
  const double T = p * ph.rcp_R * ir;
  const double un = u * nx + v * ny + w * nz;
  const double ux = u - un * nx, uy = v - un * ny, uz = w - un * nz;
  const double u2 = ux * ux + uy * uy + uz * uz;
  tau[0] = tau[1] = tau[2] = 0.0;
  *qw = 0.0;
  *ok = true;
  if (!(u2 > 0.0)) return;
  const double um = sqrt(u2);
  const double r = cbrt(ph.Pr);
  const double Taw = T + r * u2 / (2.0 * ph.cp);
  double Tw, uvd;
  if (ph.T_wall > 0.0) {
    Tw = ph.T_wall;
    const double b = (Taw - Tw) / (Tw * um);
    const double a2 = r / (2.0 * ph.cp * Tw);
    const double a = sqrt(a2);
    const double q = sqrt(b * b + 4.0 * a2);
    uvd = (asin((2.0 * a2 * um - b) / q) + asin(b / q)) / a;
  } else {
    Tw = Taw;
    const double a = sqrt(r / (2.0 * ph.cp * Tw));
    uvd = asin(a * um) / a;
  }
  const double rhow = rho * T / Tw;
  const double muw = ph.sutherland ? sutherland<double>(ph, Tw) : ph.mu;
  const double ut = t_warm ? solve_utau_warm(ph.law, uvd, ph.hwm, muw / rhow, ph.kappa, ph.B, ph.wm_maxit, *t_warm,
                                             t_warm, ok)
                           : solve_utau(ph.law, uvd, ph.hwm, muw / rhow, ph.kappa, ph.B, ph.wm_maxit, ok);
  const double tw = rhow * ut * ut / um;
  tau[0] = tw * ux; tau[1] = tw * uy; tau[2] = tw * uz;
  if (ph.T_wall > 0.0) *qw = -(ph.cp / ph.Pr) * (rhow * ut * ut) * (Taw - Tw) / um;
}

// ---------------------------------------------------------------------------
// Even/odd form of a line contraction y_q = sum_m M_qm x_m whose matrix is
// centro-antisymmetric (M_{N-q,N-m} = -M_qm; the LGL derivative matrix D and
// (w_m / w_q) D_mq are).  With xe_m = x_m + x_{N-m} and xo_m = x_m - x_{N-m}
// for m < n/2,
//   E_q = sum_m (M_qm + M_q,N-m) / 2 xe_m,   O_q = sum_m (M_qm - M_q,N-m) / 2 xo_m,
//   y_q = E_q + O_q,   y_{N-q} = O_q - E_q          (q < n/2, n even),
// n/2 products per output instead of n.  The node at line position q < n/2
// forms E_q, its mirror node N - q forms O_q, and the two swap them with a
// shuffle: used with N = 7 in the warp layout of k_lift, where the mirror
// node along xi, eta, zeta is lane ^ 7, ^ 8, ^ 16.
// ---------------------------------------------------------------------------
template <int N>
struct LineEO {
  static constexpr int n = N + 1, h = n / 2;
  static_assert(n % 2 == 0, "even/odd form needs an even number of nodes");
  // table [n][h]: rows q < h hold (M_qm + M_q,N-m) / 2, rows q >= h hold
  // (M_q'm - M_q',N-m) / 2 with q' = N - q
  __device__ static double coef(const double* M, int t) {
    const int q = t / h, mm = t % h;
    const int r = q < h ? q : N - q;
    const double a = M[r * n + mm], b = M[r * n + N - mm];
    return q < h ? 0.5 * (a + b) : 0.5 * (a - b);
  }
  // the same table for the transpose of M
  __device__ static double coef_t(const double* M, int t) {
    const int q = t / h, mm = t % h;
    const int r = q < h ? q : N - q;
    const double a = M[mm * n + r], b = M[(N - mm) * n + r];
    return q < h ? 0.5 * (a + b) : 0.5 * (a - b);
  }
  // node at line position pos on the line along dir through node p (at q)
  __device__ static int at(int p, int dir, int q, int pos) {
    return p + (pos - q) * (dir == 0 ? 1 : (dir == 1 ? n : n * n));
  }
  // the value a node stores at its line position: xe_q (q < h) or xo_{N-q}
  template <class R>
  __device__ static R half(int q, R x, R x_mirror) { return fma(q < h ? R(1) : R(-1), x, x_mirror); }
  template <class R>
  __device__ static R mirror(R x, int dir) {
    return __shfl_xor_sync(0xffffffffu, x, dir == 0 ? 7 : (dir == 1 ? 8 : 16));
  }
  // y at this node from the stored halves sH of the line and the table sM
  template <class R>
  __device__ static R apply(const R* sM, const R* sH, int p, int dir, int q) {
    const bool lo = q < h;
    R P = 0;
#pragma unroll
    for (int mm = 0; mm < h; ++mm) P = fma(sM[q * h + mm], sH[at(p, dir, q, lo ? mm : N - mm)], P);
    return fma(lo ? R(1) : R(-1), mirror(P, dir), P);
  }
};

// ---------------------------------------------------------------------------
// k_lift: one CTA of n^3 threads per element.
// ---------------------------------------------------------------------------
// 2 (W* - W) of the BR1 lifting at node ab of face l of element e (own
// node q, own values Wo in the lifted form): the neighbour's trace (interior
// and halo faces), the exterior state (inflow / outflow) or the mirror state
// (slip wall)
template <int N, typename R>
__device__ __forceinline__ void lift_face_jump(const double* __restrict__ U, const MeshDev<R>& m, const PhysDev& ph,
                                               size_t S, int e, int l, int ab, int q, int nb, R Wo0, R Wo1, R Wo2,
                                               R Wo3, R dd[4]) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  R d0, d1, d2, d3;
  if (nb >= 0) {
    const NbrNode<N> nn = neighbour_node<N>(m, e, l, ab);
    const size_t gn = (size_t)nn.e * n3 + fnode<N>(nn.l, nn.ab % n, nn.ab / n);
    R u, v, w, T;
    if constexpr (std::is_same<R, float>::value) {
      velocity_temperature32s(load_prim32(m.W32, S, gn), ph, u, v, w, T);
    } else if (m.W64) {
      u = m.W64[S + gn]; v = m.W64[2 * S + gn]; w = m.W64[3 * S + gn]; T = m.W64[6 * S + gn];
    } else {
      velocity_temperature<R>(U[gn], U[S + gn], U[2 * S + gn], U[3 * S + gn], U[4 * S + gn], ph, u, v, w, T);
    }
    d0 = u - Wo0; d1 = v - Wo1; d2 = w - Wo2; d3 = T - Wo3;
  } else if (nb <= -16) {
    // halo face: the remote element's trace from the halo buffer (in the
    // master's face-node order)
    const int abm = omap_ab<N>((m.elem_face[e * 6 + l] >> 1) & 7, ab);
    const double* src = m.halo_U + (size_t)chk_idx(-16 - nb, m.n_halo, m.status) * 5 * n2 + abm;
    R u, v, w, T;
    if constexpr (std::is_same<R, double>::value) {
      if (m.W64) {
        // as the remote element's stored primitives (same function)
        const Prim<double> q = primitive_T(src[0], src[n2], src[2 * n2], src[3 * n2], src[4 * n2], ph, T);
        u = q.u; v = q.v; w = q.w;
      } else {
        velocity_temperature<R>(src[0], src[n2], src[2 * n2], src[3 * n2], src[4 * n2], ph, u, v, w, T);
      }
    } else {
      velocity_temperature32s_of(src[0], src[n2], src[2 * n2], src[3 * n2], src[4 * n2], ph, u, v, w, T);
    }
    d0 = u - Wo0; d1 = v - Wo1; d2 = w - Wo2; d3 = T - Wo3;
  } else if (nb != -1) {
    // inflow / outflow: 2 (W* - W) = W(exterior) - W
    const size_t gq = (size_t)e * n3 + q;
    double Ui[5], Ub[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Ui[v] = U[v * S + gq];
    ghost_state(ph, nb, Ui, Ub);
    R u, v, w, T;
    if constexpr (std::is_same<R, float>::value)
      velocity_temperature32s_of(Ub[0], Ub[1], Ub[2], Ub[3], Ub[4], ph, u, v, w, T);
    else
      velocity_temperature<R>(Ub[0], Ub[1], Ub[2], Ub[3], Ub[4], ph, u, v, w, T);
    d0 = u - Wo0; d1 = v - Wo1; d2 = w - Wo2; d3 = T - Wo3;
  } else {
    // mirror: 2 (W* - W) = -2 (u . n) n, T unchanged (n: own outward unit normal)
    const size_t gq = (size_t)e * n3 + q;
    const int dir = l >> 1;
    const R a0 = m.Ja[(size_t)(dir * 3 + 0) * S + gq], a1 = m.Ja[(size_t)(dir * 3 + 1) * S + gq],
            a2 = m.Ja[(size_t)(dir * 3 + 2) * S + gq];
    const R is = R(1) / sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    const R nx = a0 * is, ny = a1 * is, nz = a2 * is;  // sign irrelevant: (u.n) n
    const R un2 = R(-2) * (Wo0 * nx + Wo1 * ny + Wo2 * nz);
    d0 = un2 * nx; d1 = un2 * ny; d2 = un2 * nz; d3 = R(0);
  }
  dd[0] = d0; dd[1] = d1; dd[2] = d2; dd[3] = d3;
}

// Two floats in one 64-bit register pair, operands of the packed FP32
// instructions of sm_100 and later (add/sub/mul/fma.rn.f32x2: one instruction
// for two lanes, each rounded to nearest as its scalar form, so that the
// error-free transformations stay exact lane by lane).
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// the FP32 lifting kernel's line coefficients (D and Dvisc, rounded to FP32)
// as packed broadcasts (c, c): a line thread contracts two variables at once
template <int N>
struct LiftPk {
  f32x2 d[(N + 1) * (N + 1)], dv[(N + 1) * (N + 1)];
};

// Resident CTAs per SM asked of the register allocator for the lifting
// kernel: two for CTAs of up to 512 threads, three for the FP32 kernel at
// N = 7 (42 registers; its line phases leave the other threads waiting at a
// barrier, which a third CTA per SM covers)
template <int N, typename R>
constexpr int lift_min_blocks() {
  return ((N + 1) * (N + 1) * (N + 1) > 512) ? 1 : ((N == 7 && std::is_same<R, float>::value) ? 3 : 2);
}

template <int N, typename R>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1), (lift_min_blocks<N, R>()))
k_lift(const double* __restrict__ U, const MeshDev<R> m, const PhysDev ph, const Tables<N> tab,
       const LiftPk<N> pk, R* __restrict__ Rv, R* __restrict__ Gf) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  // FP64, N = 7: line contractions in even/odd form (LineEO), with the thread
  // of each node sharing a warp with its three mirror nodes (the FP32 kernel is
  // not bound by its multiply-adds: the extra barriers and shuffles cost more)
  constexpr bool EO = (n == 8) && std::is_same<R, double>::value;
  // FP32, N = 7: the line contractions by two threads per line, two
  // variables each (n outputs from the line's n values held in registers, the
  // coefficients as operands from the kernel parameters) instead of one thread
  // per node (n shared-memory loads per output, the kernel's bound), the node
  // slots swizzled (lift_slot8)
  constexpr bool LT = (n == 8) && std::is_same<R, float>::value;
  auto ws = [](int node) {
    if constexpr (LT) return lift_slot8(node);
    else return node;
  };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sW = reinterpret_cast<R*>(smem_raw);      // [4][n3]
  R* sC = sW + 4 * n3;                          // [6][4][n2]
  R* sG = sC + 24 * n2;                         // [3][4][n3]
  R* sD = sG + 12 * n3;                         // [n2]  (EO: [n][n/2] even/odd rows of D)
  R* sDv = sD + n2;                             // [n2]  (EO: the same for Dvisc)
  R* siw = sDv + n2;                            // [n]
  const int e = blockIdx.x, tid = threadIdx.x;
  int i, j, k;
  if constexpr (EO) {
    // warp w = a + 4 b holds the xi-lines i = 0..7 at j in {a, N - a} and
    // k in {b, N - b}: the mirror node along xi, eta, zeta is lane ^ 7, ^ 8, ^ 16
    const int lane = tid & 31, w = tid >> 5, a = w & 3, b = w >> 2;
    i = lane & 7;
    j = (lane & 8) ? N - a : a;
    k = (lane & 16) ? N - b : b;
  } else {
    i = tid % n; j = (tid / n) % n; k = tid / n2;
  }
  const int p = i + n * (j + n * k);  // this thread's node
  const size_t S = (size_t)m.K * n3;
  const size_t g = (size_t)e * n3 + p;
  if constexpr (EO) {
    if (tid < n * (n / 2)) {
      sD[tid] = (R)LineEO<N>::coef(tab.D, tid);
      sDv[tid] = (R)LineEO<N>::coef(tab.Dvisc, tid);
    }
  } else {
    for (int t = tid; t < n2; t += n3) { sD[t] = (R)tab.D[t]; sDv[t] = (R)tab.Dvisc[t]; }
  }
  if (tid < n) siw[tid] = (R)tab.iw[tid];
  // own primitives W = (u, v, w, T)
  {
    R u, v, w, T;
    if constexpr (std::is_same<R, float>::value) {
      velocity_temperature32s(load_prim32(m.W32, S, g), ph, u, v, w, T);  // T: T - T_lift
    } else if (m.W64) {
      // the FP64 primitives k_prim64 stored for this evaluation
      u = m.W64[S + g]; v = m.W64[2 * S + g]; w = m.W64[3 * S + g]; T = m.W64[6 * S + g];
    } else {
      velocity_temperature<R>(U[g], U[S + g], U[2 * S + g], U[3 * S + g], U[4 * S + g], ph, u, v, w, T);
    }
    const int sp = ws(p);
    sW[sp] = u; sW[n3 + sp] = v; sW[2 * n3 + sp] = w; sW[3 * n3 + sp] = T;
  }
  __syncthreads();
  // 2 (W* - W) at the six faces (BR1 average with the neighbour, or the
  // mirror state at a slip wall); the factor 1/2 goes with the 1/w of the
  // surface correction
  for (int t = tid; t < 6 * n2; t += n3) {
    const int l = t / n2, ab = t - l * n2, a = ab % n, b = ab / n;
    const int q = fnode<N>(l, a, b);
    const int nb = m.nbr[e * 6 + l];
    const int sq = ws(q);
    const R Wo0 = sW[sq], Wo1 = sW[n3 + sq], Wo2 = sW[2 * n3 + sq], Wo3 = sW[3 * n3 + sq];
    R dd[4];
    lift_face_jump<N, R>(U, m, ph, S, e, l, ab, q, nb, Wo0, Wo1, Wo2, Wo3, dd);
    const R d0 = dd[0], d1 = dd[1], d2 = dd[2], d3 = dd[3];
    sC[(l * 4 + 0) * n2 + ab] = d0; sC[(l * 4 + 1) * n2 + ab] = d1;
    sC[(l * 4 + 2) * n2 + ab] = d2; sC[(l * 4 + 3) * n2 + ab] = d3;
  }
  __syncthreads();
  // gradients in reference space
  R dW[3][4];
  if constexpr (EO) {
    const int qd[3] = {i, j, k};
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        sG[(dir * 4 + v) * n3 + p] = LineEO<N>::half(qd[dir], sW[v * n3 + p],
                                                      sW[v * n3 + LineEO<N>::at(p, dir, qd[dir], N - qd[dir])]);
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
        dW[dir][v] = LineEO<N>::apply(sD, sG + (dir * 4 + v) * n3, p, dir, qd[dir]);
  } else if constexpr (LT) {
    // thread tid < 6 n2 takes two of the four variables (v0, v0 + 1) on line
    // L of direction dir and writes the reference-space derivatives of its n
    // nodes into sG
    if (tid < 6 * n2) {
      const int dir = tid / (2 * n2), r = tid - dir * 2 * n2, v0 = 2 * (r / n2), L = r % n2;
      const int n0 = dir == 0 ? n * L : (dir == 1 ? (L % n) + n2 * (L / n) : L);
      // node n0 + q stride has slot slot(n0) ^ slot(q stride) (the slot map
      // is linear in the index bits, and n0 has no bits of the line's axis)
      const int s0 = lift_slot8(n0);
      int sl[n];
#pragma unroll
      for (int q = 0; q < n; ++q)
        sl[q] = s0 ^ (dir == 0 ? lift_slot8(q) : (dir == 1 ? lift_slot8(q * n) : lift_slot8(q * n2)));
      // the two variables in the lanes of packed FMAs (each lane the scalar
      // FMA chain's roundings)
      f32x2 x[n];
#pragma unroll
      for (int q = 0; q < n; ++q) x[q] = pk2(sW[v0 * n3 + sl[q]], sW[(v0 + 1) * n3 + sl[q]]);
#pragma unroll
      for (int q = 0; q < n; ++q) {
        f32x2 y = pk2(0.f, 0.f);
#pragma unroll
        for (int mm = 0; mm < n; ++mm) y = fma2(pk.d[q * n + mm], x[mm], y);
        float y0, y1;
        upk2(y, y0, y1);
        sG[(dir * 4 + v0) * n3 + sl[q]] = y0;
        sG[(dir * 4 + v0 + 1) * n3 + sl[q]] = y1;
      }
    }
    __syncthreads();
    const int sp = lift_slot8(p);
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v) dW[dir][v] = sG[(dir * 4 + v) * n3 + sp];
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      R s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
      for (int mm = 0; mm < n; ++mm) {
        s0 += sD[i * n + mm] * sW[v * n3 + mm + n * (j + n * k)];
        s1 += sD[j * n + mm] * sW[v * n3 + i + n * (mm + n * k)];
        s2 += sD[k * n + mm] * sW[v * n3 + i + n * (j + n * mm)];
      }
      dW[0][v] = s0; dW[1][v] = s1; dW[2][v] = s2;
    }
  }
  // surface corrections of the reference-space gradient: (W* - W) (+-1 / w)
  // at the first and last node of each line (with n s = +-Ja^dir they give
  // the (W* - W) (n s)_d / w terms of the physical gradient); sC holds
  // 2 (W* - W), so the weights are shw = 1 / (2 w)
  const R shw0 = R(0.5) * siw[0], shwN = R(0.5) * siw[N];
  auto surf = [&](int dir, int l, int ab, R sgn_iw) {
#pragma unroll
    for (int v = 0; v < 4; ++v) dW[dir][v] += sgn_iw * sC[(l * 4 + v) * n2 + ab];
  };
  // (one branch per direction: a warp holds nodes of both end faces of the
  // lines along xi, and the masked lanes of a branch cost as much as active ones)
  if (i == 0 || i == N) surf(0, i == 0 ? 0 : 1, j + n * k, i == 0 ? -shw0 : shwN);
  if (j == 0 || j == N) surf(1, j == 0 ? 2 : 3, i + n * k, j == 0 ? -shw0 : shwN);
  if (k == 0 || k == N) surf(2, k == 0 ? 4 : 5, i + n * j, k == 0 ? -shw0 : shwN);
  // viscous flux Fv_d = (0, tau_1d, tau_2d, tau_3d, tau_jd u_j + k dT/dx_d)
  R mu = cR<R>(ph.mu, ph.f32c.mu), kc = cR<R>(ph.kcond, ph.f32c.kcond);
  if (ph.sutherland) {
    // (FP32: the lifted temperature is T - T_lift)
    mu = sutherland<R>(ph, sW[3 * n3 + ws(p)] + cR<R>(0.0, ph.f32c.T_lift));
    kc = mu * cR<R>(ph.cp_Pr, ph.f32c.cp_Pr);
  }
  const R uu = sW[ws(p)], vv = sW[n3 + ws(p)], ww = sW[2 * n3 + ws(p)];
  // contravariant G^dir = sum_d Ja^dir_d Fv_d
  R G[3][4];
  // symmetric stress: tau_ab = mu (q_ba + q_ab) - (2/3) mu div delta_ab
  auto stress = [&](const R q[3][4], R tau[3][3]) {
    const R div = q[0][0] + q[1][1] + q[2][2];
    const R mdiv = R(2.0 / 3.0) * mu * div, mu2 = R(2) * mu;
    tau[0][0] = mu2 * q[0][0] - mdiv;
    tau[1][1] = mu2 * q[1][1] - mdiv;
    tau[2][2] = mu2 * q[2][2] - mdiv;
    tau[0][1] = tau[1][0] = mu * (q[0][1] + q[1][0]);
    tau[0][2] = tau[2][0] = mu * (q[0][2] + q[2][0]);
    tau[1][2] = tau[2][1] = mu * (q[1][2] + q[2][1]);
  };
  if constexpr (std::is_same<R, double>::value) {
    // FP64: the metric products come precomputed (metrics are fixed, the
    // FP64 pipe is the bound).  Velocity gradients q[d][c] = du_c/dx_d =
    // sum_dir (Ja^dir_d / J) dW_dir; the energy row as
    //   G^dir_E = sum_c u_c G^dir_c + k (Ja^dir . grad T),
    //   Ja^dir . grad T = sum_m ((Ja^dir . Ja^m) / J) dT_m
    R q[3][4], hT[3];
    {
      R jj[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) jj[c] = m.JaJ[(size_t)c * S + g];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 3; ++v)
          q[d][v] = jj[0 * 3 + d] * dW[0][v] + jj[1 * 3 + d] * dW[1][v] + jj[2 * 3 + d] * dW[2][v];
      R mm[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) mm[c] = m.Mj[(size_t)c * S + g];
      hT[0] = mm[0] * dW[0][3] + mm[3] * dW[1][3] + mm[4] * dW[2][3];
      hT[1] = mm[3] * dW[0][3] + mm[1] * dW[1][3] + mm[5] * dW[2][3];
      hT[2] = mm[4] * dW[0][3] + mm[5] * dW[1][3] + mm[2] * dW[2][3];
    }
    R tau[3][3];
    stress(q, tau);
    R ja[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) ja[c] = m.Ja[(size_t)c * S + g];
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
#pragma unroll
      for (int v = 0; v < 3; ++v)
        G[dir][v] = ja[dir * 3 + 0] * tau[v][0] + ja[dir * 3 + 1] * tau[v][1] + ja[dir * 3 + 2] * tau[v][2];
      G[dir][3] = uu * G[dir][0] + vv * G[dir][1] + ww * G[dir][2] + kc * hT[dir];
    }
  } else {
    // own metrics (loaded here, after the contractions, to keep them out of
    // the registers live across those)
    R ja[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) ja[c] = m.Ja[(size_t)c * S + g];
    const R iJ = m.invJ[g];
    // physical gradients q[d][v] = (1/J) sum_dir Ja^dir_d dW_dir
    R q[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R j0 = iJ * ja[0 * 3 + d], j1 = iJ * ja[1 * 3 + d], j2 = iJ * ja[2 * 3 + d];
#pragma unroll
      for (int v = 0; v < 4; ++v) q[d][v] = j0 * dW[0][v] + j1 * dW[1][v] + j2 * dW[2][v];
    }
    R tau[3][3];
    stress(q, tau);
    R Fv[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Fv[d][0] = tau[0][d]; Fv[d][1] = tau[1][d]; Fv[d][2] = tau[2][d];
      Fv[d][3] = tau[0][d] * uu + tau[1][d] * vv + tau[2][d] * ww + kc * q[d][3];
    }
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        G[dir][v] = ja[dir * 3 + 0] * Fv[0][v] + ja[dir * 3 + 1] * Fv[1][v] + ja[dir * 3 + 2] * Fv[2][v];
  }
  // own outward viscous flux at face nodes: Gf[e][l][v][ab] = +-G^{l/2}
  auto gface = [&](int l, int ab, R sgn) {
    R* dst = Gf + ((size_t)e * 6 + l) * 4 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v * n2] = sgn * G[l >> 1][v];
  };
  if (i == 0) gface(0, j + n * k, R(-1));
  if (i == N) gface(1, j + n * k, R(1));
  if (j == 0) gface(2, i + n * k, R(-1));
  if (j == N) gface(3, i + n * k, R(1));
  if (k == 0) gface(4, i + n * j, R(-1));
  if (k == N) gface(5, i + n * j, R(1));
  // weak-form viscous volume term R_v = sum_dir sum_m (w_m / w_i) D_mi G^dir_m
  if constexpr (EO) {
    const int qd[3] = {i, j, k};
    __syncthreads();  // the gradient contractions have read sG
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        sG[(dir * 4 + v) * n3 + p] = LineEO<N>::half(qd[dir], G[dir][v], LineEO<N>::mirror(G[dir][v], dir));
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      R s = 0;
#pragma unroll
      for (int dir = 0; dir < 3; ++dir) s += LineEO<N>::apply(sDv, sG + (dir * 4 + v) * n3, p, dir, qd[dir]);
      Rv[(size_t)v * S + g] = s;
    }
  } else if constexpr (LT) {
    __syncthreads();  // the nodes have read their derivatives from sG
    const int sp = lift_slot8(p);
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v) sG[(dir * 4 + v) * n3 + sp] = G[dir][v];
    __syncthreads();
    // two threads per line: its direction's part of R_v at its n nodes, in
    // place (a line's slots of its direction and variables belong to its
    // thread alone)
    if (tid < 6 * n2) {
      const int dir = tid / (2 * n2), r = tid - dir * 2 * n2, v0 = 2 * (r / n2), L = r % n2;
      const int n0 = dir == 0 ? n * L : (dir == 1 ? (L % n) + n2 * (L / n) : L);
      const int s0 = lift_slot8(n0);
      int sl[n];
#pragma unroll
      for (int q = 0; q < n; ++q)
        sl[q] = s0 ^ (dir == 0 ? lift_slot8(q) : (dir == 1 ? lift_slot8(q * n) : lift_slot8(q * n2)));
      f32x2 x[n];
#pragma unroll
      for (int q = 0; q < n; ++q)
        x[q] = pk2(sG[(dir * 4 + v0) * n3 + sl[q]], sG[(dir * 4 + v0 + 1) * n3 + sl[q]]);
#pragma unroll
      for (int q = 0; q < n; ++q) {
        f32x2 y = pk2(0.f, 0.f);
#pragma unroll
        for (int mm = 0; mm < n; ++mm) y = fma2(pk.dv[q * n + mm], x[mm], y);
        float y0, y1;
        upk2(y, y0, y1);
        sG[(dir * 4 + v0) * n3 + sl[q]] = y0;
        sG[(dir * 4 + v0 + 1) * n3 + sl[q]] = y1;
      }
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v)
      Rv[(size_t)v * S + g] = sG[(0 * 4 + v) * n3 + sp] + sG[(1 * 4 + v) * n3 + sp] + sG[(2 * 4 + v) * n3 + sp];
  } else {
#pragma unroll
    for (int dir = 0; dir < 3; ++dir)
#pragma unroll
      for (int v = 0; v < 4; ++v) sG[(dir * 4 + v) * n3 + p] = G[dir][v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      R s = 0;
#pragma unroll
      for (int mm = 0; mm < n; ++mm) {
        s += sDv[i * n + mm] * sG[(0 * 4 + v) * n3 + mm + n * (j + n * k)];
        s += sDv[j * n + mm] * sG[(1 * 4 + v) * n3 + i + n * (mm + n * k)];
        s += sDv[k * n + mm] * sG[(2 * 4 + v) * n3 + i + n * (j + n * mm)];
      }
      Rv[(size_t)v * S + g] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// k_face: one thread per node of an interior face.  In FP64 the halo faces of
// a partitioned mesh follow the interior faces in the same launch, so that one
// code path forms the flux of both kinds (and a halo face's flux equals,
// bitwise, the one a single-domain run forms for the same face).
// ---------------------------------------------------------------------------
template <int N, typename R>
__global__ void __launch_bounds__(256)
k_face(const double* __restrict__ U, const MeshDev<R> m, const PhysDev ph, const R* __restrict__ Gf,
       R* __restrict__ Fs) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  constexpr bool D = std::is_same<R, double>::value;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int f0 = tid / n2, ab = tid - f0 * n2;
  if (f0 >= m.n_interior + (D ? m.n_halo : 0)) return;
  const bool is_halo = D && f0 >= m.n_interior;
  const int f = is_halo ? m.F - m.n_halo + (f0 - m.n_interior) : f0;
  const int4 fc = m.faces[f];
  const size_t S = (size_t)m.K * n3;
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const R nx = (R)m.fgeo[fg], ny = (R)m.fgeo[FN + fg], nz = (R)m.fgeo[2 * FN + fg], s = (R)m.fgeo[3 * FN + fg];
  R F[5];
  const R* gA;
  const R* gB;
  if constexpr (!D) {
    const int abS = omap_ab<N>(fc.w >> 3, ab), lS = fc.w & 7;
    const int eM = chk_idx(fc.x, m.K, m.status), eS = chk_idx(fc.z, m.K, m.status);
    const size_t gM = (size_t)eM * n3 + fnode<N>(fc.y, ab % n, ab / n);
    const size_t gS = (size_t)eS * n3 + fnode<N>(lS, abS % n, abS / n);
    gA = Gf + ((size_t)eM * 6 + fc.y) * 4 * n2 + ab;
    gB = Gf + ((size_t)eS * 6 + lS) * 4 * n2 + abS;
    const Prim<float> A = load_prim32(m.W32, S, gM), B = load_prim32(m.W32, S, gS);
    const Lo3 la = load_lo32(m.W32, S, gM), lb = load_lo32(m.W32, S, gS);
    // U_B - U_A for the Lax-Friedrichs dissipation, differenced in FP64 (from
    // rounded FP32 states the difference would carry an error of eps |U|)
    float dU[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (ph.surf_flux == 1) {
#pragma unroll
      for (int v = 0; v < 5; ++v) dU[v] = d2f_bits(U[v * S + gS] - U[v * S + gM]);
    }
    if (ph.fs_diff) {
      store_face_delta(ph, A, B, la, lb, dU, nx, ny, nz, s, gA, gB, R(0.5), Fs + (size_t)f * 10 * n2 + ab, n2, true);
      return;
    }
    riemann_d<float>(ph, unshift32(A, ph), unshift32(B, ph), dU, nx, ny, nz, F);
  } else {
    // both sides' FP64 primitives: from the stored array in the viscous form,
    // else (and for a remote trace) by primitive_T, whose one compiled body
    // also writes that array
    Prim<double> A, B;
    double dU[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, T;
    const bool llf = ph.surf_flux == 1;
    if (!is_halo) {
      const int abS = omap_ab<N>(fc.w >> 3, ab), lS = fc.w & 7;
      const int eM = chk_idx(fc.x, m.K, m.status), eS = chk_idx(fc.z, m.K, m.status);
      const size_t gM = (size_t)eM * n3 + fnode<N>(fc.y, ab % n, ab / n);
      const size_t gS = (size_t)eS * n3 + fnode<N>(lS, abS % n, abS / n);
      gA = Gf + ((size_t)eM * 6 + fc.y) * 4 * n2 + ab;
      gB = Gf + ((size_t)eS * 6 + lS) * 4 * n2 + abS;
      if (m.W64) {
        A = load_prim64(m.W64, S, gM);
        B = load_prim64(m.W64, S, gS);
      } else {
        A = primitive_T(U[gM], U[S + gM], U[2 * S + gM], U[3 * S + gM], U[4 * S + gM], ph, T);
        B = primitive_T(U[gS], U[S + gS], U[2 * S + gS], U[3 * S + gS], U[4 * S + gS], ph, T);
      }
      if (llf) {
#pragma unroll
        for (int v = 0; v < 5; ++v) dU[v] = U[v * S + gS] - U[v * S + gM];
      }
    } else {
      // fc = (local element, local face, halo index, local side is master
      // | 8 o_own); ab is the master's face-node index, abl the local one
      const int h = f0 - m.n_interior;
      const int abl = omap_ab<N>(orient_inv(fc.w >> 3), ab);
      const int eL = chk_idx(fc.x, m.K, m.status);
      const size_t gL = (size_t)eL * n3 + fnode<N>(fc.y, abl % n, abl / n);
      const double* rU = m.halo_U + (size_t)h * 5 * n2 + ab;
      const bool master = (fc.w & 1) != 0;
      const Prim<double> loc =
          m.W64 ? load_prim64(m.W64, S, gL)
                : primitive_T(U[gL], U[S + gL], U[2 * S + gL], U[3 * S + gL], U[4 * S + gL], ph, T);
      const Prim<double> rem = primitive_T(rU[0], rU[n2], rU[2 * n2], rU[3 * n2], rU[4 * n2], ph, T);
      A = master ? loc : rem;
      B = master ? rem : loc;
      const R* gl = Gf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
      const R* gr = m.halo_G + (size_t)h * 4 * n2 + ab;
      gA = master ? gl : gr;
      gB = master ? gr : gl;
      if (llf) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const double d = rU[v * n2] - U[v * S + gL];
          dU[v] = master ? d : -d;
        }
      }
    }
    riemann_d<double>(ph, A, B, dU, nx, ny, nz, F);
  }
  R* out = Fs + (size_t)f * 5 * n2 + ab;
  out[0] = F[0] * s;
  if (ph.viscous) {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(v + 1) * n2] = F[v + 1] * s - R(0.5) * (gA[v * n2] - gB[v * n2]);
  } else {
#pragma unroll
    for (int v = 1; v < 5; ++v) out[v * n2] = F[v] * s;
  }
}

// ---------------------------------------------------------------------------
// Halo faces of a partitioned mesh, FP32-mixed form (FP64: in k_face).  Both
// ranks of a shared face evaluate its flux from the same master and slave
// traces (one side from the halo buffer) with the master's normal.
// ---------------------------------------------------------------------------
template <int N, typename R>
__global__ void __launch_bounds__(256)
k_halo_face(const double* __restrict__ U, const MeshDev<R> m, const PhysDev ph, const R* __restrict__ Gf,
            R* __restrict__ Fs) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = tid / n2, ab = tid - h * n2;
  if (h >= m.n_halo) return;
  const int f = m.F - m.n_halo + h;
  // (local element, local face, halo index, local is master | 8 o_own); ab
  // is the master's face-node index, abl the local one
  const int4 fc = m.faces[f];
  const size_t S = (size_t)m.K * n3;
  const int abl = omap_ab<N>(orient_inv(fc.w >> 3), ab);
  const int eL = chk_idx(fc.x, m.K, m.status);
  const size_t gL = (size_t)eL * n3 + fnode<N>(fc.y, abl % n, abl / n);
  const double* rU = m.halo_U + (size_t)h * 5 * n2 + ab;
  const bool master = (fc.w & 1) != 0;
  double UA[5], UB[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double loc = U[v * S + gL], rem = rU[v * n2];
    UA[v] = master ? loc : rem;
    UB[v] = master ? rem : loc;
  }
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const R nx = (R)m.fgeo[fg], ny = (R)m.fgeo[FN + fg], nz = (R)m.fgeo[2 * FN + fg], s = (R)m.fgeo[3 * FN + fg];
  Prim<R> As, Bs;
  Lo3 la, lb;
  const Prim<R> A = trace_prims<R>(UA, ph, &As, &la), B = trace_prims<R>(UB, ph, &Bs, &lb);
  if constexpr (std::is_same<R, float>::value) {
    if (ph.fs_diff) {
      float dU[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) dU[v] = d2f_bits(UB[v] - UA[v]);
      const R* gl = Gf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
      const R* gr = m.halo_G + (size_t)h * 4 * n2 + ab;
      store_face_delta(ph, As, Bs, la, lb, dU, nx, ny, nz, s, master ? gl : gr, master ? gr : gl, 0.5f,
                       Fs + (size_t)f * 10 * n2 + ab, n2, true);
      return;
    }
  }
  R F[5];
  riemann<R, double>(ph, A, UA, B, UB, nx, ny, nz, F);
  R* out = Fs + (size_t)f * 5 * n2 + ab;
  out[0] = F[0] * s;
  if (ph.viscous) {
    const R* gl = Gf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
    const R* gr = m.halo_G + (size_t)h * 4 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const R gA = master ? gl[v * n2] : gr[v * n2], gB = master ? gr[v * n2] : gl[v * n2];
      out[(v + 1) * n2] = F[v + 1] * s - R(0.5) * (gA - gB);
    }
  } else {
#pragma unroll
    for (int v = 1; v < 5; ++v) out[v * n2] = F[v] * s;
  }
}

// the local traces of the halo faces: state (before the lifting) and own
// outward viscous flux (after it), in the halo-buffer layout (the master's
// face-node order)
template <int N, typename R>
__global__ void __launch_bounds__(256)
k_halo_pack(const double* __restrict__ U, const MeshDev<R> m, const R* __restrict__ Gf, double* __restrict__ sendU,
            R* __restrict__ sendG) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = tid / n2, ab = tid - h * n2;
  if (h >= m.n_halo) return;
  const int4 fc = m.faces[m.F - m.n_halo + h];
  // ab is the index in the master's face-node order; abl the local one
  const int abl = omap_ab<N>(orient_inv(fc.w >> 3), ab);
  const int eL = chk_idx(fc.x, m.K, m.status);
  if (sendU) {
    const size_t S = (size_t)m.K * n3;
    const size_t gL = (size_t)eL * n3 + fnode<N>(fc.y, abl % n, abl / n);
#pragma unroll
    for (int v = 0; v < 5; ++v) sendU[((size_t)h * 5 + v) * n2 + ab] = U[v * S + gL];
  }
  if (sendG) {
    const R* gl = Gf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
#pragma unroll
    for (int v = 0; v < 4; ++v) sendG[((size_t)h * 4 + v) * n2 + ab] = gl[v * n2];
  }
}

// ---------------------------------------------------------------------------
// k_bc: one thread per node of an inflow or outflow face: the Riemann flux
// between the interior trace and the exterior state, and the interior viscous
// flux (the BR1 average with an exterior side that carries the same flux).
// ---------------------------------------------------------------------------
template <int N, typename R>
__global__ void __launch_bounds__(256)
k_bc(const double* __restrict__ U, const MeshDev<R> m, const PhysDev ph, const R* __restrict__ Gf,
     R* __restrict__ Fs) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int bf = tid / n2, ab = tid - bf * n2;
  if (bf >= m.n_bc) return;
  const int f = m.n_interior + m.n_wall + bf;
  int4 fc = m.faces[f];
  fc.x = chk_idx(fc.x, m.K, m.status);
  const size_t S = (size_t)m.K * n3;
  const size_t gM = (size_t)fc.x * n3 + fnode<N>(fc.y, ab % n, ab / n);
  double UA[5], UB[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) UA[v] = U[v * S + gM];
  ghost_state(ph, fc.z, UA, UB);
  Prim<R> As, Bs;  // FP32: the storage form, for the flux-difference form
  Lo3 la, lb;
  const Prim<R> A = trace_prims<R>(UA, ph, &As, &la), B = trace_prims<R>(UB, ph, &Bs, &lb);
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const R nx = (R)m.fgeo[fg], ny = (R)m.fgeo[FN + fg], nz = (R)m.fgeo[2 * FN + fg], s = (R)m.fgeo[3 * FN + fg];
  if constexpr (std::is_same<R, float>::value) {
    if (ph.fs_diff) {
      float dU[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) dU[v] = d2f_bits(UB[v] - UA[v]);
      store_face_delta(ph, As, Bs, la, lb, dU, nx, ny, nz, s, Gf + ((size_t)fc.x * 6 + fc.y) * 4 * n2 + ab, nullptr,
                       1.f,
                       Fs + (size_t)f * 10 * n2 + ab, n2, false);
      return;
    }
  }
  R F[5];
  riemann<R, double>(ph, A, UA, B, UB, nx, ny, nz, F);
  R* out = Fs + (size_t)f * 5 * n2 + ab;
  out[0] = F[0] * s;
  if (ph.viscous) {
    const R* gA = Gf + ((size_t)fc.x * 6 + fc.y) * 4 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(v + 1) * n2] = F[v + 1] * s - gA[v * n2];
  } else {
#pragma unroll
    for (int v = 1; v < 5; ++v) out[v * n2] = F[v] * s;
  }
}

// ---------------------------------------------------------------------------
// k_wall: one thread per node of a wall face (slip wall + wall model).
// The work per node is long (sample interpolation over n^3 nodes, Newton
// iterations of transcendental functions) and the nodes are few, so blocks
// are one warp: the launch spreads over all SMs instead of filling a few.
// ---------------------------------------------------------------------------
constexpr int WALL_THREADS = 32;

template <int N, typename R>
__global__ void __launch_bounds__(WALL_THREADS)
k_wall(const double* __restrict__ U, const MeshDev<R> m, const PhysDev ph, R* __restrict__ Fs,
       double* __restrict__ tau_out, int* __restrict__ status) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int wf = tid / n2, ab = tid - wf * n2;
  if (wf >= m.n_wall) return;
  const int f = m.n_interior + wf;
  int4 fc = m.faces[f];
  fc.x = chk_idx(fc.x, m.K, m.status);
  const size_t S = (size_t)m.K * n3;
  const size_t gM = (size_t)fc.x * n3 + fnode<N>(fc.y, ab % n, ab / n);
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const double nxd = m.fgeo[fg], nyd = m.fgeo[FN + fg], nzd = m.fgeo[2 * FN + fg], sd = m.fgeo[3 * FN + fg];
  double UA[5], UB[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) UA[v] = U[v * S + gM];
  const double mn = UA[1] * nxd + UA[2] * nyd + UA[3] * nzd;
  UB[0] = UA[0]; UB[1] = UA[1] - 2.0 * mn * nxd; UB[2] = UA[2] - 2.0 * mn * nyd;
  UB[3] = UA[3] - 2.0 * mn * nzd; UB[4] = UA[4];
  Prim<R> As, Bs;  // FP32: the storage form, for the flux-difference form
  Lo3 la, lb;
  const Prim<R> A = trace_prims<R>(UA, ph, &As, &la), B = trace_prims<R>(UB, ph, &Bs, &lb);
  R F[5];
  int fss = 5;  // surface-flux values per face node (10: FP32 difference form)
  if constexpr (std::is_same<R, float>::value) {
    if (ph.fs_diff) {
      float dU[5], DB[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) dU[v] = d2f_bits(UB[v] - UA[v]);
      face_flux_delta(ph, As, Bs, la, lb, dU, (R)nxd, (R)nyd, (R)nzd, F, DB);
      fss = 10;
    }
  }
  if (fss == 5) riemann<R, double>(ph, A, UA, B, UB, (R)nxd, (R)nyd, (R)nzd, F);
  double tau[3] = {0.0, 0.0, 0.0}, qw = 0.0;
  if constexpr (std::is_same<R, float>::value) {
    if (ph.viscous) {
      // FP32 form: interpolation of the conservative state formed from the
      // stage's FP32 primitives, with the energy taken relative to
      // p_ref / (gamma - 1) (the interpolation weights sum to one), then the
      // FP32 wall model
      const size_t slot = (size_t)wf * n2 + ab;
      const int es = chk_idx(m.ws_elem[slot], m.K, m.status);
      const double* Ld = m.ws_lag + slot * 3 * n;
      float L[3 * n];
#pragma unroll
      for (int x = 0; x < 3 * n; ++x) L[x] = (float)Ld[x];
      const float rg = ph.f32c.rgm1;
      float Us[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int kk = 0; kk < n; ++kk)
        for (int jj = 0; jj < n; ++jj) {
          const float ljk = L[n + jj] * L[2 * n + kk];
          float row[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
          for (int ii = 0; ii < n; ++ii) {
            const Prim<float> q = load_prim32_full(m.W32, S, (size_t)es * n3 + ii + n * (jj + n * kk), ph);
            const float li = L[ii];
            row[0] += li * q.rho;
            row[1] += li * (q.rho * q.u);
            row[2] += li * (q.rho * q.v);
            row[3] += li * (q.rho * q.w);
            row[4] += li * (q.p * rg + 0.5f * q.rho * (q.u * q.u + q.v * q.v + q.w * q.w));
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) Us[v] += ljk * row[v];
        }
      const float ir = 1.0f / Us[0];
      const float u = Us[1] * ir, v = Us[2] * ir, w = Us[3] * ir;
      const float pp = (float)ph.gm1 * (Us[4] - 0.5f * Us[0] * (u * u + v * v + w * w));  // p - p_ref
      const float Ts = (pp + ph.f32c.p_ref) * ph.f32c.rcp_R * ir;
      float tf[3], qf;
      bool ok;
      wall_stress_f(ph, Us[0], u, v, w, Ts, (float)nxd, (float)nyd, (float)nzd, tf, &qf, &ok);
      if (!ok) atomicOr(status, ST_WM_NOCONV);
      tau[0] = tf[0]; tau[1] = tf[1]; tau[2] = tf[2]; qw = qf;
      if (tau_out) {
        tau_out[slot * 3 + 0] = tau[0]; tau_out[slot * 3 + 1] = tau[1]; tau_out[slot * 3 + 2] = tau[2];
      }
    }
  } else if (ph.viscous) {
    // sample state at h_wm: tensor-product Lagrange interpolation of U
    const size_t slot = (size_t)wf * n2 + ab;
    const int es = chk_idx(m.ws_elem[slot], m.K, m.status);
    const double* L = m.ws_lag + slot * 3 * n;
    double Us[5] = {0, 0, 0, 0, 0};
    for (int kk = 0; kk < n; ++kk)
      for (int jj = 0; jj < n; ++jj) {
        const double ljk = L[n + jj] * L[2 * n + kk];
        double row[5] = {0, 0, 0, 0, 0};
        for (int ii = 0; ii < n; ++ii) {
          const size_t gs = (size_t)es * n3 + ii + n * (jj + n * kk);
#pragma unroll
          for (int v = 0; v < 5; ++v) row[v] += L[ii] * U[v * S + gs];
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) Us[v] += ljk * row[v];
      }
    bool ok;
    if (m.wm_t) {
      double tw = m.wm_t[slot];
      wall_stress(ph, Us, nxd, nyd, nzd, tau, &qw, &ok, &tw);
      m.wm_t[slot] = tw;
    } else {
      wall_stress(ph, Us, nxd, nyd, nzd, tau, &qw, &ok);
    }
    if (!ok) atomicOr(status, ST_WM_NOCONV);
    if (tau_out) {
      tau_out[slot * 3 + 0] = tau[0]; tau_out[slot * 3 + 1] = tau[1]; tau_out[slot * 3 + 2] = tau[2];
    }
  }
  // viscous wall flux Fv . n = (0, -tau_w t, 0): the wall decelerates the flow
  R* out = Fs + (size_t)f * fss * n2 + ab;
  const R s = (R)sd;
  out[0] = F[0] * s;
  out[n2] = F[1] * s + (R)(tau[0] * sd);
  out[2 * n2] = F[2] * s + (R)(tau[1] * sd);
  out[3 * n2] = F[3] * s + (R)(tau[2] * sd);
  out[4 * n2] = F[4] * s - (R)(qw * sd);  // viscous energy flux along the outward normal: q_w
}

// ---------------------------------------------------------------------------
// k_volume: one CTA per element.  MODE 0 writes Ut; MODE 1 applies the LSERK4
// stage to U and dU in place.
//
// Split-form volume integral with symmetric pairs: the two-point flux is
// symmetric, F#(i, m) = F#(m, i), so each unordered pair of a line is
// evaluated once.  A line of n nodes occupies n consecutive lanes of a warp
// (32 / n lines per warp); at distance d lane i evaluates the pair
// (i, i + d mod n), keeps DVS_{i,m} F and hands F to lane m by a shuffle,
// which applies DVS_{m,i}.  One pass per direction; the three passes meet in
// a shared-memory residual.  With per-node sums S_x = x_i + x_m the flux is
// F0 * 8 = S_rho (S_u . S_a) and F1..4 * 16 = m S_u + S_p4 S_a, m S_h, so
// the scale factors fold into the coefficient tables (DVS/8 and DVS/16).
// EC selects the entropy-conserving flux; its nodes hold (rho, u, v, w,
// 8 beta p', beta, |u|^2, 1 / beta, 1 / rho) and each pair takes two
// logarithmic means (series in t, or the logarithm for far-apart values).
// ---------------------------------------------------------------------------
struct StageArgs {
  double A, B, dt;
  int read_dU;
  int write_w32;  // FP32-mixed form: store the updated state's primitives into W32
};

// Shared-memory slot of a node in the volume kernel's per-node arrays.  A
// direction pass gives each line of n nodes n consecutive lanes; in natural
// order the 8 lanes of a zeta line at N = 7 read addresses 64 apart, all in one
// bank (8-way conflicts), and those of an eta line conflict 2-way.  At N = 7
// the nodes are swizzled (XOR of index bits) so that the lanes of every
// direction's loads and of the thread-per-node prologue and epilogue hit
// distinct banks: 32 four-byte banks per warp for FP32, 16 eight-byte bank
// pairs per half warp for FP64.
template <int N, class R>
__device__ __forceinline__ int vslot(int node) {
  if constexpr (N != 7) {
    return node;
  } else {
    const int i = node & 7, j = (node >> 3) & 7, k = node >> 6;
    if constexpr (sizeof(R) == 4) {
      // bank bits (i0, i1, i2^j2^k2, j0^k0, j1^k1); row (j2, k)
      const int bank = (i & 3) | ((((i ^ j ^ k) >> 2) & 1) << 2) | (((j ^ k) & 3) << 3);
      return (((j >> 2) | (k << 1)) << 5) | bank;
    } else {
      // bank-pair bits (i0, i1^j1^k1, i2^j2^k2, j0^k0); row (j1, j2, k)
      const int bank = (i & 1) | ((i ^ j ^ k) & 6) | (((j ^ k) & 1) << 3);
      return ((((j >> 1) & 3) | (k << 2)) << 4) | bank;
    }
  }
}

// Metric sums a_i + a_m (a = Ja^dir) of the pairs that the FP64 volume kernel
// evaluates at N = 7, per element 16128 doubles: the pairs (pos, pos + d mod 8)
// at cyclic distance d = 1..3 of line L (0..63) along dir at
// pair_main(e, dir, c, d, L, pos), and the pairs (pa, pa + 4) at
// pair_half(K, e, dir, c, L, pa) after all of those.  The volume kernel reads
// them instead of summing the two nodes' metrics (3 FP64 additions of a pair's
// 30), the FP64 pipe being its bound.
__host__ __device__ __forceinline__ size_t pair_main(int e, int dir, int c, int d, int L, int pos) {
  return ((((size_t)e * 3 + dir) * 3 + c) * 3 + (d - 1)) * 512 + (size_t)L * 8 + pos;
}
__host__ __device__ __forceinline__ size_t pair_half(int K, int e, int dir, int c, int L, int pa) {
  return (size_t)K * 13824 + (((size_t)e * 3 + dir) * 3 + c) * 256 + (size_t)L * 4 + pa;
}
__host__ __device__ __forceinline__ int line_node8(int dir, int L, int q) {
  return dir == 0 ? q + 8 * L : (dir == 1 ? (L % 8) + 8 * q + 64 * (L / 8) : L + 64 * q);
}

// one thread per (element, direction, component, line)
static __global__ void k_pair_metric_sums(int K, const double* __restrict__ Ja, double* __restrict__ out) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)K * 3 * 3 * 64) return;
  const int L = (int)(tid % 64), c = (int)((tid / 64) % 3), dir = (int)((tid / 192) % 3), e = (int)(tid / 576);
  const size_t S = (size_t)K * 512;
  const double* a = Ja + (size_t)(dir * 3 + c) * S + (size_t)e * 512;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = a[line_node8(dir, L, q)];
#pragma unroll
  for (int d = 1; d <= 3; ++d)
#pragma unroll
    for (int pos = 0; pos < 8; ++pos) out[pair_main(e, dir, c, d, L, pos)] = x[pos] + x[(pos + d) & 7];
#pragma unroll
  for (int pa = 0; pa < 4; ++pa) out[pair_half(K, e, dir, c, L, pa)] = x[pa] + x[pa + 4];
}

// the values of one node that the two-point flux of a direction reads
template <class R>
struct VolNode {
  R rho, u, v, w, p4, hh, p2, ib, irh, a0, a1, a2;
};

template <int N>
struct VolShape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int LPW = 32 / n;                        // lines per warp
  static constexpr int WARPS_LINES = (n2 + LPW - 1) / LPW;  // warps for one direction
  static constexpr int WARPS_NODES = (n3 + 31) / 32;
  static constexpr int THREADS = 32 * (WARPS_LINES > WARPS_NODES ? WARPS_LINES : WARPS_NODES);
  // shared memory (in units of R): 7 prim slots (9 with the entropy-
  // conserving flux, 10 in the FP32 form of the KEP fluxes: the low parts of
  // the velocity), 9 metric, 5 residual per node, three coefficient tables, 1/w
  static constexpr int SMEM_R = 21 * n3 + 3 * n2 + n;
  static constexpr int SMEM_R_EC = 23 * n3 + 3 * n2 + n;
  static constexpr int SMEM_R_F32 = 24 * n3 + 3 * n2 + n;
};

// Resident CTAs per SM asked of the register allocator: two for CTAs of up to
// 512 threads (64 registers at N = 7; measured 5 % faster in FP64 than one CTA
// at 106 registers, 1.6x faster for the FP32 entropy-conserving kernel than one
// CTA at 104, and 1.3 % faster for the FP64 entropy-conserving kernel than one
// CTA at 126 registers, in spite of its spills).
template <int N, typename R, bool EC>
constexpr int vol_min_blocks() {
  return (N == 7 && !EC && std::is_same<R, float>::value) ? 3 : ((VolShape<N>::THREADS * 64 * 2 <= 65536) ? 2 : 1);
}

template <int N, typename R, int MODE, bool EC>
__global__ void __launch_bounds__(VolShape<N>::THREADS, (vol_min_blocks<N, R, EC>()))
k_volume(const double* __restrict__ Uin, const MeshDev<R> m, const PhysDev ph, const Tables<N> tab,
         const R* __restrict__ Rv, const R* __restrict__ Fs, double* __restrict__ Out,
         double* __restrict__ dU, double* __restrict__ Uout, const StageArgs st, int* __restrict__ status) {
  using Sh = VolShape<N>;
  constexpr int n = Sh::n, n2 = Sh::n2, n3 = Sh::n3, T = Sh::THREADS, LPW = Sh::LPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool F32 = std::is_same<R, float>::value;
  // FP64 at N = 7: the pairs' metric sums read from m.pairA
  constexpr bool PSUM = std::is_same<R, double>::value && n == 8;
  constexpr int QS = EC ? 9 : (F32 ? 10 : 7);
  R* sQ = reinterpret_cast<R*>(smem_raw);  // [QS][n3]: rho u v w 4p' h|e 2p (KG) (+ FP32: ul vl wl); EC see above
  R* sA = sQ + QS * n3;                     // [9][n3]: Ja (dir*3+comp)
  R* sR = sA + 9 * n3;                      // [5][n3]: residual
  R* sC8 = sR + 5 * n3;                     // [n2]: DVS / 8
  R* sC16 = sC8 + n2;                       // [n2]: DVS / 16
  R* sC1 = sC16 + n2;                       // [n2]: DVS
  R* siw = sC1 + n2;                        // [n]
  const int e = blockIdx.x, t = threadIdx.x;
  const size_t S = (size_t)m.K * n3;
  const bool kg = ph.vol_flux == 1;
  // FP32 Pirozzoli form: flux differences G(i -> m) and per-side surface
  // differences F* - F(U_i) (see flux_delta)
  const bool dif = std::is_same<R, float>::value && !EC && ph.fs_diff;
  for (int x = t; x < n2; x += T) {
    sC8[x] = (R)tab.DVS8[x];
    sC16[x] = (R)(0.5 * tab.DVS8[x]);
    sC1[x] = (R)(8.0 * tab.DVS8[x]);
  }
  if (t < n) siw[t] = (R)tab.iw[t];
  // prologue: node t (the FP32-mixed form reads the stage's FP32 primitives
  // and loads the FP64 state only in the epilogue)
  double Uo[5];
  if (t < n3) {
    const size_t g = (size_t)e * n3 + t;
    Prim<R> q;
    if constexpr (F32) {
      // the difference form works on the storage form (shifted rho, h) and
      // the velocity's low parts
      q = dif ? load_prim32(m.W32, S, g) : load_prim32_full(m.W32, S, g, ph);
      if constexpr (!EC) {
        if (dif) {
          const int ts = vslot<N, R>(t);
          const Lo3 l = load_lo32(m.W32, S, g);
          sQ[7 * n3 + ts] = l.u; sQ[8 * n3 + ts] = l.v; sQ[9 * n3 + ts] = l.w;
        }
      }
    } else if (m.W64) {
      q = load_prim64(m.W64, S, g);
    } else {
      q = primitive<R>(Uin[g], Uin[S + g], Uin[2 * S + g], Uin[3 * S + g], Uin[4 * S + g], ph);
    }
    const int ts = vslot<N, R>(t);
    sQ[ts] = q.rho; sQ[n3 + ts] = q.u; sQ[2 * n3 + ts] = q.v; sQ[3 * n3 + ts] = q.w;
    sQ[4 * n3 + ts] = dif ? q.p : R(4) * q.p;
    if constexpr (EC) {
      const R pf = q.p + cR<R>(ph.p_ref, ph.f32c.p_ref);
      const R beta = R(0.5) * q.rho * rcp_t<R>(pf);
      const R irho = rcp_t<R>(q.rho);
      sQ[4 * n3 + ts] = R(8) * beta * q.p;
      sQ[5 * n3 + ts] = beta;
      sQ[6 * n3 + ts] = q.u * q.u + q.v * q.v + q.w * q.w;
      sQ[7 * n3 + ts] = pf * irho;      // 1 / (2 beta)
      sQ[8 * n3 + ts] = R(0.5) * irho;  // 1 / (2 rho)
    } else if (!kg) {
      sQ[5 * n3 + ts] = q.h;
    } else {
      const R pf = q.p + cR<R>(ph.p_ref, ph.f32c.p_ref);
      sQ[5 * n3 + ts] = q.h - pf / q.rho;  // e = E / rho
      sQ[6 * n3 + ts] = R(2) * pf;
    }
    // (FP64 at N = 7: the pairs' metric sums come from m.pairA instead)
    if constexpr (!PSUM) {
#pragma unroll
      for (int c = 0; c < 9; ++c) sA[c * n3 + ts] = m.Ja[(size_t)c * S + g];
    }
  }
  __syncthreads();
  // three direction passes over the lines
  {
    const int warp = t >> 5, lane = t & 31;
    const int seg = lane / n, pos = lane - seg * n;
    const int L0 = warp * LPW + seg;
    const bool active = (seg < LPW) && (L0 < n2);
    const int L = active ? L0 : 0;
    const int base = seg * n;  // first lane of the segment
    const int la = L % n, lb = L / n;
    // node at position q of this lane's line along dir (a warp holds the same
    // lines L in every direction)
    auto node_at = [&](int dir, int q) {
      return dir == 0 ? q + n * L : (dir == 1 ? la + n * q + n2 * lb : L + n2 * q);
    };
    auto load_node = [&](int nd, int dir) {
      const int node = vslot<N, R>(nd);
      VolNode<R> X;
      X.rho = sQ[node]; X.u = sQ[n3 + node]; X.v = sQ[2 * n3 + node]; X.w = sQ[3 * n3 + node];
      X.p4 = sQ[4 * n3 + node]; X.hh = sQ[5 * n3 + node];
      X.p2 = (kg || EC) ? sQ[6 * n3 + node] : R(0);
      X.ib = EC ? sQ[7 * n3 + node] : R(0);
      X.irh = EC ? sQ[8 * n3 + node] : R(0);
      if constexpr (!PSUM) {
        X.a0 = sA[(dir * 3 + 0) * n3 + node]; X.a1 = sA[(dir * 3 + 1) * n3 + node];
        X.a2 = sA[(dir * 3 + 2) * n3 + node];
      } else {
        X.a0 = X.a1 = X.a2 = R(0);
      }
      return X;
    };
    // symmetric two-point flux F#(A, B) . 4 {Ja} in the scaled form of the
    // coefficient tables (mass row against DVS / 8, the others against DVS / 16)
    // (Sa: the sum of the two nodes' metrics, given or formed here)
    auto sym_flux_s = [&](const VolNode<R>& A, const VolNode<R>& B, R Sa0, R Sa1, R Sa2, R F[5]) {
      const R Sr = A.rho + B.rho, Su = A.u + B.u, Sv = A.v + B.v, Sw = A.w + B.w;
      const R Sp = A.p4 + B.p4;
      const R ua = Su * Sa0 + Sv * Sa1 + Sw * Sa2;  // 4 {u}.{a}
      if constexpr (EC) {
        // nodes hold ib = 1 / (2 beta) and irh = 1 / (2 rho), so that with
        // Sh = ib_A + ib_B (half the sum of the inverse temperatures):
        //   rho_ln = Sr G / 2;  rgm1 / beta_ln = Sh Qg / 2 (Qg = 2 rgm1 Q);
        //   1 / (bA + bB) = Sh Rh / 2 (Rh = Rb / 2)
        const R Dr = A.rho - B.rho, Db = A.hh - B.hh, Sh = A.ib + B.ib;
        const R tr = Dr * Dr * (A.irh * B.irh);
        const R tb = Db * Db * (A.ib * B.ib);
        const R G = tr < LogMeanCut<R>::v ? logmean_G<R>(tr) : R(2) * Dr / (Sr * log1p(Dr / B.rho));
        R Qg, Rh;
        if (tb < LogMeanCut<R>::v) {
          auto qc = [&](int c) { return cR<R>(ph.ec_q[c], ph.f32c.ec_q[c]); };
          Qg = qc(0) + tb * (qc(1) + tb * (qc(2) + tb * (qc(3) + tb * qc(4))));
          Rh = R(0.5) + tb * (R(-0.5) + tb * (R(0.5) + tb * (R(-0.5) + tb * R(0.5))));
        } else {
          Qg = R(2) * cR<R>(ph.rgm1, ph.f32c.rgm1) * log1p(Db / B.hh) / (Db * Sh);
          Rh = R(1) / (Sh * (A.hh + B.hh));
        }
        const R mf = Sr * G * ua;                 // 8 F_rho
        const R Spt = Sh * Rh * Sp;               // 8 (p~ - p_ref)
        F[0] = mf;
        F[1] = mf * Su + Spt * Sa0;               // 16 F_m
        F[2] = mf * Sv + Spt * Sa1;
        F[3] = mf * Sw + Spt * Sa2;
        // 16 F_E = 2 mf (1 / (2 (gamma-1) beta_ln) + |{u}|^2 - {|u|^2} / 2) + 4 p~ (4 {u}.{a})
        //        = mf X / 2 + (Spt / 2 + 4 p_ref) (4 {u}.{a})
        const R X = Sh * Qg + Su * Su + Sv * Sv + Sw * Sw - A.p2 - B.p2;
        F[4] = R(0.5) * mf * X + (R(0.5) * Spt + R(4) * cR<R>(ph.p_ref, ph.f32c.p_ref)) * ua;
      } else {
        const R mf = Sr * ua;                     // 8 F0
        F[0] = mf;
        F[1] = mf * Su + Sp * Sa0;                // 16 F1
        F[2] = mf * Sv + Sp * Sa1;
        F[3] = mf * Sw + Sp * Sa2;
        F[4] = mf * (A.hh + B.hh);                // 16 F4
        if (kg) F[4] += (A.p2 + B.p2) * ua;
      }
    };
    auto sym_flux = [&](const VolNode<R>& A, const VolNode<R>& B, R F[5]) {
      sym_flux_s(A, B, A.a0 + B.a0, A.a1 + B.a1, A.a2 + B.a2, F);
    };
    auto sums_main = [&](int dir, int d, R Sa[3]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) Sa[c] = m.pairA[pair_main(e, dir, c, d, L, pos)];
    };
    auto sums_half = [&](int dir, int Lx, int pa, R Sa[3]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) Sa[c] = m.pairA[pair_half(m.K, e, dir, c, Lx, pa)];
    };
    // FP64, N = 7: the n/2 pairs at distance n/2 of a line would be formed twice
    // (once in each lane); instead the distance-n/2 step of the xi pass forms
    // the xi pairs in lanes pos < n/2 and the eta pairs in lanes pos >= n/2
    // (swapped by a shuffle), and the one of the eta pass, in the first half
    // of the warps, the zeta pairs of its own lines (lanes pos < n/2) and of
    // the lines of warp + WARPS_LINES/2 (lanes pos >= n/2, through shared
    // memory: the xi metrics, no longer read after the xi pass).  A lane
    // carries that pair's flux for its next pass's node in `carry`.
    // A node's sum runs through the passes: the xi pass starts it with the
    // weak viscous divergence R_v, the eta and zeta passes from the sum the
    // previous pass stored (with the carried pair's term as its first FMA).
    constexpr bool HALF = std::is_same<R, double>::value && n == 8 && Sh::WARPS_LINES % 2 == 0;
    constexpr int DMAX = HALF ? n / 2 - 1 : n / 2;
    constexpr int HW = Sh::WARPS_LINES / 2, NX = HW * LPW * (n / 2);
    R* sX = sA;  // [5][NX] zeta pair fluxes handed to the second half of the warps
    R carry[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int me = node_at(dir, pos);
      const int ms = vslot<N, R>(me);
      const VolNode<R> A = load_node(me, dir);
      // FP32 difference form: the low parts of this lane's node velocity
      float Aul = 0.f, Avl = 0.f, Awl = 0.f;
      if constexpr (F32 && !EC) {
        if (dif) { Aul = sQ[7 * n3 + ms]; Avl = sQ[8 * n3 + ms]; Awl = sQ[9 * n3 + ms]; }
      }
      R acc[5];
      if (dir == 0) {
        acc[0] = R(0);
        const R* rv = Rv + (size_t)e * n3 + me;
#pragma unroll
        for (int v = 1; v < 5; ++v) acc[v] = ph.viscous ? rv[(size_t)(v - 1) * S] : R(0);
      } else if constexpr (HALF) {
        const int px = pos ^ (n / 2);
        const R c8 = sC8[pos * n + px], c16 = sC16[pos * n + px];
        if (dir == 2 && warp >= HW) {
          const int x = ((warp - HW) * LPW + seg) * (n / 2) + (pos & (n / 2 - 1));
#pragma unroll
          for (int v = 0; v < 5; ++v) carry[v] = sX[v * NX + x];
        }
        acc[0] = fma(c8, carry[0], sR[ms]);
#pragma unroll
        for (int v = 1; v < 5; ++v) acc[v] = fma(c16, carry[v], sR[v * n3 + ms]);
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] = sR[v * n3 + ms];
      }
#pragma unroll
      for (int d = 1; d <= DMAX; ++d) {
        const int pm = pos + d < n ? pos + d : pos + d - n;
        const int q = node_at(dir, pm);
        if constexpr (std::is_same<R, float>::value && !EC) {
          if (dif) {
            const NodeF mi{A.rho, A.u, A.v, A.w, A.p4, A.hh, Aul, Avl, Awl};
            // the partner node's values from the lane that holds it (lane
            // base + pm of this line's segment)
            const int lq = base + pm;
            auto sh = [&](float x) { return __shfl_sync(0xffffffffu, x, lq); };
            const NodeF mq{sh(A.rho), sh(A.u), sh(A.v), sh(A.w), sh(A.p4), sh(A.hh), sh(Aul), sh(Avl), sh(Awl)};
            const float aq0 = sh(A.a0), aq1 = sh(A.a1), aq2 = sh(A.a2);
            float G[5], Gq[5];
            const float c1 = sC1[pos * n + pm];
            if (2 * d != n) {
              // and G(q -> i) for the partner lane (pos + d); receive G(i -> pos - d)
              flux_delta_pair(mi, mq, A.a0, A.a1, A.a2, aq0, aq1, aq2, ph.f32c.rho_ref, ph.f32c.h_ref, G, Gq);
#pragma unroll
              for (int v = 0; v < 5; ++v) acc[v] += c1 * G[v];
              const int src = base + (pos - d >= 0 ? pos - d : pos - d + n);
              const float r1 = sC1[pos * n + (src - base)];
#pragma unroll
              for (int v = 0; v < 5; ++v) acc[v] += r1 * __shfl_sync(0xffffffffu, Gq[v], src);
            } else {
              flux_delta(mi, mq, A.a0, A.a1, A.a2, aq0 - A.a0, aq1 - A.a1, aq2 - A.a2, ph.f32c.rho_ref,
                         ph.f32c.h_ref, G);
#pragma unroll
              for (int v = 0; v < 5; ++v) acc[v] += c1 * G[v];
            }
            continue;
          }
        }
        R F[5];
        if constexpr (PSUM) {
          R Sa[3];
          sums_main(dir, d, Sa);
          sym_flux_s(A, load_node(q, dir), Sa[0], Sa[1], Sa[2], F);
        } else {
          sym_flux(A, load_node(q, dir), F);
        }
        const R c8 = sC8[pos * n + pm], c16 = sC16[pos * n + pm];
        acc[0] += c8 * F[0];
#pragma unroll
        for (int v = 1; v < 5; ++v) acc[v] += c16 * F[v];
        if (2 * d != n) {
          // hand the pair flux to the partner lane (pos + d); receive the one
          // of lane (pos - d)
          const int src = base + (pos - d >= 0 ? pos - d : pos - d + n);
          const int ps = src - base;
          const R r8 = sC8[pos * n + ps], r16 = sC16[pos * n + ps];
          acc[0] += r8 * __shfl_sync(0xffffffffu, F[0], src);
#pragma unroll
          for (int v = 1; v < 5; ++v) acc[v] += r16 * __shfl_sync(0xffffffffu, F[v], src);
        }
      }
      if constexpr (HALF) {
        constexpr int h = n / 2;
        const int px = pos ^ h;  // partner at distance n/2
        const R c8 = sC8[pos * n + px], c16 = sC16[pos * n + px];
        if (dir == 0) {
          const bool lo = pos < h;
          const int dd = lo ? 0 : 1, pa = pos & (h - 1);
          R F[5];
          if constexpr (PSUM) {
            R Sa[3];
            sums_half(dd, L, pa, Sa);
            sym_flux_s(load_node(node_at(dd, pa), dd), load_node(node_at(dd, pa + h), dd), Sa[0], Sa[1], Sa[2], F);
          } else {
            sym_flux(load_node(node_at(dd, pa), dd), load_node(node_at(dd, pa + h), dd), F);
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const R Fx = __shfl_xor_sync(0xffffffffu, F[v], h);
            acc[v] += (v == 0 ? c8 : c16) * (lo ? F[v] : Fx);
            carry[v] = lo ? Fx : F[v];
          }
        } else if (dir == 1 && warp < HW) {
          const bool lo = pos < h;
          const int pa = pos & (h - 1);
          const int Lz = lo ? L : L + HW * LPW;  // zeta line of this warp or of warp + HW
          R F[5];
          if constexpr (PSUM) {
            R Sa[3];
            sums_half(2, Lz, pa, Sa);
            sym_flux_s(load_node(Lz + n2 * pa, 2), load_node(Lz + n2 * (pa + h), 2), Sa[0], Sa[1], Sa[2], F);
          } else {
            sym_flux(load_node(Lz + n2 * pa, 2), load_node(Lz + n2 * (pa + h), 2), F);
          }
          const int x = (warp * LPW + seg) * h + pa;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const R Fx = __shfl_xor_sync(0xffffffffu, F[v], h);
            carry[v] = lo ? F[v] : Fx;
            if (!lo) sX[v * NX + x] = F[v];
          }
        }
      }
      if (active) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sR[v * n3 + ms] = acc[v];
      }
      __syncthreads();
    }
  }
  if (t >= n3) return;
  // epilogue: one node per thread.  At N = 7 the two warps of a zeta layer
  // hold the eta rows {0, N, 1, 2} and {3, 4, 5, 6}, so that only the first
  // runs the (masked) eta-face branch of the surface integral
  int i, j, k;
  if constexpr (n == 8 && T == n3) {
    const int w = t >> 5, r = (t >> 3) & 3;
    i = t & 7;
    k = w >> 1;
    j = (w & 1) ? 3 + r : (r == 0 ? 0 : (r == 1 ? N : r - 1));
  } else {
    i = t % n; j = (t / n) % n; k = t / n2;
  }
  const int nd = i + n * (j + n * k);
  const size_t g = (size_t)e * n3 + nd;
  // the element's own state, for the register update (read again here rather
  // than kept in registers through the passes)
#pragma unroll
  for (int v = 0; v < 5; ++v) Uo[v] = Uin[v * S + g];
  R acc[5];  // the passes' sums (with R_v)
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = sR[v * n3 + vslot<N, R>(nd)];
  // surface integral: + sgn * Fs / w_perp on the faces that touch the node
  auto surf = [&](int l, int ab, R iw) {
    const int code = m.elem_face[e * 6 + l];
    const int f = chk_idx(code >> 4, m.F, m.status);
    const R sg = (code & 1) ? -iw : iw;
    ab = omap_ab<N>((code >> 1) & 7, ab);  // the node's index in the master's face order
    // difference form: the face's own side, F* - F(U_side), in rows 5 n2 apart
    const R* src = dif ? Fs + (size_t)f * 10 * n2 + ((code & 1) ? 5 * n2 : 0) + ab : Fs + (size_t)f * 5 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += sg * src[v * n2];
  };
  // one branch per direction (masked lanes of a branch cost as much as active ones)
  if (i == 0 || i == N) surf(i == 0 ? 0 : 1, j + n * k, i == 0 ? siw[0] : siw[N]);
  if (j == 0 || j == N) surf(j == 0 ? 2 : 3, i + n * k, j == 0 ? siw[0] : siw[N]);
  if (k == 0 || k == N) surf(k == 0 ? 4 : 5, i + n * j, k == 0 ? siw[0] : siw[N]);
  // Ut = -(1/J) acc + S, S = (0, f, f . u)
  const R iJ = m.invJ[g];
  const bool force = ph.has_force != 0;
  double src[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (force) {
    const double ir = 1.0 / Uo[0];
    src[1] = ph.f[0]; src[2] = ph.f[1]; src[3] = ph.f[2];
    src[4] = (ph.f[0] * Uo[1] + ph.f[1] * Uo[2] + ph.f[2] * Uo[3]) * ir;
  }
  if (MODE == 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Out[v * S + g] = -(double)(iJ * acc[v]) + src[v];
  } else {
    // dU = A dU + dt Ut = A dU + (-dt / J) acc + dt S;  U = U + B dU
    // (the FP32-mixed form forms the increment dt Ut in FP32, the accuracy of
    // its Ut, and keeps the register update in FP64)
    const double c = -st.dt * (double)iJ;
    const R cf = F32 ? (R)(-st.dt) * iJ : R(0);
    bool bad = false;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double d;
      if constexpr (F32) d = f2d_bits(cf * acc[v]);
      else d = c * (double)acc[v];
      if (force) d = fma(st.dt, src[v], d);
      if (st.read_dU) d = fma(st.A, dU[v * S + g], d);
      const double un = fma(st.B, d, Uo[v]);
      dU[v * S + g] = d;
      Uout[v * S + g] = un;
      Uo[v] = un;
      bad |= !finite_bits(un);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    // the next stage's FP32 primitives, from the updated FP64 state
    if constexpr (F32) {
      if (st.write_w32) {
        Lo3 l;
        const Prim<float> q = prim32_shifted(Uo[0], Uo[1], Uo[2], Uo[3], Uo[4], ph, &l);
        store_prim32(m.W32, S, g, q, l);
      }
    }
  }
}

}  // namespace dg
