// adjoint.cuh -- vector-Jacobian product of the DGSEM operator (FP64).
//
// Given a cotangent lam of Ut = DG_Operator(U), computes gU = (dUt/dU)^T lam
// and g_theta = (dUt/d(kappa, B))^T lam for the wall-law constants.  The
// kernels run the forward operator's structure backwards:
//   k_adj_face   interior face nodes: cotangent of the surface flux from the
//                two sides' lam, the Riemann flux in hand-written reverse mode
//                (face_flux_vjp), and the cotangents of the two sides'
//                viscous face fluxes;
//   k_adj_wall   wall face nodes: the same through the mirror state, and the
//                wall-model derivative (forward-mode duals over the sample
//                state; implicit function theorem for the law of the wall)
//                with respect to the sample state and (kappa, B);
//   k_adj_element one CTA per element: transposed split-form volume integral
//                (hand-derived, symmetric pairs with shuffles), transposed
//                viscous divergence and viscous flux, transposed BR1 lifting,
//                transposed primitive recovery, source term;
//   k_adj_gather  adds the per-face contributions of the face kernels and of
//                the neighbours' lifting to every node;
//   k_adj_scatter adds the wall-model sample cotangents to the sample
//                elements (Lagrange weights; atomics).
#pragma once
#include "kernels.cuh"

namespace dg {

// ---------------------------------------------------------------------------
// forward-mode dual number (value, one directional derivative)
// ---------------------------------------------------------------------------
struct DualD {
  double v, d;
  __device__ DualD() : v(0.0), d(0.0) {}
  __device__ DualD(double x) : v(x), d(0.0) {}
  __device__ DualD(double x, double dx) : v(x), d(dx) {}
};
__device__ __forceinline__ DualD operator+(DualD a, DualD b) { return DualD(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ DualD operator-(DualD a, DualD b) { return DualD(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ DualD operator-(DualD a) { return DualD(-a.v, -a.d); }
__device__ __forceinline__ DualD operator*(DualD a, DualD b) { return DualD(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ DualD operator/(DualD a, DualD b) {
  const double r = a.v / b.v;
  return DualD(r, (a.d - r * b.d) / b.v);
}
__device__ __forceinline__ DualD operator+(DualD a, double b) { return DualD(a.v + b, a.d); }
__device__ __forceinline__ DualD operator+(double a, DualD b) { return DualD(a + b.v, b.d); }
__device__ __forceinline__ DualD operator-(DualD a, double b) { return DualD(a.v - b, a.d); }
__device__ __forceinline__ DualD operator-(double a, DualD b) { return DualD(a - b.v, -b.d); }
__device__ __forceinline__ DualD operator*(DualD a, double b) { return DualD(a.v * b, a.d * b); }
__device__ __forceinline__ DualD operator*(double a, DualD b) { return DualD(a * b.v, a * b.d); }
__device__ __forceinline__ DualD operator/(DualD a, double b) { return DualD(a.v / b, a.d / b); }
__device__ __forceinline__ DualD operator/(double a, DualD b) {
  const double r = a / b.v;
  return DualD(r, -r * b.d / b.v);
}
__device__ __forceinline__ DualD& operator+=(DualD& a, DualD b) { a = a + b; return a; }
__device__ __forceinline__ DualD& operator-=(DualD& a, DualD b) { a = a - b; return a; }
__device__ __forceinline__ bool operator<(DualD a, DualD b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>=(DualD a, DualD b) { return a.v >= b.v; }
__device__ __forceinline__ DualD sqrt(DualD a) {
  const double s = ::sqrt(a.v);
  return DualD(s, a.d / (2.0 * s));
}
__device__ __forceinline__ DualD fabs(DualD a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ DualD asin(DualD a) { return DualD(::asin(a.v), a.d / ::sqrt(1.0 - a.v * a.v)); }

// ---------------------------------------------------------------------------
// wall-model JVP: tau (3) with its derivative along the duals of Us and
// (dk, dB) for the law constants.  u_tau comes from the primal solver; its
// derivative from the implicit function theorem on F(t) = t + ln L(e^t) -
// ln Re_h = 0, Re_h = h u_VD / nu_w.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void law_param_derivs(int law, double w, double kap, double B, double* Lk,
                                                 double* LB) {
  if (law == 1) {
    const double e1 = exp(-w / 11.0), e2 = exp(-0.33 * w);
    const double brk = 1.0 - e1 - (w / 11.0) * e2;
    const double dC = -(1.0 - log(kap)) / (kap * kap);
    *Lk = (w / (1.0 + kap * w)) / kap - log1p(kap * w) / (kap * kap) + dC * brk;
    *LB = brk;
  } else {
    const double x = kap * w, eb = exp(-kap * B), ex = exp(x);
    const double x3 = x * x * x / 6.0;
    const double P = ex - 1.0 - x - 0.5 * x * x - x3 - 0.25 * x * x3;
    const double Pp = ex - 1.0 - x - 0.5 * x * x - x3;
    *Lk = -B * eb * P + eb * Pp * w;
    *LB = -kap * eb * P;
  }
}

// qw (may be null): the wall heat flux of isothermal walls (0 for adiabatic ones)
static __device__ void wall_stress_jvp(const PhysDev& ph, const DualD Us[5], double dk, double dB, double nx,
                                double ny, double nz, DualD tau[3], bool* ok, DualD* qw = nullptr) {
  const DualD rho = Us[0], ir = 1.0 / rho;
  const DualD u = Us[1] * ir, v = Us[2] * ir, w = Us[3] * ir;
  const DualD p = ph.gm1 * (Us[4] - 0.5 * rho * (u * u + v * v + w * w));
  const DualD T = p * ph.rcp_R * ir;
  const DualD un = u * nx + v * ny + w * nz;
  const DualD ux = u - un * nx, uy = v - un * ny, uz = w - un * nz;
  const DualD u2 = ux * ux + uy * uy + uz * uz;
  tau[0] = tau[1] = tau[2] = DualD(0.0);
  if (qw) *qw = DualD(0.0);
  *ok = true;
  if (!(u2.v > 0.0)) return;
  const DualD um = sqrt(u2);
  const double r = cbrt(ph.Pr);
  const DualD Taw = T + r * u2 / (2.0 * ph.cp);
  // the Van Driest transform: adiabatic (T_w = T_aw) or, at an isothermal
  // wall, the closed form of the Crocco-Busemann integral (as wall_stress)
  DualD Tw, uvd;
  if (ph.T_wall > 0.0) {
    Tw = DualD(ph.T_wall);
    const DualD b = (Taw - Tw) / (Tw * um);
    const DualD a2 = r / (2.0 * ph.cp * Tw);
    const DualD aa = sqrt(a2);
    const DualD q = sqrt(b * b + 4.0 * a2);
    uvd = (asin((2.0 * a2 * um - b) / q) + asin(b / q)) / aa;
  } else {
    Tw = Taw;
    const DualD a = sqrt(r / (2.0 * ph.cp * Tw));
    uvd = asin(a * um) / a;
  }
  const DualD rhow = rho * T / Tw;
  // wall viscosity: constant, or Sutherland's law at the wall temperature
  const DualD muw = ph.sutherland ? ph.suth_C * Tw * sqrt(Tw) / (Tw + ph.suth_S) : DualD(ph.mu);
  const DualD nuw = muw / rhow;
  const double ut = solve_utau(ph.law, uvd.v, ph.hwm, nuw.v, ph.kappa, ph.B, ph.wm_maxit, ok);
  // explicit variable of the law at the solution
  const double wv = ph.law == 1 ? ut * ph.hwm / nuw.v : uvd.v / ut;
  double L, wdL, Lk, LB;
  law_eval(ph.law, wv, ph.kappa, ph.B, &L, &wdL);
  law_param_derivs(ph.law, wv, ph.kappa, ph.B, &Lk, &LB);
  const double Ft = 1.0 + wdL / L;
  const double dlnRe = uvd.d / uvd.v - nuw.d / nuw.v;
  const double dt = -((Lk * dk + LB * dB) / L - dlnRe) / Ft;
  const double dut = ph.law == 1 ? ut * (dt + nuw.d / nuw.v) : ut * (uvd.d / uvd.v - dt);
  const DualD utD(ut, dut);
  const DualD tw = rhow * utD * utD / um;
  tau[0] = tw * ux; tau[1] = tw * uy; tau[2] = tw * uz;
  if (qw && ph.T_wall > 0.0) *qw = -(ph.cp / ph.Pr) * (rhow * utD * utD) * (Taw - Tw) / um;
}

// ---------------------------------------------------------------------------
// transposed primitive recoveries
// ---------------------------------------------------------------------------
// Q = (rho, u, v, w, p - p_ref, h): gU += (dQ/dU)^T gQ
__device__ __forceinline__ void prim_vjp(const double U[5], const PhysDev& ph, const double gQ[6], double gU[5]) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const double q2 = u * u + v * v + w * w;
  const double p = ph.gm1 * (U[4] - 0.5 * U[0] * q2);
  const double h = (U[4] + p) * ir;
  const double g1 = ph.gm1;
  const double gp = gQ[4], gh = gQ[5];
  gU[0] += gQ[0] - (gQ[1] * u + gQ[2] * v + gQ[3] * w) * ir + gp * 0.5 * g1 * q2 + gh * (0.5 * g1 * q2 - h) * ir;
  gU[1] += gQ[1] * ir - gp * g1 * u - gh * g1 * u * ir;
  gU[2] += gQ[2] * ir - gp * g1 * v - gh * g1 * v * ir;
  gU[3] += gQ[3] * ir - gp * g1 * w - gh * g1 * w * ir;
  gU[4] += gp * g1 + gh * (1.0 + g1) * ir;
}

// W = (u, v, w, T): gU += (dW/dU)^T gW
__device__ __forceinline__ void vt_vjp(const double U[5], const PhysDev& ph, const double gW[4], double gU[5]) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const double q2 = u * u + v * v + w * w;
  const double p = ph.gm1 * (U[4] - 0.5 * U[0] * q2);
  const double T = p * ph.rcp_R * ir;
  const double c = ph.gm1 * ph.rcp_R * ir;  // dT/dE
  gU[0] += -(gW[0] * u + gW[1] * v + gW[2] * w) * ir + gW[3] * (0.5 * q2 * c - T * ir);
  gU[1] += gW[0] * ir - gW[3] * c * u;
  gU[2] += gW[1] * ir - gW[3] * c * v;
  gU[3] += gW[2] * ir - gW[3] * c * w;
  gU[4] += gW[3] * c;
}

// ---------------------------------------------------------------------------
// Reverse mode of the inviscid interface flux F*(U_A, U_B; n) (two-point
// Pirozzoli or entropy-conserving two-point flux plus the central / Lax-Friedrichs /
// Roe-Harten dissipation,
// as riemann<double> forms it): gUA += (dF*/dU_A)^T gF, gUB += (dF*/dU_B)^T gF.
// One forward sweep keeps the intermediates, one backward sweep applies the
// chain rule to them in reverse order (about three flux evaluations, against
// ten forward-mode dual sweeps).  |x| takes the derivative sign(x) with
// sign(0) = +1, as the dual numbers do.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sgn1(double x) { return x < 0.0 ? -1.0 : 1.0; }

// Logarithmic mean L(a, b) = (a - b) / ln(a / b) and its partial derivatives:
// dL/da = (1 - L / a) / ln(a / b), dL/db = (L / b - 1) / ln(a / b); for nearby
// values (u = ((a - b) / (a + b))^2 below the forward kernels' cut) from the
// series L = (s / 2) g(u) with g' = -1/3 - 8u/45 - 132u^2/945 and
// du/da = 4 (a - b) b / s^3, du/db = -4 (a - b) a / s^3.
__device__ __forceinline__ void logmean_d(double a, double b, double* L, double* La, double* Lb) {
  const double s = a + b, d = a - b, f = d / s, u = f * f;
  if (u < LogMeanCut<double>::v) {
    const double g = logmean_g<double>(u);
    const double gp = -(1.0 / 3.0 + u * (8.0 / 45.0 + u * (132.0 / 945.0)));
    const double c = 2.0 * d * gp / (s * s);
    *L = 0.5 * s * g;
    *La = 0.5 * g + c * b;
    *Lb = 0.5 * g - c * a;
  } else {
    const double l = log1p(d / b);
    *L = d / l;
    *La = (1.0 - *L / a) / l;
    *Lb = (*L / b - 1.0) / l;
  }
}

// Reverse mode of Chandrashekar's entropy-conserving two-point flux along a
// (twopoint_ec): gA, gB += (dF/dq_A)^T mu, (dF/dq_B)^T mu for the primitives
// q = (rho, u, v, w, p - p_ref) of the two nodes.  With beta = rho / (2 p),
//   f0 = L(rho) ua, ua = {u}.a, p~' = (bA p'A + bB p'B) / (bA + bB),
//   F = (f0, f0 {u} + p~' a, f0 X + (p~' + p_ref) ua),
//   X = 1 / (2 (gamma - 1) L(beta)) + |{u}|^2 - ({|u|^2}) / 2.
__device__ __forceinline__ void ec_flux_vjp(const PhysDev& ph, const Prim<double>& A, const Prim<double>& B,
                                            double a0, double a1, double a2, const double mu[5], double gA[5],
                                            double gB[5]) {
  const double pref = ph.p_ref;
  const double PA = A.p + pref, PB = B.p + pref;
  const double bA = 0.5 * A.rho / PA, bB = 0.5 * B.rho / PB;
  double Lr, Lra, Lrb, Lb, Lba, Lbb;
  logmean_d(A.rho, B.rho, &Lr, &Lra, &Lrb);
  logmean_d(bA, bB, &Lb, &Lba, &Lbb);
  const double Mb = 1.0 / Lb, rb = 1.0 / (bA + bB);
  const double u = 0.5 * (A.u + B.u), v = 0.5 * (A.v + B.v), w = 0.5 * (A.w + B.w);
  const double ua = u * a0 + v * a1 + w * a2;
  const double pt = (bA * A.p + bB * B.p) * rb;
  const double f0 = Lr * ua;
  const double k2 = 0.25 * (A.u * A.u + A.v * A.v + A.w * A.w + B.u * B.u + B.v * B.v + B.w * B.w);
  const double X = 0.5 * Mb * ph.rgm1 + (u * u + v * v + w * w) - k2;
  // backward sweep
  const double gf0 = mu[0] + mu[1] * u + mu[2] * v + mu[3] * w + mu[4] * X;
  const double gpt = mu[1] * a0 + mu[2] * a1 + mu[3] * a2 + mu[4] * ua;
  const double gua = gf0 * Lr + mu[4] * (pt + pref);
  const double gLr = gf0 * ua;
  const double gX = mu[4] * f0;
  const double gu = mu[1] * f0 + 2.0 * u * gX + a0 * gua;
  const double gv = mu[2] * f0 + 2.0 * v * gX + a1 * gua;
  const double gw = mu[3] * f0 + 2.0 * w * gX + a2 * gua;
  const double gLb = -Mb * Mb * (0.5 * ph.rgm1 * gX);
  double gbA = gpt * rb * (A.p - pt) + gLb * Lba;
  double gbB = gpt * rb * (B.p - pt) + gLb * Lbb;
  double gpA = gpt * rb * bA, gpB = gpt * rb * bB;
  // beta = rho / (2 P): d/drho = 1 / (2 P), d/dP = -beta / P
  gA[0] += gLr * Lra + gbA * 0.5 / PA;
  gB[0] += gLr * Lrb + gbB * 0.5 / PB;
  gpA -= gbA * bA / PA;
  gpB -= gbB * bB / PB;
  // velocities: {u} and the kinetic-energy term k2
  gA[1] += 0.5 * gu - 0.5 * gX * A.u; gB[1] += 0.5 * gu - 0.5 * gX * B.u;
  gA[2] += 0.5 * gv - 0.5 * gX * A.v; gB[2] += 0.5 * gv - 0.5 * gX * B.v;
  gA[3] += 0.5 * gw - 0.5 * gX * A.w; gB[3] += 0.5 * gw - 0.5 * gX * B.w;
  gA[4] += gpA; gB[4] += gpB;
}

static __device__ void face_flux_vjp(const PhysDev& ph, const double UA[5], const double UB[5], double nx,
                                     double ny, double nz, const double gF[5], double gUA[5], double gUB[5]) {
  const Prim<double> A = primitive<double>(UA[0], UA[1], UA[2], UA[3], UA[4], ph);
  const Prim<double> B = primitive<double>(UB[0], UB[1], UB[2], UB[3], UB[4], ph);
  // cotangents of the primitives (rho, u, v, w, p - p_ref, h) of each side
  double qA[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, qB[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (ph.vol_flux == 2) {
    // the entropy-conserving flux as the central part (Sec. 4's scheme)
    ec_flux_vjp(ph, A, B, nx, ny, nz, gF, qA, qB);
  } else {
    // two-point flux: m = {rho} ({u}.n); F = (m, m {u} + {p} n, m {h})
    const double rho = 0.5 * (A.rho + B.rho), u = 0.5 * (A.u + B.u), v = 0.5 * (A.v + B.v), w = 0.5 * (A.w + B.w);
    const double hb = 0.5 * (A.h + B.h);
    const double un = u * nx + v * ny + w * nz, m = rho * un;
    const double gm = gF[0] + gF[1] * u + gF[2] * v + gF[3] * w + gF[4] * hb;
    const double gun = gm * rho;
    const double g[6] = {gm * un, gF[1] * m + gun * nx, gF[2] * m + gun * ny, gF[3] * m + gun * nz,
                         gF[1] * nx + gF[2] * ny + gF[3] * nz, gF[4] * m};
#pragma unroll
    for (int x = 0; x < 6; ++x) { qA[x] += 0.5 * g[x]; qB[x] += 0.5 * g[x]; }
  }
  if (ph.surf_flux == 1) {
    // F -= lam (U_B - U_A), lam = max(|u_n| + c) / 2 over the sides
    const double pref = ph.p_ref, gam = ph.gamma;
    const double cA = ::sqrt(gam * (A.p + pref) / A.rho), cB = ::sqrt(gam * (B.p + pref) / B.rho);
    const double unA = A.u * nx + A.v * ny + A.w * nz, unB = B.u * nx + B.v * ny + B.w * nz;
    const double lA = ::fabs(unA) + cA, lB = ::fabs(unB) + cB;
    const double lam = 0.5 * (lA >= lB ? lA : lB);
    double glam = 0.0;
#pragma unroll
    for (int x = 0; x < 5; ++x) {
      glam -= gF[x] * (UB[x] - UA[x]);
      gUA[x] += lam * gF[x];
      gUB[x] -= lam * gF[x];
    }
    const bool a_side = lA >= lB;
    double* q = a_side ? qA : qB;
    const double un = a_side ? unA : unB, c = a_side ? cA : cB;
    const Prim<double>& X = a_side ? A : B;
    const double gl = 0.5 * glam, gn = gl * sgn1(un);
    q[1] += gn * nx; q[2] += gn * ny; q[3] += gn * nz;
    // c = sqrt(gamma (p + p_ref) / rho)
    q[4] += gl * gam / (2.0 * c * X.rho);
    q[0] -= gl * c / (2.0 * X.rho);
  } else if (ph.surf_flux == 2) {
    // forward sweep of the Roe dissipation with Harten's fix (F -= D / 2)
    const double gam = ph.gamma;
    const double sA = ::sqrt(A.rho), sB = ::sqrt(B.rho);
    const double is = 1.0 / (sA + sB);
    const double rt = sA * sB;
    const double Nu = sA * A.u + sB * B.u, Nv = sA * A.v + sB * B.v, Nw = sA * A.w + sB * B.w;
    const double NH = sA * A.h + sB * B.h;
    const double u = Nu * is, v = Nv * is, w = Nw * is, H = NH * is;
    const double q2 = u * u + v * v + w * w;
    const double c2 = (gam - 1.0) * (H - 0.5 * q2);
    const double c = ::sqrt(c2);
    const double un = u * nx + v * ny + w * nz;
    const double dr = B.rho - A.rho, dp = B.p - A.p;
    const double du = B.u - A.u, dv = B.v - A.v, dw = B.w - A.w;
    const double dun = du * nx + dv * ny + dw * nz;
    const double i2c2 = 0.5 / c2;
    const double P1 = dp - rt * c * dun, P5 = dp + rt * c * dun;
    const double a1 = P1 * i2c2, a2 = dr - dp / c2, a5 = P5 * i2c2;
    const double l1o = ::fabs(un - c), l2 = ::fabs(un), l5o = ::fabs(un + c);
    const double del = 0.1 * c;
    const bool h1 = l1o < del, h5 = l5o < del;
    const double l1 = h1 ? (l1o * l1o + del * del) / (2.0 * del) : l1o;
    const double l5 = h5 ? (l5o * l5o + del * del) / (2.0 * del) : l5o;
    const double w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5, ws = l2 * rt;
    const double dut = du - dun * nx, dvt = dv - dun * ny, dwt = dw - dun * nz;
    const double X4 = u * du + v * dv + w * dw - un * dun;
    // backward sweep
    const double g0 = -0.5 * gF[0], g1 = -0.5 * gF[1], g2 = -0.5 * gF[2], g3 = -0.5 * gF[3], g4 = -0.5 * gF[4];
    const double g13 = g1 * nx + g2 * ny + g3 * nz;  // sum_d gD_d n_d
    double gw1 = g0 + g1 * (u - c * nx) + g2 * (v - c * ny) + g3 * (w - c * nz) + g4 * (H - c * un);
    double gw2 = g0 + g1 * u + g2 * v + g3 * w + g4 * (0.5 * q2);
    double gw5 = g0 + g1 * (u + c * nx) + g2 * (v + c * ny) + g3 * (w + c * nz) + g4 * (H + c * un);
    const double gws = g1 * dut + g2 * dvt + g3 * dwt + g4 * X4;
    const double wsum = w1 + w2 + w5;
    double gu = g1 * wsum + g4 * ws * du, gv = g2 * wsum + g4 * ws * dv, gw = g3 * wsum + g4 * ws * dw;
    double gc = g13 * (w5 - w1) + g4 * un * (w5 - w1);
    double gun = g4 * c * (w5 - w1) - g4 * ws * dun;
    double gH = g4 * (w1 + w5);
    double gq2 = g4 * 0.5 * w2;
    double gdu = g1 * ws + g4 * ws * u, gdv = g2 * ws + g4 * ws * v, gdw = g3 * ws + g4 * ws * w;
    double gdun = -ws * g13 - g4 * ws * un;
    // ws = l2 rt; w_k = l_k a_k
    double gl2 = gws * rt + gw2 * a2, grt = gws * l2;
    double gl1 = gw1 * a1, gl5 = gw5 * a5;
    const double ga1 = gw1 * l1, ga2 = gw2 * l2, ga5 = gw5 * l5;
    // Harten: l = (l_o^2 + del^2) / (2 del) below del
    double gdel = 0.0;
    if (h1) { gdel += gl1 * (0.5 - l1o * l1o / (2.0 * del * del)); gl1 *= l1o / del; }
    if (h5) { gdel += gl5 * (0.5 - l5o * l5o / (2.0 * del * del)); gl5 *= l5o / del; }
    gc += 0.1 * gdel;
    // l1 = |un - c|, l2 = |un|, l5 = |un + c|
    const double s1 = sgn1(un - c), s5 = sgn1(un + c);
    gun += gl1 * s1 + gl2 * sgn1(un) + gl5 * s5;
    gc += -gl1 * s1 + gl5 * s5;
    // a1 = P1 i2c2, a5 = P5 i2c2, a2 = dr - dp / c2
    double gdp = (ga1 + ga5) * i2c2 - ga2 / c2;
    const double gdr = ga2;
    const double gP = (ga5 - ga1) * i2c2;  // d/d(rt c dun) of P5 and -P1
    grt += gP * c * dun;
    gc += gP * rt * dun;
    gdun += gP * rt * c;
    const double gi2c2 = ga1 * P1 + ga5 * P5;
    double gc2 = ga2 * dp / (c2 * c2) - gi2c2 * 0.5 / (c2 * c2);
    // dun, un
    gdu += gdun * nx; gdv += gdun * ny; gdw += gdun * nz;
    gu += gun * nx; gv += gun * ny; gw += gun * nz;
    // c = sqrt(c2), c2 = (gamma - 1)(H - q2 / 2), q2 = |u|^2
    gc2 += gc / (2.0 * c);
    gH += gc2 * (gam - 1.0);
    gq2 -= 0.5 * (gam - 1.0) * gc2;
    gu += 2.0 * u * gq2; gv += 2.0 * v * gq2; gw += 2.0 * w * gq2;
    // Roe averages x = N_x is, N_x = sA x_A + sB x_B
    const double gis = gu * Nu + gv * Nv + gw * Nw + gH * NH;
    double gsA = (gu * A.u + gv * A.v + gw * A.w + gH * A.h) * is + grt * sB - gis * is * is;
    double gsB = (gu * B.u + gv * B.v + gw * B.w + gH * B.h) * is + grt * sA - gis * is * is;
    qA[1] += gu * sA * is; qA[2] += gv * sA * is; qA[3] += gw * sA * is; qA[5] += gH * sA * is;
    qB[1] += gu * sB * is; qB[2] += gv * sB * is; qB[3] += gw * sB * is; qB[5] += gH * sB * is;
    // jumps
    qB[0] += gdr; qA[0] -= gdr;
    qB[4] += gdp; qA[4] -= gdp;
    qB[1] += gdu; qA[1] -= gdu;
    qB[2] += gdv; qA[2] -= gdv;
    qB[3] += gdw; qA[3] -= gdw;
    // s = sqrt(rho)
    qA[0] += gsA / (2.0 * sA);
    qB[0] += gsB / (2.0 * sB);
  }
  prim_vjp(UA, ph, qA, gUA);
  prim_vjp(UB, ph, qB, gUB);
}

// ---------------------------------------------------------------------------
// k_adj_face: one thread per node of an interior face, then (partitioned
// meshes) of a halo face.  A halo face's flux enters this rank's bracket on
// its own side only; the cotangents of the remote side's state and outward
// viscous flux go to sendU / sendG [n_halo][5 or 4][n2] (master's face-node
// order) for the peer.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_adj_face(const double* __restrict__ U, const double* __restrict__ lam, const MeshDev<double> m,
           const PhysDev ph, double iw, double* __restrict__ gUf, double* __restrict__ gGf,
           double* __restrict__ sendU, double* __restrict__ sendG) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = tid / n2, ab = tid - f * n2;
  if (f >= m.n_interior + (sendU ? m.n_halo : 0)) return;
  if (f >= m.n_interior) {
    // fc = (local element, local face, halo index, local side is master | 8 o_own)
    const int h = f - m.n_interior, fh = m.F - m.n_halo + h;
    const int4 fc = m.faces[fh];
    const int abl = omap_ab<N>(orient_inv(fc.w >> 3), ab);
    const int eL = chk_idx(fc.x, m.K, m.status);
    const bool master = (fc.w & 1) != 0;
    const size_t S = (size_t)m.K * n3;
    const size_t gL = (size_t)eL * n3 + fnode<N>(fc.y, abl % n, abl / n);
    const double jL = m.invJ[gL];
    const double* rU = m.halo_U + (size_t)h * 5 * n2 + ab;
    double gFs[5], UL[5], UR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      gFs[v] = (master ? -lam[v * S + gL] : lam[v * S + gL]) * jL * iw;
      UL[v] = U[v * S + gL];
      UR[v] = rU[v * n2];
    }
    const size_t FN = (size_t)m.F * n2, fg = (size_t)fh * n2 + ab;
    const double nx = m.fgeo[fg], ny = m.fgeo[FN + fg], nz = m.fgeo[2 * FN + fg], s = m.fgeo[3 * FN + fg];
    if (ph.viscous) {
      // Fs = F* s - (Gf_M - Gf_S) / 2
      double* dL = gGf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        dL[v * n2] = (master ? -0.5 : 0.5) * gFs[v + 1];
        sendG[((size_t)h * 4 + v) * n2 + ab] = (master ? 0.5 : -0.5) * gFs[v + 1];
      }
    }
    double gF[5], gA[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gB[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int v = 0; v < 5; ++v) gF[v] = gFs[v] * s;
    face_flux_vjp(ph, master ? UL : UR, master ? UR : UL, nx, ny, nz, gF, gA, gB);
    double* oL = gUf + ((size_t)eL * 6 + fc.y) * 5 * n2 + abl;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      oL[v * n2] = master ? gA[v] : gB[v];
      sendU[((size_t)h * 5 + v) * n2 + ab] = master ? gB[v] : gA[v];
    }
    return;
  }
  int4 fc = m.faces[f];
  fc.x = chk_idx(fc.x, m.K, m.status);
  fc.z = chk_idx(fc.z, m.K, m.status);
  const size_t S = (size_t)m.K * n3;
  const size_t gM = (size_t)fc.x * n3 + fnode<N>(fc.y, ab % n, ab / n);
  // ab indexes the master's face nodes; abS the slave's (orientation fc.w >> 3)
  const int abS = omap_ab<N>(fc.w >> 3, ab), lS = fc.w & 7;
  const size_t gS = (size_t)fc.z * n3 + fnode<N>(lS, abS % n, abS / n);
  const double jM = m.invJ[gM], jS = m.invJ[gS];
  double gFs[5], UA[5], UB[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    // Fs enters the bracket of the master with +1/w and of the slave with -1/w;
    // the bracket's cotangent is -lam/J
    gFs[v] = (-lam[v * S + gM] * jM + lam[v * S + gS] * jS) * iw;
    UA[v] = U[v * S + gM];
    UB[v] = U[v * S + gS];
  }
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const double nx = m.fgeo[fg], ny = m.fgeo[FN + fg], nz = m.fgeo[2 * FN + fg], s = m.fgeo[3 * FN + fg];
  if (ph.viscous) {
    // Fs = F* s - (Gf_M - Gf_S) / 2
    double* dM = gGf + ((size_t)fc.x * 6 + fc.y) * 4 * n2 + ab;
    double* dS = gGf + ((size_t)fc.z * 6 + lS) * 4 * n2 + abS;
#pragma unroll
    for (int v = 0; v < 4; ++v) { dM[v * n2] = -0.5 * gFs[v + 1]; dS[v * n2] = 0.5 * gFs[v + 1]; }
  }
  double gF[5], gA[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gB[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 5; ++v) gF[v] = gFs[v] * s;
  face_flux_vjp(ph, UA, UB, nx, ny, nz, gF, gA, gB);
  double* oM = gUf + ((size_t)fc.x * 6 + fc.y) * 5 * n2 + ab;
  double* oS = gUf + ((size_t)fc.z * 6 + lS) * 5 * n2 + abS;
#pragma unroll
  for (int v = 0; v < 5; ++v) { oM[v * n2] = gA[v]; oS[v * n2] = gB[v]; }
}

// ---------------------------------------------------------------------------
// k_adj_wall: one thread per node of a wall face.  Also accumulates
// g_theta = sum_nodes (dFs/dtheta)^T gFs.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_adj_wall(const double* __restrict__ U, const double* __restrict__ lam, const MeshDev<double> m,
           const PhysDev ph, double iw, double* __restrict__ gUf, double* __restrict__ gGf,
           double* __restrict__ gUs, double* __restrict__ gtheta, int* __restrict__ status) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int wf = tid / n2, ab = tid - wf * n2;
  double gk = 0.0, gb = 0.0;
  if (wf < m.n_wall) {
    const int f = m.n_interior + wf;
    int4 fc = m.faces[f];
    fc.x = chk_idx(fc.x, m.K, m.status);
    const size_t S = (size_t)m.K * n3;
    const size_t gM = (size_t)fc.x * n3 + fnode<N>(fc.y, ab % n, ab / n);
    const double jM = m.invJ[gM];
    double gFs[5], UA[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      gFs[v] = -lam[v * S + gM] * jM * iw;
      UA[v] = U[v * S + gM];
    }
    const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
    const double nx = m.fgeo[fg], ny = m.fgeo[FN + fg], nz = m.fgeo[2 * FN + fg], s = m.fgeo[3 * FN + fg];
    if (ph.viscous) {
      double* dM = gGf + ((size_t)fc.x * 6 + fc.y) * 4 * n2 + ab;
#pragma unroll
      for (int v = 0; v < 4; ++v) dM[v * n2] = 0.0;
    }
    // inviscid flux through the mirror state U_B = (rho, m - 2 (m.n) n, E):
    // gU = gA + (dU_B/dU)^T gB
    double g[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gB[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gF[5], UB[5];
    {
      const double mn = UA[1] * nx + UA[2] * ny + UA[3] * nz;
      UB[0] = UA[0]; UB[1] = UA[1] - 2.0 * mn * nx; UB[2] = UA[2] - 2.0 * mn * ny; UB[3] = UA[3] - 2.0 * mn * nz;
      UB[4] = UA[4];
#pragma unroll
      for (int v = 0; v < 5; ++v) gF[v] = gFs[v] * s;
      face_flux_vjp(ph, UA, UB, nx, ny, nz, gF, g, gB);
      const double gbn = gB[1] * nx + gB[2] * ny + gB[3] * nz;
      g[0] += gB[0]; g[4] += gB[4];
      g[1] += gB[1] - 2.0 * gbn * nx; g[2] += gB[2] - 2.0 * gbn * ny; g[3] += gB[3] - 2.0 * gbn * nz;
    }
    double* oM = gUf + ((size_t)fc.x * 6 + fc.y) * 5 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) oM[v * n2] = g[v];
    // wall model: Fs_mom += tau s
    const size_t slot = (size_t)wf * n2 + ab;
    if (ph.viscous) {
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
      const double gt0 = gFs[1] * s, gt1 = gFs[2] * s, gt2 = gFs[3] * s, gt4 = -gFs[4] * s;
      bool ok = true;
#pragma unroll 1
      for (int k = 0; k < 7; ++k) {
        DualD Ud[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Ud[v] = DualD(Us[v], k == v ? 1.0 : 0.0);
        DualD tau[3], qwd;
        bool okk;
        wall_stress_jvp(ph, Ud, k == 5 ? 1.0 : 0.0, k == 6 ? 1.0 : 0.0, nx, ny, nz, tau, &okk, &qwd);
        ok = ok && okk;
        // (the wall flux: Fs_mom += tau s, Fs_E -= q_w s)
        const double gdot = tau[0].d * gt0 + tau[1].d * gt1 + tau[2].d * gt2 + qwd.d * gt4;
        if (k < 5) gUs[slot * 5 + k] = gdot;
        else if (k == 5) gk = gdot;
        else gb = gdot;
      }
      if (!ok) atomicOr(status, ST_WM_NOCONV);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) gUs[slot * 5 + v] = 0.0;
    }
  }
  // block reduction of the two parameter cotangents
  if (gtheta) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gk += __shfl_down_sync(0xffffffffu, gk, o);
      gb += __shfl_down_sync(0xffffffffu, gb, o);
    }
    if ((threadIdx.x & 31) == 0 && (gk != 0.0 || gb != 0.0)) {
      atomicAdd(&gtheta[0], gk);
      atomicAdd(&gtheta[1], gb);
    }
  }
}

// ---------------------------------------------------------------------------
// k_adj_bc: one thread per node of an inflow or outflow face.  The forward
// flux Fs = F*(U, U_B(U)) s - (0, Gf) with the exterior state U_B: the
// prescribed inflow state (a constant), or at an outflow the interior
// density and momentum with the energy of the prescribed pressure,
// E_B = p_out / (gamma - 1) + |m|^2 / (2 rho).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_adj_bc(const double* __restrict__ U, const double* __restrict__ lam, const MeshDev<double> m, const PhysDev ph,
         double iw, double* __restrict__ gUf, double* __restrict__ gGf) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int bf = tid / n2, ab = tid - bf * n2;
  if (bf >= m.n_bc) return;
  const int f = m.n_interior + m.n_wall + bf;
  int4 fc = m.faces[f];
  fc.x = chk_idx(fc.x, m.K, m.status);
  const size_t S = (size_t)m.K * n3;
  const size_t gM = (size_t)fc.x * n3 + fnode<N>(fc.y, ab % n, ab / n);
  const double jM = m.invJ[gM];
  double gFs[5], UA[5], UB[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    gFs[v] = -lam[v * S + gM] * jM * iw;
    UA[v] = U[v * S + gM];
  }
  ghost_state(ph, fc.z, UA, UB);
  const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
  const double nx = m.fgeo[fg], ny = m.fgeo[FN + fg], nz = m.fgeo[2 * FN + fg], s = m.fgeo[3 * FN + fg];
  if (ph.viscous) {
    double* dM = gGf + ((size_t)fc.x * 6 + fc.y) * 4 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 4; ++v) dM[v * n2] = -gFs[v + 1];
  }
  double gF[5], g[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, gB[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 5; ++v) gF[v] = gFs[v] * s;
  face_flux_vjp(ph, UA, UB, nx, ny, nz, gF, g, gB);
  if (fc.z == -3) {
    // dE_B/drho = -|m|^2 / (2 rho^2), dE_B/dm = m / rho
    const double ir = 1.0 / UA[0];
    const double m2 = UA[1] * UA[1] + UA[2] * UA[2] + UA[3] * UA[3];
    g[0] += gB[0] - 0.5 * m2 * ir * ir * gB[4];
#pragma unroll
    for (int v = 1; v < 4; ++v) g[v] += gB[v] + UA[v] * ir * gB[4];
  }
  double* oM = gUf + ((size_t)fc.x * 6 + fc.y) * 5 * n2 + ab;
#pragma unroll
  for (int v = 0; v < 5; ++v) oM[v * n2] = g[v];
}

// ---------------------------------------------------------------------------
// k_adj_halo_in: the peers' cotangents of this rank's outward viscous fluxes
// at the halo faces (recvG, master's face-node order) into gGf.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_adj_halo_in(const MeshDev<double> m, const double* __restrict__ recvG, double* __restrict__ gGf) {
  constexpr int n = N + 1, n2 = n * n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = tid / n2, ab = tid - h * n2;
  if (h >= m.n_halo) return;
  const int4 fc = m.faces[m.F - m.n_halo + h];
  const int abl = omap_ab<N>(orient_inv(fc.w >> 3), ab);
  const int eL = chk_idx(fc.x, m.K, m.status);
  double* dL = gGf + ((size_t)eL * 6 + fc.y) * 4 * n2 + abl;
#pragma unroll
  for (int v = 0; v < 4; ++v) dL[v * n2] += recvG[((size_t)h * 4 + v) * n2 + ab];
}

// ---------------------------------------------------------------------------
// k_adj_element: one CTA per element.  Writes the element's own part of gU
// and, for every interior face, the lifting cotangent of the neighbour's
// face nodes (gWf[e][l]: for the node across face l).
// ---------------------------------------------------------------------------
template <int N>
struct AdjShape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int THREADS = VolShape<N>::THREADS;
  // doubles per node: Q 6 (reused with 6 more for H 12 after the pair
  // phase), lam~ 5, Ja 9, W 4, gQ 6; 24 n2 face corrections; D, DVS, Dvisc
  // tables, 1/w
  static constexpr int SMEM_D = 36 * n3 + 24 * n2 + 3 * n2 + n;
};

// EC: the entropy-conserving volume flux; SUTH: Sutherland's law (own
// instantiations: the reverse mode of the entropy-conserving pair flux and
// the temperature-dependent viscosity need registers that the Pirozzoli,
// constant-viscosity kernel would otherwise spill)
template <int N, bool EC, bool SUTH>
__global__ void __launch_bounds__(AdjShape<N>::THREADS)
k_adj_element(const double* __restrict__ U, const double* __restrict__ lam, const MeshDev<double> m,
              const PhysDev ph, const Tables<N> tab, const double* __restrict__ gGf, double* __restrict__ gU,
              double* __restrict__ gWf, double* __restrict__ gHaloU) {
  using Sh = AdjShape<N>;
  constexpr int n = Sh::n, n2 = Sh::n2, n3 = Sh::n3, T = Sh::THREADS, LPW = VolShape<N>::LPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sQ = reinterpret_cast<double*>(smem_raw);  // [6][n3] (pair phase)
  double* sH = sQ;                                     // [3][4][n3] (viscous phase, reuses Q)
  double* sL = sQ + 12 * n3;                           // [5][n3] lam~ = -lam / J
  double* sA = sL + 5 * n3;                            // [9][n3]
  double* sW = sA + 9 * n3;                            // [4][n3] u v w T
  double* sGQ = sW + 4 * n3;                           // [6][n3]
  double* sC = sGQ + 6 * n3;                           // [6][4][n2]
  double* sD = sC + 24 * n2;                           // [n2]
  double* sDVS = sD + n2;                              // [n2] w_a DVS_ab
  double* sDv = sDVS + n2;                             // [n2]
  double* siw = sDv + n2;                              // [n]
  const int e = blockIdx.x, t = threadIdx.x;
  const size_t S = (size_t)m.K * n3;
  // N = 7: the viscous part's line contractions in even/odd form (as in the
  // lifting kernel): sD holds the tables of D and of D^T, sDv that of Dvisc^T
  constexpr bool EO = (n == 8) && (T == n3);
  for (int x = t; x < n2; x += T) {
    sDVS[x] = 8.0 * tab.DVS8[x] / tab.iw[x / n];
    if constexpr (EO) {
      if (x < n * (n / 2)) {
        sD[x] = LineEO<N>::coef(tab.D, x);
        sD[n * (n / 2) + x] = LineEO<N>::coef_t(tab.D, x);
        sDv[x] = LineEO<N>::coef_t(tab.Dvisc, x);
      }
    } else {
      sD[x] = tab.D[x];
      sDv[x] = tab.Dvisc[x];
    }
  }
  if (t < n) siw[t] = tab.iw[t];
  if (t < n3) {
    const size_t g = (size_t)e * n3 + t;
    double Uo[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Uo[v] = U[v * S + g];
    const Prim<double> q = primitive<double>(Uo[0], Uo[1], Uo[2], Uo[3], Uo[4], ph);
    sQ[t] = q.rho; sQ[n3 + t] = q.u; sQ[2 * n3 + t] = q.v; sQ[3 * n3 + t] = q.w;
    sQ[4 * n3 + t] = q.p; sQ[5 * n3 + t] = q.h;
    const double iJ = m.invJ[g];
#pragma unroll
    for (int v = 0; v < 5; ++v) sL[v * n3 + t] = -lam[v * S + g] * iJ;
#pragma unroll
    for (int c = 0; c < 9; ++c) sA[c * n3 + t] = m.Ja[(size_t)c * S + g];
    double uu, vv, ww, TT;
    velocity_temperature<double>(Uo[0], Uo[1], Uo[2], Uo[3], Uo[4], ph, uu, vv, ww, TT);
    sW[t] = uu; sW[n3 + t] = vv; sW[2 * n3 + t] = ww; sW[3 * n3 + t] = TT;
  }
  __syncthreads();
  // ---- transposed split-form volume integral (symmetric pairs)
  {
    const int warp = t >> 5, lane = t & 31;
    const int seg = lane / n, pos = lane - seg * n;
    const int L0 = warp * LPW + seg;
    const bool active = (seg < LPW) && (L0 < n2);
    const int L = active ? L0 : 0;
    const int base = seg * n;
    // The pair terms are linear in the combined cotangent
    //   mu = DVS_im lam~_i + DVS_mi lam~_m = w_i DVS_im (lam~_i / w_i - lam~_m / w_m)
    // (w_i DVS_im = -w_m DVS_mi off the diagonal, the SBP property), so each
    // pass first stores lam~ / w along its direction and a pair forms the
    // difference; the factor w_i DVS_im (table sDVS) scales its terms as they
    // are summed, for the partner lane's pair w_m DVS_mi.
    double* sLt = sQ + 6 * n3;  // [5][n3] lam~ / w (the unused half of the Q slots)
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      const int a = L % n, b = L / n;
      auto node = [&](int q) {
        return dir == 0 ? q + n * L : (dir == 1 ? a + n * q + n2 * b : L + n2 * q);
      };
      const int me = node(pos);
      if (active) {
        const double iwp = siw[pos];
#pragma unroll
        for (int v = 0; v < 5; ++v) sLt[v * n3 + me] = sL[v * n3 + me] * iwp;
      }
      __syncthreads();
      // the pair terms below carry constant factors (1/8 for rho, u, v, w,
      // 1/4 for p, 1/16 for h) that are applied once per node after the sums
      double g0 = 0, g1 = 0, g2 = 0, g3 = 0, g4 = 0, g5 = 0;
      if constexpr (EC) {
        // entropy-conserving flux: the two nodes of a pair get different
        // cotangents (the logarithmic means are symmetric, their partial
        // derivatives are not); the lane keeps its node's share and hands the
        // partner's share (pos + d) over by a shuffle
#pragma unroll 1
        for (int d = 1; d <= n / 2; ++d) {
          const int pm = pos + d < n ? pos + d : pos + d - n;
          const int q = node(pm);
          const Prim<double> Pa{sQ[me], sQ[n3 + me], sQ[2 * n3 + me], sQ[3 * n3 + me], sQ[4 * n3 + me], 0.0};
          const Prim<double> Pb{sQ[q], sQ[n3 + q], sQ[2 * n3 + q], sQ[3 * n3 + q], sQ[4 * n3 + q], 0.0};
          const double a0 = 0.5 * (sA[(dir * 3 + 0) * n3 + me] + sA[(dir * 3 + 0) * n3 + q]);
          const double a1 = 0.5 * (sA[(dir * 3 + 1) * n3 + me] + sA[(dir * 3 + 1) * n3 + q]);
          const double a2 = 0.5 * (sA[(dir * 3 + 2) * n3 + me] + sA[(dir * 3 + 2) * n3 + q]);
          double mu[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) mu[v] = sLt[v * n3 + me] - sLt[v * n3 + q];
          double gA[5] = {0, 0, 0, 0, 0}, gB[5] = {0, 0, 0, 0, 0};
          ec_flux_vjp(ph, Pa, Pb, a0, a1, a2, mu, gA, gB);
          const double cw = sDVS[pos * n + pm];
          g0 = fma(cw, gA[0], g0); g1 = fma(cw, gA[1], g1); g2 = fma(cw, gA[2], g2);
          g3 = fma(cw, gA[3], g3); g4 = fma(cw, gA[4], g4);
          if (2 * d != n) {
            const int src = base + (pos - d >= 0 ? pos - d : pos - d + n);
            const double cs = sDVS[(src - base) * n + pos];
            g0 = fma(cs, __shfl_sync(0xffffffffu, gB[0], src), g0);
            g1 = fma(cs, __shfl_sync(0xffffffffu, gB[1], src), g1);
            g2 = fma(cs, __shfl_sync(0xffffffffu, gB[2], src), g2);
            g3 = fma(cs, __shfl_sync(0xffffffffu, gB[3], src), g3);
            g4 = fma(cs, __shfl_sync(0xffffffffu, gB[4], src), g4);
          }
        }
      } else {
#pragma unroll
      for (int d = 1; d <= n / 2; ++d) {
        const int pm = pos + d < n ? pos + d : pos + d - n;
        const int q = node(pm);
        // sums of the two nodes' values: {x} = Sx / 2
        const double Sr = sQ[me] + sQ[q];
        const double Su = sQ[n3 + me] + sQ[n3 + q], Sv = sQ[2 * n3 + me] + sQ[2 * n3 + q],
                     Sw = sQ[3 * n3 + me] + sQ[3 * n3 + q];
        const double Sh = sQ[5 * n3 + me] + sQ[5 * n3 + q];
        const double Sa0 = sA[(dir * 3 + 0) * n3 + me] + sA[(dir * 3 + 0) * n3 + q];
        const double Sa1 = sA[(dir * 3 + 1) * n3 + me] + sA[(dir * 3 + 1) * n3 + q];
        const double Sa2 = sA[(dir * 3 + 2) * n3 + me] + sA[(dir * 3 + 2) * n3 + q];
        double mu[5];  // mu / (w_i DVS_im)
#pragma unroll
        for (int v = 0; v < 5; ++v) mu[v] = sLt[v * n3 + me] - sLt[v * n3 + q];
        // F0 = {rho} qa, Fk = {rho} qa {u_k} + {p} {a_k}, F4 = {rho} qa {h}, qa = {u}.{a} = Q / 4;
        // tt = mu . dF/d({rho} qa) = mu0 + (mu1 Su + mu2 Sv + mu3 Sw + mu4 Sh) / 2;
        // half of each average's cotangent goes to each node:
        //   g_rho = Q tt / 8, g_u_k = Sr (tt Sa_k + Q mu_k / 2) / 8, g_p = (mu . Sa) / 4,
        //   g_h = Sr Q mu4 / 16
        const double Q = Su * Sa0 + Sv * Sa1 + Sw * Sa2;
        const double tt = fma(0.5, mu[1] * Su + mu[2] * Sv + mu[3] * Sw + mu[4] * Sh, mu[0]);
        const double hQ = 0.5 * Q;
        const double h0 = Q * tt;
        const double h1 = Sr * fma(tt, Sa0, hQ * mu[1]);
        const double h2 = Sr * fma(tt, Sa1, hQ * mu[2]);
        const double h3 = Sr * fma(tt, Sa2, hQ * mu[3]);
        const double h4 = mu[1] * Sa0 + mu[2] * Sa1 + mu[3] * Sa2;
        const double h5 = Sr * Q * mu[4];
        const double cw = sDVS[pos * n + pm];
        g0 = fma(cw, h0, g0); g1 = fma(cw, h1, g1); g2 = fma(cw, h2, g2);
        g3 = fma(cw, h3, g3); g4 = fma(cw, h4, g4); g5 = fma(cw, h5, g5);
        if (2 * d != n) {
          const int src = base + (pos - d >= 0 ? pos - d : pos - d + n);
          const double cs = sDVS[(src - base) * n + pos];
          g0 = fma(cs, __shfl_sync(0xffffffffu, h0, src), g0);
          g1 = fma(cs, __shfl_sync(0xffffffffu, h1, src), g1);
          g2 = fma(cs, __shfl_sync(0xffffffffu, h2, src), g2);
          g3 = fma(cs, __shfl_sync(0xffffffffu, h3, src), g3);
          g4 = fma(cs, __shfl_sync(0xffffffffu, h4, src), g4);
          g5 = fma(cs, __shfl_sync(0xffffffffu, h5, src), g5);
        }
      }
      g0 *= 0.125; g1 *= 0.125; g2 *= 0.125; g3 *= 0.125; g4 *= 0.25; g5 *= 0.0625;
      }  // Pirozzoli
      if (active) {
        if (dir == 0) {
          sGQ[me] = g0; sGQ[n3 + me] = g1; sGQ[2 * n3 + me] = g2; sGQ[3 * n3 + me] = g3;
          sGQ[4 * n3 + me] = g4; sGQ[5 * n3 + me] = g5;
        } else {
          sGQ[me] += g0; sGQ[n3 + me] += g1; sGQ[2 * n3 + me] += g2; sGQ[3 * n3 + me] += g3;
          sGQ[4 * n3 + me] += g4; sGQ[5 * n3 + me] += g5;
        }
      }
      __syncthreads();
    }
  }
  // ---- viscous part: recompute the lifted gradients, then transpose
  // this thread's node from here on (N = 7: warp a + 4 b holds the xi lines at
  // eta in {a, N - a} and zeta in {b, N - b}, so that a node's mirror nodes
  // along xi, eta, zeta are lanes ^ 7, ^ 8, ^ 16 of its own warp)
  int i, j, k;
  if constexpr (EO) {
    const int lane = t & 31, w = t >> 5, a = w & 3, b = w >> 2;
    i = lane & 7;
    j = (lane & 8) ? N - a : a;
    k = (lane & 16) ? N - b : b;
  } else {
    i = t % n; j = (t / n) % n; k = t / n2;
  }
  const int p = i + n * (j + n * k);
  double* sX = sQ;  // [3][4][n3] even/odd half sums (the Q slots, free after the pair phase)
  double gWo[4] = {0, 0, 0, 0};
  double gText = 0.0;  // cotangent of the outflow exterior temperature p_out / (rho R)
  if (ph.viscous) {
    // W* - W at the faces (as in the forward lifting)
    for (int x = t; x < 6 * n2; x += T) {
      const int l = x / n2, ab = x - l * n2, a = ab % n, b = ab / n;
      const int q = fnode<N>(l, a, b);
      const int nb = m.nbr[e * 6 + l];
      double d[4];
      if (nb >= 0) {
        const NbrNode<N> nn = neighbour_node<N>(m, e, l, ab);
        const size_t gn = (size_t)nn.e * n3 + fnode<N>(nn.l, nn.ab % n, nn.ab / n);
        double un, vn, wn, Tn;
        velocity_temperature<double>(U[gn], U[S + gn], U[2 * S + gn], U[3 * S + gn], U[4 * S + gn], ph, un, vn,
                                     wn, Tn);
        d[0] = 0.5 * (un - sW[q]); d[1] = 0.5 * (vn - sW[n3 + q]); d[2] = 0.5 * (wn - sW[2 * n3 + q]);
        d[3] = 0.5 * (Tn - sW[3 * n3 + q]);
      } else if (nb <= -16) {
        // halo face: the remote element's trace (master's face-node order)
        const int abm = omap_ab<N>((m.elem_face[e * 6 + l] >> 1) & 7, ab);
        const double* src = m.halo_U + (size_t)chk_idx(-16 - nb, m.n_halo, m.status) * 5 * n2 + abm;
        double un, vn, wn, Tn;
        velocity_temperature<double>(src[0], src[n2], src[2 * n2], src[3 * n2], src[4 * n2], ph, un, vn, wn, Tn);
        d[0] = 0.5 * (un - sW[q]); d[1] = 0.5 * (vn - sW[n3 + q]); d[2] = 0.5 * (wn - sW[2 * n3 + q]);
        d[3] = 0.5 * (Tn - sW[3 * n3 + q]);
      } else if (nb == -2 || nb == -3) {
        // inflow / outflow: W* - W = (W(exterior) - W) / 2
        const size_t gq = (size_t)e * n3 + q;
        double Ui[5], Ub[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Ui[v] = U[v * S + gq];
        ghost_state(ph, nb, Ui, Ub);
        double ub, vb, wb, Tb;
        velocity_temperature<double>(Ub[0], Ub[1], Ub[2], Ub[3], Ub[4], ph, ub, vb, wb, Tb);
        d[0] = 0.5 * (ub - sW[q]); d[1] = 0.5 * (vb - sW[n3 + q]); d[2] = 0.5 * (wb - sW[2 * n3 + q]);
        d[3] = 0.5 * (Tb - sW[3 * n3 + q]);
      } else {
        const int dir = l >> 1;
        const double a0 = sA[(dir * 3 + 0) * n3 + q], a1 = sA[(dir * 3 + 1) * n3 + q], a2 = sA[(dir * 3 + 2) * n3 + q];
        const double is = 1.0 / ::sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        const double nx = a0 * is, ny = a1 * is, nz = a2 * is;
        const double un = sW[q] * nx + sW[n3 + q] * ny + sW[2 * n3 + q] * nz;
        d[0] = -un * nx; d[1] = -un * ny; d[2] = -un * nz; d[3] = 0.0;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) sC[(l * 4 + v) * n2 + ab] = d[v];
    }
    __syncthreads();
    double H[3][4];
    if (t < n3) {
      const size_t g = (size_t)e * n3 + p;
      const int qd[3] = {i, j, k};
      double ja[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) ja[c] = sA[c * n3 + p];
      // forward gradients q[d][v]: reference-space derivatives, the BR1
      // surface corrections on them, then the metric transform (with the
      // stored Ja / J, which also maps gq back to the reference space below)
      double dW[3][4];
      if constexpr (EO) {
#pragma unroll
        for (int dir = 0; dir < 3; ++dir)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            sX[(dir * 4 + v) * n3 + p] =
                LineEO<N>::half(qd[dir], sW[v * n3 + p], sW[v * n3 + LineEO<N>::at(p, dir, qd[dir], N - qd[dir])]);
        __syncthreads();
#pragma unroll
        for (int dir = 0; dir < 3; ++dir)
#pragma unroll
          for (int v = 0; v < 4; ++v) dW[dir][v] = LineEO<N>::apply(sD, sX + (dir * 4 + v) * n3, p, dir, qd[dir]);
        __syncthreads();
        // the half sums of lam~ for the transposed weak divergence below
#pragma unroll
        for (int dir = 0; dir < 3; ++dir)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            sX[(dir * 4 + v) * n3 + p] = LineEO<N>::half(
                qd[dir], sL[(v + 1) * n3 + p], sL[(v + 1) * n3 + LineEO<N>::at(p, dir, qd[dir], N - qd[dir])]);
        __syncthreads();
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
          for (int mm = 0; mm < n; ++mm) {
            s0 += sD[i * n + mm] * sW[v * n3 + mm + n * (j + n * k)];
            s1 += sD[j * n + mm] * sW[v * n3 + i + n * (mm + n * k)];
            s2 += sD[k * n + mm] * sW[v * n3 + i + n * (j + n * mm)];
          }
          dW[0][v] = s0; dW[1][v] = s1; dW[2][v] = s2;
        }
      }
      auto surf = [&](int dir, int l, int ab, double sgn_iw) {
#pragma unroll
        for (int v = 0; v < 4; ++v) dW[dir][v] += sgn_iw * sC[(l * 4 + v) * n2 + ab];
      };
      if (i == 0 || i == N) surf(0, i == 0 ? 0 : 1, j + n * k, i == 0 ? -siw[0] : siw[N]);
      if (j == 0 || j == N) surf(1, j == 0 ? 2 : 3, i + n * k, j == 0 ? -siw[0] : siw[N]);
      if (k == 0 || k == N) surf(2, k == 0 ? 4 : 5, i + n * j, k == 0 ? -siw[0] : siw[N]);
      double jj[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) jj[c] = m.JaJ[(size_t)c * S + g];
      double q[3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          q[d][v] = jj[0 * 3 + d] * dW[0][v] + jj[1 * 3 + d] * dW[1][v] + jj[2 * 3 + d] * dW[2][v];
      // cotangent of the contravariant viscous flux G^dir at this node:
      // from R_v = sum_i Dvisc_i,m G_m (transposed) and from the face fluxes
      double gG[3][4];
      if constexpr (EO) {
#pragma unroll
        for (int dir = 0; dir < 3; ++dir)
#pragma unroll
          for (int v = 0; v < 4; ++v) gG[dir][v] = LineEO<N>::apply(sDv, sX + (dir * 4 + v) * n3, p, dir, qd[dir]);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
          for (int ii = 0; ii < n; ++ii) {
            s0 += sDv[ii * n + i] * sL[(v + 1) * n3 + ii + n * (j + n * k)];
            s1 += sDv[ii * n + j] * sL[(v + 1) * n3 + i + n * (ii + n * k)];
            s2 += sDv[ii * n + k] * sL[(v + 1) * n3 + i + n * (j + n * ii)];
          }
          gG[0][v] = s0; gG[1][v] = s1; gG[2][v] = s2;
        }
      }
      auto gface = [&](int l, int ab, double sgn) {
        const double* src = gGf + ((size_t)e * 6 + l) * 4 * n2 + ab;
#pragma unroll
        for (int v = 0; v < 4; ++v) gG[l >> 1][v] += sgn * src[v * n2];
      };
      if (i == 0) gface(0, j + n * k, -1.0);
      if (i == N) gface(1, j + n * k, 1.0);
      if (j == 0) gface(2, i + n * k, -1.0);
      if (j == N) gface(3, i + n * k, 1.0);
      if (k == 0) gface(4, i + n * j, -1.0);
      if (k == N) gface(5, i + n * j, 1.0);
      // G^dir = sum_d Ja^dir_d Fv_d  ->  gFv_d = sum_dir Ja^dir_d gG^dir
      double gF[3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 4; ++v) gF[d][v] = ja[0 * 3 + d] * gG[0][v] + ja[1 * 3 + d] * gG[1][v] + ja[2 * 3 + d] * gG[2][v];
      // viscous flux Fv_d = (tau_0d, tau_1d, tau_2d, tau_jd u_j + k q[d][T]);
      // with Sutherland's law mu(T) and k = mu(T) cp / Pr (Sec. 4), whose
      // derivatives dmu/dT = mu (3 / (2T) - 1 / (T + S)) give T a cotangent too
      double mu = ph.mu, kc = ph.kcond, dmu = 0.0;
      if constexpr (SUTH) {
        const double Tn = sW[3 * n3 + p];
        mu = sutherland<double>(ph, Tn);
        dmu = mu * (1.5 / Tn - 1.0 / (Tn + ph.suth_S));
        kc = mu * ph.cp_Pr;
      }
      const double div = q[0][0] + q[1][1] + q[2][2];
      double tau[3][3];
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) tau[aa][bb] = mu * (q[bb][aa] + q[aa][bb]) - (aa == bb ? 2.0 / 3.0 * mu * div : 0.0);
      const double uvw[3] = {sW[p], sW[n3 + p], sW[2 * n3 + p]};
      double gq[3][4] = {{0}};
      double gtau[3][3];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj)
#pragma unroll
        for (int d = 0; d < 3; ++d) gtau[jj][d] = gF[d][jj] + gF[d][3] * uvw[jj];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) gWo[jj] += tau[jj][0] * gF[0][3] + tau[jj][1] * gF[1][3] + tau[jj][2] * gF[2][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) gq[d][3] += kc * gF[d][3];
      double gdiv = 0.0;
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          gq[bb][aa] += mu * gtau[aa][bb];
          gq[aa][bb] += mu * gtau[aa][bb];
        }
        gdiv -= 2.0 / 3.0 * mu * gtau[aa][aa];
      }
      gq[0][0] += gdiv; gq[1][1] += gdiv; gq[2][2] += gdiv;
      if constexpr (SUTH) {
        // tau = mu(T) S(q), heat flux k(T) q_T: T's cotangent
        double gT = 0.0;
#pragma unroll
        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
          for (int bb = 0; bb < 3; ++bb) gT += gtau[aa][bb] * tau[aa][bb];
        gT *= dmu / mu;
#pragma unroll
        for (int d = 0; d < 3; ++d) gT += dmu * ph.cp_Pr * gF[d][3] * q[d][3];
        gWo[3] += gT;
      }
      // lifting transposed: q = (1/J)(sum_dir Ja^dir dW_dir + surface), so the
      // cotangent of the reference-space gradient is H^dir = (Ja^dir / J) . gq
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          H[dir][v] = jj[dir * 3 + 0] * gq[0][v] + jj[dir * 3 + 1] * gq[1][v] + jj[dir * 3 + 2] * gq[2][v];
          if constexpr (!EO) sH[(dir * 4 + v) * n3 + p] = H[dir][v];
        }
      // surface terms: dW_dir += (W* - W) (+-1 / w) at the line ends
      auto surf_t = [&](int l, int ab, double sgn_iw) {
        const int dir = l >> 1;
        double tv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) tv[v] = sgn_iw * H[dir][v];
        const int nb = m.nbr[e * 6 + l];
        if (nb >= 0) {
          // W* - W = (W_nbr - W) / 2
#pragma unroll
          for (int v = 0; v < 4; ++v) gWo[v] -= 0.5 * tv[v];
          double* dst = gWf + ((size_t)e * 6 + l) * 4 * n2 + ab;
#pragma unroll
          for (int v = 0; v < 4; ++v) dst[v * n2] = 0.5 * tv[v];
        } else if (nb <= -16) {
          // halo face: the remote node's share, through its W(U), to the peer
          // (gHaloU holds the face kernel's share already)
#pragma unroll
          for (int v = 0; v < 4; ++v) gWo[v] -= 0.5 * tv[v];
          const int abm = omap_ab<N>((m.elem_face[e * 6 + l] >> 1) & 7, ab);
          const size_t hb = (size_t)chk_idx(-16 - nb, m.n_halo, m.status) * 5 * n2 + abm;
          double Ur[5], gr[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          const double gWr[4] = {0.5 * tv[0], 0.5 * tv[1], 0.5 * tv[2], 0.5 * tv[3]};
#pragma unroll
          for (int v = 0; v < 5; ++v) Ur[v] = m.halo_U[hb + v * n2];
          vt_vjp(Ur, ph, gWr, gr);
#pragma unroll
          for (int v = 0; v < 5; ++v) gHaloU[hb + v * n2] += gr[v];
        } else if (nb == -2) {
          // inflow: the exterior state is the prescribed one
#pragma unroll
          for (int v = 0; v < 4; ++v) gWo[v] -= 0.5 * tv[v];
        } else if (nb == -3) {
          // outflow: the exterior velocity is the interior one (W* - W = 0),
          // the exterior temperature p_out / (rho R)
          gWo[3] -= 0.5 * tv[3];
          gText += 0.5 * tv[3];
        } else {
          // W* - W = -(u . n) n (mirror), T unchanged
          const double a0 = ja[dir * 3 + 0], a1 = ja[dir * 3 + 1], a2 = ja[dir * 3 + 2];
          const double is = 1.0 / ::sqrt(a0 * a0 + a1 * a1 + a2 * a2);
          const double nx = a0 * is, ny = a1 * is, nz = a2 * is;
          const double tn = tv[0] * nx + tv[1] * ny + tv[2] * nz;
          gWo[0] -= tn * nx; gWo[1] -= tn * ny; gWo[2] -= tn * nz;
        }
      };
      if (i == 0 || i == N) surf_t(i == 0 ? 0 : 1, j + n * k, i == 0 ? -siw[0] : siw[N]);
      if (j == 0 || j == N) surf_t(j == 0 ? 2 : 3, i + n * k, j == 0 ? -siw[0] : siw[N]);
      if (k == 0 || k == N) surf_t(k == 0 ? 4 : 5, i + n * j, k == 0 ? -siw[0] : siw[N]);
    }
    __syncthreads();
    if constexpr (EO) {  // (every thread holds a node: T == n3)
      // gW_m += sum_dir sum_i D_{i, m} H^dir_i along the lines through m (D^T
      // in even/odd form; the half sums from this node's H and its mirror's)
      const int qd[3] = {i, j, k};
#pragma unroll
      for (int dir = 0; dir < 3; ++dir)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          sX[(dir * 4 + v) * n3 + p] = LineEO<N>::half(qd[dir], H[dir][v], LineEO<N>::mirror(H[dir][v], dir));
      __syncthreads();
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double s = 0;
#pragma unroll
        for (int dir = 0; dir < 3; ++dir)
          s += LineEO<N>::apply(sD + n * (n / 2), sX + (dir * 4 + v) * n3, p, dir, qd[dir]);
        gWo[v] += s;
      }
    } else if (t < n3) {
      // gW_m += sum_dir sum_i D_{i, m} H^dir_i along the lines through m
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double s = 0;
#pragma unroll
        for (int ii = 0; ii < n; ++ii) {
          s += sD[ii * n + i] * sH[(0 * 4 + v) * n3 + ii + n * (j + n * k)];
          s += sD[ii * n + j] * sH[(1 * 4 + v) * n3 + i + n * (ii + n * k)];
          s += sD[ii * n + k] * sH[(2 * 4 + v) * n3 + i + n * (j + n * ii)];
        }
        gWo[v] += s;
      }
    }
  }
  if (t >= n3) return;
  // ---- own part of gU: primitives, lifting variables and the source term
  const size_t g = (size_t)e * n3 + p;
  double Uo[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Uo[v] = U[v * S + g];
  double gQ[6];
#pragma unroll
  for (int v = 0; v < 6; ++v) gQ[v] = sGQ[v * n3 + p];
  double out[5] = {0, 0, 0, 0, 0};
  prim_vjp(Uo, ph, gQ, out);
  if (ph.viscous) vt_vjp(Uo, ph, gWo, out);
  if (gText != 0.0) out[0] -= gText * ph.p_out * ph.rcp_R / (Uo[0] * Uo[0]);
  if (ph.f[0] != 0.0 || ph.f[1] != 0.0 || ph.f[2] != 0.0) {
    // S_E = f . m / rho
    const double l4 = lam[4 * S + g], ir = 1.0 / Uo[0];
    out[0] -= l4 * (ph.f[0] * Uo[1] + ph.f[1] * Uo[2] + ph.f[2] * Uo[3]) * ir * ir;
    out[1] += l4 * ph.f[0] * ir; out[2] += l4 * ph.f[1] * ir; out[3] += l4 * ph.f[2] * ir;
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) gU[v * S + g] = out[v];
}

// ---------------------------------------------------------------------------
// k_adj_gather: one thread per node; adds the face kernels' state cotangents
// and the neighbours' lifting cotangents (through W(U) of this node).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(256)
k_adj_gather(const double* __restrict__ U, const MeshDev<double> m, const PhysDev ph,
             const double* __restrict__ gUf, const double* __restrict__ gWf, const double* __restrict__ recvGU,
             double* __restrict__ gU) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const size_t S = (size_t)m.K * n3;
  const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= S) return;
  const int e = (int)(g / n3), t = (int)(g - (size_t)e * n3);
  const int i = t % n, j = (t / n) % n, k = t / n2;
  double add[5] = {0, 0, 0, 0, 0}, gW[4] = {0, 0, 0, 0};
  bool any_w = false;
  auto face = [&](int l, int ab) {
    const double* src = gUf + ((size_t)e * 6 + l) * 5 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) add[v] += src[v * n2];
    const int nb = m.nbr[e * 6 + l];
    if (ph.viscous && nb >= 0) {
      const NbrNode<N> nn = neighbour_node<N>(m, e, l, ab);
      const double* w = gWf + ((size_t)nn.e * 6 + nn.l) * 4 * n2 + nn.ab;
#pragma unroll
      for (int v = 0; v < 4; ++v) gW[v] += w[v * n2];
      any_w = true;
    } else if (recvGU && nb <= -16) {
      // a halo face: the peer's cotangent of this node's state (its face
      // flux and its lifting, master's face-node order)
      const int abm = omap_ab<N>((m.elem_face[e * 6 + l] >> 1) & 7, ab);
      const double* r = recvGU + (size_t)chk_idx(-16 - nb, m.n_halo, m.status) * 5 * n2 + abm;
#pragma unroll
      for (int v = 0; v < 5; ++v) add[v] += r[v * n2];
    }
  };
  if (i == 0) face(0, j + n * k);
  if (i == N) face(1, j + n * k);
  if (j == 0) face(2, i + n * k);
  if (j == N) face(3, i + n * k);
  if (k == 0) face(4, i + n * j);
  if (k == N) face(5, i + n * j);
  if (any_w) {
    double Uo[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Uo[v] = U[v * S + g];
    vt_vjp(Uo, ph, gW, add);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) gU[v * S + g] += add[v];
}

// ---------------------------------------------------------------------------
// k_adj_scatter: wall-model sample cotangents to the sample element's nodes.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_adj_scatter(const MeshDev<double> m, const double* __restrict__ gUs, double* __restrict__ gU) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= m.n_wall * n2) return;
  const size_t S = (size_t)m.K * n3;
  const int es = chk_idx(m.ws_elem[slot], m.K, m.status);
  const double* L = m.ws_lag + (size_t)slot * 3 * n;
  double gs[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) gs[v] = gUs[(size_t)slot * 5 + v];
  if (gs[0] == 0.0 && gs[1] == 0.0 && gs[2] == 0.0 && gs[3] == 0.0 && gs[4] == 0.0) return;
  for (int kk = 0; kk < n; ++kk)
    for (int jj = 0; jj < n; ++jj)
      for (int ii = 0; ii < n; ++ii) {
        const double wgt = L[ii] * L[n + jj] * L[2 * n + kk];
        const size_t gn = (size_t)es * n3 + ii + n * (jj + n * kk);
#pragma unroll
        for (int v = 0; v < 5; ++v) atomicAdd(&gU[v * S + gn], wgt * gs[v]);
      }
}

// ---------------------------------------------------------------------------
// k_wall_loss: mean wall shear L = sum_slots wq tau_x / sum wq (wq: surface
// quadrature weight w_a w_b s of the wall node), accumulated into loss[0].
// With grad != 0 also dL/dUs per slot (into gUs, for k_adj_scatter) and
// dL/d(kappa, B) (into gtheta).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128)
k_wall_loss(const double* __restrict__ U, const MeshDev<double> m, const PhysDev ph, const double* __restrict__ wq,
            double inv_total, int grad, double* __restrict__ loss, double* __restrict__ gUs,
            double* __restrict__ gtheta, int* __restrict__ status) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  double lv = 0.0, gk = 0.0, gb = 0.0;
  if (slot < m.n_wall * n2) {
    const int f = m.n_interior + slot / n2;
    const int ab = slot % n2;
    const size_t S = (size_t)m.K * n3;
    const size_t FN = (size_t)m.F * n2, fg = (size_t)f * n2 + ab;
    const double nx = m.fgeo[fg], ny = m.fgeo[FN + fg], nz = m.fgeo[2 * FN + fg];
    const int es = chk_idx(m.ws_elem[slot], m.K, m.status);
    const double* L = m.ws_lag + (size_t)slot * 3 * n;
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
    const double wgt = wq[slot] * inv_total;
    bool ok = true;
    const int seeds = grad ? 7 : 1;
#pragma unroll 1
    for (int k = 0; k < seeds; ++k) {
      DualD Ud[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) Ud[v] = DualD(Us[v], grad && k == v ? 1.0 : 0.0);
      DualD tau[3];
      bool okk;
      wall_stress_jvp(ph, Ud, grad && k == 5 ? 1.0 : 0.0, grad && k == 6 ? 1.0 : 0.0, nx, ny, nz, tau, &okk);
      ok = ok && okk;
      if (k == 0) lv = wgt * tau[0].v;
      if (grad) {
        if (k < 5) gUs[(size_t)slot * 5 + k] = wgt * tau[0].d;
        else if (k == 5) gk = wgt * tau[0].d;
        else gb = wgt * tau[0].d;
      }
    }
    if (!ok) atomicOr(status, ST_WM_NOCONV);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lv += __shfl_down_sync(0xffffffffu, lv, o);
    gk += __shfl_down_sync(0xffffffffu, gk, o);
    gb += __shfl_down_sync(0xffffffffu, gb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(loss, lv);
    if (grad && gtheta) { atomicAdd(&gtheta[0], gk); atomicAdd(&gtheta[1], gb); }
  }
}

// y = a x + b y over n doubles
static __global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (b == 0.0 ? 0.0 : b * y[i]) + a * x[i];
}

}  // namespace dg
