// dgsem_oracle.cpp -- plain, slow FP64 CPU reference of the DGSEM operator.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: it exists so that tests/, the smoke check and the timed
// CPU baseline of bench.py have an independent answer to compare against.
// It shares no code, header or table with the CUDA library.
//
// What it computes (paper: Sec. 2.2 "split-form DG scheme" on Legendre-
// Gauss-Lobatto nodes; Sec. 4 "split DGSE formulation", fourth-order
// low-storage Runge-Kutta, Roe solver with Harten entropy fix, ideal gas;
// Sec. 3.1 wall-stress coupling; Sec. 3.2 Spalding law, Van Driest transform,
// Algorithms 1 and 2):
//   Ut = DG_Operator(U) for the 3D compressible Navier-Stokes equations in
//   strong form on curvilinear hexahedra, followed by the LSERK4 update.
// The paper gives no operator equations; this is the textbook DGSEM written
// out step by step (one loop per definition, no symmetry tricks, no fusion).
// Where the paper leaves a point open (lifted variables, flux forms, boundary
// states, the wall model's sampling and Newton stopping rule, the logarithmic
// mean, Sutherland constants), the reading taken is stated at the function
// that implements it; the library implements the same readings independently.
//
// Everything is templated on the scalar type T so that a forward-mode dual
// number gives exact Jacobian-vector products (used to check the adjoint).
//
// Parity status of each function: pinned by tests/test_oracle_*.py against
// closed forms, identities (SBP, metric identities, free-stream, conservation,
// kinetic-energy and entropy conservation, boundary flux balances), tabulated
// data (Spalding's printed constants, air viscosities), a manufactured
// solution and finite differences.  Nothing here is "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORA_REAL
#define ORA_REAL double
#endif

namespace ora {

// Base floating-point type of the whole oracle: double for the FP64 oracle
// (the CPU baseline and every pin), long double for the extended-precision
// build used as the parity reference.
typedef ORA_REAL real;

// ---------------------------------------------------------------------------
// Forward-mode dual number (value, one directional derivative).
// ---------------------------------------------------------------------------
struct Dual {
  real v, d;
  Dual(real x = 0.0, real dx = 0.0) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  real r = a.v / b.v;
  return Dual(r, (a.d - r * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { real s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual exp(Dual a) { real e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual log1p(Dual a) { return Dual(std::log1p(a.v), a.d / (1.0 + a.v)); }
inline Dual asin(Dual a) { return Dual(std::asin(a.v), a.d / std::sqrt(1.0 - a.v * a.v)); }
inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }

inline real val(real x) { return x; }
inline real val(const Dual& x) { return x.v; }
inline real der(real) { return 0.0; }
inline real der(const Dual& x) { return x.d; }

using std::sqrt; using std::exp; using std::log; using std::log1p; using std::asin; using std::fabs;

// ---------------------------------------------------------------------------
// Enumerations (same numeric values as the public C ABI documents).
// ---------------------------------------------------------------------------
enum VolFlux { VOL_KEP_PIROZZOLI = 0, VOL_KEP_KENNEDY_GRUBER = 1, VOL_EC_CHANDRASHEKAR = 2 };
enum SurfFlux { SURF_CENTRAL = 0, SURF_LLF = 1, SURF_ROE = 2 };
enum WallLaw { LAW_SPALDING = 0, LAW_REICHARDT = 1 };
// neighbour codes of boundary faces: slip wall with the wall model (Sec. 3),
// Dirichlet inflow and subsonic pressure outflow (Sec. 4's cascade boundaries)
enum BoundaryCode { BC_WALL = -1, BC_INFLOW = -2, BC_OUTFLOW = -3 };

// ---------------------------------------------------------------------------
// 1. Legendre-Gauss-Lobatto nodes/weights and the nodal derivative matrix.
//    Nodes: x = +-1 and the roots of P_N'(x) (Newton, P_N'' from the Legendre
//    ODE).  Weights: w_i = 2 / (N (N+1) P_N(x_i)^2).
//    D_ij = l_j'(x_i) from barycentric weights; D_ii = -sum_{j!=i} D_ij.
// ---------------------------------------------------------------------------
static void legendre(int N, real x, real* P, real* dP) {
  // P_N(x) and P_N'(x) by the three-term recurrence.
  real p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= N; ++k) {
    real p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    real d2 = d0 + (2.0 * k - 1.0) * p1;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

void lgl(int N, std::vector<real>& x, std::vector<real>& w, std::vector<real>& D) {
  const int n = N + 1;
  x.assign(n, 0.0); w.assign(n, 0.0); D.assign(n * n, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    real xi = -std::cos(M_PI * i / N);  // Chebyshev-Lobatto start
    for (int it = 0; it < 100; ++it) {
      real P, dP;
      legendre(N, xi, &P, &dP);
      real d2P = (2.0 * xi * dP - N * (N + 1.0) * P) / (1.0 - xi * xi);
      real step = dP / d2P;
      xi -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[i] = xi;
  }
  // symmetrise (nodes are symmetric about 0)
  for (int i = 0; i < n / 2; ++i) {
    real a = 0.5 * (x[N - i] - x[i]);
    x[i] = -a; x[N - i] = a;
  }
  if (n % 2 == 1) x[N / 2] = 0.0;
  for (int i = 0; i < n; ++i) {
    real P, dP;
    legendre(N, x[i], &P, &dP);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
  std::vector<real> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (x[j] - x[k]);
  for (int i = 0; i < n; ++i) {
    real s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * n + j];
    }
    D[i * n + i] = -s;
  }
}

// Lagrange basis l_j(s) and l_j'(s) on the nodes x, by the product formula.
static void lagrange(const std::vector<real>& x, real s, real* l, real* dl) {
  const int n = (int)x.size();
  for (int j = 0; j < n; ++j) {
    real p = 1.0, dp = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == j) continue;
      real f = (s - x[k]) / (x[j] - x[k]);
      dp = dp * f + p / (x[j] - x[k]);
      p *= f;
    }
    l[j] = p;
    if (dl) dl[j] = dp;
  }
}

// LSERK4: Carpenter & Kennedy (1994) five-stage, fourth-order 2N-storage
// scheme (paper Sec. 4: "fourth-order low-storage Runge-Kutta").
static const real RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                               -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0,
                               -1275806237668.0 / 842570457699.0};
static const real RK_B[5] = {1432997174477.0 / 9575080441755.0,
                               5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0,
                               3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const real RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                               2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0,
                               2802321613138.0 / 2924317926251.0};

// ---------------------------------------------------------------------------
// Physical parameters and options.
// ---------------------------------------------------------------------------
template <class T>
struct Phys {
  real gamma = 1.4, R = 1.0, mu = 0.0, Pr = 0.72;
  real f[3] = {0.0, 0.0, 0.0};  // constant body force per unit volume
  T kappa = 0.41, B = 5.2;        // wall-law constants
  real suth_S = 0.0, T_ref = 1.0;  // Sutherland constant and reference temperature (S <= 0: constant mu)
  real U_in[5] = {1.0, 0.0, 0.0, 0.0, 1.0};  // Dirichlet inflow state (conservative)
  real p_out = 1.0;                          // outflow pressure
  real T_wall = 0.0;                         // isothermal wall temperature (<= 0: adiabatic walls)
  real hwm = 0.1;               // wall-model sampling distance
};
struct Opts {
  int vol_flux = VOL_KEP_PIROZZOLI;
  int surf_flux = SURF_LLF;
  int viscous = 1;
  int law = LAW_REICHARDT;
};

// ---------------------------------------------------------------------------
// Mesh: nodes X[c][e][p] (p = i + n (j + n k)), neighbours nbr[e][l]
// (l = 0:-xi 1:+xi 2:-eta 3:+eta 4:-zeta 5:+zeta; value >= 0 is the
// neighbour element, negative values are boundary codes, -1 a wall-modelled
// slip wall).  A conforming hexahedral mesh joins face l of e to face
// nface[e][l] of the neighbour, whose face-local node (a', b') coincides with
// node (a, b) of face l by the orientation code o = orient[e][l]:
//   (s, t) = (o & 1) ? (b, a) : (a, b);  a' = (o & 2) ? N - s : s;
//   b' = (o & 4) ? N - t : t
// (face-local coordinates as in face_node below).  A structured mesh has
// nface = l ^ 1 and o = 0 everywhere.
// ---------------------------------------------------------------------------
struct Mesh {
  int N = 0, n = 0, n2 = 0, n3 = 0, K = 0;
  std::vector<real> xi, w, D;
  std::vector<real> X;    // [3][K*n3]
  std::vector<int> nbr;     // [K*6]
  std::vector<int> nface;   // [K*6] neighbour's local face
  std::vector<int> orient;  // [K*6] orientation code (see above)
  std::vector<real> Ja;   // [(e*n3+p)*9 + dir*3 + comp]
  std::vector<real> J;    // [e*n3+p]
  // wall model: one slot per wall face node, ordered by (e, l, b, a)
  std::vector<int> wslot;   // [K*6] first slot of that face or -1
  std::vector<int> ws_elem; // sample element
  std::vector<real> ws_ref;   // sample reference coordinates [slot*3]
  std::vector<real> ws_l;     // Lagrange weights [slot*3*n]
  int nwall = 0;
  // Optional evaluation subset (empty: every element).  Ut is computed for
  // the elements in mask_out only; the lifting for those and their
  // neighbours (mask_grad); primitives and metrics for one more ring
  // (mask_q).  Used to sample meshes too large to evaluate whole.
  std::vector<char> mask_out, mask_grad, mask_q;
};

inline bool in_mask(const std::vector<char>& m, int e) { return m.empty() || m[e]; }

inline int node(const Mesh& M, int i, int j, int k) { return i + M.n * (j + M.n * k); }
inline void ijk(const Mesh& M, int p, int& i, int& j, int& k) {
  i = p % M.n; j = (p / M.n) % M.n; k = p / M.n2;
}
// volume node of face-local node (a, b) on local face l
inline int face_node(const Mesh& M, int l, int a, int b) {
  const int N = M.N;
  switch (l) {
    case 0: return node(M, 0, a, b);
    case 1: return node(M, N, a, b);
    case 2: return node(M, a, 0, b);
    case 3: return node(M, a, N, b);
    case 4: return node(M, a, b, 0);
    default: return node(M, a, b, N);
  }
}
inline real face_sign(int l) { return (l & 1) ? 1.0 : -1.0; }

// the node of the neighbour's face that coincides with node (a, b) of face
// l of e (interior faces only)
inline void neighbour_node(const Mesh& M, int e, int l, int a, int b, int* nb, int* q) {
  const int o = M.orient[e * 6 + l];
  const int s = (o & 1) ? b : a, t = (o & 1) ? a : b;
  const int a2 = (o & 2) ? M.N - s : s, b2 = (o & 4) ? M.N - t : t;
  *nb = M.nbr[e * 6 + l];
  *q = face_node(M, M.nface[e * 6 + l], a2, b2);
}

// inverse of an orientation code
inline int orient_inverse(int o) {
  return (o & 1) ? (1 | (((o >> 2) & 1) << 1) | (((o >> 1) & 1) << 2)) : o;
}

// The side of an interior face whose metrics give the face normal and whose
// node order indexes the face (reading R21, generalised to any pair of local
// faces): the side with the odd local face (+xi, +eta, +zeta) when the two
// local faces differ in parity, else the side with the smaller (element,
// face) pair.
inline bool is_master(const Mesh& M, int e, int l) {
  const int nb = M.nbr[e * 6 + l], l2 = M.nface[e * 6 + l];
  if ((l & 1) != (l2 & 1)) return (l & 1) != 0;
  return e * 6 + l < nb * 6 + l2;
}

static bool build_metrics(Mesh& M, std::string& err) {
  const int n = M.n, n3 = M.n3, K = M.K;
  M.Ja.assign((size_t)K * n3 * 9, 0.0);
  M.J.assign((size_t)K * n3, 0.0);
  std::vector<real> dX(9 * n3), v(3 * n3);
  for (int e = 0; e < K; ++e) {
    if (!in_mask(M.mask_q, e)) continue;
    // Coordinates relative to the element's first node: rows of D sum to
    // zero and curl(c grad X_m) = 0 for a constant c, so derivatives and the
    // curl form are unchanged in exact arithmetic, while the roundoff no
    // longer depends on where the element sits in the domain (periodic
    // images of one face then get the same metrics to roundoff).
    auto Xc = [&](int c, int p) {
      return M.X[(size_t)c * K * n3 + (size_t)e * n3 + p] - M.X[(size_t)c * K * n3 + (size_t)e * n3];
    };
    // dX[(c*3+dir)*n3+p] = d x_c / d xi_dir
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < n3; ++p) {
        int i, j, k; ijk(M, p, i, j, k);
        real s0 = 0, s1 = 0, s2 = 0;
        for (int m = 0; m < n; ++m) {
          s0 += M.D[i * n + m] * Xc(c, node(M, m, j, k));
          s1 += M.D[j * n + m] * Xc(c, node(M, i, m, k));
          s2 += M.D[k * n + m] * Xc(c, node(M, i, j, m));
        }
        dX[(c * 3 + 0) * n3 + p] = s0;
        dX[(c * 3 + 1) * n3 + p] = s1;
        dX[(c * 3 + 2) * n3 + p] = s2;
      }
    for (int p = 0; p < n3; ++p) {
      real a[3][3];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) a[c][d] = dX[(c * 3 + d) * n3 + p];
      real det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                   a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                   a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
      M.J[(size_t)e * n3 + p] = det;
      if (!(det > 0.0)) {
        err = "non-positive Jacobian in element " + std::to_string(e);
        return false;
      }
    }
    // Curl form (Kopriva 2006): (J a^i)_nn = -xhat_i . curl_xi( X_l grad_xi X_m ),
    // (nn, m, l) cyclic.
    for (int nn = 0; nn < 3; ++nn) {
      const int mm = (nn + 1) % 3, ll = (nn + 2) % 3;
      for (int p = 0; p < n3; ++p)
        for (int d = 0; d < 3; ++d) v[d * n3 + p] = Xc(ll, p) * dX[(mm * 3 + d) * n3 + p];
      for (int p = 0; p < n3; ++p) {
        int i, j, k; ijk(M, p, i, j, k);
        real dv[3][3] = {{0}};  // dv[d][dir] = d v_d / d xi_dir
        for (int d = 0; d < 3; ++d)
          for (int m = 0; m < n; ++m) {
            dv[d][0] += M.D[i * n + m] * v[d * n3 + node(M, m, j, k)];
            dv[d][1] += M.D[j * n + m] * v[d * n3 + node(M, i, m, k)];
            dv[d][2] += M.D[k * n + m] * v[d * n3 + node(M, i, j, m)];
          }
        real* ja = &M.Ja[((size_t)e * n3 + p) * 9];
        ja[0 * 3 + nn] = -(dv[2][1] - dv[1][2]);
        ja[1 * 3 + nn] = -(dv[0][2] - dv[2][0]);
        ja[2 * 3 + nn] = -(dv[1][0] - dv[0][1]);
      }
    }
  }
  return true;
}

static bool check_connectivity(const Mesh& M, std::string& err) {
  const int K = M.K, n3 = M.n3;
  real scale = 0.0;
  for (real x : M.X) scale = std::max(scale, std::fabs(x));
  scale = std::max<real>(scale, 1.0);
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l) {
      int nb = M.nbr[e * 6 + l];
      if (nb < BC_OUTFLOW || nb >= K) { err = "bad neighbour id"; return false; }
      if (nb < 0) continue;
      const int l2 = M.nface[e * 6 + l], o = M.orient[e * 6 + l];
      if (l2 < 0 || l2 > 5 || o < 0 || o > 7) { err = "bad neighbour face or orientation"; return false; }
      if (nb == e && l2 == l) { err = "a face cannot be its own neighbour"; return false; }
      if (M.nbr[nb * 6 + l2] != e || M.nface[nb * 6 + l2] != l || M.orient[nb * 6 + l2] != orient_inverse(o)) {
        err = "non-reciprocal connectivity";
        return false;
      }
      // faces must coincide up to one translation (periodic image)
      real shift[3];
      for (int b = 0; b < M.n; ++b)
        for (int a = 0; a < M.n; ++a) {
          int p = face_node(M, l, a, b), q, nbq;
          neighbour_node(M, e, l, a, b, &nbq, &q);
          for (int c = 0; c < 3; ++c) {
            real dx = M.X[(size_t)c * K * n3 + (size_t)nb * n3 + q] -
                        M.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
            if (a == 0 && b == 0) shift[c] = dx;
            else if (std::fabs(dx - shift[c]) > 1e-9 * scale) {
              err = "faces do not match (not watertight) at element " + std::to_string(e);
              return false;
            }
          }
        }
    }
  return true;
}

// Wall-model sampling points (reading of Sec. 3.1: the wall model samples
// the LES solution at distance h_wm from the wall): for every wall face node
// the point x_w - h_wm * n_out is located by Newton on each candidate
// element's polynomial mapping.  The first element that contains it
// (max |xi| <= 1 + 1e-8) is used, searching the wall element's column first
// (the wall element, then its neighbours across the faces opposite the wall,
// up to 3 layers) and then all elements by ascending index: points on a face
// shared by two elements (e.g. above an edge node of the wall face) then get
// one well-defined element although the DG solution is discontinuous there.
static bool locate_point(const Mesh& M, int e, const real xs[3], real ref[3]) {
  const int n = M.n, n3 = M.n3, K = M.K;
  real r[3] = {0.0, 0.0, 0.0};
  std::vector<real> l0(n), l1(n), l2(n), d0(n), d1(n), d2(n);
  for (int it = 0; it < 60; ++it) {
    lagrange(M.xi, r[0], l0.data(), d0.data());
    lagrange(M.xi, r[1], l1.data(), d1.data());
    lagrange(M.xi, r[2], l2.data(), d2.data());
    real x[3] = {0, 0, 0}, Jm[3][3] = {{0}};
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int p = node(M, i, j, k);
          for (int c = 0; c < 3; ++c) {
            real Xv = M.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
            x[c] += Xv * l0[i] * l1[j] * l2[k];
            Jm[c][0] += Xv * d0[i] * l1[j] * l2[k];
            Jm[c][1] += Xv * l0[i] * d1[j] * l2[k];
            Jm[c][2] += Xv * l0[i] * l1[j] * d2[k];
          }
        }
    real res[3] = {xs[0] - x[0], xs[1] - x[1], xs[2] - x[2]};
    // solve Jm * dr = res by Cramer's rule
    real det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                 Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                 Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
    if (det == 0.0) return false;
    real dr[3];
    for (int c = 0; c < 3; ++c) {
      real A[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) A[a][b] = (b == c) ? res[a] : Jm[a][b];
      dr[c] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
    }
    real step = 0.0;
    for (int c = 0; c < 3; ++c) {
      r[c] += dr[c];
      r[c] = std::max<real>(-3.0, std::min<real>(3.0, r[c]));
      step = std::max(step, std::fabs(dr[c]));
    }
    if (step < 1e-15) break;
  }
  for (int c = 0; c < 3; ++c) ref[c] = r[c];
  return true;
}

static bool build_wall_samples(Mesh& M, real hwm, std::string& err) {
  const int n = M.n, n3 = M.n3, K = M.K;
  M.wslot.assign((size_t)K * 6, -1);
  int slots = 0;
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l)
      if (M.nbr[e * 6 + l] == BC_WALL) { M.wslot[e * 6 + l] = slots; slots += M.n2; }
  M.nwall = slots;
  M.ws_elem.assign(slots, -1);
  M.ws_ref.assign((size_t)slots * 3, 0.0);
  M.ws_l.assign((size_t)slots * 3 * n, 0.0);
  if (slots == 0) return true;
  // element bounding boxes
  std::vector<real> bmin((size_t)K * 3, 1e300), bmax((size_t)K * 3, -1e300);
  for (int e = 0; e < K; ++e)
    for (int p = 0; p < n3; ++p)
      for (int c = 0; c < 3; ++c) {
        real x = M.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
        bmin[e * 3 + c] = std::min(bmin[e * 3 + c], x);
        bmax[e * 3 + c] = std::max(bmax[e * 3 + c], x);
      }
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l) {
      int s0 = M.wslot[e * 6 + l];
      if (s0 < 0 || !in_mask(M.mask_q, e)) continue;
      const int dir = l / 2;
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          int p = face_node(M, l, a, b);
          const real* ja = &M.Ja[((size_t)e * n3 + p) * 9 + dir * 3];
          real s = std::sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
          real xs[3];
          for (int c = 0; c < 3; ++c) {
            real nout = face_sign(l) * ja[c] / s;
            xs[c] = M.X[(size_t)c * K * n3 + (size_t)e * n3 + p] - hwm * nout;
          }
          int best = -1; real bref[3] = {0, 0, 0};
          // first the wall element's column: the wall element, then its
          // neighbours across the faces opposite the wall (up to 3 layers;
          // in each element the face opposite the one it was entered by)
          for (int c2 = e, layer = 0, lin = l; c2 >= 0 && layer < 4 && best < 0; ++layer) {
            real ref[3];
            if (locate_point(M, c2, xs, ref)) {
              real rm = std::max(std::fabs(ref[0]), std::max(std::fabs(ref[1]), std::fabs(ref[2])));
              if (rm <= 1.0 + 1e-8) {
                best = c2;
                for (int c = 0; c < 3; ++c) bref[c] = ref[c];
              }
            }
            const int lout = lin ^ 1, nxt = M.nbr[c2 * 6 + lout];
            if (nxt >= 0) lin = M.nface[c2 * 6 + lout];
            c2 = nxt;
          }
          // else the lowest-index element containing the point
          for (int c2 = 0; c2 < K && best < 0; ++c2) {
            bool inside = true;
            for (int c = 0; c < 3; ++c) {
              real marg = 0.05 * (bmax[c2 * 3 + c] - bmin[c2 * 3 + c]) + 1e-12;
              if (xs[c] < bmin[c2 * 3 + c] - marg || xs[c] > bmax[c2 * 3 + c] + marg) inside = false;
            }
            if (!inside) continue;
            real ref[3];
            if (!locate_point(M, c2, xs, ref)) continue;
            real rm = std::max(std::fabs(ref[0]), std::max(std::fabs(ref[1]), std::fabs(ref[2])));
            if (rm <= 1.0 + 1e-8) {  // first (lowest-index) element containing the point
              best = c2;
              for (int c = 0; c < 3; ++c) bref[c] = ref[c];
              break;
            }
          }
          if (best < 0) {
            err = "wall-model sample point outside the mesh (element " + std::to_string(e) + ")";
            return false;
          }
          int slot = s0 + a + n * b;
          M.ws_elem[slot] = best;
          for (int c = 0; c < 3; ++c) {
            M.ws_ref[slot * 3 + c] = bref[c];
            lagrange(M.xi, bref[c], &M.ws_l[((size_t)slot * 3 + c) * n], nullptr);
          }
        }
    }
  return true;
}

// ---------------------------------------------------------------------------
// 3. Primitive variables (ideal gas, paper Sec. 4).
// ---------------------------------------------------------------------------
template <class T>
struct Prim { T rho, u[3], p, T_, h; };  // h = (E + p) / rho

template <class T>
inline Prim<T> prim_of(const Phys<T>& P, const T U[5]) {
  Prim<T> q;
  q.rho = U[0];
  for (int c = 0; c < 3; ++c) q.u[c] = U[1 + c] / U[0];
  T kin = 0.5 * U[0] * (q.u[0] * q.u[0] + q.u[1] * q.u[1] + q.u[2] * q.u[2]);
  q.p = (P.gamma - 1.0) * (U[4] - kin);
  q.T_ = q.p / (U[0] * P.R);
  q.h = (U[4] + q.p) / U[0];
  return q;
}

// ---------------------------------------------------------------------------
// 5. Fluxes.  a is a (not necessarily unit) direction vector.
// ---------------------------------------------------------------------------
// Euler flux F(U) . a
template <class T>
void euler_flux(const Prim<T>& q, const T U[5], const real a[3], T F[5]) {
  T un = q.u[0] * a[0] + q.u[1] * a[1] + q.u[2] * a[2];
  F[0] = q.rho * un;
  for (int c = 0; c < 3; ++c) F[1 + c] = q.rho * un * q.u[c] + q.p * a[c];
  F[4] = (U[4] + q.p) * un;
}

// Logarithmic mean (a - b) / ln(a / b), written as (a - b) / log1p((a - b) / b)
// so that it stays accurate when a and b are close; a == b gives a.
template <class T>
T logmean(const T& a, const T& b) {
  if (val(a) == val(b)) return 0.5 * (a + b);
  T d = a - b;
  return d / log1p(d / b);
}

// Two-point flux F#(UL, UR) . a.
//  Pirozzoli (KEP):      {rho}{u.a},  {rho}{u.a}{u} + {p} a,  {rho}{u.a}{h}
//  Kennedy-Gruber (KEP): {rho}{u.a},  {rho}{u.a}{u} + {p} a,  {rho}{u.a}{e} + {p}{u.a}
//  Chandrashekar (entropy conserving and KEP, the paper's Sec. 4 scheme):
//    beta = rho / (2 p), rho^ = ln-mean(rho), beta^ = ln-mean(beta),
//    p~ = {rho} / (2 {beta}),  F_rho = rho^ {u}.a,  F_m = p~ a + {u} F_rho,
//    F_E = F_rho (1 / (2 (gamma - 1) beta^) - {|u|^2} / 2) + {u} . F_m
template <class T>
void twopoint_flux(int kind, real gamma, const Prim<T>& L, const T UL[5], const Prim<T>& R, const T UR[5],
                   const real a[3], T F[5]) {
  T u[3];
  for (int c = 0; c < 3; ++c) u[c] = 0.5 * (L.u[c] + R.u[c]);
  T ua = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];
  if (kind == VOL_EC_CHANDRASHEKAR) {
    T bL = L.rho / (2.0 * L.p), bR = R.rho / (2.0 * R.p);
    T rho_ln = logmean(L.rho, R.rho), b_ln = logmean(bL, bR);
    T pt = 0.5 * (L.rho + R.rho) / (bL + bR);
    T u2 = 0.5 * (L.u[0] * L.u[0] + L.u[1] * L.u[1] + L.u[2] * L.u[2] +
                  R.u[0] * R.u[0] + R.u[1] * R.u[1] + R.u[2] * R.u[2]);
    F[0] = rho_ln * ua;
    for (int c = 0; c < 3; ++c) F[1 + c] = pt * a[c] + u[c] * F[0];
    F[4] = F[0] * (1.0 / (2.0 * (gamma - 1.0) * b_ln) - 0.5 * u2) + u[0] * F[1] + u[1] * F[2] + u[2] * F[3];
    return;
  }
  T rho = 0.5 * (L.rho + R.rho);
  T p = 0.5 * (L.p + R.p);
  F[0] = rho * ua;
  for (int c = 0; c < 3; ++c) F[1 + c] = rho * ua * u[c] + p * a[c];
  if (kind == VOL_KEP_PIROZZOLI) {
    T h = 0.5 * (L.h + R.h);
    F[4] = rho * ua * h;
  } else {
    T e = 0.5 * (UL[4] / L.rho + UR[4] / R.rho);
    F[4] = rho * ua * e + p * ua;
  }
}

// dynamic viscosity: constant, or Sutherland mu (T / T_ref)^(3/2) (T_ref + S) / (T + S)
template <class T>
T viscosity(const Phys<T>& P, const T& Tt) {
  if (!(P.suth_S > 0.0)) return T(P.mu);
  T x = Tt / P.T_ref;
  return P.mu * x * sqrt(x) * (P.T_ref + P.suth_S) / (Tt + P.suth_S);
}

// Viscous flux Fv(U, grad W) . a  with grad W = g[d][w], W = (u, v, w, T).
//   Fv_d = (0, tau_1d, tau_2d, tau_3d, tau_jd u_j + k dT/dx_d)
//   tau_ij = mu (du_i/dx_j + du_j/dx_i) - 2/3 mu (div u) delta_ij
template <class T>
void viscous_flux(const Phys<T>& P, const Prim<T>& q, const T g[3][4], const real a[3], T F[5]) {
  const T mu = viscosity(P, q.T_);
  const real cp = P.gamma * P.R / (P.gamma - 1.0);
  const T kcond = mu * cp / P.Pr;
  T div = g[0][0] + g[1][1] + g[2][2];
  T tau[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      tau[i][j] = mu * (g[j][i] + g[i][j]);
      if (i == j) tau[i][j] -= (2.0 / 3.0) * mu * div;
    }
  F[0] = 0.0;
  for (int i = 0; i < 3; ++i) F[1 + i] = tau[i][0] * a[0] + tau[i][1] * a[1] + tau[i][2] * a[2];
  T e = 0.0;
  for (int d = 0; d < 3; ++d) {
    T work = tau[0][d] * q.u[0] + tau[1][d] * q.u[1] + tau[2][d] * q.u[2] + kcond * g[d][3];
    e += work * a[d];
  }
  F[4] = e;
}

// Numerical inviscid flux along the unit normal nh (master orientation).
//  central: F#(UL, UR) . nh
//  LLF:     central - 1/2 lambda_max (UR - UL)
//  Roe:     central - 1/2 sum_k |lambda_k| alpha_k r_k, Roe averages, Harten
//           entropy fix |l| <- (l^2 + d^2) / (2 d) for |l| < d = 0.1 c~ on the
//           two acoustic waves.
template <class T>
void riemann(const Phys<T>& P, int vol_kind, int kind, const Prim<T>& L, const T UL[5],
             const Prim<T>& R, const T UR[5], const real nh[3], T F[5]) {
  twopoint_flux(vol_kind, P.gamma, L, UL, R, UR, nh, F);
  if (kind == SURF_CENTRAL) return;
  const real g = P.gamma;
  if (kind == SURF_LLF) {
    T unL = L.u[0] * nh[0] + L.u[1] * nh[1] + L.u[2] * nh[2];
    T unR = R.u[0] * nh[0] + R.u[1] * nh[1] + R.u[2] * nh[2];
    T cL = sqrt(g * L.p / L.rho), cR = sqrt(g * R.p / R.rho);
    T lamL = fabs(unL) + cL, lamR = fabs(unR) + cR;
    T lam = val(lamL) >= val(lamR) ? lamL : lamR;
    for (int v = 0; v < 5; ++v) F[v] -= 0.5 * lam * (UR[v] - UL[v]);
    return;
  }
  // Roe
  T sL = sqrt(L.rho), sR = sqrt(R.rho);
  T rt = sL * sR;
  T ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * L.u[c] + sR * R.u[c]) / (sL + sR);
  T Ht = (sL * L.h + sR * R.h) / (sL + sR);
  T q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  T c2 = (g - 1.0) * (Ht - 0.5 * q2);
  T ct = sqrt(c2);
  T un = ut[0] * nh[0] + ut[1] * nh[1] + ut[2] * nh[2];
  T drho = R.rho - L.rho, dp = R.p - L.p;
  T du[3];
  for (int c = 0; c < 3; ++c) du[c] = R.u[c] - L.u[c];
  T dun = du[0] * nh[0] + du[1] * nh[1] + du[2] * nh[2];
  T a1 = (dp - rt * ct * dun) / (2.0 * c2);
  T a2 = drho - dp / c2;
  T a5 = (dp + rt * ct * dun) / (2.0 * c2);
  T l1 = fabs(un - ct), l2 = fabs(un), l5 = fabs(un + ct);
  T delta = 0.1 * ct;
  if (val(l1) < val(delta)) l1 = (l1 * l1 + delta * delta) / (2.0 * delta);
  if (val(l5) < val(delta)) l5 = (l5 * l5 + delta * delta) / (2.0 * delta);
  T Dd[5];
  // wave 1: (1, u - c n, H - c un)
  Dd[0] = l1 * a1;
  for (int c = 0; c < 3; ++c) Dd[1 + c] = l1 * a1 * (ut[c] - ct * nh[c]);
  Dd[4] = l1 * a1 * (Ht - ct * un);
  // entropy wave: (1, u, |u|^2 / 2)
  Dd[0] += l2 * a2;
  for (int c = 0; c < 3; ++c) Dd[1 + c] += l2 * a2 * ut[c];
  Dd[4] += l2 * a2 * 0.5 * q2;
  // wave 5: (1, u + c n, H + c un)
  Dd[0] += l5 * a5;
  for (int c = 0; c < 3; ++c) Dd[1 + c] += l5 * a5 * (ut[c] + ct * nh[c]);
  Dd[4] += l5 * a5 * (Ht + ct * un);
  // two shear waves: rho~ (0, du - dun n, u~ . du - un dun)
  for (int c = 0; c < 3; ++c) Dd[1 + c] += l2 * rt * (du[c] - dun * nh[c]);
  Dd[4] += l2 * rt * (ut[0] * du[0] + ut[1] * du[1] + ut[2] * du[2] - un * dun);
  for (int v = 0; v < 5; ++v) F[v] -= 0.5 * Dd[v];
}

// ---------------------------------------------------------------------------
// 12. Wall model: Van Driest transform (adiabatic, Crocco-Busemann) and the
//     algebraic laws of the wall, solved by Newton for u_tau.
// ---------------------------------------------------------------------------
// law value u+(y+) (Reichardt) or y+(u+) (Spalding as printed in Sec. 3.2:
// y+ = u+ + e^{-kB} [e^{k u+} - sum_{p=0..4} (k u+)^p / p!]).
template <class T>
T reichardt(const T& yp, const T& kappa, const T& B) {
  T C = B - log(kappa) / kappa;
  return log(1.0 + kappa * yp) / kappa +
         C * (1.0 - exp(-yp / 11.0) - (yp / 11.0) * exp(-0.33 * yp));
}
template <class T>
T spalding(const T& up, const T& kappa, const T& B) {
  T ku = kappa * up;
  return up + exp(-kappa * B) *
                  (exp(ku) - 1.0 - ku - ku * ku / 2.0 - ku * ku * ku / 6.0 - ku * ku * ku * ku / 24.0);
}

// Solve the law for u_tau given the (transformed) velocity u, the sampling
// height h and the wall kinematic viscosity nu (SolveWallStress of
// Algorithms 1-2).  With Re_h = h u / nu = u+ y+, each law is written in its
// explicit variable w (y+ for Reichardt, u+ for Spalding) as
//   F(t) = t + ln L(e^t) - ln Re_h = 0,   w = e^t,
// L(w) = u+(y+) (Reichardt) or y+(u+) (Spalding).  F is increasing in t and
// close to linear at both ends (viscous sublayer: F ~ 2t; log layer: ln L
// ~ kappa w or ln w), so Newton converges from the laminar estimate
// t0 = ln(Re_h)/2 (u+ = y+).  The root is bracketed first; Newton steps that
// leave the bracket are replaced by bisection; stop after a Newton step
// |dt| <= 1e-12 max(1, |t|) (its error is O(dt^2)) or a bracket of 2e-15.
// u_tau = y+ nu / h (Reichardt) or u / u+ (Spalding).
// Returns the iterations used, or -1 after 200 without convergence.
template <class T>
T law_residual(int law, const T& t, const T& lnRe, const T& kappa, const T& B) {
  T w = exp(t);
  T L = (law == LAW_REICHARDT) ? reichardt(w, kappa, B) : spalding(w, kappa, B);
  return t + log(L) - lnRe;
}

template <class T>
int solve_utau(int law, const T& u, real h, const T& nu, const T& kappa, const T& B, T& ut) {
  if (!(val(u) > 0.0)) { ut = 0.0; return 0; }
  const real lnRe = std::log(h * val(u) / val(nu));
  const Dual kD(val(kappa)), BD(val(B)), lnReD(lnRe);
  auto F_of = [&](real t, real* dF) {
    Dual F = law_residual(law, Dual(t, 1.0), lnReD, kD, BD);
    *dF = F.d;
    return F.v;
  };
  real dF;
  real lo = 0.5 * lnRe, hi = lo, stepb = 1.0;
  int it = 0;
  while (!(F_of(lo, &dF) < 0.0) && it < 200) { lo -= stepb; stepb *= 2.0; ++it; }
  stepb = 1.0;
  while (!(F_of(hi, &dF) > 0.0) && it < 200) { hi += stepb; stepb *= 2.0; ++it; }
  real t = 0.5 * lnRe;
  if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
  bool done = false;
  for (; it < 200; ++it) {
    real Ft = F_of(t, &dF);
    if (Ft == 0.0) { done = true; ++it; break; }
    if (Ft < 0.0) lo = t; else hi = t;
    real next = t - Ft / dF;
    const bool newton = (next >= lo && next <= hi);
    if (!newton) next = 0.5 * (lo + hi);
    real step = std::fabs(next - t);
    t = next;
    const real scale = std::max<real>(1.0, std::fabs(t));
    // a Newton step of size d leaves an error of order d^2: 1e-12 suffices
    if ((newton && step <= 1e-12 * scale) || hi - lo <= 2e-15 * scale) { done = true; ++it; break; }
  }
  if (!done) { ut = 0.0; return -1; }
  T tT = t;
  if (!std::is_same<T, real>::value) {
    // derivative of the root by the implicit function theorem:
    // dt = -(dF/dparams . dparams) / (dF/dt) at fixed t
    real Ft_t;
    F_of(t, &Ft_t);
    T lnReT = log(h * u / nu);
    T FT = law_residual(law, T(t), lnReT, kappa, B);
    tT = T(t) - (FT - T(val(FT))) / Ft_t;
  }
  if (law == LAW_REICHARDT) ut = exp(tT) * nu / h;
  else ut = u / exp(tT);
  return it;
}

// Wall-model viscous flux at a wall node: returns Fv*.n_out (momentum part)
// and the wall shear vector tau_w * t (t = unit wall-parallel sample velocity).
//
// Isothermal wall (T_wall > 0; Sec. 3.1 names the wall heat flux q_w, the
// model is a reading): the Crocco-Busemann relation through the wall layer,
//   T(u) = T_w + (T_aw - T_w) u / u_s - r u^2 / (2 cp),  T_aw = T_s + r u_s^2 / (2 cp),
// which meets T_w at the wall and T_s at the sample.  The Van Driest velocity
// u_VD = int_0^{u_s} sqrt(T_w / T(u)) du, with T / T_w = 1 + b u - a^2 u^2,
// b = (T_aw - T_w) / (T_w u_s), a^2 = r / (2 cp T_w), integrates to
//   u_VD = [asin((2 a^2 u_s - b) / q) + asin(b / q)] / a,  q = sqrt(b^2 + 4 a^2),
// (b = 0: the adiabatic asin(a u_s) / a), and the wall heat flux into the
// fluid is q_w = -k_w dT/dy = -k_w (dT/du)(0) tau_w / mu_w
//   = -(cp / Pr) tau_w (T_aw - T_w) / u_s.
// qw receives q_w (0 for adiabatic walls); it is the energy component of the
// viscous flux along the outward normal.
template <class T>
int wall_flux(const Phys<T>& P, int law, const Prim<T>& s, const real nout[3], T fm[3], T tauvec[3], T* qw) {
  const real cp = P.gamma * P.R / (P.gamma - 1.0);
  const real r = std::cbrt(P.Pr);
  T un = s.u[0] * nout[0] + s.u[1] * nout[1] + s.u[2] * nout[2];
  T upar[3];
  for (int c = 0; c < 3; ++c) upar[c] = s.u[c] - un * nout[c];
  T u2 = upar[0] * upar[0] + upar[1] * upar[1] + upar[2] * upar[2];
  for (int c = 0; c < 3; ++c) { fm[c] = 0.0; tauvec[c] = 0.0; }
  *qw = T(0.0);
  if (!(val(u2) > 0.0)) return 0;
  T umag = sqrt(u2);
  T Tw, uvd;
  T Taw = s.T_ + r * u2 / (2.0 * cp);
  if (P.T_wall > 0.0) {
    Tw = T(P.T_wall);
    T b = (Taw - Tw) / (Tw * umag);
    T a2 = r / (2.0 * cp * Tw);
    T a = sqrt(a2);
    T q = sqrt(b * b + 4.0 * a2);
    uvd = (asin((2.0 * a2 * umag - b) / q) + asin(b / q)) / a;
  } else {
    Tw = Taw;  // adiabatic: the wall takes the recovery temperature
    T a = sqrt(r / (2.0 * cp * Tw));
    uvd = asin(a * umag) / a;
  }
  T rhow = s.rho * s.T_ / Tw;
  T nuw = viscosity(P, Tw) / rhow;
  T ut;
  int it = solve_utau(law, uvd, P.hwm, nuw, P.kappa, P.B, ut);
  T tw = rhow * ut * ut;
  for (int c = 0; c < 3; ++c) {
    T tc = upar[c] / umag;
    tauvec[c] = tw * tc;
    fm[c] = -tw * tc;
  }
  if (P.T_wall > 0.0) *qw = -(cp / P.Pr) * tw * (Taw - Tw) / umag;
  return it < 0 ? -1 : 0;
}

// ---------------------------------------------------------------------------
// The operator.
// ---------------------------------------------------------------------------
template <class T>
struct Work {
  std::vector<Prim<T>> q;        // [K*n3]
  std::vector<T> grad;           // [(e*n3+p)*12 + d*4 + w]
  std::vector<T> G;              // contravariant viscous flux [(e*n3+p)*15 + dir*5 + v]
  std::vector<T> wflux;          // wall-model momentum flux [slot*3]
  std::vector<T> wtau;           // wall shear vector [slot*3]
  std::vector<T> wq;             // wall heat flux into the fluid [slot]
  std::vector<int> wstat;
};

template <class T>
inline void load_U(const Mesh& M, const T* U, int e, int p, T u[5]) {
  const size_t s = (size_t)M.K * M.n3;
  for (int v = 0; v < 5; ++v) u[v] = U[v * s + (size_t)e * M.n3 + p];
}

// mirror state for a slip wall: normal velocity reversed
template <class T>
void mirror(const T U[5], const real nh[3], T Ub[5]) {
  T mn = U[1] * nh[0] + U[2] * nh[1] + U[3] * nh[2];
  Ub[0] = U[0];
  for (int c = 0; c < 3; ++c) Ub[1 + c] = U[1 + c] - 2.0 * mn * nh[c];
  Ub[4] = U[4];
}

// exterior (ghost) state of a boundary face: the wall's mirror state, the
// prescribed inflow state, or the interior density and velocity with the
// prescribed outflow pressure
template <class T>
void ghost_state(const Phys<T>& P, int code, const T U[5], const real nh[3], T Ub[5]) {
  if (code == BC_WALL) {
    mirror(U, nh, Ub);
  } else if (code == BC_INFLOW) {
    for (int v = 0; v < 5; ++v) Ub[v] = T(P.U_in[v]);
  } else {
    for (int v = 0; v < 4; ++v) Ub[v] = U[v];
    Ub[4] = P.p_out / (P.gamma - 1.0) + 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
  }
}

// master side's unit normal and surface element of face l of e at node (a,b)
static void face_geometry(const Mesh& M, int e, int l, int a, int b, real nh[3], real* s, bool* own_is_master) {
  int nb = M.nbr[e * 6 + l];
  int me = e, ml = l;
  bool master = true;
  int p = face_node(M, l, a, b);
  if (nb >= 0 && !is_master(M, e, l)) {
    neighbour_node(M, e, l, a, b, &me, &p);
    ml = M.nface[e * 6 + l];
    master = false;
  }
  const real* ja = &M.Ja[((size_t)me * M.n3 + p) * 9 + (ml / 2) * 3];
  real ss = std::sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
  for (int c = 0; c < 3; ++c) nh[c] = face_sign(ml) * ja[c] / ss;
  *s = ss;
  *own_is_master = master;
}

template <class T>
int time_derivative(const Mesh& M, const Phys<T>& P, const Opts& O, const T* U, real t, T* Ut,
                    Work<T>& W) {
  (void)t;
  const int n = M.n, n3 = M.n3, K = M.K;
  const size_t S = (size_t)K * n3;
  W.q.resize(S);
  // 3. primitives
#pragma omp parallel for schedule(static)
  for (int e = 0; e < K; ++e)
    if (in_mask(M.mask_q, e))
    for (int p = 0; p < n3; ++p) {
      T u[5]; load_U(M, U, e, p, u);
      W.q[(size_t)e * n3 + p] = prim_of(P, u);
    }
  // 4. BR1 lifting of W = (u, v, w, T), non-conservative strong form
  if (O.viscous) {
    W.grad.assign(S * 12, T(0.0));
#pragma omp parallel for schedule(static)
    for (int e = 0; e < K; ++e)
      if (in_mask(M.mask_grad, e))
      for (int p = 0; p < n3; ++p) {
        int i, j, k; ijk(M, p, i, j, k);
        const real* ja = &M.Ja[((size_t)e * n3 + p) * 9];
        const real invJ = 1.0 / M.J[(size_t)e * n3 + p];
        auto Wv = [&](int ee, int pp, int w) -> T {
          const Prim<T>& q = W.q[(size_t)ee * n3 + pp];
          return w < 3 ? q.u[w] : q.T_;
        };
        for (int w = 0; w < 4; ++w) {
          T dxi[3] = {0.0, 0.0, 0.0};
          for (int m = 0; m < n; ++m) {
            dxi[0] += M.D[i * n + m] * Wv(e, node(M, m, j, k), w);
            dxi[1] += M.D[j * n + m] * Wv(e, node(M, i, m, k), w);
            dxi[2] += M.D[k * n + m] * Wv(e, node(M, i, j, m), w);
          }
          for (int d = 0; d < 3; ++d) {
            T s = ja[0 * 3 + d] * dxi[0] + ja[1 * 3 + d] * dxi[1] + ja[2 * 3 + d] * dxi[2];
            W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w] = s * invJ;
          }
        }
        // surface corrections (W* - W) n s / w_perp for every face touching p
        int fl[6], nf = 0;
        if (i == 0) fl[nf++] = 0;
        if (i == M.N) fl[nf++] = 1;
        if (j == 0) fl[nf++] = 2;
        if (j == M.N) fl[nf++] = 3;
        if (k == 0) fl[nf++] = 4;
        if (k == M.N) fl[nf++] = 5;
        for (int f = 0; f < nf; ++f) {
          int l = fl[f], dir = l / 2;
          int a, b;
          if (dir == 0) { a = j; b = k; } else if (dir == 1) { a = i; b = k; } else { a = i; b = j; }
          real wperp = M.w[dir == 0 ? i : (dir == 1 ? j : k)];
          real ns[3];
          for (int c = 0; c < 3; ++c) ns[c] = face_sign(l) * ja[dir * 3 + c];
          T Wo[4], Wn[4];
          for (int w = 0; w < 4; ++w) Wo[w] = Wv(e, p, w);
          int nb = M.nbr[e * 6 + l];
          if (nb >= 0) {
            int q;
            neighbour_node(M, e, l, a, b, &nb, &q);
            for (int w = 0; w < 4; ++w) Wn[w] = Wv(nb, q, w);
          } else if (nb == BC_WALL) {
            // slip wall: mirror state (normal velocity reversed, same T)
            real ss = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
            real nh[3] = {ns[0] / ss, ns[1] / ss, ns[2] / ss};
            T un = Wo[0] * nh[0] + Wo[1] * nh[1] + Wo[2] * nh[2];
            for (int c = 0; c < 3; ++c) Wn[c] = Wo[c] - 2.0 * un * nh[c];
            Wn[3] = Wo[3];
          } else {
            // inflow / outflow: W of the exterior state
            real ss = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
            real nh[3] = {ns[0] / ss, ns[1] / ss, ns[2] / ss};
            T u[5], ub[5];
            load_U(M, U, e, p, u);
            ghost_state(P, nb, u, nh, ub);
            Prim<T> qb = prim_of(P, ub);
            for (int c = 0; c < 3; ++c) Wn[c] = qb.u[c];
            Wn[3] = qb.T_;
          }
          for (int w = 0; w < 4; ++w) {
            T Ws = 0.5 * (Wo[w] + Wn[w]);
            for (int d = 0; d < 3; ++d)
              W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w] += (Ws - Wo[w]) * ns[d] * invJ / wperp;
          }
        }
      }
    // contravariant viscous fluxes G^dir = Fv . Ja^dir at every node
    W.G.assign(S * 15, T(0.0));
#pragma omp parallel for schedule(static)
    for (int e = 0; e < K; ++e)
      if (in_mask(M.mask_grad, e))
      for (int p = 0; p < n3; ++p) {
        T g[3][4];
        for (int d = 0; d < 3; ++d)
          for (int w = 0; w < 4; ++w) g[d][w] = W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w];
        const real* ja = &M.Ja[((size_t)e * n3 + p) * 9];
        for (int dir = 0; dir < 3; ++dir)
          viscous_flux(P, W.q[(size_t)e * n3 + p], g, &ja[dir * 3], &W.G[((size_t)e * n3 + p) * 15 + dir * 5]);
      }
  }
  // 12. wall model at every wall face node
  W.wflux.assign((size_t)M.nwall * 3, T(0.0));
  W.wtau.assign((size_t)M.nwall * 3, T(0.0));
  W.wq.assign((size_t)M.nwall, T(0.0));
  W.wstat.assign(M.nwall, 0);
  if (O.viscous && M.nwall > 0) {
#pragma omp parallel for schedule(static)
    for (int e = 0; e < K; ++e)
      if (in_mask(M.mask_out, e))
      for (int l = 0; l < 6; ++l) {
        int s0 = M.wslot[e * 6 + l];
        if (s0 < 0) continue;
        for (int b = 0; b < n; ++b)
          for (int a = 0; a < n; ++a) {
            int slot = s0 + a + n * b;
            int es = M.ws_elem[slot];
            const real* l0 = &M.ws_l[((size_t)slot * 3 + 0) * n];
            const real* l1 = &M.ws_l[((size_t)slot * 3 + 1) * n];
            const real* l2 = &M.ws_l[((size_t)slot * 3 + 2) * n];
            T Us[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int kk = 0; kk < n; ++kk)
              for (int jj = 0; jj < n; ++jj)
                for (int ii = 0; ii < n; ++ii) {
                  T u[5]; load_U(M, U, es, node(M, ii, jj, kk), u);
                  real lw = l0[ii] * l1[jj] * l2[kk];
                  for (int v = 0; v < 5; ++v) Us[v] += lw * u[v];
                }
            Prim<T> qs = prim_of(P, Us);
            real nh[3], s; bool own;
            face_geometry(M, e, l, a, b, nh, &s, &own);
            T fm[3], tv[3], qwv;
            W.wstat[slot] = wall_flux(P, O.law, qs, nh, fm, tv, &qwv);
            W.wq[slot] = qwv;
            for (int c = 0; c < 3; ++c) {
              W.wflux[(size_t)slot * 3 + c] = fm[c];
              W.wtau[(size_t)slot * 3 + c] = tv[c];
            }
          }
      }
  }
  // 6-8. volume integral, surface integral, Jacobian scaling, source
#pragma omp parallel for schedule(static)
  for (int e = 0; e < K; ++e)
    if (in_mask(M.mask_out, e))
    for (int p = 0; p < n3; ++p) {
      int i, j, k; ijk(M, p, i, j, k);
      const int idx[3] = {i, j, k};
      T Uo[5]; load_U(M, U, e, p, Uo);
      const Prim<T>& qo = W.q[(size_t)e * n3 + p];
      const real* jao = &M.Ja[((size_t)e * n3 + p) * 9];
      T V[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int dir = 0; dir < 3; ++dir)
        for (int m = 0; m < n; ++m) {
          int pm = dir == 0 ? node(M, m, j, k) : (dir == 1 ? node(M, i, m, k) : node(M, i, j, m));
          const real Dim = M.D[idx[dir] * n + m];
          const real* jam = &M.Ja[((size_t)e * n3 + pm) * 9];
          real abar[3];
          for (int c = 0; c < 3; ++c) abar[c] = 0.5 * (jao[dir * 3 + c] + jam[dir * 3 + c]);
          T Um[5]; load_U(M, U, e, pm, Um);
          T F[5];
          twopoint_flux(O.vol_flux, P.gamma, qo, Uo, W.q[(size_t)e * n3 + pm], Um, abar, F);
          for (int v = 0; v < 5; ++v) V[v] += 2.0 * Dim * F[v];
          if (O.viscous)
            for (int v = 0; v < 5; ++v) V[v] -= Dim * W.G[((size_t)e * n3 + pm) * 15 + dir * 5 + v];
        }
      // surface terms
      int fl[6], nf = 0;
      if (i == 0) fl[nf++] = 0;
      if (i == M.N) fl[nf++] = 1;
      if (j == 0) fl[nf++] = 2;
      if (j == M.N) fl[nf++] = 3;
      if (k == 0) fl[nf++] = 4;
      if (k == M.N) fl[nf++] = 5;
      for (int f = 0; f < nf; ++f) {
        int l = fl[f], dir = l / 2;
        int a, b;
        if (dir == 0) { a = j; b = k; } else if (dir == 1) { a = i; b = k; } else { a = i; b = j; }
        real wperp = M.w[idx[dir]];
        real nh[3], s; bool own_master;
        face_geometry(M, e, l, a, b, nh, &s, &own_master);
        int nb = M.nbr[e * 6 + l];
        // master / slave states
        T Um[5], Us[5];
        Prim<T> qm, qs;
        T gm[3][4], gs[3][4];
        if (nb >= 0) {
          int q;
          neighbour_node(M, e, l, a, b, &nb, &q);
          T Un[5]; load_U(M, U, nb, q, Un);
          const Prim<T>& qn = W.q[(size_t)nb * n3 + q];
          if (own_master) {
            for (int v = 0; v < 5; ++v) { Um[v] = Uo[v]; Us[v] = Un[v]; }
            qm = qo; qs = qn;
          } else {
            for (int v = 0; v < 5; ++v) { Um[v] = Un[v]; Us[v] = Uo[v]; }
            qm = qn; qs = qo;
          }
          if (O.viscous)
            for (int d = 0; d < 3; ++d)
              for (int w = 0; w < 4; ++w) {
                T go = W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w];
                T gn = W.grad[((size_t)nb * n3 + q) * 12 + d * 4 + w];
                gm[d][w] = own_master ? go : gn;
                gs[d][w] = own_master ? gn : go;
              }
        } else {
          for (int v = 0; v < 5; ++v) Um[v] = Uo[v];
          ghost_state(P, nb, Uo, nh, Us);
          qm = qo; qs = prim_of(P, Us);
        }
        T Fi[5];
        riemann(P, O.vol_flux, O.surf_flux, qm, Um, qs, Us, nh, Fi);
        T Fv[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (O.viscous) {
          if (nb >= 0) {
            T Fa[5], Fb[5];
            viscous_flux(P, qm, gm, nh, Fa);
            viscous_flux(P, qs, gs, nh, Fb);
            for (int v = 0; v < 5; ++v) Fv[v] = 0.5 * (Fa[v] + Fb[v]);
          } else if (nb == BC_WALL) {
            int slot = M.wslot[e * 6 + l] + a + n * b;
            for (int c = 0; c < 3; ++c) Fv[1 + c] = W.wflux[(size_t)slot * 3 + c];
            Fv[4] = W.wq[slot];
          } else {
            // inflow / outflow: the interior viscous flux
            T go[3][4];
            for (int d = 0; d < 3; ++d)
              for (int w = 0; w < 4; ++w) go[d][w] = W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w];
            viscous_flux(P, qo, go, nh, Fv);
          }
        }
        const real sg = own_master ? 1.0 : -1.0;
        // own flux along own outward metric normal
        real ns[3];
        for (int c = 0; c < 3; ++c) ns[c] = face_sign(l) * jao[dir * 3 + c];
        T Fo[5];
        euler_flux(qo, Uo, ns, Fo);
        if (O.viscous) {
          T go[3][4];
          for (int d = 0; d < 3; ++d)
            for (int w = 0; w < 4; ++w) go[d][w] = W.grad[((size_t)e * n3 + p) * 12 + d * 4 + w];
          T Gv[5];
          viscous_flux(P, qo, go, ns, Gv);
          for (int v = 0; v < 5; ++v) Fo[v] -= Gv[v];
        }
        for (int v = 0; v < 5; ++v) V[v] += (sg * (Fi[v] - Fv[v]) * s - Fo[v]) / wperp;
      }
      const real invJ = 1.0 / M.J[(size_t)e * n3 + p];
      T src[5] = {0.0, P.f[0], P.f[1], P.f[2],
                  P.f[0] * qo.u[0] + P.f[1] * qo.u[1] + P.f[2] * qo.u[2]};
      for (int v = 0; v < 5; ++v) Ut[v * S + (size_t)e * n3 + p] = -V[v] * invJ + src[v];
    }
  for (int s = 0; s < M.nwall; ++s)
    if (W.wstat[s] < 0) return -1;
  return 0;
}

// mean wall shear (x component of tau_w t, quadrature-weighted over walls)
template <class T>
T wall_shear_loss(const Mesh& M, const Phys<T>& P, const Opts& O, const T* U, Work<T>& W, int* status) {
  Opts o2 = O; o2.viscous = 1;
  std::vector<T> Ut((size_t)5 * M.K * M.n3);
  *status = time_derivative(M, P, o2, U, 0.0, Ut.data(), W);
  T num = 0.0; real den = 0.0;
  for (int e = 0; e < M.K; ++e)
    for (int l = 0; l < 6; ++l) {
      int s0 = M.wslot[e * 6 + l];
      if (s0 < 0) continue;
      for (int b = 0; b < M.n; ++b)
        for (int a = 0; a < M.n; ++a) {
          real nh[3], s; bool own;
          face_geometry(M, e, l, a, b, nh, &s, &own);
          real wt = M.w[a] * M.w[b] * s;
          num += wt * W.wtau[(size_t)(s0 + a + M.n * b) * 3 + 0];
          den += wt;
        }
    }
  if (den == 0.0) return T(0.0);
  return num / den;
}

// explicit time step (reading: dt = CFL * 2/(2N+1) * min_p J / sum_dir(|u.Ja| + c |Ja|))
static real time_step(const Mesh& M, const Phys<real>& P, const real* U, real cfl) {
  real best = 1e300;
  for (int e = 0; e < M.K; ++e)
    for (int p = 0; p < M.n3; ++p) {
      real u[5]; load_U(M, U, e, p, u);
      Prim<real> q = prim_of(P, u);
      real c = std::sqrt(P.gamma * q.p / q.rho);
      const real* ja = &M.Ja[((size_t)e * M.n3 + p) * 9];
      real lam = 0.0;
      for (int d = 0; d < 3; ++d) {
        real un = q.u[0] * ja[d * 3] + q.u[1] * ja[d * 3 + 1] + q.u[2] * ja[d * 3 + 2];
        real jn = std::sqrt(ja[d * 3] * ja[d * 3] + ja[d * 3 + 1] * ja[d * 3 + 1] + ja[d * 3 + 2] * ja[d * 3 + 2]);
        lam += std::fabs(un) + c * jn;
      }
      best = std::min(best, M.J[(size_t)e * M.n3 + p] / lam);
    }
  return cfl * 2.0 / (2.0 * M.N + 1.0) * best;
}

// one LSERK4 stage: dU = A_s dU + dt Ut(U, t + c_s dt); U = U + B_s dU
template <class T>
int rk_stage(const Mesh& M, const Phys<T>& P, const Opts& O, T* U, T* dU, int s, real t, real dt,
             Work<T>& W) {
  const size_t S5 = (size_t)5 * M.K * M.n3;
  std::vector<T> Ut(S5);
  int st = time_derivative(M, P, O, U, t + RK_C[s] * dt, Ut.data(), W);
  for (size_t x = 0; x < S5; ++x) {
    dU[x] = RK_A[s] * dU[x] + dt * Ut[x];
    U[x] = U[x] + RK_B[s] * dU[x];
  }
  return st;
}

struct Ctx {
  Mesh M;
  Phys<real> P;
  Opts O;
  Work<real> W;
  Work<Dual> WD;
  std::string err;
};

}  // namespace ora

// ---------------------------------------------------------------------------
// C interface for the Python test harness (ctypes).
// phys = [gamma, R, mu, Pr, fx, fy, fz, kappa, B, hwm]
// opts = [vol_flux, surf_flux, viscous, law]
// ---------------------------------------------------------------------------
using namespace ora;

static Phys<Dual> dual_phys(const Phys<real>& P, real dk, real dB) {
  Phys<Dual> Q;
  Q.gamma = P.gamma; Q.R = P.R; Q.mu = P.mu; Q.Pr = P.Pr;
  for (int c = 0; c < 3; ++c) Q.f[c] = P.f[c];
  Q.kappa = Dual(P.kappa, dk); Q.B = Dual(P.B, dB); Q.hwm = P.hwm;
  Q.suth_S = P.suth_S; Q.T_ref = P.T_ref;
  for (int v = 0; v < 5; ++v) Q.U_in[v] = P.U_in[v];
  Q.p_out = P.p_out;
  Q.T_wall = P.T_wall;
  return Q;
}

// conversions at the C boundary (the interface is double in both builds)
static std::vector<real> to_real(const double* a, size_t n) { return std::vector<real>(a, a + n); }
static void to_double(const std::vector<real>& a, double* out) {
  for (size_t x = 0; x < a.size(); ++x) out[x] = (double)a[x];
}

extern "C" {

int ora_lgl(int N, double* xi, double* w, double* D) {
  if (N < 1 || N > 32) return -1;
  std::vector<real> x, ww, DD;
  lgl(N, x, ww, DD);
  to_double(x, xi); to_double(ww, w); to_double(DD, D);
  return 0;
}

int ora_lserk4(double* A, double* B, double* c) {
  for (int s = 0; s < 5; ++s) { A[s] = (double)RK_A[s]; B[s] = (double)RK_B[s]; c[s] = (double)RK_C[s]; }
  return 0;
}

int ora_real_digits(void) { return std::numeric_limits<real>::digits; }

void ora_set_threads(int nt) {
#ifdef _OPENMP
  omp_set_num_threads(nt > 0 ? nt : 1);
#else
  (void)nt;
#endif
}

int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static void* create_impl(int N, int K, const double* X, const int* nbr, const int* nface, const int* orient,
                         const double* phys, const int* opts, int n_sel, const int* sel, char* err, int errlen) {
  Ctx* c = new Ctx();
  Mesh& M = c->M;
  M.N = N; M.n = N + 1; M.n2 = M.n * M.n; M.n3 = M.n2 * M.n; M.K = K;
  lgl(N, M.xi, M.w, M.D);
  M.X = to_real(X, (size_t)3 * K * M.n3);
  M.nbr.assign(nbr, nbr + (size_t)6 * K);
  // neighbour faces and orientations (null: the structured default l ^ 1, 0)
  M.nface.assign((size_t)6 * K, 0);
  M.orient.assign((size_t)6 * K, 0);
  for (size_t x = 0; x < (size_t)6 * K; ++x) {
    M.nface[x] = nface ? nface[x] : (int)(x % 6) ^ 1;
    M.orient[x] = orient ? orient[x] : 0;
  }
  if (n_sel > 0) {
    // the selected elements, their neighbours, and one more ring
    M.mask_out.assign(K, 0); M.mask_grad.assign(K, 0); M.mask_q.assign(K, 0);
    for (int x = 0; x < n_sel; ++x)
      if (sel[x] >= 0 && sel[x] < K) M.mask_out[sel[x]] = 1;
    auto grow = [&](const std::vector<char>& a, std::vector<char>& b) {
      for (int e = 0; e < K; ++e)
        if (a[e]) {
          b[e] = 1;
          for (int l = 0; l < 6; ++l)
            if (M.nbr[e * 6 + l] >= 0) b[M.nbr[e * 6 + l]] = 1;
        }
    };
    grow(M.mask_out, M.mask_grad);
    grow(M.mask_grad, M.mask_q);
  }
  c->P.gamma = phys[0]; c->P.R = phys[1]; c->P.mu = phys[2]; c->P.Pr = phys[3];
  c->P.f[0] = phys[4]; c->P.f[1] = phys[5]; c->P.f[2] = phys[6];
  c->P.kappa = phys[7]; c->P.B = phys[8]; c->P.hwm = phys[9];
  c->P.suth_S = phys[10]; c->P.T_ref = phys[11];
  for (int v = 0; v < 5; ++v) c->P.U_in[v] = phys[12 + v];
  c->P.p_out = phys[17];
  c->P.T_wall = phys[18];
  c->O.vol_flux = opts[0]; c->O.surf_flux = opts[1]; c->O.viscous = opts[2]; c->O.law = opts[3];
  std::string e;
  bool ok = check_connectivity(M, e) && build_metrics(M, e) && build_wall_samples(M, c->P.hwm, e);
  if (!ok) {
    if (err && errlen > 0) { std::snprintf(err, errlen, "%s", e.c_str()); }
    delete c;
    return nullptr;
  }
  return c;
}

// nface, orient: neighbour faces and orientation codes [K][6] (see Mesh), or
// null for the structured default (face l ^ 1, orientation 0).
void* ora_create(int N, int K, const double* X, const int* nbr, const int* nface, const int* orient,
                 const double* phys, const int* opts, char* err, int errlen) {
  return create_impl(N, K, X, nbr, nface, orient, phys, opts, 0, nullptr, err, errlen);
}

// As ora_create, but Ut is evaluated only on the n_sel selected elements
// (other entries of the output stay 0).
void* ora_create_subset(int N, int K, const double* X, const int* nbr, const int* nface, const int* orient,
                        const double* phys, const int* opts, int n_sel, const int* sel, char* err, int errlen) {
  return create_impl(N, K, X, nbr, nface, orient, phys, opts, n_sel, sel, err, errlen);
}

void ora_destroy(void* h) { delete (Ctx*)h; }

int ora_get_metrics(void* h, double* Ja, double* J) {
  Ctx* c = (Ctx*)h;
  to_double(c->M.Ja, Ja);
  to_double(c->M.J, J);
  return 0;
}

int ora_num_wall(void* h) { return ((Ctx*)h)->M.nwall; }

int ora_get_wall_samples(void* h, int* elem, double* ref) {
  Ctx* c = (Ctx*)h;
  for (int s = 0; s < c->M.nwall; ++s) {
    elem[s] = c->M.ws_elem[s];
    for (int d = 0; d < 3; ++d) ref[s * 3 + d] = (double)c->M.ws_ref[s * 3 + d];
  }
  return 0;
}

// Lagrange weights of the wall-model samples: l[slot][3][n] (per reference
// direction, the weights of the n nodes at the sample's coordinate).
int ora_get_wall_weights(void* h, double* l) {
  Ctx* c = (Ctx*)h;
  const size_t cnt = (size_t)c->M.nwall * 3 * c->M.n;
  for (size_t x = 0; x < cnt; ++x) l[x] = (double)c->M.ws_l[x];
  return 0;
}

static size_t state_size(const Ctx* c) { return (size_t)5 * c->M.K * c->M.n3; }

int ora_time_derivative(void* h, const double* U, double t, double* Ut) {
  Ctx* c = (Ctx*)h;
  const size_t S5 = state_size(c);
  std::vector<real> u = to_real(U, S5), ut(S5);
  int st = time_derivative(c->M, c->P, c->O, u.data(), t, ut.data(), c->W);
  to_double(ut, Ut);
  return st;
}

// Wall heat flux q_w into the fluid at every wall slot for state U (tests).
int ora_wall_heat(void* h, const double* U, double* qw) {
  Ctx* c = (Ctx*)h;
  const size_t S5 = state_size(c);
  std::vector<real> u = to_real(U, S5), ut(S5);
  int st = time_derivative(c->M, c->P, c->O, u.data(), 0.0, ut.data(), c->W);
  for (int s2 = 0; s2 < c->M.nwall; ++s2) qw[s2] = (double)c->W.wq[s2];
  return st;
}

// Jacobian-vector product: dUt = (dUt/dU) dU + (dUt/dkappa) dk + (dUt/dB) dB
int ora_jvp(void* h, const double* U, const double* dU, double dk, double dB, double t, double* Ut,
            double* dUt) {
  Ctx* c = (Ctx*)h;
  const size_t S5 = state_size(c);
  std::vector<Dual> Ud(S5), Utd(S5);
  for (size_t x = 0; x < S5; ++x) Ud[x] = Dual(U[x], dU ? dU[x] : 0.0);
  Phys<Dual> P = dual_phys(c->P, dk, dB);
  int st = time_derivative(c->M, P, c->O, Ud.data(), t, Utd.data(), c->WD);
  for (size_t x = 0; x < S5; ++x) { Ut[x] = (double)Utd[x].v; dUt[x] = (double)Utd[x].d; }
  return st;
}

int ora_rk_stage(void* h, double* U, double* dU, int s, double t, double dt) {
  Ctx* c = (Ctx*)h;
  if (s < 0 || s > 4) return -1;
  const size_t S5 = state_size(c);
  std::vector<real> u = to_real(U, S5), du = to_real(dU, S5);
  int st = rk_stage(c->M, c->P, c->O, u.data(), du.data(), s, t, dt, c->W);
  to_double(u, U); to_double(du, dU);
  return st;
}

int ora_rk_steps(void* h, double* U, double t0, double dt, int nsteps) {
  Ctx* c = (Ctx*)h;
  const size_t S5 = state_size(c);
  std::vector<real> u = to_real(U, S5), du(S5, 0.0);
  int st = 0;
  for (int it = 0; it < nsteps; ++it) {
    std::fill(du.begin(), du.end(), real(0.0));
    for (int s = 0; s < 5; ++s) st |= rk_stage(c->M, c->P, c->O, u.data(), du.data(), s, t0 + it * dt, dt, c->W);
  }
  to_double(u, U);
  return st;
}

int ora_dt(void* h, const double* U, double cfl, double* dt) {
  Ctx* c = (Ctx*)h;
  std::vector<real> u = to_real(U, state_size(c));
  *dt = (double)time_step(c->M, c->P, u.data(), cfl);
  return 0;
}

int ora_wall_shear(void* h, const double* U, double* loss) {
  Ctx* c = (Ctx*)h;
  int st = 0;
  std::vector<real> u = to_real(U, state_size(c));
  *loss = (double)wall_shear_loss(c->M, c->P, c->O, u.data(), c->W, &st);
  return st;
}

// Forward-mode derivative of the mean wall shear after nsteps LSERK4 steps
// from U0 along (dU0, dk, dB).
int ora_rollout_jvp(void* h, const double* U0, const double* dU0, double dk, double dB, int nsteps,
                    double dt, double* loss, double* dloss) {
  Ctx* c = (Ctx*)h;
  const size_t S5 = state_size(c);
  std::vector<Dual> U(S5), dU(S5);
  for (size_t x = 0; x < S5; ++x) U[x] = Dual(U0[x], dU0 ? dU0[x] : 0.0);
  Phys<Dual> P = dual_phys(c->P, dk, dB);
  int st = 0;
  for (int it = 0; it < nsteps; ++it) {
    std::fill(dU.begin(), dU.end(), Dual(0.0));
    for (int s = 0; s < 5; ++s) st |= rk_stage(c->M, P, c->O, U.data(), dU.data(), s, it * dt, dt, c->WD);
  }
  int st2 = 0;
  Dual L = wall_shear_loss(c->M, P, c->O, U.data(), c->WD, &st2);
  *loss = (double)L.v; *dloss = (double)L.d;
  return st | st2;
}

// kinetic energy (1/|Omega|) sum w J rho |u|^2 / 2
int ora_kinetic_energy(void* h, const double* U, double* ke) {
  Ctx* c = (Ctx*)h;
  const Mesh& M = c->M;
  real num = 0.0, vol = 0.0;
  for (int e = 0; e < M.K; ++e)
    for (int p = 0; p < M.n3; ++p) {
      int i, j, k; ijk(M, p, i, j, k);
      real wJ = M.w[i] * M.w[j] * M.w[k] * M.J[(size_t)e * M.n3 + p];
      real u[5];
      for (int v = 0; v < 5; ++v) u[v] = U[(size_t)v * M.K * M.n3 + (size_t)e * M.n3 + p];
      num += wJ * 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
      vol += wJ;
    }
  *ke = (double)(num / vol);
  return 0;
}

// Wall law solve for tests: returns u_tau and iterations (law pins).
int ora_solve_utau(int law, double u, double h, double nu, double kappa, double B, double* ut) {
  real x;
  int it = solve_utau<real>(law, u, h, nu, kappa, B, x);
  *ut = (double)x;
  return it;
}

double ora_law_value(int law, double x, double kappa, double B) {
  return (double)(law == LAW_REICHARDT ? reichardt<real>(x, kappa, B) : spalding<real>(x, kappa, B));
}

// Wall flux at one sample state (tests): U5 conservative, nout unit normal.
int ora_wall_flux(const double* phys, int law, const double* U5, const double* nout, double* fm, double* tau,
                  double* qw) {
  Phys<real> P;
  P.gamma = phys[0]; P.R = phys[1]; P.mu = phys[2]; P.Pr = phys[3];
  P.kappa = phys[7]; P.B = phys[8]; P.hwm = phys[9];
  P.suth_S = phys[10]; P.T_ref = phys[11]; P.T_wall = phys[18];
  real u[5], nh[3], f[3], t[3], q_w;
  for (int v = 0; v < 5; ++v) u[v] = U5[v];
  for (int c = 0; c < 3; ++c) nh[c] = nout[c];
  Prim<real> q = prim_of(P, u);
  int st = wall_flux(P, law, q, nh, f, t, &q_w);
  for (int c = 0; c < 3; ++c) { fm[c] = (double)f[c]; tau[c] = (double)t[c]; }
  if (qw) *qw = (double)q_w;
  return st;
}

// Dynamic viscosity at temperature T (tests).
double ora_viscosity(const double* phys, double T) {
  Phys<real> P;
  P.mu = phys[2]; P.suth_S = phys[10]; P.T_ref = phys[11];
  return (double)viscosity(P, (real)T);
}

// Single numerical flux evaluation (tests): returns F*(UL, UR; nh).
int ora_riemann(const double* phys, int vol_kind, int kind, const double* UL, const double* UR,
                const double* nh, double* F) {
  Phys<real> P;
  P.gamma = phys[0]; P.R = phys[1];
  real ul[5], ur[5], n3[3], f[5];
  for (int v = 0; v < 5; ++v) { ul[v] = UL[v]; ur[v] = UR[v]; }
  for (int c = 0; c < 3; ++c) n3[c] = nh[c];
  Prim<real> L = prim_of(P, ul), R = prim_of(P, ur);
  riemann(P, vol_kind, kind, L, ul, R, ur, n3, f);
  for (int v = 0; v < 5; ++v) F[v] = (double)f[v];
  return 0;
}

}  // extern "C"
