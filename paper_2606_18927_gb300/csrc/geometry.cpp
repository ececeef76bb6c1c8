// geometry.cpp -- host-side mesh preprocessing (see geometry.h).
#include "geometry.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>
#include <thread>

namespace dg {

// ---------------------------------------------------------------------------
// Double-double arithmetic (Dekker / Knuth error-free transformations): the
// nodes, the derivative matrix and the metric terms are computed with a
// ~106-bit significand and rounded to double once.  The curl-form metrics
// chain two derivative applications (entries up to N(N+1)/4) and lose
// ~|D|^2 ulps in plain double; the kernels multiply them by O(p0) and O(h)
// flux values at low Mach number.
// ---------------------------------------------------------------------------
struct dd {
  double hi = 0.0, lo = 0.0;
  dd() = default;
  dd(double h) : hi(h), lo(0.0) {}
  dd(double h, double l) : hi(h), lo(l) {}
};
static inline dd two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
static inline dd fast_two_sum(double a, double b) {
  const double s = a + b;
  return dd(s, b - (s - a));
}
static inline dd two_prod(double a, double b) {
  const double p = a * b;
  return dd(p, std::fma(a, b, -p));
}
static inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
static inline dd operator-(dd a, dd b) { return a + (-b); }
static inline dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd operator/(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = a - b * dd(q1);
  const double q2 = r.hi / b.hi;
  r = r - b * dd(q2);
  const double q3 = r.hi / b.hi;
  return fast_two_sum(q1, q2) + dd(q3);
}
static inline dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd(0.0);
  const double x = std::sqrt(a.hi);
  const dd y(x);
  return y + (a - y * y) / dd(2.0 * x);  // one Newton step
}

static void run_parallel(int count, const std::function<void(int, int)>& fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<unsigned>(hw ? hw : 1, 64);
  if (count < 64 || nt <= 1) { fn(0, count); return; }
  std::vector<std::thread> pool;
  const int chunk = (count + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int b = t * chunk, e = std::min(count, b + chunk);
    if (b < e) pool.emplace_back(fn, b, e);
  }
  for (auto& th : pool) th.join();
}

static void legendre_pair(int N, dd x, dd* PN, dd* PNm1) {
  dd a(1.0), b = x;  // P_0, P_1
  if (N == 0) { *PN = dd(1.0); *PNm1 = dd(0.0); return; }
  for (int k = 2; k <= N; ++k) {
    dd c = (dd(2.0 * k - 1.0) * x * b - dd(k - 1.0) * a) / dd((double)k);
    a = b; b = c;
  }
  *PN = b; *PNm1 = a;
}

// nodes, weights and D in double-double (Dd) and rounded (x, w, D)
static void make_basis_dd(int N, std::vector<dd>& x, std::vector<dd>& w, std::vector<dd>& D) {
  const int n = N + 1;
  x.assign(n, dd(0.0)); w.assign(n, dd(0.0)); D.assign(n * n, dd(0.0));
  // Chebyshev-Gauss-Lobatto start, then x <- x - (x P_N - P_{N-1}) / ((N+1) P_N)
  // (a Newton step on (1 - x^2) P_N'(x) written through the recurrence).
  for (int i = 1; i < N; ++i) {
    dd xi(std::cos(M_PI * (N - i) / N));
    for (int it = 0; it < 100; ++it) {
      dd P, Q;
      legendre_pair(N, xi, &P, &Q);
      dd dx = (xi * P - Q) / (dd(N + 1.0) * P);
      xi = xi - dx;
      if (std::fabs(dx.hi) <= 1e-32) break;
    }
    x[i] = xi;
  }
  x[0] = dd(-1.0); x[N] = dd(1.0);
  for (int i = 0; i < n / 2; ++i) {  // exact symmetry
    dd m = (x[N - i] - x[i]) * dd(0.5);
    x[i] = -m; x[N - i] = m;
  }
  if (n % 2) x[N / 2] = dd(0.0);
  std::vector<dd> PN(n);
  for (int i = 0; i < n; ++i) {
    dd P, Q;
    legendre_pair(N, x[i], &P, &Q);
    PN[i] = P;
    w[i] = dd(2.0) / (dd(N * (N + 1.0)) * P * P);
  }
  // closed form: D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j,
  // D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j) D[i * n + j] = PN[i] / (PN[j] * (x[i] - x[j]));
  D[0] = dd(-N * (N + 1.0) / 4.0);
  D[N * n + N] = dd(N * (N + 1.0) / 4.0);
}

Basis make_basis(int N) {
  Basis B;
  B.N = N; B.n = N + 1;
  std::vector<dd> x, w, D;
  make_basis_dd(N, x, w, D);
  B.x.resize(B.n); B.w.resize(B.n); B.D.resize(B.n * B.n);
  for (int i = 0; i < B.n; ++i) { B.x[i] = x[i].hi; B.w[i] = w[i].hi; }
  for (int i = 0; i < B.n * B.n; ++i) B.D[i] = D[i].hi;
  return B;
}

void lagrange_at(const Basis& b, double s, double* l) {
  const int n = b.n;
  // barycentric weights
  double num = 0.0;
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (b.x[j] - b.x[k]);
  for (int j = 0; j < n; ++j)
    if (s == b.x[j]) {
      for (int k = 0; k < n; ++k) l[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  for (int j = 0; j < n; ++j) {
    l[j] = lam[j] / (s - b.x[j]);
    num += l[j];
  }
  for (int j = 0; j < n; ++j) l[j] /= num;
}

// --------------------------------------------------------------------------
static bool metrics(Geometry& g, std::string& err) {
  const int n = g.n, n3 = g.n3, K = g.K;
  std::vector<dd> bx, bw, D;
  make_basis_dd(g.N, bx, bw, D);
  g.Ja.assign((size_t)K * n3 * 9, 0.0);
  g.J.assign((size_t)K * n3, 0.0);
  std::vector<int> bad(K, 0);
  run_parallel(K, [&](int e0, int e1) {
    std::vector<dd> xl(3 * n3), dx(9 * n3), v(3 * n3);
    auto dxi = [&](const dd* f, int dir, int p) {
      const int i = p % n, j = (p / n) % n, k = p / (n * n);
      dd s(0.0);
      if (dir == 0) for (int m = 0; m < n; ++m) s = s + D[i * n + m] * f[m + n * (j + n * k)];
      else if (dir == 1) for (int m = 0; m < n; ++m) s = s + D[j * n + m] * f[i + n * (m + n * k)];
      else for (int m = 0; m < n; ++m) s = s + D[k * n + m] * f[i + n * (j + n * m)];
      return s;
    };
    for (int e = e0; e < e1; ++e) {
      // element-local coordinates (relative to the element's first node): the
      // curl form and the derivatives are unchanged by a constant shift
      for (int c = 0; c < 3; ++c) {
        const double x0 = g.X[(size_t)c * K * n3 + (size_t)e * n3];
        for (int p = 0; p < n3; ++p) xl[c * n3 + p] = two_sum(g.X[(size_t)c * K * n3 + (size_t)e * n3 + p], -x0);
      }
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d)
          for (int p = 0; p < n3; ++p) dx[(c * 3 + d) * n3 + p] = dxi(&xl[c * n3], d, p);
      for (int p = 0; p < n3; ++p) {
        dd m[3][3];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) m[c][d] = dx[(c * 3 + d) * n3 + p];
        const dd det = m[0][0] * (m[1][1] * m[2][2] - m[2][1] * m[1][2]) -
                       m[1][0] * (m[0][1] * m[2][2] - m[2][1] * m[0][2]) +
                       m[2][0] * (m[0][1] * m[1][2] - m[1][1] * m[0][2]);
        g.J[(size_t)e * n3 + p] = det.hi;
        if (!(det.hi > 0.0)) bad[e] = 1;
      }
      // Ja^i_c = -(curl_xi (x_l grad_xi x_m))_i with (c, m, l) cyclic
      for (int c = 0; c < 3; ++c) {
        const int mm = (c + 1) % 3, ll = (c + 2) % 3;
        for (int d = 0; d < 3; ++d)
          for (int p = 0; p < n3; ++p) v[d * n3 + p] = xl[ll * n3 + p] * dx[(mm * 3 + d) * n3 + p];
        for (int p = 0; p < n3; ++p) {
          double* ja = &g.Ja[((size_t)e * n3 + p) * 9];
          ja[0 * 3 + c] = (dxi(&v[1 * n3], 2, p) - dxi(&v[2 * n3], 1, p)).hi;
          ja[1 * 3 + c] = (dxi(&v[2 * n3], 0, p) - dxi(&v[0 * n3], 2, p)).hi;
          ja[2 * 3 + c] = (dxi(&v[0 * n3], 1, p) - dxi(&v[1 * n3], 0, p)).hi;
        }
      }
    }
  });
  for (int e = 0; e < K; ++e)
    if (bad[e]) {
      char buf[128];
      std::snprintf(buf, sizeof buf, "non-positive Jacobian in element %d", e);
      err = buf;
      return false;
    }
  return true;
}

static bool faces(Geometry& g, std::string& err) {
  const int n = g.n, n2 = g.n2, n3 = g.n3, K = g.K;
  double scale = 1.0;
  for (double x : g.X) scale = std::max(scale, std::fabs(x));
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l) {
      const int nb = g.nbr[e * 6 + l];
      if ((nb < BC_CODE_MIN && nb > HALO_BASE) || nb >= K) { err = "neighbour index out of range"; return false; }
      if (nb < 0) continue;
      const int l2 = g.nface[e * 6 + l], o = g.orient[e * 6 + l];
      if (l2 < 0 || l2 > 5 || o < 0 || o > 7) { err = "bad neighbour face or orientation code"; return false; }
      if (nb == e && l2 == l) { err = "a face cannot be its own neighbour"; return false; }
      if (g.nbr[nb * 6 + l2] != e || g.nface[nb * 6 + l2] != l || g.orient[nb * 6 + l2] != orient_inverse(o)) {
        err = "connectivity is not reciprocal";
        return false;
      }
      // the two sides must coincide up to a single translation
      double sh[3] = {0, 0, 0};
      for (int ab = 0; ab < n2; ++ab) {
        int a2, b2;
        orient_map(o, n - 1, ab % n, ab / n, &a2, &b2);
        const int p = face_node(n, l, ab % n, ab / n), q = face_node(n, l2, a2, b2);
        for (int c = 0; c < 3; ++c) {
          const double d = g.X[(size_t)c * K * n3 + (size_t)nb * n3 + q] - g.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
          if (ab == 0) sh[c] = d;
          else if (std::fabs(d - sh[c]) > 1e-9 * scale) {
            err = "face nodes of neighbouring elements do not match";
            return false;
          }
        }
      }
    }
  g.faces.clear();
  g.elem_face.assign((size_t)K * 6, -1);
  // interior faces, listed from their masters in (element, face) order
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l) {
      const int nb = g.nbr[e * 6 + l];
      if (nb < 0) continue;
      const int l2 = g.nface[e * 6 + l], o = g.orient[e * 6 + l];
      if (!face_is_master(e, l, nb, l2)) continue;
      const int id = (int)g.faces.size();
      g.faces.push_back({e, l, nb, l2, o});
      g.elem_face[e * 6 + l] = 16 * id;
      g.elem_face[nb * 6 + l2] = 16 * id + 2 * orient_inverse(o) + 1;
    }
  g.n_interior = (int)g.faces.size();
  // boundary faces: walls first, then inflow / outflow faces (eS = the code)
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l)
      if (g.nbr[e * 6 + l] == BC_CODE_WALL) {
        const int id = (int)g.faces.size();
        g.faces.push_back({e, l, BC_CODE_WALL, -1, 0});
        g.elem_face[e * 6 + l] = 16 * id;
      }
  g.n_wall = (int)g.faces.size() - g.n_interior;
  for (int e = 0; e < K; ++e)
    for (int l = 0; l < 6; ++l) {
      const int nb = g.nbr[e * 6 + l];
      if (nb < 0 && nb != BC_CODE_WALL && nb > HALO_BASE) {
        const int id = (int)g.faces.size();
        g.faces.push_back({e, l, nb, -1, 0});
        g.elem_face[e * 6 + l] = 16 * id;
      }
    }
  g.n_bc = (int)g.faces.size() - g.n_interior - g.n_wall;
  // halo faces, in halo-index order.  The local element is the face's master
  // by the rule of face_is_master: when its local face and the remote one
  // (nface) differ in parity, the odd one; else the partitioner decides from
  // the global element ids and marks the master side with bit 3 (value 8)
  // of the orientation code.  Traces cross in the master's face-node order.
  {
    std::vector<int> hid;
    for (int e = 0; e < K; ++e)
      for (int l = 0; l < 6; ++l)
        if (g.nbr[e * 6 + l] <= HALO_BASE) hid.push_back(e * 6 + l);
    std::sort(hid.begin(), hid.end(), [&](int a, int b) { return g.nbr[a] > g.nbr[b]; });
    for (size_t i = 0; i < hid.size(); ++i) {
      const int e = hid[i] / 6, l = hid[i] % 6, h = HALO_BASE - g.nbr[hid[i]];
      if (h != (int)i) { err = "halo face indices must be 0 .. n_halo-1, each once"; return false; }
      const int id = (int)g.faces.size();
      const int l2 = g.nface[e * 6 + l], oc = g.orient[e * 6 + l];
      if (l2 < 0 || l2 > 5 || oc < 0 || oc > 15) { err = "bad halo face or orientation code"; return false; }
      const int master = ((l & 1) != (l2 & 1)) ? (l & 1) : ((oc >> 3) & 1);
      const int o_own = master ? 0 : (oc & 7);  // own face nodes -> the master's
      g.faces.push_back({e, l, h, master, o_own});
      g.elem_face[e * 6 + l] = 16 * id + 2 * o_own + (master ? 0 : 1);
    }
    g.n_halo = (int)hid.size();
  }
  const size_t F = g.faces.size();
  g.fgeo.assign(4 * F * n2, 0.0);
  const size_t F_halo0 = F - (size_t)g.n_halo;
  for (size_t f = 0; f < F; ++f) {
    const Face& fc = g.faces[f];
    // the master's outward normal; a halo face whose local element is the
    // slave takes the negated own normal until the master's is installed
    double sgn = (fc.lM & 1) ? 1.0 : -1.0;
    const bool halo_slave = f >= F_halo0 && fc.lS == 0;
    if (halo_slave) sgn = -sgn;
    for (int ab = 0; ab < n2; ++ab) {
      // (a halo face's slave side: its own node at the master's index ab)
      int a = ab % n, b = ab / n;
      if (halo_slave) orient_map(orient_inverse(fc.o), n - 1, ab % n, ab / n, &a, &b);
      const int p = face_node(n, fc.lM, a, b);
      const double* ja = &g.Ja[((size_t)fc.eM * n3 + p) * 9 + (fc.lM / 2) * 3];
      const dd s = dd_sqrt(dd(ja[0]) * dd(ja[0]) + dd(ja[1]) * dd(ja[1]) + dd(ja[2]) * dd(ja[2]));
      for (int c = 0; c < 3; ++c) g.fgeo[(size_t)c * F * n2 + f * n2 + ab] = sgn * (dd(ja[c]) / s).hi;
      g.fgeo[3 * F * n2 + f * n2 + ab] = s.hi;
    }
  }
  return true;
}

// Newton on the element map x(r) = sum X_ijk l_i(r0) l_j(r1) l_k(r2); the
// derivative of the interpolant uses l_j'(s) = sum_k l_k(s) D_kj.
static bool invert_map(const Geometry& g, int e, const double xs[3], double r[3]) {
  const int n = g.n, n3 = g.n3, K = g.K;
  const std::vector<double>& D = g.basis.D;
  std::vector<double> L(3 * n), dL(3 * n);
  r[0] = r[1] = r[2] = 0.0;
  for (int it = 0; it < 80; ++it) {
    for (int a = 0; a < 3; ++a) {
      lagrange_at(g.basis, r[a], &L[a * n]);
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += L[a * n + k] * D[k * n + j];
        dL[a * n + j] = s;
      }
    }
    double x[3] = {0, 0, 0}, A[3][3] = {{0}};
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int p = i + n * (j + n * k);
          const double l0 = L[i], l1 = L[n + j], l2 = L[2 * n + k];
          for (int c = 0; c < 3; ++c) {
            const double X = g.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
            x[c] += X * l0 * l1 * l2;
            A[c][0] += X * dL[i] * l1 * l2;
            A[c][1] += X * l0 * dL[n + j] * l2;
            A[c][2] += X * l0 * l1 * dL[2 * n + k];
          }
        }
    // r += A^{-1} (xs - x) by the adjugate
    double inv[3][3];
    inv[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    inv[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    inv[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    inv[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    inv[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    inv[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    inv[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    inv[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    inv[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    const double det = A[0][0] * inv[0][0] + A[0][1] * inv[1][0] + A[0][2] * inv[2][0];
    if (det == 0.0 || !std::isfinite(det)) return false;
    const double res[3] = {xs[0] - x[0], xs[1] - x[1], xs[2] - x[2]};
    double step = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double d = (inv[a][0] * res[0] + inv[a][1] * res[1] + inv[a][2] * res[2]) / det;
      r[a] = std::min(3.0, std::max(-3.0, r[a] + d));
      step = std::max(step, std::fabs(d));
    }
    if (step < 1e-15) break;
  }
  return true;
}

static bool wall_samples(Geometry& g, double hwm, std::string& err) {
  const int n = g.n, n2 = g.n2, n3 = g.n3, K = g.K;
  const int F = (int)g.faces.size();
  g.ws_elem.assign((size_t)g.n_wall * n2, -1);
  g.ws_ref.assign((size_t)g.n_wall * n2 * 3, 0.0);
  g.ws_lag.assign((size_t)g.n_wall * n2 * 3 * n, 0.0);
  if (g.n_wall == 0) return true;
  std::vector<double> lo((size_t)K * 3, 1e300), hi((size_t)K * 3, -1e300);
  for (int e = 0; e < K; ++e)
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < n3; ++p) {
        const double x = g.X[(size_t)c * K * n3 + (size_t)e * n3 + p];
        lo[e * 3 + c] = std::min(lo[e * 3 + c], x);
        hi[e * 3 + c] = std::max(hi[e * 3 + c], x);
      }
  for (int wf = 0; wf < g.n_wall; ++wf) {
    const int f = g.n_interior + wf;
    const Face& fc = g.faces[f];
    // candidate elements: neighbourhood of the wall element (3 layers)
    std::vector<int> cand{fc.eM};
    for (int layer = 0; layer < 3; ++layer) {
      const size_t m = cand.size();
      for (size_t c = 0; c < m; ++c)
        for (int l = 0; l < 6; ++l) {
          const int nb = g.nbr[cand[c] * 6 + l];
          if (nb >= 0 && std::find(cand.begin(), cand.end(), nb) == cand.end()) cand.push_back(nb);
        }
    }
    std::sort(cand.begin(), cand.end());
    // search order: the wall element's column first (the wall element, then
    // its neighbours across the faces opposite the wall, up to 3 layers; a
    // choice that does not depend on element numbering or partitioning), then
    // the remaining candidates by ascending index
    std::vector<int> order;
    for (int c = fc.eM, layer = 0, lin = fc.lM; c >= 0 && layer < 4; ++layer) {
      order.push_back(c);
      // the face opposite the one the column entered this element by
      const int lout = lin ^ 1, nxt = g.nbr[c * 6 + lout];
      if (nxt >= 0) lin = g.nface[c * 6 + lout];
      c = nxt;
    }
    for (int c : cand)
      if (std::find(order.begin(), order.end(), c) == order.end()) order.push_back(c);
    for (int ab = 0; ab < n2; ++ab) {
      const int p = face_node(n, fc.lM, ab % n, ab / n);
      double xs[3];
      for (int c = 0; c < 3; ++c)
        xs[c] = g.X[(size_t)c * K * n3 + (size_t)fc.eM * n3 + p] - hwm * g.fgeo[(size_t)c * F * n2 + (size_t)f * n2 + ab];
      // the first element in that order containing the point (within 1e-8 in
      // the reference coordinates): points on a shared face get one element
      int best = -1;
      double br[3] = {0, 0, 0};
      for (int e : order) {
        bool in = true;
        for (int c = 0; c < 3; ++c) {
          const double pad = 0.05 * (hi[e * 3 + c] - lo[e * 3 + c]) + 1e-12;
          in = in && xs[c] >= lo[e * 3 + c] - pad && xs[c] <= hi[e * 3 + c] + pad;
        }
        if (!in) continue;
        double r[3];
        if (!invert_map(g, e, xs, r)) continue;
        const double mx = std::max(std::fabs(r[0]), std::max(std::fabs(r[1]), std::fabs(r[2])));
        if (mx <= 1.0 + 1e-8) {
          best = e;
          br[0] = r[0]; br[1] = r[1]; br[2] = r[2];
          break;
        }
      }
      if (best < 0) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "wall-model sample point of element %d is not inside the mesh", fc.eM);
        err = buf;
        return false;
      }
      const size_t slot = (size_t)wf * n2 + ab;
      g.ws_elem[slot] = best;
      for (int a = 0; a < 3; ++a) {
        g.ws_ref[slot * 3 + a] = br[a];
        lagrange_at(g.basis, br[a], &g.ws_lag[(slot * 3 + a) * n]);
      }
    }
  }
  return true;
}

std::string build_geometry(Geometry& g, int N, int K, const double* X, const int* nbr, const int* nface,
                           const int* orient, double hwm) {
  g.N = N; g.n = N + 1; g.n2 = g.n * g.n; g.n3 = g.n2 * g.n; g.K = K;
  g.basis = make_basis(N);
  g.X.assign(X, X + (size_t)3 * K * g.n3);
  g.nbr.assign(nbr, nbr + (size_t)6 * K);
  g.nface.resize((size_t)6 * K);
  g.orient.resize((size_t)6 * K);
  for (size_t x = 0; x < (size_t)6 * K; ++x) {
    g.nface[x] = nface ? nface[x] : (int)(x % 6) ^ 1;
    g.orient[x] = orient ? orient[x] : 0;
  }
  std::string err;
  if (!metrics(g, err)) return err;
  if (!faces(g, err)) return err;
  if (!wall_samples(g, hwm, err)) return err;
  return "";
}

}  // namespace dg
