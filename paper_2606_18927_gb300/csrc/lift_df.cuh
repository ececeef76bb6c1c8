// BR1 lifting, viscous flux and weak viscous divergence of the FP64 operator
// at N = 7 in double-float arithmetic: every FP64 value of the kernel is an
// unevaluated sum hi + lo of two floats, and the arithmetic is built from
// error-free transformations on the FP32 pipe (which on GB300 issues 64 times
// as many lanes per clock as the FP64 pipe):
//   TwoSum (Knuth): s = a + b, e = (a - (s - b')) + (b - b'), b' = s - a;
//   TwoProd by FMA: p = a b, e = fma(a, b, -p);
//   products of two double-floats (Dekker's product with the cross terms
//   a_hi b_lo + a_lo b_hi folded into the FMA), and sums of products
//   accumulated as in Ogita, Rump and Oishi's Dot2 (the high parts by
//   TwoSum, every rounding error and low part into a second float).
// The relative rounding of a double-float operation is about 2^-47 against
// FP64's 2^-53.  The viscous terms are a small part of Ut (1/Re), so their
// rounding at that level stays far below the operator's FP64 parity bound;
// the temperature is lifted relative to T_ref = p_ref / (rho_ref R) (its
// gradient is the same) so that no O(T) value is rounded.  The inviscid
// volume term, whose rounding the derivative amplifies against Ut, stays in
// FP64.
#pragma once

#include "kernels.cuh"

namespace dg {

struct DFl {
  float hi, lo;
};

__device__ __forceinline__ DFl df_of(double x) {
  float lo;
  const float hi = d2f_bits(x, &lo);
  return DFl{hi, lo};
}

__device__ __forceinline__ double df_to(DFl a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, t) with |t| small against |s|: the nearest float and the remainder
__device__ __forceinline__ DFl df_norm(float s, float t) {
  const float h = __fadd_rn(s, t);
  return DFl{h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ DFl df_add(DFl a, DFl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DFl df_neg(DFl a) { return DFl{-a.hi, -a.lo}; }
__device__ __forceinline__ DFl df_sub(DFl a, DFl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DFl df_mul(DFl a, DFl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}

// sum of products: s the TwoSum-exact sum of the products' high parts, t the
// rest (product errors, cross terms, the sums' errors)
struct DFAcc {
  float s, t;
};

__device__ __forceinline__ void acc_fma(DFAcc& A, DFl c, DFl x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, e);
  e = __fmaf_rn(c.lo, x.hi, e);
  float s, r;
  two_sum(A.s, p, s, r);
  A.s = s;
  A.t = __fadd_rn(A.t, __fadd_rn(e, r));
}

__device__ __forceinline__ void acc_add(DFAcc& A, DFl x) {
  float s, r;
  two_sum(A.s, x.hi, s, r);
  A.s = s;
  A.t = __fadd_rn(A.t, __fadd_rn(x.lo, r));
}

__device__ __forceinline__ DFl acc_val(const DFAcc& A) { return df_norm(A.s, A.t); }

__device__ __forceinline__ DFl dot3(DFl a0, DFl b0, DFl a1, DFl b1, DFl a2, DFl b2) {
  DFAcc A{0.f, 0.f};
  acc_fma(A, a0, b0);
  acc_fma(A, a1, b1);
  acc_fma(A, a2, b2);
  return acc_val(A);
}

__device__ __forceinline__ DFl df_ld(const float2* p) {
  const float2 v = *p;
  return DFl{v.x, v.y};
}
__device__ __forceinline__ void df_st(float2* p, DFl a) { *p = make_float2(a.hi, a.lo); }

// two double-floats side by side: (hi0, hi1) and (lo0, lo1)
struct DF2 {
  f32x2 hi, lo;
};

// TwoSum and its mirror TwoDiff (a - b, the TwoSum of a and -b), lane by lane
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2& s, f32x2& e) {
  s = add2(a, b);
  const f32x2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_diff2(f32x2 a, f32x2 b, f32x2& s, f32x2& e) {
  s = sub2(a, b);
  const f32x2 bb = sub2(s, a);
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
__device__ __forceinline__ DF2 df_norm2(f32x2 s, f32x2 t) {
  const f32x2 h = add2(s, t);
  return DF2{h, sub2(t, sub2(h, s))};
}
__device__ __forceinline__ DF2 df_add2(DF2 a, DF2 b) {
  f32x2 s, e;
  two_sum2(a.hi, b.hi, s, e);
  return df_norm2(s, add2(e, add2(a.lo, b.lo)));
}
__device__ __forceinline__ DF2 df_sub2(DF2 a, DF2 b) {
  f32x2 s, e;
  two_diff2(a.hi, b.hi, s, e);
  return df_norm2(s, add2(e, sub2(a.lo, b.lo)));
}

// Dot2 step A += c x with the coefficient given as (c_hi, -c_hi, -c_lo), both
// lanes alike: the product's error is formed negated, -(c x - p) =
// fma(-c_hi, x_hi, p) - c_hi x_lo - c_lo x_hi, which rounds exactly as the
// scalar acc_fma's positive form (rounding to nearest is symmetric)
struct DFAcc2 {
  f32x2 s, t;
};
__device__ __forceinline__ void acc_fma2(DFAcc2& A, f32x2 ch, f32x2 chn, f32x2 cln, DF2 x) {
  const f32x2 p = mul2(ch, x.hi);
  f32x2 en = fma2(chn, x.hi, p);
  en = fma2(chn, x.lo, en);
  en = fma2(cln, x.hi, en);
  f32x2 s, r;
  two_sum2(A.s, p, s, r);
  A.s = s;
  A.t = add2(A.t, sub2(r, en));
}

__device__ __forceinline__ DF2 df2_ld(const float4* p) {
  const float4 v = *p;
  return DF2{pk2(v.x, v.y), pk2(v.z, v.w)};
}
__device__ __forceinline__ void df2_st(float4* p, DF2 a) {
  float h0, h1, l0, l1;
  upk2(a.hi, h0, h1);
  upk2(a.lo, l0, l1);
  *p = make_float4(h0, h1, l0, l1);
}
// variable 0 or 1 of a stored pair (hi0, hi1, lo0, lo1)
__device__ __forceinline__ DFl df_ld4(const float4* p, int which) {
  const float4 v = *p;
  return which ? DFl{v.y, v.w} : DFl{v.x, v.z};
}

// even/odd line coefficients of the lifting (D) and of the weak divergence
// (w_m / w_i D_mi) as packed broadcasts (c_hi, -c_hi, -c_lo), LineEO::coef order
template <int N>
struct LiftDfCoef {
  static constexpr int NE = (N + 1) * ((N + 1) / 2);
  f32x2 g[3][NE], v[3][NE];
};

// shared memory of k_lift_df (in float2): W 4 n3, face jumps 24 n2, G 12 n3
template <int N>
struct LiftDfShape {
  static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  static constexpr int SMEM_F2 = 16 * n3 + 24 * n2;
};

// node slot: lift_slot8 at N = 7 (bank-conflict free for the node- and
// line-ordered warps), the natural order otherwise
template <int N>
__device__ __forceinline__ int df_slot(int node) {
  if constexpr (N == 7) return lift_slot8(node);
  else return node;
}

// One CTA of n^3 threads per element (odd N: the even/odd contractions need
// an even node count): the roles of k_lift (own face fluxes Gf and the weak
// divergence R_v, both FP64 in memory) with the line contractions on two
// threads per line, two variables each.
template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1), ((N + 1) * (N + 1) * (N + 1) <= 512 ? 2 : 1))
k_lift_df(const double* __restrict__ U, const MeshDev<double> m, const PhysDev ph, const Tables<N> tab,
          const LiftDfCoef<N> cf, double* __restrict__ Rv, double* __restrict__ Gf) {
  static_assert(N % 2 == 1, "the double-float lifting kernel needs an even node count");
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the four lifted variables in two pairs (u, v), (w, T - T_ref), each slot
  // one float4 (hi0, hi1, lo0, lo1): a line thread contracts both variables
  // of a pair with packed instructions
  float4* sW = reinterpret_cast<float4*>(smem_raw);          // [2][n3]
  float2* sC = reinterpret_cast<float2*>(sW + 2 * n3);       // [6][4][n2] 2 (W* - W)
  float4* sG = reinterpret_cast<float4*>(sC + 24 * n2);      // [3][2][n3]
  const int e = blockIdx.x, tid = threadIdx.x;
  const int i = tid % n, j = (tid / n) % n, k = tid / n2;
  const int p = tid;
  const size_t S = (size_t)m.K * n3;
  const size_t g = (size_t)e * n3 + p;
  const int sp = df_slot<N>(p);
  // own primitives (stored as (hi, lo) pairs by k_prim64)
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const float2 a = m.lift_W2[2 * pr * S + g], b = m.lift_W2[(2 * pr + 1) * S + g];
    sW[pr * n3 + sp] = make_float4(a.x, b.x, a.y, b.y);
  }
  // 2 (W* - W) at the six faces, in FP64 from the stored primitives (the
  // jumps are differences of nearby values: exact or nearly so), then split
  for (int t = tid; t < 6 * n2; t += n3) {
    const int l = t / n2, ab = t - l * n2, a = ab % n, b = ab / n;
    const int q = fnode<N>(l, a, b);
    const int nb = m.nbr[e * 6 + l];
    const size_t gq = (size_t)e * n3 + q;
    double dd[4];
    lift_face_jump<N, double>(U, m, ph, S, e, l, ab, q, nb, m.W64[S + gq], m.W64[2 * S + gq], m.W64[3 * S + gq],
                              m.W64[6 * S + gq], dd);
#pragma unroll
    for (int v = 0; v < 4; ++v) df_st(&sC[(l * 4 + v) * n2 + ab], df_of(dd[v]));
  }
  __syncthreads();
  // line contraction by thread tid < 6 n2: the variable pair pr (both
  // variables in the lanes of the packed instructions) on line L of direction
  // dir, y_q = sum_m C_qm x_m for the n nodes, in place or into dst; in
  // even/odd form (C centro-antisymmetric: with xe_m = x_m + x_{N-m},
  // xo_m = x_m - x_{N-m}, E_q = sum_{m<n/2} Ce_qm xe_m, O_q = sum Co_qm xo_m:
  // y_q = E_q + O_q, y_{N-q} = O_q - E_q; tables as LineEO::coef)
  auto line_pass = [&](const float4* src, float4* dst, bool divergence) {
    constexpr int h = n / 2;
    for (int task = tid; task < 6 * n2; task += n3) {
      const int dir = task / (2 * n2), r = task - dir * 2 * n2, pr = r / n2, L = r % n2;
      const int n0 = dir == 0 ? n * L : (dir == 1 ? (L % n) + n2 * (L / n) : L);
      const int stride = dir == 0 ? 1 : (dir == 1 ? n : n2);
      int sl[n];
      if constexpr (N == 7) {
        const int s0 = lift_slot8(n0);
#pragma unroll
        for (int q = 0; q < n; ++q)
          sl[q] = s0 ^ (dir == 0 ? lift_slot8(q) : (dir == 1 ? lift_slot8(q * n) : lift_slot8(q * n2)));
      } else {
#pragma unroll
        for (int q = 0; q < n; ++q) sl[q] = n0 + q * stride;
      }
      const f32x2(*c)[LiftDfCoef<N>::NE] = divergence ? cf.v : cf.g;
      const float4* xs = src + (divergence ? (dir * 2 + pr) : pr) * n3;
      float4* ys = dst + (dir * 2 + pr) * n3;
      DF2 xe[h], xo[h];
#pragma unroll
      for (int mm = 0; mm < h; ++mm) {
        const DF2 a = df2_ld(&xs[sl[mm]]), b = df2_ld(&xs[sl[N - mm]]);
        xe[mm] = df_add2(a, b);
        xo[mm] = df_sub2(a, b);
      }
#pragma unroll
      for (int q = 0; q < h; ++q) {
        DFAcc2 E{0ull, 0ull}, O{0ull, 0ull};
#pragma unroll
        for (int mm = 0; mm < h; ++mm) {
          const int te = q * h + mm, to = (N - q) * h + mm;
          acc_fma2(E, c[0][te], c[1][te], c[2][te], xe[mm]);
          acc_fma2(O, c[0][to], c[1][to], c[2][to], xo[mm]);
        }
        f32x2 s, e;
        two_sum2(O.s, E.s, s, e);
        const DF2 yq = df_norm2(s, add2(add2(O.t, E.t), e));
        two_diff2(O.s, E.s, s, e);
        const DF2 ym = df_norm2(s, add2(sub2(O.t, E.t), e));
        df2_st(&ys[sl[q]], yq);
        df2_st(&ys[sl[N - q]], ym);
      }
    }
  };
  // reference-space gradients
  line_pass(sW, sG, false);
  __syncthreads();
  DFl dW[3][4];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir)
#pragma unroll
    for (int v = 0; v < 4; ++v) dW[dir][v] = df_ld4(&sG[(dir * 2 + (v >> 1)) * n3 + sp], v & 1);
  // surface corrections: sC holds 2 (W* - W), the weights are 1 / (2 w)
  const DFl shw0 = df_of(0.5 * tab.iw[0]), shwN = df_of(0.5 * tab.iw[N]);
  auto surf = [&](int dir, int l, int ab, DFl sw) {
#pragma unroll
    for (int v = 0; v < 4; ++v) dW[dir][v] = df_add(dW[dir][v], df_mul(sw, df_ld(&sC[(l * 4 + v) * n2 + ab])));
  };
  if (i == 0 || i == N) surf(0, i == 0 ? 0 : 1, j + n * k, i == 0 ? df_neg(shw0) : shwN);
  if (j == 0 || j == N) surf(1, j == 0 ? 2 : 3, i + n * k, j == 0 ? df_neg(shw0) : shwN);
  if (k == 0 || k == N) surf(2, k == 0 ? 4 : 5, i + n * j, k == 0 ? df_neg(shw0) : shwN);
  // viscosity and conductivity (FP64, then split)
  double mu_d = ph.mu, kc_d = ph.kcond;
  if (ph.sutherland) {
    mu_d = sutherland<double>(ph, m.W64[6 * S + g]);
    kc_d = mu_d * ph.cp_Pr;
  }
  const DFl mu = df_of(mu_d), kc = df_of(kc_d), mu2 = df_of(2.0 * mu_d), mu23 = df_of(2.0 / 3.0 * mu_d);
  // velocity gradients q[d][c] = sum_dir (Ja^dir_d / J) dW_dir and the
  // contravariant temperature gradients hT[dir] = sum_m ((Ja^dir . Ja^m) / J) dT_m
  DFl q[3][3], hT[3];
  {
    DFl jj[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) jj[c] = df_ld(&m.lift_M2[(size_t)(9 + c) * S + g]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) q[d][c] = dot3(jj[d], dW[0][c], jj[3 + d], dW[1][c], jj[6 + d], dW[2][c]);
  }
  {
    DFl mm[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) mm[c] = df_ld(&m.lift_M2[(size_t)(18 + c) * S + g]);
    hT[0] = dot3(mm[0], dW[0][3], mm[3], dW[1][3], mm[4], dW[2][3]);
    hT[1] = dot3(mm[3], dW[0][3], mm[1], dW[1][3], mm[5], dW[2][3]);
    hT[2] = dot3(mm[4], dW[0][3], mm[5], dW[1][3], mm[2], dW[2][3]);
  }
  // stress tau_ab = mu (q_ba + q_ab) - (2/3) mu div delta_ab
  DFl tau[3][3];
  {
    const DFl div = df_add(df_add(q[0][0], q[1][1]), q[2][2]);
    const DFl mdiv = df_mul(mu23, div);
#pragma unroll
    for (int a = 0; a < 3; ++a) tau[a][a] = df_sub(df_mul(mu2, q[a][a]), mdiv);
    tau[0][1] = tau[1][0] = df_mul(mu, df_add(q[0][1], q[1][0]));
    tau[0][2] = tau[2][0] = df_mul(mu, df_add(q[0][2], q[2][0]));
    tau[1][2] = tau[2][1] = df_mul(mu, df_add(q[1][2], q[2][1]));
  }
  // contravariant viscous fluxes G^dir = sum_d Ja^dir_d Fv_d; energy row
  // G^dir_E = sum_c u_c G^dir_c + k (Ja^dir . grad T)
  DFl G[3][4];
  {
    const DFl uu = df_ld4(&sW[sp], 0), vv = df_ld4(&sW[sp], 1), ww = df_ld4(&sW[n3 + sp], 0);
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      const DFl a0 = df_ld(&m.lift_M2[(size_t)(dir * 3 + 0) * S + g]),
                a1 = df_ld(&m.lift_M2[(size_t)(dir * 3 + 1) * S + g]),
                a2 = df_ld(&m.lift_M2[(size_t)(dir * 3 + 2) * S + g]);
#pragma unroll
      for (int v = 0; v < 3; ++v) G[dir][v] = dot3(a0, tau[v][0], a1, tau[v][1], a2, tau[v][2]);
      DFAcc A{0.f, 0.f};
      acc_fma(A, uu, G[dir][0]);
      acc_fma(A, vv, G[dir][1]);
      acc_fma(A, ww, G[dir][2]);
      acc_fma(A, kc, hT[dir]);
      G[dir][3] = acc_val(A);
    }
  }
  // own outward viscous flux at face nodes: Gf[e][l][v][ab] = +-G^{l/2}
  auto gface = [&](int l, int ab, double sgn) {
    double* dst = Gf + ((size_t)e * 6 + l) * 4 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v * n2] = sgn * df_to(G[l >> 1][v]);
  };
  if (i == 0) gface(0, j + n * k, -1.0);
  if (i == N) gface(1, j + n * k, 1.0);
  if (j == 0) gface(2, i + n * k, -1.0);
  if (j == N) gface(3, i + n * k, 1.0);
  if (k == 0) gface(4, i + n * j, -1.0);
  if (k == N) gface(5, i + n * j, 1.0);
  // weak-form viscous volume term R_v = sum_dir sum_m (w_m / w_i) D_mi G^dir_m
  __syncthreads();  // the nodes have read their derivatives from sG
#pragma unroll
  for (int dir = 0; dir < 3; ++dir)
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const DFl a = G[dir][2 * pr], b = G[dir][2 * pr + 1];
      sG[(dir * 2 + pr) * n3 + sp] = make_float4(a.hi, b.hi, a.lo, b.lo);
    }
  __syncthreads();
  line_pass(sG, sG, true);  // in place: a line's slots belong to its thread
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    DFAcc A{0.f, 0.f};
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) acc_add(A, df_ld4(&sG[(dir * 2 + (v >> 1)) * n3 + sp], v & 1));
    Rv[(size_t)v * S + g] = df_to(acc_val(A));
  }
}

}  // namespace dg
