// ops_impl.cuh -- host launch code for one polynomial degree (included by
// op_n<N>.cu with DG_N defined).
#pragma once

#include <cstring>
#include <algorithm>
#include <type_traits>

#include "adjoint.cuh"
#include "kernels.cuh"
#include "lift_df.cuh"
#include "ops.h"

namespace dg {

template <int N>
static Tables<N> make_tables(const double* D, const double* w) {
  constexpr int n = N + 1;
  Tables<N> t;
  for (int i = 0; i < n; ++i) {
    t.iw[i] = 1.0 / w[i];
    for (int m = 0; m < n; ++m) {
      double dvs = 2.0 * D[i * n + m];
      if (i == m && i == 0) dvs += 1.0 / w[0];
      if (i == m && i == N) dvs -= 1.0 / w[N];
      t.D[i * n + m] = D[i * n + m];
      t.DVS8[i * n + m] = dvs / 8.0;
      t.Dvisc[i * n + m] = w[m] / w[i] * D[m * n + i];
      t.D32[i * n + m] = (float)t.D[i * n + m];
      t.Dvisc32[i * n + m] = (float)t.Dvisc[i * n + m];
      t.D32lo[i * n + m] = (float)(t.D[i * n + m] - (double)t.D32[i * n + m]);
      t.Dvisc32lo[i * n + m] = (float)(t.Dvisc[i * n + m] - (double)t.Dvisc32[i * n + m]);
    }
  }
  // even/odd tables [n][n/2] (as LineEO::coef): rows q < n/2 hold
  // (M_qm + M_q,N-m) / 2, rows q >= n/2 (M_q'm - M_q',N-m) / 2 with q' = N - q
  constexpr int h = n / 2;
  for (int t2 = 0; t2 < n * h; ++t2) {
    const int q = t2 / h, mm = t2 % h, r = q < h ? q : N - q;
    auto co = [&](const double* M) {
      const double a = M[r * n + mm], b = M[r * n + N - mm];
      return q < h ? 0.5 * (a + b) : 0.5 * (a - b);
    };
    const double cd = co(t.D), cv = co(t.Dvisc);
    t.Deo32[t2] = (float)cd; t.Deo32lo[t2] = (float)(cd - (double)t.Deo32[t2]);
    t.Dveo32[t2] = (float)cv; t.Dveo32lo[t2] = (float)(cv - (double)t.Dveo32[t2]);
  }
  return t;
}

// the double-float lifting's line coefficients as packed broadcasts
// (c_hi, -c_hi, -c_lo) of the even/odd tables
static inline unsigned long long bcast2(float x) {
  unsigned int b;
  std::memcpy(&b, &x, 4);
  return (unsigned long long)b | ((unsigned long long)b << 32);
}
template <int N>
static LiftDfCoef<N> make_lift_df_coef(const Tables<N>& t) {
  LiftDfCoef<N> c;
  for (int i = 0; i < LiftDfCoef<N>::NE; ++i) {
    c.g[0][i] = bcast2(t.Deo32[i]);
    c.g[1][i] = bcast2(-t.Deo32[i]);
    c.g[2][i] = bcast2(-t.Deo32lo[i]);
    c.v[0][i] = bcast2(t.Dveo32[i]);
    c.v[1][i] = bcast2(-t.Dveo32[i]);
    c.v[2][i] = bcast2(-t.Dveo32lo[i]);
  }
  return c;
}

template <int N>
static LiftPk<N> make_lift_pk(const Tables<N>& t) {
  LiftPk<N> c;
  for (int i = 0; i < (N + 1) * (N + 1); ++i) {
    c.d[i] = bcast2(t.D32[i]);
    c.dv[i] = bcast2(t.Dvisc32[i]);
  }
  return c;
}

template <int N, typename R>
static int run_typed(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  MeshDev<R> m{};
  m.K = a.K; m.F = a.F; m.n_interior = a.n_interior; m.n_wall = a.n_wall; m.n_bc = a.n_bc;
  m.Ja = static_cast<const R*>(a.Ja); m.invJ = static_cast<const R*>(a.invJ);
  m.fgeo = a.fgeo; m.nbr = a.nbr; m.elem_face = a.elem_face; m.faces = a.faces;
  m.ws_elem = a.ws_elem; m.ws_lag = a.ws_lag;
  m.status = a.status;
  m.W32 = std::is_same<R, float>::value ? a.W32 : nullptr;
  // FP64 viscous form: the primitives stored by k_prim64 (before the lifting
  // kernel) and the lifting kernel's metric products
  m.W64 = std::is_same<R, double>::value && ph.viscous ? a.W64 : nullptr;
  m.JaJ = a.JaJ; m.Mj = a.Mj;
  if (std::is_same<R, double>::value && ph.viscous && (!a.JaJ || !a.Mj))
    return (int)cudaErrorInvalidValue;
  m.lift_M2 = a.lift_M2; m.lift_W2 = a.lift_W2;
  m.pairA = a.pairA;
  if (N == 7 && std::is_same<R, double>::value && !a.pairA) return (int)cudaErrorInvalidValue;
  m.wm_t = a.wm_t;
  m.n_halo = a.n_halo; m.halo_U = a.halo_U; m.halo_G = static_cast<const R*>(a.halo_G);
  const Tables<N> tab = make_tables<N>(a.D, a.w);
  R* Rv = static_cast<R*>(a.Rv);
  R* Gf = static_cast<R*>(a.Gf);
  R* Fs = static_cast<R*>(a.Fs);
  const size_t smem_lift = (size_t)(16 * n3 + 26 * n2 + n) * sizeof(R);
  const size_t smem_vol = (size_t)(ph.vol_flux == 2 ? VolShape<N>::SMEM_R_EC
                                   : (std::is_same<R, float>::value ? VolShape<N>::SMEM_R_F32 : VolShape<N>::SMEM_R)) *
                          sizeof(R);
  constexpr int vol_threads = VolShape<N>::THREADS;
  // per device and cheap: set on every call
  cudaFuncSetAttribute(k_lift<N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_lift);
  const bool ec = ph.vol_flux == 2;
  if (ec) {
    cudaFuncSetAttribute(k_volume<N, R, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_vol);
    cudaFuncSetAttribute(k_volume<N, R, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_vol);
  } else {
    cudaFuncSetAttribute(k_volume<N, R, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_vol);
    cudaFuncSetAttribute(k_volume<N, R, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_vol);
  }
  const int phase = a.phase ? a.phase : 7;
  const unsigned halo_blocks = (unsigned)(((long long)a.n_halo * n2 + 255) / 256);
  if ((phase & 1) && a.n_halo > 0 && a.send_U)
    k_halo_pack<N, R><<<halo_blocks, 256, 0, s>>>(a.Uin, m, Gf, a.send_U, nullptr);
  if (!(phase & 6)) return (int)cudaGetLastError();
  // the wall kernel reads only U and writes only the wall faces' fluxes, so
  // it may run beside the lifting and the interior faces
  const bool fork = a.side != nullptr && a.n_wall > 0;
  const cudaStream_t ws = fork ? a.side : s;
  auto wall = [&]() {
    if (a.n_wall == 0) return;
    const int threads = WALL_THREADS;
    const long long work = (long long)a.n_wall * n2;
    k_wall<N, R><<<(unsigned)((work + threads - 1) / threads), threads, 0, ws>>>(a.Uin, m, ph, Fs, a.tau, a.status);
  };
  if (phase & 2) {
    // the FP32 primitives first: the FP32 wall kernel reads them
    if (std::is_same<R, float>::value && !a.w32_valid) {
      const long long S = (long long)a.K * n3;
      k_prim32<<<(unsigned)std::min<long long>((S + 255) / 256, 152 * 16), 256, 0, s>>>(S, a.Uin, ph, a.W32);
    }
    if (fork) {
      cudaEventRecord(a.fork, s);
      cudaStreamWaitEvent(a.side, a.fork, 0);
      if (a.ev) cudaEventRecord(a.ev[3], ws);
      wall();
      if (a.ev) cudaEventRecord(a.ev[4], ws);
      cudaEventRecord(a.join, a.side);
    }
    if (a.ev) cudaEventRecord(a.ev[0], s);
    // the FP64 primitives of the input (timed with the lifting kernel, their
    // first reader; kept between evaluations of an unchanged state)
    if (m.W64 && !a.w64_valid) {
      const long long S = (long long)a.K * n3;
      k_prim64<<<(unsigned)std::min<long long>((S + 255) / 256, 152 * 16), 256, 0, s>>>(
          S, a.Uin, ph, m.W64, (ph.lift_df && N % 2 == 1) ? a.lift_W2 : nullptr);
    }
    if (ph.viscous) {
      bool done = false;
      if constexpr (N % 2 == 1 && std::is_same<R, double>::value) {
        // the double-float lifting (it reads the stored primitives and metric products)
        if (ph.lift_df && m.W64 && m.lift_M2 && m.lift_W2) {
          const size_t smem_df = (size_t)LiftDfShape<N>::SMEM_F2 * sizeof(float2);
          cudaFuncSetAttribute(k_lift_df<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_df);
          k_lift_df<N><<<a.K, n3, smem_df, s>>>(a.Uin, m, ph, tab, make_lift_df_coef<N>(tab), Rv, Gf);
          done = true;
        }
      }
      if (!done) k_lift<N, R><<<a.K, n3, smem_lift, s>>>(a.Uin, m, ph, tab, make_lift_pk<N>(tab), Rv, Gf);
    }
    if (a.ev) cudaEventRecord(a.ev[1], s);
    if (a.n_halo > 0 && a.send_G && ph.viscous)
      k_halo_pack<N, R><<<halo_blocks, 256, 0, s>>>(a.Uin, m, Gf, nullptr, static_cast<R*>(a.send_G));
  }
  if (!(phase & 4)) return (int)cudaGetLastError();
  // FP64: k_face also takes the halo faces (after the interior ones)
  constexpr bool halo_in_face = std::is_same<R, double>::value;
  const long long face_work = (long long)(a.n_interior + (halo_in_face ? a.n_halo : 0)) * n2;
  if (face_work > 0) {
    const int threads = 256;
    k_face<N, R><<<(unsigned)((face_work + threads - 1) / threads), threads, 0, s>>>(a.Uin, m, ph, Gf, Fs);
  }
  if (a.n_bc > 0) {
    const int threads = 256;
    const long long work = (long long)a.n_bc * n2;
    k_bc<N, R><<<(unsigned)((work + threads - 1) / threads), threads, 0, s>>>(a.Uin, m, ph, Gf, Fs);
  }
  if (!halo_in_face && a.n_halo > 0) k_halo_face<N, R><<<halo_blocks, 256, 0, s>>>(a.Uin, m, ph, Gf, Fs);
  if (a.ev) cudaEventRecord(a.ev[2], s);
  if (fork) {
    cudaStreamWaitEvent(s, a.join, 0);
  } else {
    if (a.ev) cudaEventRecord(a.ev[3], s);
    wall();
    if (a.ev) cudaEventRecord(a.ev[4], s);
  }
  if (a.ev) cudaEventRecord(a.ev[5], s);
  StageArgs st{a.A, a.B, a.dt, a.read_dU, std::is_same<R, float>::value && a.mode == 1 ? 1 : 0};
  if (a.mode == 0 && !ec)
    k_volume<N, R, 0, false><<<a.K, vol_threads, smem_vol, s>>>(a.Uin, m, ph, tab, Rv, Fs, a.Out, nullptr, nullptr,
                                                                st, a.status);
  else if (a.mode == 0)
    k_volume<N, R, 0, true><<<a.K, vol_threads, smem_vol, s>>>(a.Uin, m, ph, tab, Rv, Fs, a.Out, nullptr, nullptr,
                                                               st, a.status);
  else if (!ec)
    k_volume<N, R, 1, false><<<a.K, vol_threads, smem_vol, s>>>(a.Uin, m, ph, tab, Rv, Fs, nullptr, a.dU, a.Uout,
                                                                st, a.status);
  else
    k_volume<N, R, 1, true><<<a.K, vol_threads, smem_vol, s>>>(a.Uin, m, ph, tab, Rv, Fs, nullptr, a.dU, a.Uout,
                                                               st, a.status);
  if (a.ev) cudaEventRecord(a.ev[6], s);
  return (int)cudaGetLastError();
}

template <int N>
static int run_vjp_typed(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  MeshDev<double> m{};
  m.K = a.K; m.F = a.F; m.n_interior = a.n_interior; m.n_wall = a.n_wall; m.n_bc = a.n_bc;
  m.Ja = static_cast<const double*>(a.Ja); m.invJ = static_cast<const double*>(a.invJ);
  m.fgeo = a.fgeo; m.nbr = a.nbr; m.elem_face = a.elem_face; m.faces = a.faces;
  m.ws_elem = a.ws_elem; m.ws_lag = a.ws_lag;
  m.status = a.status;
  m.JaJ = a.JaJ; m.Mj = a.Mj;
  m.n_halo = a.n_halo; m.halo_U = a.halo_U; m.halo_G = static_cast<const double*>(a.halo_G);
  if (ph.viscous && !a.JaJ) return (int)cudaErrorInvalidValue;
  const Tables<N> tab = make_tables<N>(a.D, a.w);
  const double iw = tab.iw[0];
  const size_t smem = (size_t)AdjShape<N>::SMEM_D * sizeof(double);
  // the adjoint element kernel's instantiation: entropy-conserving flux,
  // Sutherland's law
  auto element = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return kern;
  };
  const bool ec = ph.vol_flux == 2, su = ph.sutherland != 0;
  auto kel = ec ? (su ? element(k_adj_element<N, true, true>) : element(k_adj_element<N, true, false>))
                : (su ? element(k_adj_element<N, false, true>) : element(k_adj_element<N, false, false>));
  // Partitioned meshes run in four phases around three exchanges (the
  // reverse of the evaluation's): 1 packs the state traces of the halo
  // faces (send_U); 2 the face, wall and boundary kernels, which leave the
  // cotangents of the peers' viscous-flux traces in send_G and of their
  // state traces in send_U; 3 adds the peers' viscous-flux cotangents
  // (halo_G) and runs the element kernel, which adds its lifting's share to
  // send_U; 4 gathers, with the peers' state cotangents (halo_U).
  const bool part = a.n_halo > 0;
  const int phase = part ? a.phase : 14;
  double* sendU = part ? a.send_U : nullptr;
  double* sendG = part ? static_cast<double*>(a.send_G) : nullptr;
  const unsigned halo_blocks = (unsigned)(((long long)a.n_halo * n2 + 127) / 128);
  if (phase == 1) {
    k_halo_pack<N, double><<<(unsigned)(((long long)a.n_halo * n2 + 255) / 256), 256, 0, s>>>(
        a.Uin, m, static_cast<const double*>(nullptr), a.send_U, static_cast<double*>(nullptr));
    return (int)cudaGetLastError();
  }
  if (phase == 2 || phase == 14) {
    const long long work = (long long)(a.n_interior + (part ? a.n_halo : 0)) * n2;
    if (work > 0)
      k_adj_face<N><<<(unsigned)((work + 127) / 128), 128, 0, s>>>(a.Uin, a.lam, m, ph, iw, a.gUf, a.gGf, sendU,
                                                                   sendG);
    if (a.n_wall > 0) {
      const long long ww = (long long)a.n_wall * n2;
      k_adj_wall<N><<<(unsigned)((ww + WALL_THREADS - 1) / WALL_THREADS), WALL_THREADS, 0, s>>>(
          a.Uin, a.lam, m, ph, iw, a.gUf, a.gGf, a.gUs, a.gtheta, a.status);
    }
    if (a.n_bc > 0) {
      const long long wb = (long long)a.n_bc * n2;
      k_adj_bc<N><<<(unsigned)((wb + 127) / 128), 128, 0, s>>>(a.Uin, a.lam, m, ph, iw, a.gUf, a.gGf);
    }
  }
  if (phase == 3 || phase == 14) {
    if (part && ph.viscous) k_adj_halo_in<N><<<halo_blocks, 128, 0, s>>>(m, m.halo_G, a.gGf);
    kel<<<a.K, AdjShape<N>::THREADS, smem, s>>>(a.Uin, a.lam, m, ph, tab, a.gGf, a.gU, a.gWf, sendU);
  }
  if (phase == 4 || phase == 14) {
    const long long S = (long long)a.K * n3;
    k_adj_gather<N><<<(unsigned)((S + 255) / 256), 256, 0, s>>>(a.Uin, m, ph, a.gUf, a.gWf,
                                                                 part ? a.halo_U : nullptr, a.gU);
    if (a.n_wall > 0 && ph.viscous) {
      const long long work = (long long)a.n_wall * n2;
      k_adj_scatter<N><<<(unsigned)((work + 127) / 128), 128, 0, s>>>(m, a.gUs, a.gU);
    }
  }
  return (int)cudaGetLastError();
}

template <int N>
static int run_wall_loss_typed(const OpArgs& a, const PhysDev& ph, const double* wq, double inv_total, int grad,
                               double* loss, cudaStream_t s) {
  constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
  MeshDev<double> m{};
  m.K = a.K; m.F = a.F; m.n_interior = a.n_interior; m.n_wall = a.n_wall; m.n_bc = a.n_bc;
  m.Ja = static_cast<const double*>(a.Ja); m.invJ = static_cast<const double*>(a.invJ);
  m.fgeo = a.fgeo; m.nbr = a.nbr; m.elem_face = a.elem_face; m.faces = a.faces;
  m.ws_elem = a.ws_elem; m.ws_lag = a.ws_lag;
  m.status = a.status;
  if (a.n_wall == 0) return 0;
  const long long work = (long long)a.n_wall * n2;
  k_wall_loss<N><<<(unsigned)((work + WALL_THREADS - 1) / WALL_THREADS), WALL_THREADS, 0, s>>>(a.Uin, m, ph, wq, inv_total, grad, loss, a.gUs,
                                                                a.gtheta, a.status);
  if (grad) {
    const long long S = 5LL * a.K * n3;
    k_axpby<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(S, 0.0, a.gU, 0.0, a.gU);
    k_adj_scatter<N><<<(unsigned)((work + 127) / 128), 128, 0, s>>>(m, a.gUs, a.gU);
  }
  return (int)cudaGetLastError();
}

}  // namespace dg

#define DG_DEFINE_N(NN)                                                              \
  namespace dg {                                                                     \
  int run_operator_n##NN(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {      \
    return a.fp32 ? run_typed<NN, float>(a, ph, s) : run_typed<NN, double>(a, ph, s); \
  }                                                                                  \
  int run_vjp_n##NN(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {           \
    return run_vjp_typed<NN>(a, ph, s);                                              \
  }                                                                                  \
  int run_wall_loss_n##NN(const OpArgs& a, const PhysDev& ph, const double* wq, double inv_total, int grad, \
                          double* loss, cudaStream_t s) {                            \
    return run_wall_loss_typed<NN>(a, ph, wq, inv_total, grad, loss, s);             \
  }                                                                                  \
  }
