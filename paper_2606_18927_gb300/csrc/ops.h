// ops.h -- internal interface between the C API and the per-degree kernel
// instantiations (one translation unit per polynomial degree N).
#pragma once
#include <cuda_runtime.h>

namespace dg {

struct PhysDev;

struct OpArgs {
  int N, K, F, n_interior, n_wall, n_bc;
  int fp32;                 // 0: double fluxes, 1: float fluxes (mixed form)
  const void* Ja;           // [9][K n^3] in the flux type
  const void* invJ;         // [K n^3] in the flux type
  const double* fgeo;
  const int* nbr;
  const int* elem_face;
  const int4* faces;
  const int* ws_elem;
  const double* ws_lag;
  const double* D;          // host basis: D[n*n], w[n]
  const double* w;
  const double* Uin;        // state read by the operator
  void* Rv;                 // scratch in the flux type
  void* Gf;
  void* Fs;
  double* tau;              // wall shear per wall node (may be null)
  int* status;
  int mode;                 // 0: Ut -> Out; 1: LSERK4 stage on dU, Uout
  double* Out;
  double* dU;
  double* Uout;
  double A, B, dt;
  int read_dU;
  cudaEvent_t* ev;          // null, or 7 events: lift [0,1], face [1,2], wall [3,4], volume [5,6]
  // optional side stream for the wall-model kernel: it forks from the main
  // stream before the lifting and joins it before the volume kernel (the
  // paper's prioritised boundary work, Sec. 2.1); null side: one stream
  cudaStream_t side;
  cudaEvent_t fork, join;
  // FP32-mixed form: [6][K n^3] FP32 primitives of Uin; w32_valid = 1 when they
  // are already those of Uin (else the operator forms them first).  A stage
  // (mode 1) leaves the primitives of Uout in W32.
  float* W32;
  int w32_valid;
  // FP64 viscous form: [7][K n^3] primitives of Uin (null: each kernel forms
  // its own); w64_valid = 1 when they are already those of Uin (else k_prim64
  // forms them before the lifting kernel)
  double* W64;
  int w64_valid;
  // FP64 viscous form: the lifting kernel's metric products, [9][K n^3] Ja / J
  // and [6][K n^3] (Ja Ja^T) / J (order 00, 11, 22, 01, 02, 12)
  const double* JaJ;
  const double* Mj;
  // the double-float lifting's (hi, lo) pairs of Ja, Ja / J, (Ja Ja^T) / J
  // [24][K n^3] and of the lifted primitives [4][K n^3] (null: not selected)
  const float2* lift_M2;
  float2* lift_W2;
  const double* pairA;  // FP64 at N = 7: the volume kernel's pair metric sums (required there)
  double* wm_t;  // wall-law warm-start values per wall node (null: cold solves)
  // partitioned meshes: n_halo halo faces (the last faces), remote traces in
  // halo_U / halo_G, local traces packed into send_U / send_G.  phase selects
  // part of an evaluation: 1 packs the state traces, 2 runs the lifting and
  // packs the viscous-flux traces, 4 the faces and the volume kernel (7: all)
  int n_halo;
  const double* halo_U;
  const void* halo_G;
  double* send_U;
  void* send_G;
  int phase;
  // adjoint (FP64): cotangent lam of Ut, output gU, and scratch
  const double* lam;
  double* gU;
  double* gUf;              // [K][6][5][n2] face-kernel state cotangents
  double* gGf;              // [K][6][4][n2] cotangents of the own face viscous fluxes
  double* gWf;              // [K][6][4][n2] lifting cotangents for the neighbour's face nodes
  double* gUs;              // [n_wall n2][5] wall-model sample cotangents
  double* gtheta;           // [2] (kappa, B), accumulated
};

// Vector-Jacobian product (FP64 contexts): gU = (dUt/dU)^T lam, gtheta += ...
int run_vjp(const OpArgs& a, const PhysDev& ph, cudaStream_t s);

// Mean wall shear of U (accumulated into loss[0]); with grad also gU
// (= dL/dU, overwritten) and gtheta (accumulated).  Uses a.Uin, a.gU, a.gUs,
// a.gtheta, a.status.
int run_wall_loss(const OpArgs& a, const PhysDev& ph, const double* wq, double inv_total, int grad,
                  double* loss, cudaStream_t s);
// y = a x + b y
int run_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s);

// Launches lift (if viscous), face, wall and volume kernels on the stream.
int run_operator(const OpArgs& a, const PhysDev& ph, cudaStream_t s);

#define DG_DECLARE_N(NN) int run_operator_n##NN(const OpArgs& a, const PhysDev& ph, cudaStream_t s); \
  int run_vjp_n##NN(const OpArgs& a, const PhysDev& ph, cudaStream_t s);                           \
  int run_wall_loss_n##NN(const OpArgs& a, const PhysDev& ph, const double* wq, double inv_total, int grad, \
                          double* loss, cudaStream_t s);
DG_DECLARE_N(1)
DG_DECLARE_N(2)
DG_DECLARE_N(3)
DG_DECLARE_N(4)
DG_DECLARE_N(5)
DG_DECLARE_N(6)
DG_DECLARE_N(7)
DG_DECLARE_N(8)
#undef DG_DECLARE_N

}  // namespace dg
