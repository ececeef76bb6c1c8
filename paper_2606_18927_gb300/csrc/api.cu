// api.cu -- C ABI of the GB300 DGSEM library (declared in include/dg.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "geometry.h"
#include "kernels.cuh"
#include "ops.h"

// Five-stage fourth-order 2N-storage Runge-Kutta scheme of Carpenter and
// Kennedy (1994), the low-storage scheme of paper Sec. 4.  These are the
// published rational coefficients.
// Default iteration cap of the law-of-the-wall solve (bracket growth and
// Newton steps together); dg_set_wall_solve_limit changes it.
static const int kWallSolveMaxIter = 200;
static const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

struct dg_ctx {
  int N = 0, n = 0, n2 = 0, n3 = 0, K = 0, F = 0;
  size_t S = 0;  // K n^3
  dg_phys phys{};
  dg_options opts{};
  dg::PhysDev ph{};
  cudaStream_t stream = nullptr;
  int device = 0;
  // side stream (highest priority) for the wall-model kernel, forked from and
  // joined back into the caller's stream around each operator evaluation
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool overlap = true;
  // FP32-mixed form: FP32 primitives [6][S]; w32_of_U says they are those of U
  float* W32 = nullptr;
  bool w32_of_U = false;
  // FP64 viscous form: primitives [6][S] formed by the lifting kernel for the
  // face and volume kernels of the same evaluation
  double* W64 = nullptr;  // FP64 viscous form: primitives [7][S]; w64_of_U says they are those of U
  bool w64_of_U = false;
  double* JaJ = nullptr;  // FP64 viscous: [9][S] Ja / J
  double* Mj = nullptr;   // FP64 viscous: [6][S] (Ja Ja^T) / J
  // double-float lifting (N = 7, FP64 viscous): (hi, lo) pairs of Ja, Ja / J,
  // (Ja Ja^T) / J [24][S] and of the lifted primitives [4][S]
  float2* lift_M2 = nullptr;
  float2* lift_W2 = nullptr;
  double* pairA = nullptr;  // FP64, N = 7: the volume kernel's pair metric sums [16128 K]
  double* wm_t = nullptr;  // wall-law warm start per wall node (NaN: none yet)
  // partitioned meshes: halo buffers [n_halo][5][n2] (state traces, FP64) and
  // [n_halo][4][n2] (viscous-flux traces, flux type), received and sent
  double* halo_U = nullptr;
  double* send_U = nullptr;
  void* halo_G = nullptr;
  void* send_G = nullptr;
  dg::Geometry geo;
  // device storage
  double* U = nullptr;
  double* dU = nullptr;
  double* io = nullptr;   // staging of a host input
  double* io2 = nullptr;  // staging of a host output
  void* Ja = nullptr;
  void* invJ = nullptr;
  double* fgeo = nullptr;
  int* nbr = nullptr;
  int* elem_face = nullptr;
  int4* faces = nullptr;
  int* ws_elem = nullptr;
  double* ws_lag = nullptr;
  void* Rv = nullptr;
  void* Gf = nullptr;
  void* Fs = nullptr;
  double* tau = nullptr;
  int* status = nullptr;
  bool state_set = false;
  std::string err;
  // wall-node surface quadrature weights w_a w_b s and their sum
  double* wq = nullptr;
  double wq_total = 0.0;
  // rollout buffers (allocated on the first dg_rollout_vjp, grown on demand)
  double* ro_ckpt = nullptr;
  int ro_cap = 0;
  double* ro_stage = nullptr;  // 5 stage inputs
  double* ro_work = nullptr;   // Uw, dUw, gA, gD, gT, lam
  double* ro_scalar = nullptr; // loss
  double* wJ = nullptr;        // w_i w_j w_k J per node (kinetic-energy integral)
  double vol = 0.0;
  // adjoint scratch (allocated on the first dg_vjp)
  double* gUf = nullptr;
  double* gGf = nullptr;
  double* gWf = nullptr;
  double* gUs = nullptr;
  double* gtheta = nullptr;
  // CUDA graph of one full LSERK4 step (five stages), captured for a given dt
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  double step_graph_dt = 0.0;
  // host batches (dg_rk_stage_batch): two device slots (state, register),
  // copy-in and copy-out streams and their events
  double* bU[2] = {nullptr, nullptr};
  double* bdU[2] = {nullptr, nullptr};
  cudaStream_t cp_in = nullptr, cp_out = nullptr;
  cudaEvent_t ev_loaded[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_freed[2] = {nullptr, nullptr};
  // optional per-kernel timing: 5 events per operator evaluation
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  size_t events_used = 0;
};

static std::string g_init_error;

namespace {

int fail(dg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_init_error = msg;
  return code;
}

int cuda_fail(dg_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t alloc(T** p, size_t count) {
  if (count == 0) { *p = nullptr; return cudaSuccess; }
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void free_all(dg_ctx* c) {
  for (cudaEvent_t ev : c->events) cudaEventDestroy(ev);
  c->events.clear();
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->step_graph = nullptr;
  c->cap_stream = nullptr;
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  c->fork_ev = c->join_ev = nullptr;
  c->side = nullptr;
  for (int k = 0; k < 2; ++k) {
    for (cudaEvent_t* ev : {&c->ev_loaded[k], &c->ev_done[k], &c->ev_freed[k]}) {
      if (*ev) cudaEventDestroy(*ev);
      *ev = nullptr;
    }
    if (c->bU[k]) cudaFree(c->bU[k]);
    if (c->bdU[k]) cudaFree(c->bdU[k]);
    c->bU[k] = c->bdU[k] = nullptr;
  }
  if (c->cp_in) cudaStreamDestroy(c->cp_in);
  if (c->cp_out) cudaStreamDestroy(c->cp_out);
  c->cp_in = c->cp_out = nullptr;
  void* ptrs[] = {c->U, c->dU, c->io, c->io2, c->Ja, c->invJ, c->fgeo, c->nbr, c->elem_face, c->faces,
                  c->ws_elem, c->ws_lag, c->Rv, c->Gf, c->Fs, c->tau, c->status,
                  c->gUf, c->gGf, c->gWf, c->gUs, c->gtheta, c->wq, c->ro_ckpt, c->ro_stage, c->ro_work,
                  c->ro_scalar, c->wJ, c->W32, c->W64, c->JaJ, c->Mj, c->lift_M2, c->lift_W2, c->pairA, c->halo_U, c->send_U,
                  c->halo_G, c->send_G,
                  c->wm_t};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// profiling events per operator evaluation (see OpArgs::ev)
constexpr size_t kEventsPerLaunch = 7;

int launch(dg_ctx* c, const double* Uin, int mode, double* Out, double A, double B, double dt, int read_dU,
           double* Uout, double* dU = nullptr, int phase = 7) {
  if (phase == 7 && c->geo.n_halo > 0)
    return fail(c, DG_ERR_ARG, "a partitioned context evaluates in phases around its halo exchanges "
                               "(dg_stage_phase, dg_time_derivative_phase)");
  dg::OpArgs a{};
  a.N = c->N; a.K = c->K; a.F = c->F; a.n_interior = c->geo.n_interior; a.n_wall = c->geo.n_wall;
  a.n_bc = c->geo.n_bc;
  a.fp32 = c->opts.precision == DG_FP32_MIXED;
  a.Ja = c->Ja; a.invJ = c->invJ; a.fgeo = c->fgeo; a.nbr = c->nbr; a.elem_face = c->elem_face;
  a.faces = c->faces; a.ws_elem = c->ws_elem; a.ws_lag = c->ws_lag;
  a.D = c->geo.basis.D.data(); a.w = c->geo.basis.w.data();
  a.Uin = Uin; a.Rv = c->Rv; a.Gf = c->Gf; a.Fs = c->Fs; a.tau = c->tau; a.status = c->status;
  a.mode = mode; a.Out = Out; a.dU = dU ? dU : c->dU; a.Uout = Uout;
  a.A = A; a.B = B; a.dt = dt; a.read_dU = read_dU;
  a.ev = nullptr;
  if (c->overlap && c->side) { a.side = c->side; a.fork = c->fork_ev; a.join = c->join_ev; }
  a.phase = phase;
  a.n_halo = c->geo.n_halo;
  a.halo_U = c->halo_U; a.halo_G = c->halo_G; a.send_U = c->send_U; a.send_G = c->send_G;
  if (c->profiling && phase == 7) {
    if (c->events_used + kEventsPerLaunch > c->events.size()) {
      for (int x = 0; x < kEventsPerLaunch * 64; ++x) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(c, e, "profiling events");
        c->events.push_back(ev);
      }
    }
    a.ev = &c->events[c->events_used];
    c->events_used += kEventsPerLaunch;
  }
  a.W32 = c->W32;
  a.w32_valid = (a.fp32 && Uin == c->U && c->w32_of_U) ? 1 : 0;
  a.W64 = c->W64;
  a.w64_valid = (c->W64 && !a.fp32 && Uin == c->U && c->w64_of_U) ? 1 : 0;
  a.JaJ = c->JaJ; a.Mj = c->Mj;
  a.lift_M2 = c->lift_M2; a.lift_W2 = c->lift_W2;
  a.pairA = c->pairA;
  a.wm_t = c->wm_t;
  int rc = dg::run_operator(a, c->ph, c->stream);
  if (rc != 0) {
    c->w32_of_U = false;
    c->w64_of_U = false;
    return cuda_fail(c, (cudaError_t)rc, "kernel launch");
  }
  // the FP32 primitives now belong to the stage's output (mode 1) or input
  if (a.fp32 && (phase & 4)) c->w32_of_U = mode == 1 ? (Uout == c->U) : (Uin == c->U);
  else if (a.fp32 && (phase & 2)) c->w32_of_U = (Uin == c->U);
  // the FP64 primitives: those of the input once phase 2 ran, stale once a
  // stage has updated the state in place
  if (!a.fp32 && c->W64 && c->opts.viscous) {
    if ((phase & 4) && mode == 1 && Uout == c->U) c->w64_of_U = false;
    else if (phase & 2) c->w64_of_U = (Uin == c->U);
  }
  return DG_OK;
}

// FP32-mixed form: form the primitives of the context's state if they are stale
int refresh_w32(dg_ctx* c) {
  if (c->opts.precision != DG_FP32_MIXED || c->w32_of_U) return DG_OK;
  const long long S = (long long)c->S;
  dg::k_prim32<<<(unsigned)std::min<long long>((S + 255) / 256, 152 * 16), 256, 0, c->stream>>>(S, c->U, c->ph,
                                                                                                 c->W32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "primitive refresh");
  c->w32_of_U = true;
  return DG_OK;
}

// A captured LSERK4 step holds the kernel arguments of its capture (the
// physical constants among them): it is recaptured at its next use.
void drop_step_graph(dg_ctx* c) {
  if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
  c->step_graph = nullptr;
}

}  // namespace

namespace dg {
int run_operator(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {
  switch (a.N) {
    case 1: return run_operator_n1(a, ph, s);
    case 2: return run_operator_n2(a, ph, s);
    case 3: return run_operator_n3(a, ph, s);
    case 4: return run_operator_n4(a, ph, s);
    case 5: return run_operator_n5(a, ph, s);
    case 6: return run_operator_n6(a, ph, s);
    case 7: return run_operator_n7(a, ph, s);
    case 8: return run_operator_n8(a, ph, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
// sum over nodes of wJ * |m|^2 / (2 rho), block reduction + one atomic per warp
__global__ void k_kinetic_energy(long long S, const double* __restrict__ U, const double* __restrict__ wJ,
                                 double* __restrict__ out) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
    const double r = U[i], m1 = U[S + i], m2 = U[2 * S + i], m3 = U[3 * S + i];
    acc += wJ[i] * 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}
// max over nodes of sum_dir (|u . Ja^dir| + c |Ja^dir|) / J (positive doubles
// order like their bit patterns, so the maximum is an integer atomicMax)
template <typename R>
__global__ void k_wave_speed(long long S, const double* __restrict__ U, const R* __restrict__ Ja,
                             const R* __restrict__ invJ, double gamma, unsigned long long* __restrict__ out) {
  double mx = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
    const double r = U[i], u = U[S + i] / r, v = U[2 * S + i] / r, w = U[3 * S + i] / r;
    const double p = (gamma - 1.0) * (U[4 * S + i] - 0.5 * r * (u * u + v * v + w * w));
    const double c = sqrt(gamma * p / r);
    double lam = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double a0 = Ja[(size_t)(d * 3) * S + i], a1 = Ja[(size_t)(d * 3 + 1) * S + i],
                   a2 = Ja[(size_t)(d * 3 + 2) * S + i];
      lam += fabs(u * a0 + v * a1 + w * a2) + c * sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    }
    mx = fmax(mx, lam * (double)invJ[i]);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}
// the FP64 <-> FP32 conversions of the FP32-mixed kernels, for their tests
__global__ void k_convert_fp32(long long n, const double* __restrict__ d, float* __restrict__ f,
                               float* __restrict__ rem, const float* __restrict__ g, double* __restrict__ gd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r;
  f[i] = d2f_bits(d[i], &r);
  rem[i] = r;
  gd[i] = f2d_bits(g[i]);
}
__global__ void k_axpby_api(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (b == 0.0 ? 0.0 : b * y[i]) + (a == 0.0 ? 0.0 : a * x[i]);
}
int run_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby_api<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y);
  return (int)cudaGetLastError();
}
int run_wall_loss(const OpArgs& a, const PhysDev& ph, const double* wq, double inv_total, int grad, double* loss,
                  cudaStream_t s) {
  switch (a.N) {
    case 1: return run_wall_loss_n1(a, ph, wq, inv_total, grad, loss, s);
    case 2: return run_wall_loss_n2(a, ph, wq, inv_total, grad, loss, s);
    case 3: return run_wall_loss_n3(a, ph, wq, inv_total, grad, loss, s);
    case 4: return run_wall_loss_n4(a, ph, wq, inv_total, grad, loss, s);
    case 5: return run_wall_loss_n5(a, ph, wq, inv_total, grad, loss, s);
    case 6: return run_wall_loss_n6(a, ph, wq, inv_total, grad, loss, s);
    case 7: return run_wall_loss_n7(a, ph, wq, inv_total, grad, loss, s);
    case 8: return run_wall_loss_n8(a, ph, wq, inv_total, grad, loss, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
int run_vjp(const OpArgs& a, const PhysDev& ph, cudaStream_t s) {
  switch (a.N) {
    case 1: return run_vjp_n1(a, ph, s);
    case 2: return run_vjp_n2(a, ph, s);
    case 3: return run_vjp_n3(a, ph, s);
    case 4: return run_vjp_n4(a, ph, s);
    case 5: return run_vjp_n5(a, ph, s);
    case 6: return run_vjp_n6(a, ph, s);
    case 7: return run_vjp_n7(a, ph, s);
    case 8: return run_vjp_n8(a, ph, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
}  // namespace dg

namespace dg {
// Operator arguments of a context for dg_time_derivative_noalloc (noalloc.cu):
// everything except the scratch pointers, plus the scratch sizes in bytes.
int noalloc_args(dg_ctx* c, const double* U, double* Ut, OpArgs* a, const PhysDev** ph, cudaStream_t* s,
                 int* device, size_t* rv_bytes, size_t* gf_bytes, size_t* fs_bytes) {
  const size_t rs = c->opts.precision == DG_FP32_MIXED ? sizeof(float) : sizeof(double);
  *a = OpArgs{};
  a->N = c->N; a->K = c->K; a->F = c->F; a->n_interior = c->geo.n_interior; a->n_wall = c->geo.n_wall;
  a->n_bc = c->geo.n_bc;
  a->n_halo = c->geo.n_halo;
  a->fp32 = c->opts.precision == DG_FP32_MIXED;
  a->Ja = c->Ja; a->invJ = c->invJ; a->fgeo = c->fgeo; a->nbr = c->nbr; a->elem_face = c->elem_face;
  a->JaJ = c->JaJ; a->Mj = c->Mj;  // geometry, owned by the context
  a->lift_M2 = nullptr; a->lift_W2 = nullptr;  // (the FP64 lifting: no stored primitives here)
  a->pairA = c->pairA;
  a->faces = c->faces; a->ws_elem = c->ws_elem; a->ws_lag = c->ws_lag;
  a->D = c->geo.basis.D.data(); a->w = c->geo.basis.w.data();
  a->Uin = U; a->status = c->status;
  a->mode = 0; a->Out = Ut;
  *ph = &c->ph;
  *s = c->stream;
  *device = c->device;
  *rv_bytes = (c->opts.viscous ? 4 * c->S : 1) * rs;
  *gf_bytes = (c->opts.viscous ? 24 * (size_t)c->K * c->n2 : 1) * rs;
  *fs_bytes = (c->ph.fs_diff ? 10 : 5) * (size_t)c->F * c->n2 * rs;
  // FP32-mixed form: the primitives go to the context's own W32 array
  // (allocated with the context); they are formed afresh from U
  a->W32 = c->W32;
  a->w32_valid = 0;
  return DG_OK;
}
// After the launches of dg_time_derivative_noalloc: in the FP32-mixed form the
// context's W32 now holds the primitives of U (if the launches succeeded), so
// they are those of the context's state only when U is the state.
void noalloc_done(dg_ctx* c, const double* U, bool ok) {
  if (c->opts.precision == DG_FP32_MIXED) c->w32_of_U = ok && (U == c->U);
}
int noalloc_fail(dg_ctx* c, int code, const std::string& msg) { return fail(c, code, msg); }
}  // namespace dg

extern "C" {

int dg_lgl_nodes(int N, double* xi, double* w) {
  if (N < 1 || N > 8 || !xi || !w) return fail(nullptr, DG_ERR_ARG, "dg_lgl_nodes: need 1 <= N <= 8 and arrays");
  dg::Basis b = dg::make_basis(N);
  std::memcpy(xi, b.x.data(), sizeof(double) * (N + 1));
  std::memcpy(w, b.w.data(), sizeof(double) * (N + 1));
  return DG_OK;
}

const char* dg_last_error(const dg_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

int dg_init_mesh(dg_ctx** out, const dg_mesh_desc* m, const dg_phys* p, const dg_options* o, void* stream) {
  if (!out || !m || !p || !o) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: null argument");
  *out = nullptr;
  if (m->N < 1 || m->N > 8) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: N must be in 1..8");
  if (m->K < 1 || !m->X || !m->nbr) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: empty mesh");
  if (o->precision != DG_FP64 && o->precision != DG_FP32_MIXED)
    return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: bad precision");
  if (o->vol_flux < 0 || o->vol_flux > 2) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: bad vol_flux");
  if (p->suth_S > 0.0 && !(p->T_ref > 0.0))
    return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: Sutherland's law needs T_ref > 0");
  if (o->surf_flux < 0 || o->surf_flux > 2) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: bad surf_flux");
  if (!(p->rho_ref >= 0.0)) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: rho_ref must be >= 0");
  if (p->law < 0 || p->law > 1) return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: bad wall law");
  if (!(p->gamma > 1.0) || !(p->R > 0.0) || !(p->mu >= 0.0) || !(p->Pr > 0.0))
    return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: bad gas constants");
  dg_ctx* c = new dg_ctx();
  c->N = m->N; c->n = m->N + 1; c->n2 = c->n * c->n; c->n3 = c->n2 * c->n; c->K = m->K;
  c->S = (size_t)c->K * c->n3;
  c->phys = *p; c->opts = *o;
  c->stream = static_cast<cudaStream_t>(stream);
  std::string gerr = dg::build_geometry(c->geo, c->N, c->K, m->X, m->nbr, m->nbr_face, m->orient, p->hwm);
  if (!gerr.empty()) { delete c; return fail(nullptr, DG_ERR_MESH, "dg_init_mesh: " + gerr); }
  if (c->geo.n_wall > 0 && o->viscous && !(p->hwm > 0.0)) {
    delete c;
    return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: wall faces need hwm > 0");
  }
  c->F = (int)c->geo.faces.size();
  if (c->geo.n_bc > 0) {
    bool has_in = false, has_out = false;
    for (int f = c->geo.n_interior + c->geo.n_wall; f < c->F; ++f) {
      has_in |= c->geo.faces[f].eS == dg::BC_CODE_INFLOW;
      has_out |= c->geo.faces[f].eS == dg::BC_CODE_OUTFLOW;
    }
    const double* ui = p->U_in;
    const double pin = (p->gamma - 1.0) * (ui[4] - 0.5 * (ui[1] * ui[1] + ui[2] * ui[2] + ui[3] * ui[3]) / ui[0]);
    if ((has_in && !(ui[0] > 0.0 && pin > 0.0)) || (has_out && !(p->p_out > 0.0))) {
      delete c;
      return fail(nullptr, DG_ERR_ARG, "dg_init_mesh: inflow faces need U_in with positive density and pressure, "
                                       "outflow faces a positive p_out");
    }
  }
  // physics constants for the kernels
  dg::PhysDev& ph = c->ph;
  ph.gamma = p->gamma; ph.gm1 = p->gamma - 1.0; ph.R = p->R; ph.mu = p->mu; ph.Pr = p->Pr;
  ph.cp = p->gamma * p->R / (p->gamma - 1.0); ph.kcond = p->mu * ph.cp / p->Pr; ph.rcp_R = 1.0 / p->R;
  ph.rgm1 = 1.0 / (p->gamma - 1.0); ph.cp_Pr = ph.cp / p->Pr;
  ph.suth_S = p->suth_S > 0.0 ? p->suth_S : 0.0;
  ph.suth_C = ph.suth_S > 0.0 ? p->mu * (p->T_ref + p->suth_S) / (p->T_ref * std::sqrt(p->T_ref)) : 0.0;
  ph.p_ref = p->p_ref;
  ph.rho_ref = p->rho_ref;
  ph.h_ref = p->rho_ref > 0.0 ? p->gamma / (p->gamma - 1.0) * p->p_ref / p->rho_ref : 0.0;
  for (int d = 0; d < 3; ++d) ph.f[d] = p->force[d];
  ph.kappa = p->kappa; ph.B = p->B; ph.hwm = p->hwm; ph.law = p->law;
  ph.vol_flux = o->vol_flux; ph.surf_flux = o->surf_flux; ph.viscous = o->viscous ? 1 : 0;
  for (int v = 0; v < 5; ++v) ph.U_in[v] = p->U_in[v];
  ph.p_out = p->p_out;
  ph.T_wall = p->T_wall;
  ph.wm_maxit = kWallSolveMaxIter;
  ph.lift_df = 0;
  ph.sutherland = ph.suth_S > 0.0 ? 1 : 0;
  ph.fs_diff = (o->precision == DG_FP32_MIXED && o->vol_flux == DG_VOL_KEP_PIROZZOLI) ? 1 : 0;
  ph.has_force = (ph.f[0] != 0.0 || ph.f[1] != 0.0 || ph.f[2] != 0.0) ? 1 : 0;
  ph.f32c.p_ref = (float)ph.p_ref; ph.f32c.rcp_R = (float)ph.rcp_R; ph.f32c.rgm1 = (float)ph.rgm1;
  ph.f32c.gamma = (float)ph.gamma; ph.f32c.mu = (float)ph.mu; ph.f32c.kcond = (float)ph.kcond;
  ph.f32c.cp_Pr = (float)ph.cp_Pr; ph.f32c.suth_C = (float)ph.suth_C; ph.f32c.suth_S = (float)ph.suth_S;
  ph.f32c.rho_ref = (float)ph.rho_ref; ph.f32c.h_ref = (float)ph.h_ref;
  {
    // Q(t) = 1 - 2t/3 + 8t^2/15 - 16t^3/35 + 128t^4/315, times 2 / (gamma - 1)
    const double qc[5] = {1.0, -2.0 / 3.0, 8.0 / 15.0, -16.0 / 35.0, 128.0 / 315.0};
    for (int c = 0; c < 5; ++c) {
      ph.ec_q[c] = 2.0 * ph.rgm1 * qc[c];
      ph.f32c.ec_q[c] = (float)ph.ec_q[c];
    }
  }
  ph.f32c.g_gm1 = (float)(p->gamma / (p->gamma - 1.0));
  ph.f32c.h_p = p->rho_ref > 0.0 ? 0.0f : (float)p->p_ref;
  ph.f32c.h_r = p->rho_ref > 0.0 ? (float)(p->p_ref / p->rho_ref) : 0.0f;
  ph.f32c.T_lift = p->rho_ref > 0.0 ? (float)(p->p_ref / (p->rho_ref * p->R)) : 0.0f;
  cudaGetDevice(&c->device);
  // device storage
  const size_t S = c->S, n2 = c->n2;
  const bool f32 = o->precision == DG_FP32_MIXED;
  const size_t rs = f32 ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(alloc(&c->U, 5 * S));
  chk(alloc(&c->dU, 5 * S));
  chk(alloc(&c->io, 5 * S));
  chk(alloc(&c->io2, 5 * S));
  chk(cudaMalloc(&c->Ja, 9 * S * rs));
  chk(cudaMalloc(&c->invJ, S * rs));
  chk(alloc(&c->fgeo, 4 * (size_t)c->F * n2));
  chk(alloc(&c->nbr, 6 * (size_t)c->K));
  chk(alloc(&c->elem_face, 6 * (size_t)c->K));
  chk(alloc(&c->faces, (size_t)c->F));
  chk(alloc(&c->ws_elem, (size_t)c->geo.n_wall * n2));
  chk(alloc(&c->ws_lag, (size_t)c->geo.n_wall * n2 * 3 * c->n));
  chk(alloc(&c->tau, (size_t)c->geo.n_wall * n2 * 3));
  chk(cudaMalloc(&c->Rv, (o->viscous ? 4 * S : 1) * rs));
  chk(cudaMalloc(&c->Gf, (o->viscous ? 24 * (size_t)c->K * n2 : 1) * rs));
  chk(cudaMalloc(&c->Fs, (ph.fs_diff ? 10 : 5) * (size_t)c->F * n2 * rs));
  if (f32) chk(alloc(&c->W32, 9 * S));  // primitives and the velocity's low parts
  if (!f32 && o->viscous) {
    chk(alloc(&c->W64, 7 * S));
    chk(alloc(&c->JaJ, 9 * S));
    chk(alloc(&c->Mj, 6 * S));
  }
  if (c->geo.n_wall > 0) {
    chk(alloc(&c->wm_t, (size_t)c->geo.n_wall * n2));
    chk(cudaMemset(c->wm_t, 0xff, (size_t)c->geo.n_wall * n2 * sizeof(double)));  // NaN: no guess yet
  }
  if (c->geo.n_halo > 0) {
    const size_t nh = (size_t)c->geo.n_halo;
    chk(alloc(&c->halo_U, nh * 5 * n2));
    chk(alloc(&c->send_U, nh * 5 * n2));
    chk(cudaMalloc(&c->halo_G, nh * 4 * n2 * rs));
    chk(cudaMalloc(&c->send_G, nh * 4 * n2 * rs));
  }
  chk(alloc(&c->status, 1));
  if (e != cudaSuccess) { free_all(c); delete c; return cuda_fail(nullptr, e, "dg_init_mesh: allocation"); }
  // uploads (metrics transposed to [9][S], comp-major for coalesced loads)
  {
    std::vector<double> ja(9 * S), ij(S);
    for (size_t x = 0; x < S; ++x) {
      for (int cc = 0; cc < 9; ++cc) ja[cc * S + x] = c->geo.Ja[x * 9 + cc];
      ij[x] = 1.0 / c->geo.J[x];
    }
    if (f32) {
      std::vector<float> ja32(ja.begin(), ja.end()), ij32(ij.begin(), ij.end());
      chk(cudaMemcpy(c->Ja, ja32.data(), ja32.size() * sizeof(float), cudaMemcpyHostToDevice));
      chk(cudaMemcpy(c->invJ, ij32.data(), ij32.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      chk(cudaMemcpy(c->Ja, ja.data(), ja.size() * sizeof(double), cudaMemcpyHostToDevice));
      chk(cudaMemcpy(c->invJ, ij.data(), ij.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (c->JaJ) {
      // the lifting kernel's metric products: Ja^n_d / J (reference to
      // physical gradient) and the symmetric (Ja^n . Ja^m) / J (the heat flux
      // projected on Ja^n straight from the reference-space gradient of T),
      // M in the order 00, 11, 22, 01, 02, 12
      // (one component at a time: the host holds one extra array of S values)
      std::vector<double> buf(S);
      for (int cc = 0; cc < 9; ++cc) {
        for (size_t x = 0; x < S; ++x) buf[x] = ja[cc * S + x] * ij[x];
        chk(cudaMemcpy(c->JaJ + cc * S, buf.data(), S * sizeof(double), cudaMemcpyHostToDevice));
      }
      static const int mn[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
      for (int r = 0; r < 6; ++r) {
        const int a = mn[r][0], b = mn[r][1];
        for (size_t x = 0; x < S; ++x) {
          double dot = 0.0;
          for (int d = 0; d < 3; ++d) dot += ja[(a * 3 + d) * S + x] * ja[(b * 3 + d) * S + x];
          buf[x] = dot * ij[x];
        }
        chk(cudaMemcpy(c->Mj + r * S, buf.data(), S * sizeof(double), cudaMemcpyHostToDevice));
      }
    }
  }
  chk(cudaMemcpy(c->fgeo, c->geo.fgeo.data(), c->geo.fgeo.size() * sizeof(double), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->nbr, c->geo.nbr.data(), c->geo.nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->elem_face, c->geo.elem_face.data(), c->geo.elem_face.size() * sizeof(int),
                 cudaMemcpyHostToDevice));
  {
    std::vector<int4> fc(c->F);
    for (int f = 0; f < c->F; ++f) {
      const dg::Face& x = c->geo.faces[f];
      // interior faces: slave face | 8 orientation; halo faces: master flag | 8 o_own
      const bool packed = (int)f < c->geo.n_interior || (int)f >= c->F - c->geo.n_halo;
      fc[f] = make_int4(x.eM, x.lM, x.eS, packed ? (x.lS | (x.o << 3)) : x.lS);
    }
    if (c->F) chk(cudaMemcpy(c->faces, fc.data(), fc.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  if (c->geo.n_wall) {
    chk(cudaMemcpy(c->ws_elem, c->geo.ws_elem.data(), c->geo.ws_elem.size() * sizeof(int), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(c->ws_lag, c->geo.ws_lag.data(), c->geo.ws_lag.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (c->geo.n_wall) {
    // surface quadrature weight of every wall node (mean wall shear)
    std::vector<double> wq((size_t)c->geo.n_wall * n2);
    const size_t FN = (size_t)c->F * n2;
    for (int wf = 0; wf < c->geo.n_wall; ++wf)
      for (size_t ab = 0; ab < n2; ++ab) {
        const size_t f = (size_t)(c->geo.n_interior + wf);
        const double sface = c->geo.fgeo[3 * FN + f * n2 + ab];
        wq[wf * n2 + ab] = c->geo.basis.w[ab % c->n] * c->geo.basis.w[ab / c->n] * sface;
        c->wq_total += wq[wf * n2 + ab];
      }
    chk(alloc(&c->wq, wq.size()));
    chk(cudaMemcpy(c->wq, wq.data(), wq.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (c->geo.n_wall) {
    // the wall-model kernel's side stream, at the device's highest priority
    int least = 0, greatest = 0;
    chk(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    chk(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, greatest));
    chk(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    chk(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
  }
  chk(cudaMemset(c->status, 0, sizeof(int)));
  chk(cudaMemset(c->dU, 0, 5 * S * sizeof(double)));
  if (e != cudaSuccess) { free_all(c); delete c; return cuda_fail(nullptr, e, "dg_init_mesh: upload"); }
  // FP64 at N = 7: the volume kernel's pair metric sums
  if (c->N == 7 && o->precision == DG_FP64) {
    e = alloc(&c->pairA, (size_t)16128 * c->K);
    if (e == cudaSuccess) {
      const long long work = (long long)c->K * 576;
      dg::k_pair_metric_sums<<<(unsigned)((work + 255) / 256), 256, 0, c->stream>>>(
          c->K, static_cast<const double*>(c->Ja), c->pairA);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) { free_all(c); delete c; return cuda_fail(nullptr, e, "dg_init_mesh: pair sums"); }
  }
  // odd N, FP64 viscous form: the double-float lifting by default
  if (c->N % 2 == 1 && o->precision == DG_FP64 && o->viscous) {
    const int rc = dg_set_lifting_arithmetic(c, 1);
    if (rc != DG_OK) {
      const std::string msg = c->err;
      free_all(c); delete c;
      return fail(nullptr, rc, "dg_init_mesh: " + msg);
    }
  }
  *out = c;
  return DG_OK;
}

int dg_destroy(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return DG_OK;
}

int dg_set_stream(dg_ctx* c, void* stream) {
  if (!c) return DG_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return DG_OK;
}

int dg_set_overlap(dg_ctx* c, int enable) {
  if (!c) return DG_ERR_ARG;
  c->overlap = enable != 0;
  return DG_OK;
}

int dg_sizes(const dg_ctx* c, int* N, int* K, long long* n_state) {
  if (!c) return DG_ERR_ARG;
  if (N) *N = c->N;
  if (K) *K = c->K;
  if (n_state) *n_state = (long long)(5 * c->S);
  return DG_OK;
}

int dg_set_state(dg_ctx* c, const double* U, int on_device) {
  if (!c || !U) return c ? fail(c, DG_ERR_ARG, "dg_set_state: null U") : DG_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(c->U, U, 5 * c->S * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_set_state");
  if (!on_device) {
    e = cudaStreamSynchronize(c->stream);  // the caller may reuse a pageable buffer
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_set_state");
  }
  c->state_set = true;
  c->w32_of_U = false;
  c->w64_of_U = false;
  // a new state starts the wall-law solves afresh (results then depend only
  // on the sequence of evaluations since the last dg_set_state)
  if (c->wm_t) {
    e = cudaMemsetAsync(c->wm_t, 0xff, (size_t)c->geo.n_wall * c->n2 * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_set_state");
  }
  return DG_OK;
}

int dg_get_state(dg_ctx* c, double* U, int on_device) {
  if (!c || !U) return c ? fail(c, DG_ERR_ARG, "dg_get_state: null U") : DG_ERR_ARG;
  if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_get_state: state not set");
  cudaError_t e = cudaMemcpyAsync(U, c->U, 5 * c->S * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_get_state");
  return DG_OK;
}

int dg_time_derivative(dg_ctx* c, const double* U, double* Ut, double t, int on_device) {
  (void)t;  // the operator is autonomous (constant body force)
  if (!c || !Ut) return c ? fail(c, DG_ERR_ARG, "dg_time_derivative: null Ut") : DG_ERR_ARG;
  const size_t bytes = 5 * c->S * sizeof(double);
  const double* Uin = U;
  cudaError_t e;
  if (!U) {
    if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_time_derivative: state not set");
    Uin = c->U;
  } else if (!on_device) {
    e = cudaMemcpyAsync(c->io, U, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_time_derivative: upload");
    Uin = c->io;
  }
  double* out = on_device ? Ut : c->io2;
  int rc = launch(c, Uin, 0, out, 0, 0, 0, 0, nullptr);
  if (rc != DG_OK) return rc;
  if (!on_device) {
    e = cudaMemcpyAsync(Ut, out, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_time_derivative: download");
  }
  return DG_OK;
}

int dg_rk_stage(dg_ctx* c, int s, double t, double dt) {
  (void)t;
  if (!c) return DG_ERR_ARG;
  if (s < 0 || s > 4) return fail(c, DG_ERR_ARG, "dg_rk_stage: stage must be 0..4");
  if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_rk_stage: state not set");
  return launch(c, c->U, 1, nullptr, kRkA[s], kRkB[s], dt, s > 0 ? 1 : 0, c->U);
}

// Independent host states through the stages, two device slots deep: the
// copy of item i + 1 in and of item i - 1 out run on their own streams (the
// two copy engines) while item i computes on the context's stream.
int dg_rk_stage_batch(dg_ctx* c, int nitems, const double* const* U_in, double* const* U_out, int nstages,
                      double t, double dt) {
  (void)t;  // the operator is autonomous (constant body force)
  if (!c) return DG_ERR_ARG;
  if (nitems < 0 || nstages < 1 || nstages > 5 || (nitems > 0 && (!U_in || !U_out)))
    return fail(c, DG_ERR_ARG, "dg_rk_stage_batch: bad item count, stage count or arrays");
  for (int i = 0; i < nitems; ++i)
    if (!U_in[i] || !U_out[i]) return fail(c, DG_ERR_ARG, "dg_rk_stage_batch: null item buffer");
  if (c->geo.n_halo > 0)
    return fail(c, DG_ERR_ARG, "dg_rk_stage_batch: a partitioned context evaluates in phases");
  if (nitems == 0) return DG_OK;
  const size_t n5 = 5 * c->S, bytes = n5 * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  if (!c->cp_in) {
    for (int k = 0; k < 2; ++k) {
      chk(alloc(&c->bU[k], n5));
      chk(alloc(&c->bdU[k], n5));
      chk(cudaEventCreateWithFlags(&c->ev_loaded[k], cudaEventDisableTiming));
      chk(cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming));
      chk(cudaEventCreateWithFlags(&c->ev_freed[k], cudaEventDisableTiming));
    }
    chk(cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking));
    chk(cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking));
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_rk_stage_batch: slots");
  }
  // the slots start after the work already queued on the context's stream
  chk(cudaEventRecord(c->ev_done[0], c->stream));
  chk(cudaStreamWaitEvent(c->cp_in, c->ev_done[0], 0));
  int rc = DG_OK;
  for (int i = 0; i < nitems && e == cudaSuccess && rc == DG_OK; ++i) {
    const int k = i & 1;
    // slot k is free once the result of item i - 2 has left it
    if (i >= 2) chk(cudaStreamWaitEvent(c->cp_in, c->ev_freed[k], 0));
    chk(cudaMemcpyAsync(c->bU[k], U_in[i], bytes, cudaMemcpyHostToDevice, c->cp_in));
    chk(cudaEventRecord(c->ev_loaded[k], c->cp_in));
    chk(cudaStreamWaitEvent(c->stream, c->ev_loaded[k], 0));
    // each item starts the wall-law solves afresh, as after dg_set_state
    if (c->wm_t) chk(cudaMemsetAsync(c->wm_t, 0xff, (size_t)c->geo.n_wall * c->n2 * sizeof(double), c->stream));
    for (int st = 0; st < nstages && e == cudaSuccess && rc == DG_OK; ++st)
      rc = launch(c, c->bU[k], 1, nullptr, kRkA[st], kRkB[st], dt, st > 0 ? 1 : 0, c->bU[k], c->bdU[k]);
    chk(cudaEventRecord(c->ev_done[k], c->stream));
    chk(cudaStreamWaitEvent(c->cp_out, c->ev_done[k], 0));
    chk(cudaMemcpyAsync(U_out[i], c->bU[k], bytes, cudaMemcpyDeviceToHost, c->cp_out));
    chk(cudaEventRecord(c->ev_freed[k], c->cp_out));
  }
  // the context's own stream continues after the last result is out
  chk(cudaEventRecord(c->ev_freed[0], c->cp_out));
  chk(cudaStreamWaitEvent(c->stream, c->ev_freed[0], 0));
  const cudaError_t es = cudaStreamSynchronize(c->cp_out);
  const cudaError_t ec = cudaStreamSynchronize(c->stream);
  if (rc != DG_OK) return rc;
  if (e == cudaSuccess) e = es != cudaSuccess ? es : ec;
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_rk_stage_batch");
  return DG_OK;
}

int dg_rk_steps(dg_ctx* c, double t, double dt, int nsteps) {
  if (!c || nsteps < 0) return c ? fail(c, DG_ERR_ARG, "dg_rk_steps: nsteps < 0") : DG_ERR_ARG;
  for (int it = 0; it < nsteps; ++it)
    for (int s = 0; s < 5; ++s) {
      int rc = dg_rk_stage(c, s, t + (it + kRkC[s]) * dt, dt);
      if (rc != DG_OK) return rc;
    }
  return DG_OK;
}

int dg_halo_buffers(dg_ctx* c, int* n_halo, void** send_U, void** recv_U, void** send_G, void** recv_G) {
  if (!c || !n_halo) return c ? fail(c, DG_ERR_ARG, "dg_halo_buffers: null n_halo") : DG_ERR_ARG;
  *n_halo = c->geo.n_halo;
  if (send_U) *send_U = c->send_U;
  if (recv_U) *recv_U = c->halo_U;
  if (send_G) *send_G = c->send_G;
  if (recv_G) *recv_G = c->halo_G;
  return DG_OK;
}

int dg_halo_geometry(dg_ctx* c, double* fgeo) {
  if (!c || !fgeo) return c ? fail(c, DG_ERR_ARG, "dg_halo_geometry: null output") : DG_ERR_ARG;
  const size_t n2 = c->n2, F = (size_t)c->F, f0 = F - (size_t)c->geo.n_halo;
  for (size_t h = 0; h < (size_t)c->geo.n_halo; ++h)
    for (int k = 0; k < 4; ++k)
      std::memcpy(fgeo + (h * 4 + k) * n2, c->geo.fgeo.data() + k * F * n2 + (f0 + h) * n2, n2 * sizeof(double));
  return DG_OK;
}

int dg_halo_set_geometry(dg_ctx* c, const double* fgeo) {
  if (!c || !fgeo) return c ? fail(c, DG_ERR_ARG, "dg_halo_set_geometry: null input") : DG_ERR_ARG;
  const size_t n2 = c->n2, F = (size_t)c->F, f0 = F - (size_t)c->geo.n_halo;
  for (size_t h = 0; h < (size_t)c->geo.n_halo; ++h) {
    if (c->geo.faces[f0 + h].lS) continue;  // the local element is the master: keep its own
    for (int k = 0; k < 4; ++k)
      std::memcpy(c->geo.fgeo.data() + k * F * n2 + (f0 + h) * n2, fgeo + (h * 4 + k) * n2, n2 * sizeof(double));
  }
  cudaError_t e = cudaMemcpy(c->fgeo, c->geo.fgeo.data(), c->geo.fgeo.size() * sizeof(double),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_halo_set_geometry");
  return DG_OK;
}

int dg_stage_phase(dg_ctx* c, int phase, int s, double t, double dt) {
  (void)t;
  if (!c) return DG_ERR_ARG;
  if (s < 0 || s > 4) return fail(c, DG_ERR_ARG, "dg_stage_phase: stage must be 0..4");
  if (phase != 1 && phase != 2 && phase != 4) return fail(c, DG_ERR_ARG, "dg_stage_phase: phase must be 1, 2 or 4");
  if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_stage_phase: state not set");
  return launch(c, c->U, 1, nullptr, kRkA[s], kRkB[s], dt, s > 0 ? 1 : 0, c->U, nullptr, phase);
}

int dg_time_derivative_phase(dg_ctx* c, int phase, const double* U, double* Ut) {
  if (!c || !Ut) return c ? fail(c, DG_ERR_ARG, "dg_time_derivative_phase: null Ut") : DG_ERR_ARG;
  if (phase != 1 && phase != 2 && phase != 4)
    return fail(c, DG_ERR_ARG, "dg_time_derivative_phase: phase must be 1, 2 or 4");
  const double* Uin = U;
  if (!U) {
    if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_time_derivative_phase: state not set");
    Uin = c->U;
  }
  return launch(c, Uin, 0, Ut, 0, 0, 0, 0, nullptr, nullptr, phase);
}

int dg_set_params(dg_ctx* c, double kappa, double B) {
  if (!c) return DG_ERR_ARG;
  if (!(kappa > 0.0)) return fail(c, DG_ERR_ARG, "dg_set_params: kappa must be positive");
  c->phys.kappa = kappa; c->phys.B = B;
  c->ph.kappa = kappa; c->ph.B = B;
  drop_step_graph(c);  // a captured step holds the old constants
  return DG_OK;
}

int dg_set_lifting_arithmetic(dg_ctx* c, int mode) {
  if (!c) return DG_ERR_ARG;
  if (mode != 0 && mode != 1) return fail(c, DG_ERR_ARG, "dg_set_lifting_arithmetic: mode must be 0 or 1");
  const bool applies = c->N % 2 == 1 && c->opts.precision == DG_FP64 && c->opts.viscous && c->JaJ && c->W64;
  if (mode == 1 && applies && !c->lift_M2) {
    // the metric arrays as (hi, lo) pairs, split once on the device
    cudaError_t e = alloc(&c->lift_M2, 24 * c->S);
    if (e == cudaSuccess) e = alloc(&c->lift_W2, 4 * c->S);
    const long long S = (long long)c->S;
    const unsigned blocks = (unsigned)std::min<long long>((9 * S + 255) / 256, 152 * 16);
    if (e == cudaSuccess) {
      dg::k_split_pairs<<<blocks, 256, 0, c->stream>>>(9 * S, static_cast<const double*>(c->Ja), c->lift_M2);
      dg::k_split_pairs<<<blocks, 256, 0, c->stream>>>(9 * S, c->JaJ, c->lift_M2 + 9 * c->S);
      dg::k_split_pairs<<<blocks, 256, 0, c->stream>>>(6 * S, c->Mj, c->lift_M2 + 18 * c->S);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      // leave no half-built pair arrays behind: the FP64 lifting stays in use
      if (c->lift_M2) cudaFree(c->lift_M2);
      if (c->lift_W2) cudaFree(c->lift_W2);
      c->lift_M2 = nullptr;
      c->lift_W2 = nullptr;
      return cuda_fail(c, e, "dg_set_lifting_arithmetic");
    }
  }
  c->ph.lift_df = mode;
  c->w64_of_U = false;  // the next evaluation forms the stored primitives (and their pairs) again
  drop_step_graph(c);
  return DG_OK;
}

int dg_set_wall_solve_limit(dg_ctx* c, int max_iter) {
  if (!c) return DG_ERR_ARG;
  if (max_iter < 1) return fail(c, DG_ERR_ARG, "dg_set_wall_solve_limit: max_iter must be >= 1");
  c->ph.wm_maxit = max_iter;
  drop_step_graph(c);
  return DG_OK;
}

// the device scalar of the reductions (time step, kinetic energy, losses)
static int ensure_scalar(dg_ctx* c) {
  if (c->ro_scalar) return DG_OK;
  cudaError_t e = alloc(&c->ro_scalar, 1);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduction scalar allocation");
  return DG_OK;
}

static int ensure_adjoint_scratch(dg_ctx* c) {
  if (c->gUf) return DG_OK;
  int rc = ensure_scalar(c);
  if (rc != DG_OK) return rc;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  const size_t kn2 = (size_t)c->K * 6 * c->n2;
  chk(alloc(&c->gUf, 5 * kn2));
  chk(alloc(&c->gGf, 4 * kn2));
  chk(alloc(&c->gWf, 4 * kn2));
  chk(alloc(&c->gUs, (size_t)c->geo.n_wall * c->n2 * 5 + 1));
  chk(alloc(&c->gtheta, 2));
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint scratch allocation");
  return DG_OK;
}

static dg::OpArgs adjoint_args(dg_ctx* c, const double* U, const double* lam, double* gU, double* gth) {
  dg::OpArgs a{};
  a.N = c->N; a.K = c->K; a.F = c->F; a.n_interior = c->geo.n_interior; a.n_wall = c->geo.n_wall;
  a.n_bc = c->geo.n_bc;
  a.Ja = c->Ja; a.invJ = c->invJ; a.fgeo = c->fgeo; a.nbr = c->nbr; a.elem_face = c->elem_face;
  a.faces = c->faces; a.ws_elem = c->ws_elem; a.ws_lag = c->ws_lag;
  a.D = c->geo.basis.D.data(); a.w = c->geo.basis.w.data();
  a.Uin = U; a.status = c->status;
  a.lam = lam; a.gU = gU; a.gUf = c->gUf; a.gGf = c->gGf; a.gWf = c->gWf; a.gUs = c->gUs; a.gtheta = gth;
  a.JaJ = c->JaJ; a.Mj = c->Mj;
  a.n_halo = c->geo.n_halo;
  a.halo_U = c->halo_U; a.halo_G = c->halo_G; a.send_U = c->send_U; a.send_G = c->send_G;
  return a;
}

static int check_adjoint_options(dg_ctx* c, const char* who) {
  if (c->opts.precision != DG_FP64)
    return fail(c, DG_ERR_NOT_IMPLEMENTED, std::string(who) + ": the adjoint is available for FP64 contexts");
  if (c->opts.vol_flux == DG_VOL_KEP_KENNEDY_GRUBER)
    return fail(c, DG_ERR_NOT_IMPLEMENTED,
                std::string(who) + ": the adjoint covers the Pirozzoli and entropy-conserving volume fluxes");
  return DG_OK;
}

int dg_time_step(dg_ctx* c, const double* U, double cfl, double* dt) {
  if (!c || !dt || !(cfl > 0.0)) return c ? fail(c, DG_ERR_ARG, "dg_time_step: bad argument") : DG_ERR_ARG;
  const double* Uin = U ? U : c->U;
  if (!U && !c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_time_step: state not set");
  int rc = ensure_scalar(c);
  if (rc != DG_OK) return rc;
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(c->ro_scalar);
  cudaError_t e = cudaMemsetAsync(slot, 0, sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_time_step");
  if (c->opts.precision == DG_FP32_MIXED)
    dg::k_wave_speed<float><<<152 * 8, 256, 0, c->stream>>>((long long)c->S, Uin, static_cast<const float*>(c->Ja),
                                                             static_cast<const float*>(c->invJ), c->phys.gamma, slot);
  else
    dg::k_wave_speed<double><<<152 * 8, 256, 0, c->stream>>>((long long)c->S, Uin, static_cast<const double*>(c->Ja),
                                                              static_cast<const double*>(c->invJ), c->phys.gamma, slot);
  double mx = 0.0;
  e = cudaMemcpyAsync(&mx, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_time_step");
  if (!(mx > 0.0)) return fail(c, DG_ERR_NONFINITE, "dg_time_step: no finite wave speed");
  *dt = cfl * 2.0 / (2.0 * c->N + 1.0) / mx;
  return DG_OK;
}

int dg_kinetic_energy(dg_ctx* c, const double* U, double* ke) {
  if (!c || !ke) return c ? fail(c, DG_ERR_ARG, "dg_kinetic_energy: null ke") : DG_ERR_ARG;
  const double* Uin = U ? U : c->U;
  if (!U && !c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_kinetic_energy: state not set");
  cudaError_t e = cudaSuccess;
  if (!c->wJ) {
    std::vector<double> w(c->S);
    const std::vector<double>& bw = c->geo.basis.w;
    c->vol = 0.0;
    for (size_t x = 0; x < c->S; ++x) {
      const int p = (int)(x % c->n3);
      w[x] = bw[p % c->n] * bw[(p / c->n) % c->n] * bw[p / c->n2] * c->geo.J[x];
      c->vol += w[x];
    }
    e = alloc(&c->wJ, c->S);
    if (e == cudaSuccess) e = cudaMemcpy(c->wJ, w.data(), c->S * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_kinetic_energy: weights");
  }
  int rc = ensure_scalar(c);
  if (rc != DG_OK) return rc;
  e = cudaMemsetAsync(c->ro_scalar, 0, sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_kinetic_energy");
  dg::k_kinetic_energy<<<152 * 8, 256, 0, c->stream>>>((long long)c->S, Uin, c->wJ, c->ro_scalar);
  double sum = 0.0;
  e = cudaMemcpyAsync(&sum, c->ro_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_kinetic_energy");
  *ke = sum / c->vol;
  return DG_OK;
}

int dg_convert_fp32(long long n, const double* d, float* f, float* rem, const float* g, double* gd) {
  if (n < 0 || (n > 0 && (!d || !f || !rem || !g || !gd))) return DG_ERR_ARG;
  if (n == 0) return DG_OK;
  dg::k_convert_fp32<<<(unsigned)((n + 255) / 256), 256>>>(n, d, f, rem, g, gd);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

int dg_wall_shear(dg_ctx* c, const double* U, double* loss) {
  if (!c || !loss) return c ? fail(c, DG_ERR_ARG, "dg_wall_shear: null loss") : DG_ERR_ARG;
  if (c->geo.n_wall == 0 || !c->opts.viscous) return fail(c, DG_ERR_ARG, "dg_wall_shear: no wall-modelled walls");
  const double* Uin = U ? U : c->U;
  if (!U && !c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_wall_shear: state not set");
  int rc = ensure_scalar(c);
  if (rc != DG_OK) return rc;
  cudaError_t e = cudaMemsetAsync(c->ro_scalar, 0, sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_wall_shear");
  dg::OpArgs a = adjoint_args(c, Uin, nullptr, nullptr, nullptr);
  rc = dg::run_wall_loss(a, c->ph, c->wq, 1.0 / c->wq_total, 0, c->ro_scalar, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_wall_shear launch");
  e = cudaMemcpyAsync(loss, c->ro_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_wall_shear");
  return DG_OK;
}

int dg_rollout_vjp(dg_ctx* c, const double* U0, int nsteps, double dt, double* loss, double* gU0, double* gtheta) {
  if (!c) return DG_ERR_ARG;
  if (!U0 || !loss || !gU0 || nsteps < 0) return fail(c, DG_ERR_ARG, "dg_rollout_vjp: bad argument");
  int rc = check_adjoint_options(c, "dg_rollout_vjp");
  if (rc != DG_OK) return rc;
  if (c->geo.n_halo > 0)
    return fail(c, DG_ERR_NOT_IMPLEMENTED, "dg_rollout_vjp: unpartitioned contexts only (a partitioned context "
                                           "steps and differentiates in phases)");
  if (c->geo.n_wall == 0 || !c->opts.viscous)
    return fail(c, DG_ERR_ARG, "dg_rollout_vjp: the loss needs wall-modelled walls");
  rc = ensure_adjoint_scratch(c);
  if (rc != DG_OK) return rc;
  const size_t S5 = 5 * c->S, bytes = S5 * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  if (nsteps > c->ro_cap || !c->ro_ckpt) {
    if (c->ro_ckpt) cudaFree(c->ro_ckpt);
    c->ro_ckpt = nullptr;
    chk(alloc(&c->ro_ckpt, S5 * (size_t)std::max(nsteps, 1)));
    c->ro_cap = std::max(nsteps, 1);
  }
  if (!c->ro_stage) chk(alloc(&c->ro_stage, 5 * S5));
  if (!c->ro_work) chk(alloc(&c->ro_work, 6 * S5));
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_rollout_vjp: buffers");
  double *Uw = c->ro_work, *dUw = Uw + S5, *gA = dUw + S5, *gD = gA + S5, *gT = gD + S5, *lamS = gT + S5;
  double* gth = gtheta ? gtheta : c->gtheta;
  cudaStream_t st = c->stream;
  chk(cudaMemsetAsync(gth, 0, 2 * sizeof(double), st));
  chk(cudaMemsetAsync(c->ro_scalar, 0, sizeof(double), st));
  chk(cudaMemcpyAsync(Uw, U0, bytes, cudaMemcpyDeviceToDevice, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_rollout_vjp");
  // forward, one checkpoint per step (A_0 = 0: U alone restarts a step)
  for (int k = 0; k < nsteps; ++k) {
    chk(cudaMemcpyAsync(c->ro_ckpt + (size_t)k * S5, Uw, bytes, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < 5; ++s) {
      rc = launch(c, Uw, 1, nullptr, kRkA[s], kRkB[s], dt, s > 0, Uw, dUw);
      if (rc != DG_OK) return rc;
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_rollout_vjp: forward");
  // loss at the final state and its gradient
  dg::OpArgs la = adjoint_args(c, Uw, nullptr, gA, gth);
  rc = dg::run_wall_loss(la, c->ph, c->wq, 1.0 / c->wq_total, 1, c->ro_scalar, st);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_rollout_vjp: loss");
  // reverse sweep through the 2N-storage recurrence
  for (int k = nsteps - 1; k >= 0; --k) {
    chk(cudaMemcpyAsync(Uw, c->ro_ckpt + (size_t)k * S5, bytes, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < 5; ++s) {
      chk(cudaMemcpyAsync(c->ro_stage + (size_t)s * S5, Uw, bytes, cudaMemcpyDeviceToDevice, st));
      if (s < 4) {
        rc = launch(c, Uw, 1, nullptr, kRkA[s], kRkB[s], dt, s > 0, Uw, dUw);
        if (rc != DG_OK) return rc;
      }
    }
    chk(cudaMemsetAsync(gD, 0, bytes, st));
    for (int s = 4; s >= 0; --s) {
      // gD += B_s gA;  lam = dt gD;  gA += J^T lam (and gtheta);  gD = A_s gD
      rc = dg::run_axpby((long long)S5, kRkB[s], gA, 1.0, gD, st);
      if (rc == 0) rc = dg::run_axpby((long long)S5, dt, gD, 0.0, lamS, st);
      if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_rollout_vjp: axpby");
      dg::OpArgs va = adjoint_args(c, c->ro_stage + (size_t)s * S5, lamS, gT, gth);
      rc = dg::run_vjp(va, c->ph, st);
      if (rc == 0) rc = dg::run_axpby((long long)S5, 1.0, gT, 1.0, gA, st);
      if (rc == 0) rc = dg::run_axpby((long long)S5, 0.0, gD, kRkA[s], gD, st);
      if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_rollout_vjp: reverse");
    }
  }
  chk(cudaMemcpyAsync(gU0, gA, bytes, cudaMemcpyDeviceToDevice, st));
  chk(cudaMemcpyAsync(loss, c->ro_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_rollout_vjp");
  return DG_OK;
}

int dg_vjp(dg_ctx* c, const double* U, const double* lam, double* gU, double* gtheta) {
  if (!c) return DG_ERR_ARG;
  if (!lam || !gU) return fail(c, DG_ERR_ARG, "dg_vjp: null lam or gU");
  int rc = check_adjoint_options(c, "dg_vjp");
  if (rc != DG_OK) return rc;
  if (c->geo.n_halo > 0)
    return fail(c, DG_ERR_ARG, "dg_vjp: a partitioned context runs the adjoint in phases (dg_vjp_phase)");
  const double* Uin = U;
  if (!Uin) {
    if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_vjp: state not set");
    Uin = c->U;
  }
  rc = ensure_adjoint_scratch(c);
  if (rc != DG_OK) return rc;
  double* gth = gtheta ? gtheta : c->gtheta;
  cudaError_t e = cudaMemsetAsync(gth, 0, 2 * sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_vjp");
  dg::OpArgs a = adjoint_args(c, Uin, lam, gU, gth);
  rc = dg::run_vjp(a, c->ph, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_vjp launch");
  return DG_OK;
}

int dg_vjp_phase(dg_ctx* c, int phase, const double* U, const double* lam, double* gU, double* gtheta) {
  if (!c) return DG_ERR_ARG;
  if (phase < 1 || phase > 4) return fail(c, DG_ERR_ARG, "dg_vjp_phase: phase must be 1, 2, 3 or 4");
  if (c->geo.n_halo == 0) return fail(c, DG_ERR_ARG, "dg_vjp_phase: for partitioned contexts (else dg_vjp)");
  if (!lam || !gU) return fail(c, DG_ERR_ARG, "dg_vjp_phase: null lam or gU");
  int rc = check_adjoint_options(c, "dg_vjp_phase");
  if (rc != DG_OK) return rc;
  const double* Uin = U;
  if (!Uin) {
    if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_vjp_phase: state not set");
    Uin = c->U;
  }
  rc = ensure_adjoint_scratch(c);
  if (rc != DG_OK) return rc;
  double* gth = gtheta ? gtheta : c->gtheta;
  if (phase == 2) {
    cudaError_t e = cudaMemsetAsync(gth, 0, 2 * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_vjp_phase");
  }
  dg::OpArgs a = adjoint_args(c, Uin, lam, gU, gth);
  a.phase = phase;
  rc = dg::run_vjp(a, c->ph, c->stream);
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "dg_vjp_phase launch");
  return DG_OK;
}

int dg_get_rk_register(dg_ctx* c, double* dU, int on_device) {
  if (!c || !dU) return c ? fail(c, DG_ERR_ARG, "dg_get_rk_register: null dU") : DG_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(dU, c->dU, 5 * c->S * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_get_rk_register");
  return DG_OK;
}

int dg_set_rk_register(dg_ctx* c, const double* dU, int on_device) {
  if (!c || !dU) return c ? fail(c, DG_ERR_ARG, "dg_set_rk_register: null dU") : DG_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(c->dU, dU, 5 * c->S * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_set_rk_register");
  return DG_OK;
}

int dg_rk_steps_graph(dg_ctx* c, double t, double dt, int nsteps) {
  (void)t;  // the operator is autonomous
  if (!c || nsteps < 0) return c ? fail(c, DG_ERR_ARG, "dg_rk_steps_graph: nsteps < 0") : DG_ERR_ARG;
  if (!c->state_set) return fail(c, DG_ERR_NOT_INIT, "dg_rk_steps_graph: state not set");
  int rc0 = refresh_w32(c);
  if (rc0 != DG_OK) return rc0;
  cudaError_t e = cudaSuccess;
  if (!c->step_graph || c->step_graph_dt != dt) {
    if (!c->cap_stream) {
      e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(c, e, "dg_rk_steps_graph: stream");
    }
    // the capture stream must see the caller's pending work on the state
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_rk_steps_graph");
    const bool prof = c->profiling;
    cudaStream_t user = c->stream;
    c->profiling = false;
    c->stream = c->cap_stream;
    // every replay starts from a state its previous step updated: the first
    // stage must form the FP64 primitives
    c->w64_of_U = false;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = DG_OK;
    if (e == cudaSuccess)
      for (int s = 0; s < 5 && rc == DG_OK; ++s)
        rc = launch(c, c->U, 1, nullptr, kRkA[s], kRkB[s], dt, s > 0 ? 1 : 0, c->U);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    c->stream = user;
    c->profiling = prof;
    if (e == cudaSuccess) e = e2;
    if (rc != DG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(c, e, "dg_rk_steps_graph: capture"); }
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
    e = cudaGraphInstantiate(&c->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { c->step_graph = nullptr; return cuda_fail(c, e, "dg_rk_steps_graph: instantiate"); }
    c->step_graph_dt = dt;
  }
  for (int it = 0; it < nsteps; ++it) {
    e = cudaGraphLaunch(c->step_graph, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "dg_rk_steps_graph: launch");
  }
  if (nsteps > 0) c->w64_of_U = false;  // the state changed under the stored primitives
  return DG_OK;
}

int dg_check_status(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_check_status");
  if (h & dg::ST_BOUNDS)
    return fail(c, DG_ERR_DEVICE_BOUNDS, "a kernel gathered an index outside its array (bounds-checking build)");
  if (h & dg::ST_NONFINITE) return fail(c, DG_ERR_NONFINITE, "non-finite value in the state");
  if (h & dg::ST_WM_NOCONV) return fail(c, DG_ERR_WM_NOCONV, "wall-model Newton iteration did not converge");
  return DG_OK;
}

int dg_profile_enable(dg_ctx* c, int enable) {
  if (!c) return DG_ERR_ARG;
  c->profiling = enable != 0;
  c->events_used = 0;
  return DG_OK;
}

int dg_profile_read(dg_ctx* c, double* ms, int* launches) {
  if (!c || !ms || !launches) return c ? fail(c, DG_ERR_ARG, "dg_profile_read: null output") : DG_ERR_ARG;
  for (int k = 0; k < 4; ++k) { ms[k] = 0.0; launches[k] = 0; }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "dg_profile_read");
  const bool visc = c->opts.viscous != 0;
  const bool work[4] = {visc, c->geo.n_interior > 0, c->geo.n_wall > 0, true};
  // lift [0,1], face [1,2], wall [3,4], volume [5,6]
  const int from[4] = {0, 1, 3, 5}, to[4] = {1, 2, 4, 6};
  for (size_t b = 0; b + kEventsPerLaunch <= c->events_used; b += kEventsPerLaunch)
    for (int k = 0; k < 4; ++k) {
      float t = 0.0f;
      e = cudaEventElapsedTime(&t, c->events[b + from[k]], c->events[b + to[k]]);
      if (e != cudaSuccess) return cuda_fail(c, e, "dg_profile_read");
      ms[k] += t;
      if (work[k]) launches[k] += 1;
    }
  c->events_used = 0;
  return DG_OK;
}

int dg_get_metrics(const dg_ctx* c, double* Ja, double* J) {
  if (!c) return DG_ERR_ARG;
  if (Ja) std::memcpy(Ja, c->geo.Ja.data(), c->geo.Ja.size() * sizeof(double));
  if (J) std::memcpy(J, c->geo.J.data(), c->geo.J.size() * sizeof(double));
  return DG_OK;
}

}  // extern "C"
