// noalloc.cu -- operator evaluation whose scratch lives in a static device
// array, for callers that must not allocate device memory when they call.
//
// dg_time_derivative keeps its inter-kernel scratch (the weak viscous
// divergence, the per-face viscous fluxes and the surface fluxes) in buffers
// that the context allocated with cudaMalloc.  This variant takes that
// scratch from g_scratch below instead: a file-scope __device__ array of
// DG_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds until
// the process exits.  It calls no allocating routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/dg.h"
#include "ops.h"

static __device__ __align__(256) unsigned char g_scratch[DG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device.  In host code the
// symbol g_scratch names a host-side stand-in, not device memory, so the
// address must come from cudaGetSymbolAddress with the device current; it is
// looked up once per device and cached.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// implemented in api.cu: fills the operator arguments from a context
namespace dg {
int noalloc_args(dg_ctx* c, const double* U, double* Ut, OpArgs* a, const PhysDev** ph, cudaStream_t* s,
                 int* device, size_t* rv_bytes, size_t* gf_bytes, size_t* fs_bytes);
void noalloc_done(dg_ctx* c, const double* U, bool ok);
int noalloc_fail(dg_ctx* c, int code, const std::string& msg);
}  // namespace dg

extern "C" int dg_time_derivative_noalloc(dg_ctx* c, const double* U, double* Ut) {
  if (!c) return DG_ERR_ARG;
  if (!U || !Ut) return dg::noalloc_fail(c, DG_ERR_ARG, "dg_time_derivative_noalloc: null U or Ut");
  dg::OpArgs a{};
  const dg::PhysDev* ph = nullptr;
  cudaStream_t stream = nullptr;
  size_t rv = 0, gf = 0, fs = 0;
  int ctx_device = 0;
  int rc = dg::noalloc_args(c, U, Ut, &a, &ph, &stream, &ctx_device, &rv, &gf, &fs);
  if (rc != DG_OK) return rc;
  if (a.n_halo > 0)
    return dg::noalloc_fail(c, DG_ERR_ARG, "dg_time_derivative_noalloc: not for partitioned contexts");
  const size_t need = align256(rv) + align256(gf) + align256(fs);
  if (need > (size_t)DG_NOALLOC_SCRATCH_BYTES)
    return dg::noalloc_fail(c, DG_ERR_ARG,
                            "dg_time_derivative_noalloc: mesh needs " + std::to_string(need) +
                                " scratch bytes, more than the static limit of " +
                                std::to_string((size_t)DG_NOALLOC_SCRATCH_BYTES));
  // The scratch array used must be the one on the context's device, and the
  // kernels run on the current device: the two must agree.
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess)
    return dg::noalloc_fail(c, DG_ERR_CUDA, std::string("dg_time_derivative_noalloc: ") + cudaGetErrorString(e));
  if (device != ctx_device)
    return dg::noalloc_fail(c, DG_ERR_ARG,
                            "dg_time_derivative_noalloc: the current device (" + std::to_string(device) +
                                ") is not the context's device (" + std::to_string(ctx_device) + ")");
  void* base = nullptr;
  e = scratch_address(ctx_device, &base);
  if (e != cudaSuccess)
    return dg::noalloc_fail(c, DG_ERR_CUDA, std::string("dg_time_derivative_noalloc: ") + cudaGetErrorString(e));
  // Every scratch word is written before it is read within one call (each
  // element writes R_v at all its nodes and its outward viscous flux at all
  // its face nodes; every face writes its surface flux), so nothing needs
  // clearing between calls.
  unsigned char* p = static_cast<unsigned char*>(base);
  a.Rv = p;
  a.Gf = p + align256(rv);
  a.Fs = p + align256(rv) + align256(gf);
  a.tau = nullptr;
  a.ev = nullptr;
  rc = dg::run_operator(a, *ph, stream);
  dg::noalloc_done(c, U, rc == 0);
  if (rc != 0)
    return dg::noalloc_fail(c, DG_ERR_CUDA,
                            std::string("dg_time_derivative_noalloc: ") + cudaGetErrorString((cudaError_t)rc));
  return DG_OK;
}
