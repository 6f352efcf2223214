// ot_prox_evaluate_noalloc: the state evaluation of ot_prox_evaluate
// (residual, objective, duality-gap certificate) for a state the caller
// holds, with every byte of scratch in a fixed device array of this file.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need an answer -- code that runs inside another framework's memory
// pool which forbids allocations outside it, or a latency-critical loop where
// cudaMalloc/cudaFree would synchronise the device.  This entry point calls
// no cudaMalloc, cudaFree or any allocating library routine.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"

namespace otp {
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
}  // namespace otp

using namespace otp;

namespace {

// Scratch layout (doubles): partials [kMaxBlocks][kNumSums], certificate
// partials [kMaxBlocks][4], sums [kNumSums], certificate [4].
constexpr int kMaxBlocks = 152 * 8;   // the evaluation grid never exceeds this
constexpr int kScratchDoubles = kMaxBlocks * (kNumSums + 4) + kNumSums + 4;
constexpr int kMaxDevices = 64;
constexpr long long kMaxElems = 2147483647LL;   // B * H * W

// Every GPU that loads the library holds this array (about 114 KB) until
// the process exits.  Host code must not use its name as an address.
static __device__ __align__(256) double g_eval_scratch[kScratchDoubles];

std::mutex g_setup_mu;
struct ScratchEntry {
  unsigned long long ctx_id;   // context the address belongs to (0 = none yet)
  double* ptr;
};
ScratchEntry g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the context current on this thread (the device's primary
// context once the runtime has set it up).  A cudaDeviceReset by the caller
// ends that context; the next one has a new id, so an address looked up in
// the old one is never reused.
int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* p = nullptr;
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) != cudaSuccess ||
        r1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) != cudaSuccess ||
        r2 != cudaDriverEntryPointSuccess)
      return fail(OT_ECUDA, "ot_prox_evaluate_noalloc: driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
    get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    get_id = reinterpret_cast<CtxGetIdFn>(q);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS)
    return fail(OT_ECUDA, "ot_prox_evaluate_noalloc: no current CUDA context");
  return OT_OK;
}

// Device address of the scratch array in the current device's context,
// looked up once per device and context (the first call on a device, and the
// first after a cudaDeviceReset, does this set-up).
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "ot_prox_evaluate_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: device %d out of range", dev);
  // makes the device's primary context current on this thread (set up if needed)
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "ot_prox_evaluate_noalloc: cudaSetDevice");
  unsigned long long ctx_id = 0;
  int rc = current_context_id(&ctx_id);
  if (rc != OT_OK) return rc;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch[dev].ctx_id != ctx_id || !g_scratch[dev].ptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "ot_prox_evaluate_noalloc: cudaGetSymbolAddress");
    g_scratch[dev].ptr = static_cast<double*>(p);
    g_scratch[dev].ctx_id = ctx_id;
  }
  *out = g_scratch[dev].ptr;
  return OT_OK;
}

}  // namespace

extern "C" int ot_prox_evaluate_noalloc(const ot_prox_params* prm, const float* p0, const float* p1,
                                        const float* Mx, const float* My, const float* x0, const float* x1,
                                        const float* r, const float* a, ot_prox_result* res, void* cuda_stream) {
  if (!prm || !res) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: params and res must be non-NULL");
  const ot_prox_params& p = *prm;
  if (p.B < 1 || p.H < 1 || p.W < 1) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: B, H, W must be >= 1");
  if ((long long)p.B * p.H * p.W > kMaxElems)
    return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: B*H*W = %lld exceeds the maximum %lld",
                (long long)p.B * p.H * p.W, kMaxElems);
  if (p.mode < 0 || p.mode > 2) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: unknown mode %d", p.mode);
  if (p.norm != OT_NORM_ISO && p.norm != OT_NORM_ANISO) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: unknown norm");
  if (p.p_exp != 1 && p.p_exp != 2) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: p_exp must be 1 or 2");
  if (!(p.mu > 0) || !(p.rho > 0)) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: mu and rho must be > 0");
  if (!p0 || !p1 || !Mx || !My || !a || (p.mode == OT_MODE_PROX && !x0) || (p.mode != OT_MODE_EVAL && !x1) ||
      (!p.balanced && !r))
    return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: a required array pointer is NULL");

  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != OT_OK) return rc;

  Geometry G;
  G.B = p.B;
  G.H = p.H;
  G.W = p.W;
  G.Wp = p.W;                       // dense caller layout
  G.plane = (long long)p.H * p.W;
  G.tiles_x = G.tiles_y = 1;
  const int nb = cert_num_blocks(G);
  if (nb > kMaxBlocks) return fail(OT_EINVAL, "ot_prox_evaluate_noalloc: %d blocks exceed the scratch", nb);
  CertCoeffs cc;
  cc.mu = p.mu;
  cc.rho = p.rho;
  cc.iso = p.norm == OT_NORM_ISO;
  cc.pexp = p.p_exp;
  cc.mode = p.mode;
  cc.balanced = p.balanced;
  double* partials = scratch;
  double* cert_partials = scratch + (size_t)kMaxBlocks * kNumSums;
  double* sums = cert_partials + (size_t)kMaxBlocks * 4;
  double* cert = sums + kNumSums;
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = launch_evaluate(G, cc, Mx, My, a, x0, x1, r, p0, p1, partials, sums, cert_partials, cert, st);
  double h[kNumSums + 4];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ot_prox_evaluate_noalloc");

  memset(res, 0, sizeof *res);
  const double sp = fmax(sqrt(h[6]), 1e-30);
  res->res_pri = sqrt(h[0]) / sp;
  double obj = h[3];
  if (!p.balanced) obj += p.mu * h[4];
  obj += h[5] / (2.0 * p.rho);
  res->objective = obj;
  res->dual_obj = h[kNumSums + 1];
  res->primal_feasible = h[kNumSums + 2];
  res->rel_gap = (res->primal_feasible - res->dual_obj) / fmax(fabs(res->primal_feasible), 1e-30);
  bool bad = h[7] > 0;
  for (int k = 0; k < 7; ++k) bad = bad || !isfinite(h[k]);
  res->status = bad ? OT_ENONFINITE : OT_OK;
  if (bad) return fail(OT_ENONFINITE, "ot_prox_evaluate_noalloc: non-finite values in the state");
  return OT_OK;
}
