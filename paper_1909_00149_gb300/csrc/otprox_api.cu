// C ABI of the Algorithm 1 solver (include/otprox.h): handle lifetime,
// argument validation, host/device copies, the stopping-check loop and
// CUDA-graph replay of a check interval.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"
#include "prox_handle.cuh"

namespace otp {
thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(OT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(OT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace otp

using namespace otp;

#define OT_CUDA(call, what)                        \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)



// Leave k SMs free of the persistent TMA iteration kernel (one CTA per SM),
// so that a one-CTA kernel on another stream can run beside it.
void prox_reserve_sms(ot_prox* h, int k) {
  int n_sm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n_sm = 152;
  const int cap = n_sm - k > 1 ? n_sm - k : 1;
  if (h->tma_grid > cap) h->tma_grid = cap;
}

extern "C" {

const char* ot_last_error(void) { return g_err.c_str(); }

void ot_prox_default_params(ot_prox_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->B = p->H = p->W = 1;
  p->mode = OT_MODE_PROX;
  p->norm = OT_NORM_ISO;
  p->balanced = 0;
  p->p_exp = 1;
  p->mu = 3.0;
  p->rho = 0.01;
  p->tau1 = p->tau2 = 0.0;
  p->tol = 1e-5;
  p->max_iter = 100000;
  p->check_every = 10;
  p->kernel = OT_KERNEL_AUTO;
  p->use_graph = 1;
  p->algorithm = OT_ALG_ALG1;
  p->precision = OT_PREC_FP32;
  p->beta = 1.0;
  p->tb_depth = 4;
}

double ot_lambda_max(int32_t H, int32_t W) {
  const double pi = 3.14159265358979323846;
  const double sh = sin(pi * (double)(H - 1) / (2.0 * (double)H));
  const double sw = sin(pi * (double)(W - 1) / (2.0 * (double)W));
  return 4.0 * sh * sh + 4.0 * sw * sw;
}

int32_t ot_n_identity_blocks(int32_t mode, int32_t balanced) {
  return (mode == OT_MODE_PROX ? 1 : 0) + (mode != OT_MODE_EVAL ? 1 : 0) + (balanced ? 0 : 1);
}

}  // extern "C"

static void destroy_graphs(ot_prox* h) {
  for (int k = 0; k < 2; ++k) {
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    h->graph[k] = nullptr;
  }
}

static StatePtrs state_ptrs(ot_prox* h, int parity) {
  StatePtrs s;
  s.Mx_in = h->Mx[parity];
  s.My_in = h->My[parity];
  s.a_in = h->a[parity];
  s.Mx_out = h->Mx[parity ^ 1];
  s.My_out = h->My[parity ^ 1];
  s.a_out = h->a[parity ^ 1];
  s.x0 = h->x0;
  s.x1 = h->x1;
  s.r = h->r;
  s.p0 = h->p0;
  s.p1 = h->p1;
  return s;
}

// Enqueue n iterations starting from ping-pong `parity`; the last one
// reduces (and the sums are finalised into dsums) when `reduce`.
static cudaError_t enqueue_admm(ot_prox* h, int n, bool reduce) {
  const int nb = admm_num_blocks(h->G);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    const bool red = reduce && (k == n - 1);
    e = admm_launch_z(h->G, h->AC, h->AP, red, h->partials, h->stream);
    if (e == cudaSuccess) e = admm_launch_rhs(h->G, h->AC, h->AP, red, h->partials + (size_t)nb * kNumSums, h->stream);
    if (e == cudaSuccess) e = dct_plan_solve(h->dct, h->AP.k, h->G.Wp, h->AP.y, h->G.Wp, h->stream);
    if (e == cudaSuccess)
      e = admm_launch_w(h->G, h->AC, h->AP, red, h->partials + (size_t)2 * nb * kNumSums, h->stream);
  }
  if (e == cudaSuccess && reduce && n > 0) e = launch_finalize_sums(h->partials, 3 * nb, h->dsums, h->stream);
  return e;
}

static TbPtrs tb_ptrs(ot_prox* h, int parity) {
  TbPtrs s;
  const int o = parity ^ 1;
  s.Mx_in = h->Mx[parity];
  s.My_in = h->My[parity];
  s.a_in = h->a[parity];
  s.x0_in = h->x0s[parity];
  s.x1_in = h->x1s[parity];
  s.r_in = h->rs[parity];
  s.Mx_out = h->Mx[o];
  s.My_out = h->My[o];
  s.a_out = h->a[o];
  s.x0_out = h->x0s[o];
  s.x1_out = h->x1s[o];
  s.r_out = h->rs[o];
  s.p0 = h->p0;
  s.p1 = h->p1;
  return s;
}

// Temporal blocking: n iterations as ceil(n / depth) passes of near-equal
// length (each <= depth), one ping-pong flip per pass.
static int tb_passes(const ot_prox* h, int n) { return (n + h->tb_depth - 1) / h->tb_depth; }

static cudaError_t enqueue_temporal(ot_prox* h, int parity, int n, bool reduce) {
  const int np = tb_passes(h, n);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < np && e == cudaSuccess; ++k) {
    const int sub = n / np + (k < n % np ? 1 : 0);
    e = launch_prox_temporal(h->prm.mode, h->prm.balanced != 0, reduce && k == np - 1, h->tb_depth, sub, h->G, h->C,
                             tb_ptrs(h, parity), h->partials, h->stream);
    parity ^= 1;
  }
  if (e == cudaSuccess && reduce && n > 0)
    e = launch_finalize_sums(h->partials, temporal_num_ctas(h->G, h->tb_depth), h->dsums, h->stream);
  return e;
}

static cudaError_t enqueue_iterations(ot_prox* h, int parity, int n, bool reduce) {
  if (h->admm) return enqueue_admm(h, n, reduce);
  if (h->tb) return n > 0 ? enqueue_temporal(h, parity, n, reduce) : cudaSuccess;
  const int mode = h->prm.mode;
  const bool bal = h->prm.balanced != 0;
  cudaError_t e = cudaSuccess;
  if (h->resident) {
    if (n <= 0) return cudaSuccess;
    e = launch_prox_resident(mode, bal, h->G, h->C, h->Mx[parity], h->My[parity], h->a[parity], h->x0, h->x1, h->r,
                             h->p0, h->p1, n, reduce, h->partials, h->stream);
    if (e != cudaSuccess || !reduce) return e;
    return launch_finalize_sums(h->partials, h->G.B, h->dsums, h->stream);
  }
  for (int k = 0; k < n; ++k) {
    const bool red = reduce && (k == n - 1);
    if (h->tma)
      e = launch_prox_tma(mode, bal, red, h->maps[parity], h->G, h->C, state_ptrs(h, parity), h->partials, h->derr,
                          h->tma_grid, h->stream);
    else
      e = launch_prox_tiled(mode, bal, red, h->G, h->C, state_ptrs(h, parity), h->partials, h->stream);
    if (e != cudaSuccess) return e;
    parity ^= 1;
  }
  if (reduce && n > 0)
    e = launch_finalize_sums(h->partials, h->tma ? h->tma_grid : tiled_num_ctas(h->G), h->dsums, h->stream);
  return e;
}

static int parity_after(const ot_prox* h, int parity, int n) {
  if (h->tb) return parity ^ (tb_passes(h, n) & 1);
  return (h->resident || h->admm) ? parity : (parity ^ (n & 1));
}

// The current ping-pong parity; with temporal blocking x0, x1, r follow it.
static void set_cur(ot_prox* h, int c) {
  h->cur = c;
  if (h->tb) {
    h->x0 = h->x0s[c];
    h->x1 = h->x1s[c];
    h->r = h->rs[c];
  }
}

// One check interval: n iterations, reduction, copy of the sums to the host.
static int run_check_interval(ot_prox* h, int n) {
  // the legacy NULL stream cannot be captured
  const bool use_graph = h->prm.use_graph && h->stream != nullptr && n == h->prm.check_every;
  const int parity = h->cur;
  if (use_graph) {
    if (!h->graph[parity] || h->graph_n != n) {
      if (h->graph_n != n) destroy_graphs(h);
      cudaGraph_t g = nullptr;
      OT_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
      cudaError_t e = enqueue_iterations(h, parity, n, true);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->hsums, h->dsums, kNumSums * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "capturing a check interval");
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->graph[parity], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      h->graph_n = n;
    }
    OT_CUDA(cudaGraphLaunch(h->graph[parity], h->stream), "cudaGraphLaunch");
  } else {
    OT_CUDA(enqueue_iterations(h, parity, n, true), "launching Algorithm 1 iterations");
    OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, kNumSums * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "copying check sums");
    OT_CUDA(cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copying the error flag");
  }
  set_cur(h, parity_after(h, parity, n));
  OT_CUDA(cudaStreamSynchronize(h->stream), "synchronising after a check interval");
  if (*h->herr) return fail(OT_ETIMEOUT, "a bounded device wait expired in the iteration kernel");
  return OT_OK;
}

// Any NaN/Inf in the iterates or the inputs shows in one of the check sums.
static bool sums_nonfinite(const double* s) {
  if (s[7] > 0) return true;
  for (int k = 0; k < 7; ++k)
    if (!isfinite(s[k])) return true;
  return false;
}

static void fill_result_from_sums(const ot_prox* h, const double* s, ot_prox_result* res) {
  const double sp = fmax(sqrt(s[6]), 1e-30);
  res->res_pri = sqrt(s[0]) / sp;
  res->res_fp = sqrt(s[1]) / fmax(sqrt(s[2]), 1e-30);
  double obj = s[3];
  if (!h->prm.balanced) obj += h->prm.mu * s[4];
  obj += s[5] / (2.0 * h->prm.rho);
  res->objective = obj;
}

static int evaluate_into(ot_prox* h, ot_prox_result* res) {
  CertCoeffs cc;
  cc.mu = h->prm.mu;
  cc.rho = h->prm.rho;
  cc.iso = h->prm.norm == OT_NORM_ISO;
  cc.pexp = h->prm.p_exp;
  cc.mode = h->prm.mode;
  cc.balanced = h->prm.balanced;
  const int c = h->cur;
  OT_CUDA(launch_evaluate(h->G, cc, h->Mx[c], h->My[c], h->a[c], h->x0, h->x1, h->r, h->p0, h->p1, h->partials,
                          h->dsums, h->cert_partials, h->dsums + kNumSums, h->stream),
          "launching the evaluation kernels");
  OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, (kNumSums + 4) * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
          "copying evaluation sums");
  OT_CUDA(cudaStreamSynchronize(h->stream), "synchronising the evaluation");
  const double* s = h->hsums;
  const double rp = res->res_fp;
  fill_result_from_sums(h, s, res);
  res->res_fp = rp;
  res->dual_obj = s[kNumSums + 1];
  res->primal_feasible = s[kNumSums + 2];
  res->rel_gap = (res->primal_feasible - res->dual_obj) / fmax(fabs(res->primal_feasible), 1e-30);
  if (sums_nonfinite(s)) return OT_ENONFINITE;
  return OT_OK;
}

// projection form: restart the splitting at w = z, u = 0 after the state
// was written from outside
static int restart_projection(ot_prox* h) {
  if (!h->admm) return OT_OK;
  for (int k = 0; k < 5; ++k)
    OT_CUDA(cudaMemcpyAsync(h->AP.w[k], h->AP.z[k], h->plane_elems * sizeof(float), cudaMemcpyDeviceToDevice,
                            h->stream),
            "restart of the projection form: w = z");
  OT_CUDA(cudaMemsetAsync(h->AP.u[0], 0, h->plane_elems * 5 * sizeof(float), h->stream),
          "restart of the projection form: u = 0");
  return OT_OK;
}

static int copy_plane_in(ot_prox* h, float* dst, const float* src) {
  const size_t wb = (size_t)h->G.W * sizeof(float);
  OT_CUDA(cudaMemcpy2DAsync(dst, (size_t)h->G.Wp * sizeof(float), src, wb, wb, (size_t)h->G.B * h->G.H,
                            cudaMemcpyDefault, h->stream),
          "copying an input plane");
  return OT_OK;
}

static int copy_plane_out(ot_prox* h, float* dst, const float* src) {
  const size_t wb = (size_t)h->G.W * sizeof(float);
  OT_CUDA(cudaMemcpy2DAsync(dst, wb, src, (size_t)h->G.Wp * sizeof(float), wb, (size_t)h->G.B * h->G.H,
                            cudaMemcpyDefault, h->stream),
          "copying an output plane");
  return OT_OK;
}

extern "C" {

int ot_prox_create(const ot_prox_params* params, void* cuda_stream, ot_prox_t* out) {
  if (!params || !out) return fail(OT_EINVAL, "ot_prox_create: params and out must be non-NULL");
  *out = nullptr;
  ot_prox_params p = *params;
  if (p.B < 1 || p.H < 1 || p.W < 1) return fail(OT_EINVAL, "ot_prox_create: B, H, W must be >= 1 (got %d, %d, %d)", p.B, p.H, p.W);
  if (p.mode < 0 || p.mode > 2) return fail(OT_EINVAL, "ot_prox_create: unknown mode %d", p.mode);
  if (p.norm != OT_NORM_ISO && p.norm != OT_NORM_ANISO) return fail(OT_EINVAL, "ot_prox_create: unknown norm %d", p.norm);
  if (p.balanced != 0 && p.balanced != 1) return fail(OT_EINVAL, "ot_prox_create: balanced must be 0 or 1");
  if (p.p_exp != 1 && p.p_exp != 2) return fail(OT_EINVAL, "ot_prox_create: p_exp must be 1 or 2");
  if (!(p.mu > 0) || !isfinite(p.mu)) return fail(OT_EINVAL, "ot_prox_create: mu must be > 0");
  if (!(p.rho > 0) || !isfinite(p.rho)) return fail(OT_EINVAL, "ot_prox_create: rho must be > 0");
  if (!(p.tol >= 0) || !isfinite(p.tol)) return fail(OT_EINVAL, "ot_prox_create: tol must be >= 0");
  if (p.max_iter < 0) return fail(OT_EINVAL, "ot_prox_create: max_iter must be >= 0");
  if (p.check_every < 1) return fail(OT_EINVAL, "ot_prox_create: check_every must be >= 1");
  if (p.kernel < 0 || p.kernel > 4) return fail(OT_EINVAL, "ot_prox_create: unknown kernel %d", p.kernel);
  if (p.kernel == OT_KERNEL_TEMPORAL && p.algorithm != OT_ALG_ALG1)
    return fail(OT_EINVAL, "ot_prox_create: OT_KERNEL_TEMPORAL runs Algorithm 1 only");
  if (p.kernel == OT_KERNEL_TEMPORAL && (p.tb_depth < 2 || p.tb_depth > 4))
    return fail(OT_EINVAL, "ot_prox_create: tb_depth must be in [2, 4] (got %d)", p.tb_depth);
  if (p.algorithm != OT_ALG_ALG1 && p.algorithm != OT_ALG_PROJECTION)
    return fail(OT_EINVAL, "ot_prox_create: unknown algorithm %d", p.algorithm);
  if (p.precision != OT_PREC_FP32 && p.precision != OT_PREC_SPLIT_BF16 && p.precision != OT_PREC_SPLIT_BF16_3)
    return fail(OT_EINVAL, "ot_prox_create: unknown precision %d", p.precision);
  if (p.algorithm == OT_ALG_PROJECTION && (!(p.beta > 0) || !isfinite(p.beta)))
    return fail(OT_EINVAL, "ot_prox_create: beta must be > 0");
  if (!isfinite(p.tau1) || !isfinite(p.tau2)) return fail(OT_EINVAL, "ot_prox_create: steps must be finite");
  // Theorem 1: tau1 tau2 < 1 / (lambda_max + n_id)
  const double L = ot_lambda_max(p.H, p.W) + (double)ot_n_identity_blocks(p.mode, p.balanced);
  if (!(L > 0)) return fail(OT_EINVAL, "ot_prox_create: ||K|| = 0 (1x1 balanced EVAL has no variables)");
  const double tdef = 0.99 / sqrt(L);
  if (p.tau1 <= 0) p.tau1 = tdef;
  if (p.tau2 <= 0) p.tau2 = tdef;
  if (p.tau1 * p.tau2 * L >= 1.0)
    return fail(OT_EINVAL, "ot_prox_create: steps violate Theorem 1: tau1*tau2*(lambda_max+%d) = %.6g >= 1",
                ot_n_identity_blocks(p.mode, p.balanced), p.tau1 * p.tau2 * L);

  Geometry G;
  G.B = p.B;
  G.H = p.H;
  G.W = p.W;
  G.Wp = (p.W + 3) / 4 * 4;
  G.plane = (long long)G.H * G.Wp;
  G.tiles_x = (G.Wp + kTW - 1) / kTW;
  G.tiles_y = (G.H + kTH - 1) / kTH;
  const double ctas = (double)G.B * G.tiles_x * G.tiles_y;
  if (ctas > 2.0e9) return fail(OT_EINVAL, "ot_prox_create: problem too large for one launch (%g tiles)", ctas);
  const size_t plane_elems = (size_t)G.B * (size_t)G.plane;
  const bool tb = p.kernel == OT_KERNEL_TEMPORAL;
  const size_t nplanes = tb ? 14 : 11;
  if ((double)plane_elems * nplanes * 4.0 > 2.6e11) return fail(OT_ENOMEM, "ot_prox_create: state would exceed device memory");

  const bool fits = resident_fits(G, p.mode, p.balanced != 0);
  bool resident = false, tma = false;
  if (p.kernel == OT_KERNEL_RESIDENT) {
    if (!fits) return fail(OT_EINVAL, "ot_prox_create: H x W = %d x %d does not fit the resident kernel", p.H, p.W);
    resident = true;
  } else if (p.kernel == OT_KERNEL_AUTO) {
    resident = fits;
    tma = !fits;
  } else if (p.kernel == OT_KERNEL_TMA) {
    tma = true;
  }
  if (p.algorithm == OT_ALG_PROJECTION || tb) resident = tma = false;

  ot_prox* h = (ot_prox*)calloc(1, sizeof(ot_prox));
  if (!h) return fail(OT_ENOMEM, "ot_prox_create: host allocation failed");
  h->prm = p;
  h->stream = (cudaStream_t)cuda_stream;
  h->G = G;
  h->plane_elems = plane_elems;
  h->resident = resident;
  h->tma = tma;
  h->admm = p.algorithm == OT_ALG_PROJECTION;
  const float t1 = (float)p.tau1;
  h->C.tau1 = t1;
  h->C.tau2 = (float)p.tau2;
  h->C.cp = (float)(p.tau1 / (p.rho + p.tau1));
  h->C.cx = (float)(p.rho / (p.rho + p.tau1));
  h->C.ca = (float)(p.rho * p.tau1 / (p.rho + p.tau1));
  h->C.mu_tau1 = (float)(p.mu * p.tau1);
  h->C.r2 = (float)(1.0 / (1.0 + 2.0 * p.mu * p.tau1));
  h->C.iso = p.norm == OT_NORM_ISO;
  h->C.pexp = p.p_exp;

  cudaError_t e = cudaMalloc(&h->slab, plane_elems * nplanes * sizeof(float));
  if (e != cudaSuccess) {
    free(h);
    return cuda_fail(e, "ot_prox_create: cudaMalloc(state)");
  }
  float* q = h->slab;
  h->Mx[0] = q; q += plane_elems;
  h->Mx[1] = q; q += plane_elems;
  h->My[0] = q; q += plane_elems;
  h->My[1] = q; q += plane_elems;
  h->a[0] = q; q += plane_elems;
  h->a[1] = q; q += plane_elems;
  h->x0 = q; q += plane_elems;
  h->x1 = q; q += plane_elems;
  h->r = q; q += plane_elems;
  h->p0 = q; q += plane_elems;
  h->p1 = q; q += plane_elems;
  h->tb = tb;
  h->tb_depth = p.tb_depth;
  h->x0s[0] = h->x0;
  h->x1s[0] = h->x1;
  h->rs[0] = h->r;
  if (tb) {
    h->x0s[1] = q; q += plane_elems;
    h->x1s[1] = q; q += plane_elems;
    h->rs[1] = q; q += plane_elems;
  }
  int n_sm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n_sm = 152;
  h->tma_grid = (int)(ctas < (double)n_sm ? ctas : n_sm);
  int n_parts = (int)(ctas > (double)G.B ? ctas : G.B);
  if (tb && temporal_num_ctas(G, p.tb_depth) > n_parts) n_parts = temporal_num_ctas(G, p.tb_depth);
  if (h->admm && 3 * admm_num_blocks(G) > n_parts) n_parts = 3 * admm_num_blocks(G);
  const int n_cert = cert_num_blocks(G);
  const int np = n_parts > n_cert ? n_parts : n_cert;
  const size_t ws_bytes = (size_t)np * kNumSums * sizeof(double) + (size_t)n_cert * 4 * sizeof(double) +
                          (kNumSums + 4) * sizeof(double) + 16;
  e = cudaMalloc(&h->partials, ws_bytes);
  if (e == cudaSuccess) {
    h->cert_partials = h->partials + (size_t)np * kNumSums;
    h->dsums = h->cert_partials + (size_t)n_cert * 4;
    h->derr = reinterpret_cast<int*>(h->dsums + kNumSums + 4);
    e = cudaMallocHost(&h->hsums, (kNumSums + 4) * sizeof(double) + 16);
    if (e == cudaSuccess) h->herr = reinterpret_cast<int*>(h->hsums + kNumSums + 4);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->partials, 0, ws_bytes, h->stream);
  if (e != cudaSuccess) {
    ot_prox_destroy(h);
    return cuda_fail(e, "ot_prox_create: workspace allocation");
  }
  if (h->admm && e == cudaSuccess) {
    e = cudaMalloc(&h->admm_slab, plane_elems * 10 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->admm_slab, 0, plane_elems * 10 * sizeof(float), h->stream);
    if (e == cudaSuccess) {
      AdmmPlanes& P = h->AP;
      P.z[0] = h->Mx[0];
      P.z[1] = h->My[0];
      P.z[2] = h->x0;
      P.z[3] = h->x1;
      P.z[4] = h->r;
      for (int k = 0; k < 5; ++k) {
        P.w[k] = h->admm_slab + (size_t)k * plane_elems;
        P.u[k] = h->admm_slab + (size_t)(5 + k) * plane_elems;
      }
      P.k = h->Mx[1];      // unused by the projection form otherwise
      P.y = h->My[1];
      P.a = h->a[0];
      P.p0 = h->p0;
      P.p1 = h->p1;
      AdmmCoeffs& C = h->AC;
      C.beta = (float)p.beta;
      C.inv_beta = (float)(1.0 / p.beta);
      C.rb = (float)(p.rho * p.beta);
      C.inv_1rb = (float)(1.0 / (1.0 + p.rho * p.beta));
      C.mu_over_beta = (float)(p.mu / p.beta);
      C.r2 = (float)(1.0 / (1.0 + 2.0 * p.mu / p.beta));
      C.iso = p.norm == OT_NORM_ISO;
      C.pexp = p.p_exp;
      C.free0 = p.mode == OT_MODE_PROX;
      C.free1 = p.mode != OT_MODE_EVAL;
      C.balanced = p.balanced;
      h->n_id = ot_n_identity_blocks(p.mode, p.balanced);
      const int rc = dct_plan_create(p.B, p.H, p.W, (double)h->n_id, p.precision, &h->dct);
      if (rc != OT_OK) {
        ot_prox_destroy(h);
        return rc;
      }
      dct_plan_set_error_flag(h->dct, h->derr);
    }
  }
  if (resident && e == cudaSuccess) e = prepare_prox_resident(p.mode, p.balanced != 0, G);
  if (tb && e == cudaSuccess) e = prepare_prox_temporal(p.mode, p.balanced != 0, p.tb_depth);
  if (tma && e == cudaSuccess) {
    e = prepare_prox_tma(p.mode, p.balanced != 0);
    int bw, bh;
    for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
      TmaMaps& m = h->maps[par];
      int rc = 0;
      tma_box(0, &bw, &bh);
      rc |= encode_plane_map(&m.a, h->a[par], G, bw, bh);
      tma_box(1, &bw, &bh);
      rc |= encode_plane_map(&m.Mx, h->Mx[par], G, bw, bh);
      rc |= encode_plane_map(&m.My, h->My[par], G, bw, bh);
      tma_box(2, &bw, &bh);
      rc |= encode_plane_map(&m.x0, h->x0, G, bw, bh);
      rc |= encode_plane_map(&m.x1, h->x1, G, bw, bh);
      rc |= encode_plane_map(&m.r, h->r, G, bw, bh);
      rc |= encode_plane_map(&m.p0, h->p0, G, bw, bh);
      rc |= encode_plane_map(&m.p1, h->p1, G, bw, bh);
      if (rc != 0) {
        ot_prox_destroy(h);
        return fail(OT_ECUDA, "ot_prox_create: cuTensorMapEncodeTiled failed (%d)", rc);
      }
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->slab, 0, plane_elems * nplanes * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ot_prox_destroy(h);
    return cuda_fail(e, "ot_prox_create: clearing the state");
  }
  *out = h;
  return OT_OK;
}

int ot_prox_get_params(ot_prox_t h, ot_prox_params* out) {
  if (!h || !out) return fail(OT_EINVAL, "ot_prox_get_params: NULL argument");
  *out = h->prm;
  return OT_OK;
}

int ot_prox_set_input(ot_prox_t h, const float* p0, const float* p1) {
  if (!h) return fail(OT_EINVAL, "ot_prox_set_input: NULL handle");
  if (!p0 || !p1) return fail(OT_EINVAL, "ot_prox_set_input: p0 and p1 must be non-NULL");
  int rc = copy_plane_in(h, h->p0, p0);
  if (rc == OT_OK) rc = copy_plane_in(h, h->p1, p1);
  return rc;
}

int ot_prox_reset(ot_prox_t h) {
  if (!h) return fail(OT_EINVAL, "ot_prox_reset: NULL handle");
  // everything but the inputs p0, p1 (the last two planes)
  OT_CUDA(cudaMemsetAsync(h->slab, 0, h->plane_elems * 9 * sizeof(float), h->stream), "ot_prox_reset");
  if (h->tb)
    OT_CUDA(cudaMemsetAsync(h->x0s[1], 0, h->plane_elems * 3 * sizeof(float), h->stream), "ot_prox_reset");
  if (h->admm)
    OT_CUDA(cudaMemsetAsync(h->admm_slab, 0, h->plane_elems * 10 * sizeof(float), h->stream), "ot_prox_reset");
  set_cur(h, 0);
  return OT_OK;
}

int ot_prox_step(ot_prox_t h, int32_t n_iter) {
  if (!h) return fail(OT_EINVAL, "ot_prox_step: NULL handle");
  if (n_iter < 0) return fail(OT_EINVAL, "ot_prox_step: n_iter must be >= 0");
  if (n_iter == 0) return OT_OK;
  OT_CUDA(enqueue_iterations(h, h->cur, n_iter, false), "ot_prox_step");
  set_cur(h, parity_after(h, h->cur, n_iter));
  return OT_OK;
}

int ot_prox_check_interval(ot_prox_t h, int32_t n_iter, ot_prox_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_prox_check_interval: NULL handle");
  if (n_iter < 1) return fail(OT_EINVAL, "ot_prox_check_interval: n_iter must be >= 1");
  const int rc = run_check_interval(h, n_iter);
  if (rc != OT_OK) return rc;
  ot_prox_result r;
  memset(&r, 0, sizeof r);
  const double* s = h->hsums;
  fill_result_from_sums(h, s, &r);
  r.iters = n_iter;
  const bool bad = sums_nonfinite(s);
  r.status = bad ? OT_ENONFINITE : OT_OK;
  if (res) *res = r;
  if (bad) return fail(OT_ENONFINITE, "ot_prox_check_interval: non-finite values in the iterates");
  return OT_OK;
}

int ot_prox_step_timed(ot_prox_t h, int32_t n_iter, double* elapsed_ms) {
  if (!h || !elapsed_ms) return fail(OT_EINVAL, "ot_prox_step_timed: NULL argument");
  if (n_iter < 0) return fail(OT_EINVAL, "ot_prox_step_timed: n_iter must be >= 0");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OT_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  if (e == cudaSuccess) e = enqueue_iterations(h, h->cur, n_iter, false);
  if (e == cudaSuccess) {
    set_cur(h, parity_after(h, h->cur, n_iter));
    e = cudaEventRecord(e1, h->stream);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "ot_prox_step_timed");
  *elapsed_ms = ms;
  return OT_OK;
}

int ot_prox_solve(ot_prox_t h, ot_prox_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_prox_solve: NULL handle");
  ot_prox_result r;
  memset(&r, 0, sizeof r);
  r.res_pri = r.res_fp = INFINITY;
  int status = OT_ENOTCONV;
  int k = 0;
  while (k < h->prm.max_iter) {
    const int n = (h->prm.max_iter - k) < h->prm.check_every ? (h->prm.max_iter - k) : h->prm.check_every;
    const int rc = run_check_interval(h, n);
    if (rc != OT_OK) return rc;
    k += n;
    const double* s = h->hsums;
    fill_result_from_sums(h, s, &r);
    r.iters = k;
    if (sums_nonfinite(s)) {
      status = OT_ENONFINITE;
      break;
    }
    if (fmax(r.res_pri, r.res_fp) <= h->prm.tol) {
      status = OT_OK;
      break;
    }
  }
  r.iters = k;
  if (status != OT_ENONFINITE) {
    const int rc = evaluate_into(h, &r);
    if (rc != OT_OK && rc != OT_ENONFINITE) return rc;
    if (rc == OT_ENONFINITE) status = OT_ENONFINITE;
  }
  r.status = status;
  if (res) *res = r;
  if (status == OT_ENOTCONV) fail(OT_ENOTCONV, "ot_prox_solve: max_iter = %d reached (res_pri %.3g, res_fp %.3g)", h->prm.max_iter, r.res_pri, r.res_fp);
  if (status == OT_ENONFINITE) fail(OT_ENONFINITE, "ot_prox_solve: non-finite values in the iterates");
  return status;
}

int ot_prox_evaluate(ot_prox_t h, ot_prox_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_prox_evaluate: NULL handle");
  ot_prox_result r;
  memset(&r, 0, sizeof r);
  const int rc = evaluate_into(h, &r);
  r.status = rc;
  if (res) *res = r;
  if (rc == OT_ENONFINITE) return fail(OT_ENONFINITE, "ot_prox_evaluate: non-finite values in the state");
  return rc;
}

int ot_prox_get_state(ot_prox_t h, float* Mx, float* My, float* x0, float* x1, float* r, float* a) {
  if (!h) return fail(OT_EINVAL, "ot_prox_get_state: NULL handle");
  const int c = h->cur;
  int rc = OT_OK;
  if (Mx && rc == OT_OK) rc = copy_plane_out(h, Mx, h->Mx[c]);
  if (My && rc == OT_OK) rc = copy_plane_out(h, My, h->My[c]);
  if (x0 && rc == OT_OK) rc = copy_plane_out(h, x0, h->prm.mode == OT_MODE_PROX ? h->x0 : h->p0);
  if (x1 && rc == OT_OK) rc = copy_plane_out(h, x1, h->prm.mode != OT_MODE_EVAL ? h->x1 : h->p1);
  if (r && rc == OT_OK) rc = copy_plane_out(h, r, h->r);
  if (a && rc == OT_OK) rc = copy_plane_out(h, a, h->a[c]);
  return rc;
}

int ot_prox_set_state(ot_prox_t h, const float* Mx, const float* My, const float* x0, const float* x1,
                      const float* r, const float* a) {
  if (!h) return fail(OT_EINVAL, "ot_prox_set_state: NULL handle");
  const int c = h->cur;
  int rc = OT_OK;
  if (Mx && rc == OT_OK) rc = copy_plane_in(h, h->Mx[c], Mx);
  if (My && rc == OT_OK) rc = copy_plane_in(h, h->My[c], My);
  if (x0 && rc == OT_OK && h->prm.mode == OT_MODE_PROX) rc = copy_plane_in(h, h->x0, x0);
  if (x1 && rc == OT_OK && h->prm.mode != OT_MODE_EVAL) rc = copy_plane_in(h, h->x1, x1);
  if (r && rc == OT_OK && !h->prm.balanced) rc = copy_plane_in(h, h->r, r);
  if (a && rc == OT_OK) rc = copy_plane_in(h, h->a[c], a);
  if (rc != OT_OK) return rc;
  // no edge beyond the last row (Mx) or the last column (My): zero flux
  const size_t fb = sizeof(float);
  if (Mx)
    OT_CUDA(cudaMemset2DAsync(h->Mx[c] + (size_t)(h->G.H - 1) * h->G.Wp, (size_t)h->G.plane * fb, 0,
                              (size_t)h->G.Wp * fb, (size_t)h->G.B, h->stream),
            "ot_prox_set_state: zeroing Mx[H-1,:]");
  if (My)
    OT_CUDA(cudaMemset2DAsync(h->My[c] + (h->G.W - 1), (size_t)h->G.Wp * fb, 0, fb, (size_t)h->G.B * h->G.H,
                              h->stream),
            "ot_prox_set_state: zeroing My[:,W-1]");
  return restart_projection(h);
}

int ot_prox_warm_start(ot_prox_t h, const float* pred, double gate) {
  if (!h || !pred) return fail(OT_EINVAL, "ot_prox_warm_start: NULL argument");
  if (!(gate >= 0.0)) return fail(OT_EINVAL, "ot_prox_warm_start: gate must be >= 0");
  const int c = h->cur;
  const bool fx0 = h->prm.mode != OT_MODE_PROX, fx1 = h->prm.mode == OT_MODE_EVAL;
  OT_CUDA(launch_warm_start(pred, h->G, h->Mx[c], h->My[c], h->prm.balanced ? nullptr : h->r, h->a[c],
                            fx0 ? nullptr : h->x0, fx1 ? nullptr : h->x1, h->p0, h->p1, (float)h->prm.rho, (float)gate,
                            h->stream),
          "ot_prox_warm_start");
  return restart_projection(h);
}

int ot_prox_destroy(ot_prox_t h) {
  if (!h) return OT_OK;
  destroy_graphs(h);
  if (h->dct) dct_plan_destroy(h->dct);
  if (h->admm_slab) cudaFree(h->admm_slab);
  if (h->slab) cudaFree(h->slab);
  if (h->partials) cudaFree(h->partials);
  if (h->hsums) cudaFreeHost(h->hsums);
  free(h);
  return OT_OK;
}

}  // extern "C"
