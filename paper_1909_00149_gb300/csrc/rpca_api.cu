// C ABI of the RPCA+UOT-DF solver (Algorithm 3, Sec. IV-B.1, Phi_t = I) and
// of the standalone singular-value thresholding (Algorithm 3 line 10).
//
// One outer iteration, in stream order:
//   rpca_pre      lines 4-9 fused; builds L + D and the prox centres
//   gram          line 10, first pass: G = (L + D)^T (L + D)
//   eig | prox    the one-CTA T x T eigensolver on a side stream, beside
//                 line 11 (n_inner warm-started Algorithm 1 iterations on
//                 the T-1 frame pairs with weight kappa/rho) on all other SMs
//   apply         line 10, second pass: Tn = (L + D) Wm
//   rpca_post     lines 12-15 and the ADMM residual sums
// then, on check iterations, one fixed-order FP64 finalize and a 64-byte copy
// to the host.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"
#include "prox_handle.cuh"

using namespace otp;

#define OT_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

struct ot_rpca {
  ot_rpca_params prm;
  cudaStream_t stream;
  RpcaGeom G;
  RpcaCoeffs C;
  float* slab;
  size_t slab_floats;
  RpcaPlanes P;
  ot_prox* prox;             // B = T-1 problems, rho_prox = kappa / rho
  // SVT workspace
  int TP;
  double* gram_partials;
  // T_pad <= 64: the fused pass between outer iterations also accumulates the
  // next iteration's Gram matrix, as FP32 partials that the same cooperative
  // launch reduces into Gm
  float* fgram;
  int fgram_parts;
  unsigned* fbar;   // the fused pass's grid barrier (count, generation), after fgram
  double* Gm;
  float* V;
  float* Wm;
  float* sig;
  int* sweeps;
  int warm;
  // residual sums
  int nb_rpca, nb_apply;
  double* partials;          // [3 * nb_rpca + nb_apply][kNumSums]: pre (parity 0), post, pre (parity 1)
  double* dsums;             // [kNumSums]
  double* hsums;             // pinned: [kNumSums] sums, then sweeps (as int) and sigma
  double y_norm;
  int have_input;
  // line 10 (SVT) and line 11 (prox) are independent given lines 4-9: the
  // SVT runs on a side stream while the prox runs on the handle's stream
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // one warm outer iteration (with its residual sums) as a graph, by the
  // ping-pong parity of the inner prox state and of the SVT output planes
  cudaGraphExec_t graph[2][2];
  int tpar;                  // flips when Tm and Tn swap
};

extern "C" {

void ot_rpca_default_params(ot_rpca_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->T = 2;
  p->H = p->W = 1;
  p->lambda = 0.02;
  p->gamma = 0.0;           // <= 0: lambda * sqrt(max(N, T))
  p->kappa = 0.005;
  p->mu = 3.0;
  p->rho = 1.0;
  p->n_inner = 1;
  p->tol = 1e-5;
  p->max_iter = 5000;
  p->check_every = 1;
  p->svt_max_sweeps = 30;
  p->prox_kernel = OT_KERNEL_AUTO;
  p->use_graph = 1;
  p->signed_fg = 0;
}

int ot_rpca_destroy(ot_rpca_t h) {
  if (!h) return OT_OK;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      if (h->graph[k][j]) cudaGraphExecDestroy(h->graph[k][j]);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->prox) ot_prox_destroy(h->prox);
  if (h->slab) cudaFree(h->slab);
  if (h->gram_partials) cudaFree(h->gram_partials);
  if (h->fgram) cudaFree(h->fgram);
  if (h->partials) cudaFree(h->partials);
  if (h->hsums) cudaFreeHost(h->hsums);
  free(h);
  return OT_OK;
}

int ot_rpca_create(const ot_rpca_params* params, void* cuda_stream, ot_rpca_t* out) {
  if (!params || !out) return fail(OT_EINVAL, "ot_rpca_create: params and out must be non-NULL");
  *out = nullptr;
  ot_rpca_params p = *params;
  if (p.T < 2 || p.T > 128) return fail(OT_EINVAL, "ot_rpca_create: T must be in [2, 128] (got %d)", p.T);
  if (p.H < 1 || p.W < 1) return fail(OT_EINVAL, "ot_rpca_create: H, W must be >= 1");
  if (!(p.lambda > 0) || !(p.kappa > 0) || !(p.mu > 0) || !(p.rho > 0))
    return fail(OT_EINVAL, "ot_rpca_create: lambda, kappa, mu, rho must be > 0");
  if (!isfinite(p.gamma)) return fail(OT_EINVAL, "ot_rpca_create: gamma must be finite");
  if (p.prox_kernel == OT_KERNEL_TEMPORAL)
    return fail(OT_EINVAL, "ot_rpca_create: the inner prox cannot use OT_KERNEL_TEMPORAL (its x planes are shared)");
  if (p.n_inner < 1) return fail(OT_EINVAL, "ot_rpca_create: n_inner must be >= 1");
  if (p.max_iter < 0 || p.check_every < 1 || p.svt_max_sweeps < 1)
    return fail(OT_EINVAL, "ot_rpca_create: max_iter >= 0, check_every >= 1, svt_max_sweeps >= 1 required");
  if (!(p.tol >= 0)) return fail(OT_EINVAL, "ot_rpca_create: tol must be >= 0");
  if (p.signed_fg != 0 && p.signed_fg != 1) return fail(OT_EINVAL, "ot_rpca_create: signed_fg must be 0 or 1");
  const double N = (double)p.H * p.W;
  if (p.gamma <= 0) p.gamma = p.lambda * sqrt(N > p.T ? N : (double)p.T);

  ot_rpca* h = (ot_rpca*)calloc(1, sizeof(ot_rpca));
  if (!h) return fail(OT_ENOMEM, "ot_rpca_create: host allocation failed");
  h->prm = p;
  h->stream = (cudaStream_t)cuda_stream;
  h->G.T = p.T;
  h->G.H = p.H;
  h->G.W = p.W;
  h->G.Wp = (p.W + 3) / 4 * 4;
  h->G.plane = (long long)p.H * h->G.Wp;
  h->C.lam = (float)p.lambda;
  h->C.rho = (float)p.rho;
  h->TP = svt_padded_T(p.T);

  // the inner prox: B = T-1 pairs (both signs' 2 (T-1) for the signed
  // foreground), weight kappa / rho (line 11)
  const int nsign = p.signed_fg ? 2 : 1;
  ot_prox_params pp;
  ot_prox_default_params(&pp);
  pp.B = nsign * (p.T - 1);
  pp.H = p.H;
  pp.W = p.W;
  pp.mode = OT_MODE_PROX;
  pp.mu = p.mu;
  pp.rho = p.kappa / p.rho;
  pp.kernel = p.prox_kernel;
  pp.use_graph = 0;
  int rc = ot_prox_create(&pp, cuda_stream, &h->prox);
  if (rc != OT_OK) {
    ot_rpca_destroy(h);
    return rc;
  }
  // one SM stays free for the one-CTA eigensolver, which runs beside line 11
  prox_reserve_sms(h->prox, 1);

  const size_t plane = (size_t)h->G.plane;
  const size_t nframe = (size_t)p.T * plane, npair = (size_t)(p.T - 1) * plane;
  // Y is the sixth plane; ot_rpca_reset zeroes everything before and after it
  h->slab_floats = (9 + 2 * (nsign - 1)) * nframe + 4 * nsign * npair;
  cudaError_t e = cudaMalloc(&h->slab, h->slab_floats * sizeof(float));
  if (e != cudaSuccess) {
    ot_rpca_destroy(h);
    return cuda_fail(e, "ot_rpca_create: cudaMalloc(state)");
  }
  float* q = h->slab;
  RpcaPlanes& P = h->P;
  P.X = q; q += nframe;
  P.L = q; q += nframe;
  P.A = q; q += nframe;
  P.Tm = q; q += nframe;
  P.D = q; q += nframe;
  P.Y = q; q += nframe;
  P.S = q; q += nframe;
  P.LD = q; q += nframe;
  P.Bz = q; q += nsign * npair;
  P.Cw = q; q += nsign * npair;
  P.zprev = q; q += nsign * npair;
  P.wprev = q; q += nsign * npair;
  P.Tn = q; q += nframe;
  if (p.signed_fg) {
    P.Sp = q; q += nframe;
    P.Sm = q; q += nframe;
  }
  P.sgn_off = (long long)npair;
  P.z = h->prox->x0;
  P.w = h->prox->x1;
  P.p0 = h->prox->p0;
  P.p1 = h->prox->p1;

  const int TP = h->TP;
  const int ng = svt_gram_blocks((long long)plane);
  h->nb_rpca = rpca_num_blocks(h->G);
  int gy = 1;
  h->nb_apply = svt_apply_blocks((long long)plane, p.T, &gy) * gy;
  const size_t svt_bytes = (size_t)ng * TP * TP * sizeof(double) + (size_t)TP * TP * sizeof(double) +
                           (size_t)3 * TP * TP * sizeof(float) + 64;
  e = cudaMalloc(&h->gram_partials, svt_bytes);
  if (e == cudaSuccess) {
    h->Gm = h->gram_partials + (size_t)ng * TP * TP;
    h->V = reinterpret_cast<float*>(h->Gm + (size_t)TP * TP);
    h->Wm = h->V + (size_t)TP * TP;
    h->sig = h->Wm + (size_t)TP * TP;
    h->sweeps = reinterpret_cast<int*>(h->sig + (size_t)TP * TP);
    e = cudaMalloc(&h->partials, ((size_t)(3 * h->nb_rpca + h->nb_apply) * kNumSums + kNumSums) * sizeof(double));
  }
  if (e == cudaSuccess) {
    h->dsums = h->partials + (size_t)(3 * h->nb_rpca + h->nb_apply) * kNumSums;
    e = cudaMallocHost(&h->hsums, (kNumSums + 2 + 128) * sizeof(double));
  }
  if (e == cudaSuccess && TP <= 64 && !p.signed_fg) {
    h->fgram_parts = rpca_gram_parts(h->G);
    const size_t nf = (size_t)h->fgram_parts * TP * TP;
    e = cudaMalloc(&h->fgram, nf * sizeof(float) + 4 * sizeof(unsigned));
    if (e == cudaSuccess) {
      h->fbar = reinterpret_cast<unsigned*>(h->fgram + nf);
      e = cudaMemsetAsync(h->fbar, 0, 4 * sizeof(unsigned), h->stream);
    }
  }
  if (e == cudaSuccess) e = svt_prepare();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->slab, 0, h->slab_floats * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ot_rpca_destroy(h);
    return cuda_fail(e, "ot_rpca_create: workspace");
  }
  *out = h;
  return OT_OK;
}

int ot_rpca_get_params(ot_rpca_t h, ot_rpca_params* out) {
  if (!h || !out) return fail(OT_EINVAL, "ot_rpca_get_params: NULL argument");
  *out = h->prm;
  return OT_OK;
}

int ot_rpca_reset(ot_rpca_t h) {
  if (!h) return fail(OT_EINVAL, "ot_rpca_reset: NULL handle");
  const size_t nframe = (size_t)h->prm.T * (size_t)h->G.plane;
  // every plane but Y, the sixth of the slab (Tm and Tn may have swapped, but
  // both lie in the zeroed ranges)
  OT_CUDA(cudaMemsetAsync(h->slab, 0, 5 * nframe * sizeof(float), h->stream), "ot_rpca_reset");
  OT_CUDA(cudaMemsetAsync(h->slab + 6 * nframe, 0, (h->slab_floats - 6 * nframe) * sizeof(float), h->stream),
          "ot_rpca_reset");
  h->warm = 0;
  return ot_prox_reset(h->prox);
}

int ot_rpca_set_input(ot_rpca_t h, const float* Y) {
  if (!h || !Y) return fail(OT_EINVAL, "ot_rpca_set_input: NULL argument");
  const size_t wb = (size_t)h->G.W * sizeof(float);
  OT_CUDA(cudaMemcpy2DAsync(h->P.Y, (size_t)h->G.Wp * sizeof(float), Y, wb, wb, (size_t)h->G.T * h->G.H,
                            cudaMemcpyDefault, h->stream),
          "ot_rpca_set_input: copy");
  OT_CUDA(rpca_launch_sumsq(h->G, h->P.Y, h->partials, h->stream), "ot_rpca_set_input: ||Y||");
  OT_CUDA(launch_finalize_sums(h->partials, h->nb_rpca, h->dsums, h->stream), "ot_rpca_set_input: ||Y||");
  OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "ot_rpca_set_input");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_rpca_set_input: sync");
  h->y_norm = sqrt(h->hsums[0]);
  if (!isfinite(h->y_norm)) return fail(OT_ENONFINITE, "ot_rpca_set_input: Y has non-finite values");
  h->have_input = 1;
  return OT_OK;
}

}  // extern "C"

// Residual partial sums: lines 4-9 of an outer iteration write the rows of
// its SVT-plane parity (0: rows [0, nb), 1: rows [2 nb, 3 nb)), lines 12-15
// the rows [nb, 2 nb), so the two regions of one iteration are adjacent.
static double* pre_rows(ot_rpca* h, int tp) { return h->partials + (size_t)(tp ? 2 * h->nb_rpca : 0) * kNumSums; }
static double* post_rows(ot_rpca* h) { return h->partials + (size_t)h->nb_rpca * kNumSums; }

// The SVT output just written (Tn) becomes the previous one (Tm) for the next
// outer iteration.
static void swap_svt_planes(ot_rpca* h) {
  float* t = h->P.Tm;
  h->P.Tm = h->P.Tn;
  h->P.Tn = t;
  h->tpar ^= 1;
}

// Lines 12-15 of this outer iteration and lines 4-9 of the next in one pass;
// for T_pad <= 64 the pass also forms this iteration's SVT output (storing it
// only with store_tn) and the next iteration's Gram matrix.
static cudaError_t launch_between(ot_rpca* h, bool store_tn) {
  if (h->fgram)
    return rpca_launch_apply_post_pre_gram(h->G, h->C, h->P, h->TP, h->Wm, store_tn ? 1 : 0,
                                           pre_rows(h, h->tpar ^ 1), h->nb_rpca, h->fgram, h->Gm, h->fbar,
                                           h->prox->derr, h->stream);
  return rpca_launch_post_pre(h->G, h->C, h->P, pre_rows(h, h->tpar ^ 1), h->stream);
}

// Enqueue n >= 1 outer iterations: lines 4-9 of the first, then per
// iteration the SVT (line 10) beside the prox (line 11), and lines 12-15
// fused with the next iteration's lines 4-9, except after the last, whose
// SVT apply and lines 12-15 run alone so the state between calls is
// Algorithm 3's.  For T_pad <= 64 the fused pass also does the SVT apply of
// its iteration (storing the output only before the last iteration, whose
// lines 12-15 compare with it) and the next iteration's Gram matrix.
// `sums` finalises the last iteration's residual sums and copies them (with
// the SVT diagnostics) to the pinned host buffer.
static int enqueue_interval(ot_rpca* h, int n, bool sums) {
  const long long plane = h->G.plane;
  const long long N = plane;   // rows of the N x T matrix: one frame plane (padding columns are zero)
  OT_CUDA(rpca_launch_pre(h->G, h->C, h->P, pre_rows(h, h->tpar), h->stream), "rpca pre");
  int last_par = h->tpar;
  for (int k = 0; k < n; ++k) {
    // line 10: the Gram matrix, from the LD just written (the fused pass
    // before iterations k > 0 has already left it in Gm)
    if (k == 0 || !h->fgram)
      OT_CUDA(svt_launch_gram(h->P.LD, plane, N, h->prm.T, h->gram_partials, h->Gm, h->prox->derr, h->stream),
              "svt gram");
    // fork: the one-CTA T x T eigensolver on the side stream, on the SM that
    // the persistent prox kernel leaves free
    OT_CUDA(cudaEventRecord(h->ev_fork, h->stream), "fork");
    OT_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0), "fork wait");
    OT_CUDA(svt_launch_eig(h->Gm, h->prm.T, h->warm, (float)(h->prm.gamma / h->prm.rho), h->prm.svt_max_sweeps,
                           svt_tolerance(h->prm.T), h->V, h->Wm, h->sig, h->sweeps, h->side),
            "svt eig");
    h->warm = 1;
    OT_CUDA(cudaEventRecord(h->ev_join, h->side), "join");
    // line 11 on the handle's stream, concurrently
    const int rc = ot_prox_step(h->prox, h->prm.n_inner);
    if (rc != OT_OK) return rc;
    // join, then the rest of line 10 and lines 12-15
    OT_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0), "join wait");
    if (k == n - 1 || !h->fgram)
      OT_CUDA(svt_launch_apply(h->P.LD, plane, N, h->prm.T, h->Wm, h->P.Tn, plane, false, nullptr, h->prox->derr,
                               h->stream),
              "svt apply");
    last_par = h->tpar;
    if (k == n - 1)
      OT_CUDA(rpca_launch_post(h->G, h->P, post_rows(h), h->stream), "rpca post");
    else
      OT_CUDA(launch_between(h, k == n - 2), "rpca post + pre");
    swap_svt_planes(h);
  }
  if (sums) {
    OT_CUDA(launch_finalize_sums(h->partials + (size_t)(last_par ? h->nb_rpca : 0) * kNumSums, 2 * h->nb_rpca,
                                 h->dsums, h->stream),
            "rpca finalize");
    OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, kNumSums * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "rpca sums copy");
    OT_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(h->hsums + kNumSums), h->sweeps, sizeof(int),
                            cudaMemcpyDeviceToHost, h->stream),
            "rpca sweeps copy");
    OT_CUDA(cudaMemcpyAsync(reinterpret_cast<float*>(h->hsums + kNumSums + 2), h->sig, h->TP * sizeof(float),
                            cudaMemcpyDeviceToHost, h->stream),
            "rpca sigma copy");
    OT_CUDA(cudaMemcpyAsync(h->prox->herr, h->prox->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
            "rpca error flag copy");
  }
  return OT_OK;
}

// The signed-foreground variant: per outer iteration lines 4-9 for both
// signs, the SVT as its own Gram, eigensolver (beside line 11 on a side
// stream) and apply, line 11 on both signs' 2 (T-1) pairs, and lines 12-15;
// the residual rows of lines 4-9 are [0, nb), of lines 12-15 [nb, 2 nb).
static int enqueue_interval_pn(ot_rpca* h, int n, bool sums) {
  const long long plane = h->G.plane;
  for (int k = 0; k < n; ++k) {
    OT_CUDA(rpca_launch_pn_pre(h->G, h->C, h->P, h->partials, h->stream), "rpca signed pre");
    OT_CUDA(svt_launch_gram(h->P.LD, plane, plane, h->prm.T, h->gram_partials, h->Gm, h->prox->derr, h->stream),
            "svt gram");
    OT_CUDA(cudaEventRecord(h->ev_fork, h->stream), "fork");
    OT_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0), "fork wait");
    OT_CUDA(svt_launch_eig(h->Gm, h->prm.T, h->warm, (float)(h->prm.gamma / h->prm.rho), h->prm.svt_max_sweeps,
                           svt_tolerance(h->prm.T), h->V, h->Wm, h->sig, h->sweeps, h->side),
            "svt eig");
    h->warm = 1;
    OT_CUDA(cudaEventRecord(h->ev_join, h->side), "join");
    const int rc = ot_prox_step(h->prox, h->prm.n_inner);
    if (rc != OT_OK) return rc;
    OT_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0), "join wait");
    OT_CUDA(svt_launch_apply(h->P.LD, plane, plane, h->prm.T, h->Wm, h->P.Tn, plane, false, nullptr, h->prox->derr,
                             h->stream),
            "svt apply");
    OT_CUDA(rpca_launch_pn_post(h->G, h->P, post_rows(h), h->stream), "rpca signed post");
    swap_svt_planes(h);
  }
  if (sums) {
    OT_CUDA(launch_finalize_sums(h->partials, 2 * h->nb_rpca, h->dsums, h->stream), "rpca finalize");
    OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, kNumSums * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "rpca sums copy");
    OT_CUDA(cudaMemcpyAsync(reinterpret_cast<int*>(h->hsums + kNumSums), h->sweeps, sizeof(int),
                            cudaMemcpyDeviceToHost, h->stream),
            "rpca sweeps copy");
    OT_CUDA(cudaMemcpyAsync(reinterpret_cast<float*>(h->hsums + kNumSums + 2), h->sig, h->TP * sizeof(float),
                            cudaMemcpyDeviceToHost, h->stream),
            "rpca sigma copy");
    OT_CUDA(cudaMemcpyAsync(h->prox->herr, h->prox->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
            "rpca error flag copy");
  }
  return OT_OK;
}

// n outer iterations.  An interval of check_every iterations with a warm
// eigensolver replays from a CUDA graph (one per starting parity of the
// inner prox state and of the SVT output planes; the graph bakes in the warm
// flag and the buffers of those parities, and always finalises the sums);
// anything else is enqueued directly.
static int enqueue_any(ot_rpca* h, int n, bool sums) {
  return h->prm.signed_fg ? enqueue_interval_pn(h, n, sums) : enqueue_interval(h, n, sums);
}

static int run_interval(ot_rpca* h, int n, bool sums) {
  const bool can_graph = h->prm.use_graph && h->stream != nullptr && h->warm && n == h->prm.check_every;
  if (!can_graph) return enqueue_any(h, n, sums);
  ot_prox* px = h->prox;
  const int par = px->cur, tp = h->tpar;
  if (!h->graph[par][tp]) {
    cudaGraph_t g = nullptr;
    OT_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "rpca graph capture");
    const int rc = enqueue_any(h, n, true);
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    // capture enqueued nothing: undo the parity bookkeeping
    px->cur = par;
    while (h->tpar != tp) swap_svt_planes(h);
    if (rc != OT_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "rpca graph capture end");
    const cudaError_t e3 = cudaGraphInstantiate(&h->graph[par][tp], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_fail(e3, "rpca graph instantiate");
  }
  OT_CUDA(cudaGraphLaunch(h->graph[par][tp], h->stream), "rpca graph launch");
  px->cur = px->resident ? par : (par ^ ((n * h->prm.n_inner) & 1));
  if (n & 1) swap_svt_planes(h);
  return OT_OK;
}

static void fill_rpca_result(const ot_rpca* h, ot_rpca_result* r) {
  const double* s = h->hsums;
  const double ny = fmax(h->y_norm, 1e-30);
  r->res_pri = sqrt(s[2] + s[3] + s[4] + s[5]) / ny;
  r->res_dual = h->prm.rho * sqrt(s[0] + s[1] + s[6] + s[7]) / ny;
  r->svt_rounds = *reinterpret_cast<const int*>(h->hsums + kNumSums);
  const float* sig = reinterpret_cast<const float*>(h->hsums + kNumSums + 2);
  int rank = 0;
  for (int i = 0; i < h->prm.T; ++i) rank += sig[i] > (float)(h->prm.gamma / h->prm.rho);
  r->svt_rank = rank;
}

static bool rpca_sums_bad(const double* s) {
  for (int k = 0; k < kNumSums; ++k)
    if (!isfinite(s[k])) return true;
  return false;
}

extern "C" {

int ot_rpca_step(ot_rpca_t h, int32_t n_outer) {
  if (!h) return fail(OT_EINVAL, "ot_rpca_step: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_rpca_step: no input (call ot_rpca_set_input)");
  if (n_outer < 0) return fail(OT_EINVAL, "ot_rpca_step: n_outer must be >= 0");
  return n_outer > 0 ? run_interval(h, n_outer, false) : OT_OK;
}

int ot_rpca_iterate_checked(ot_rpca_t h, int32_t n_outer, ot_rpca_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_rpca_iterate_checked: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_rpca_iterate_checked: no input (call ot_rpca_set_input)");
  if (n_outer < 1) return fail(OT_EINVAL, "ot_rpca_iterate_checked: n_outer must be >= 1");
  const int rc = run_interval(h, n_outer, true);
  if (rc != OT_OK) return rc;
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_rpca_iterate_checked: sync");
  if (*h->prox->herr) return fail(OT_ETIMEOUT, "a bounded device wait expired (prox kernel or grid barrier)");
  ot_rpca_result r;
  memset(&r, 0, sizeof r);
  r.iters = n_outer;
  fill_rpca_result(h, &r);
  const bool bad = rpca_sums_bad(h->hsums);
  r.status = bad ? OT_ENONFINITE : OT_OK;
  if (res) *res = r;
  if (bad) return fail(OT_ENONFINITE, "ot_rpca_iterate_checked: non-finite residuals");
  return OT_OK;
}

int ot_rpca_solve(ot_rpca_t h, ot_rpca_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_rpca_solve: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_rpca_solve: no input (call ot_rpca_set_input)");
  ot_rpca_result r;
  memset(&r, 0, sizeof r);
  r.res_pri = r.res_dual = INFINITY;
  int status = OT_ENOTCONV, k = 0;
  while (k < h->prm.max_iter) {
    const int n = (h->prm.max_iter - k) < h->prm.check_every ? (h->prm.max_iter - k) : h->prm.check_every;
    ot_rpca_result rr;
    const int rc = ot_rpca_iterate_checked(h, n, &rr);
    k += n;
    if (rc == OT_ENONFINITE) {
      r = rr;
      status = OT_ENONFINITE;
      break;
    }
    if (rc != OT_OK) return rc;
    r = rr;
    if (fmax(r.res_pri, r.res_dual) <= h->prm.tol) {
      status = OT_OK;
      break;
    }
  }
  r.iters = k;
  r.status = status;
  if (res) *res = r;
  if (status == OT_ENOTCONV)
    fail(OT_ENOTCONV, "ot_rpca_solve: max_iter = %d reached (res_pri %.3g, res_dual %.3g)", h->prm.max_iter,
         r.res_pri, r.res_dual);
  if (status == OT_ENONFINITE) fail(OT_ENONFINITE, "ot_rpca_solve: non-finite values");
  return status;
}

int ot_debug_grid_barrier(int32_t ctas, uint32_t preset_count, int32_t* err, uint32_t* generation) {
  if (!err || !generation) return fail(OT_EINVAL, "ot_debug_grid_barrier: NULL argument");
  int dev = 0, n_sm = 0;
  OT_CUDA(cudaGetDevice(&dev), "ot_debug_grid_barrier: device");
  OT_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "ot_debug_grid_barrier: SM count");
  if (ctas < 1 || ctas > n_sm) return fail(OT_EINVAL, "ot_debug_grid_barrier: ctas must be in [1, %d]", n_sm);
  int e = 0;
  unsigned gen = 0;
  OT_CUDA(grid_barrier_probe(ctas, preset_count, &e, &gen), "ot_debug_grid_barrier");
  *err = e;
  *generation = gen;
  return OT_OK;
}

// One signed-foreground outer iteration with its phases serialised and timed.
static int step_profiled_pn(ot_rpca* h, double* phase_ms) {
  constexpr int kEv = 7;
  cudaEvent_t ev[kEv] = {};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kEv && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
  const long long plane = h->G.plane;
  int rc = OT_OK;
  auto rec = [&](int k) {
    if (e == cudaSuccess && rc == OT_OK) e = cudaEventRecord(ev[k], h->stream);
  };
  rec(0);
  if (e == cudaSuccess) e = rpca_launch_pn_pre(h->G, h->C, h->P, h->partials, h->stream);
  rec(1);
  if (e == cudaSuccess)
    e = svt_launch_gram(h->P.LD, plane, plane, h->prm.T, h->gram_partials, h->Gm, h->prox->derr, h->stream);
  rec(2);
  if (e == cudaSuccess) {
    e = svt_launch_eig(h->Gm, h->prm.T, h->warm, (float)(h->prm.gamma / h->prm.rho), h->prm.svt_max_sweeps,
                       svt_tolerance(h->prm.T), h->V, h->Wm, h->sig, h->sweeps, h->stream);
    h->warm = 1;
  }
  rec(3);
  if (e == cudaSuccess) rc = ot_prox_step(h->prox, h->prm.n_inner);
  rec(4);
  if (e == cudaSuccess && rc == OT_OK)
    e = svt_launch_apply(h->P.LD, plane, plane, h->prm.T, h->Wm, h->P.Tn, plane, false, nullptr, h->prox->derr,
                         h->stream);
  rec(5);
  if (e == cudaSuccess && rc == OT_OK) {
    e = rpca_launch_pn_post(h->G, h->P, post_rows(h), h->stream);
    swap_svt_planes(h);
  }
  rec(6);
  if (e == cudaSuccess && rc == OT_OK) e = cudaEventSynchronize(ev[6]);
  // phases: pre, Gram, eig, apply, prox, post
  const int from[6] = {0, 1, 2, 4, 3, 5}, to[6] = {1, 2, 3, 5, 4, 6};
  for (int k = 0; k < 6 && e == cudaSuccess && rc == OT_OK; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[from[k]], ev[to[k]]);
    phase_ms[k] = ms;
  }
  phase_ms[6] = phase_ms[7] = 0.0;
  for (int k = 0; k < kEv; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  if (rc != OT_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "ot_rpca_step_profiled");
  return OT_OK;
}

int ot_rpca_step_profiled(ot_rpca_t h, double* phase_ms) {
  if (!h || !phase_ms) return fail(OT_EINVAL, "ot_rpca_step_profiled: NULL argument");
  if (!h->have_input) return fail(OT_EINVAL, "ot_rpca_step_profiled: no input (call ot_rpca_set_input)");
  if (h->prm.signed_fg) return step_profiled_pn(h, phase_ms);
  // the kernels of ot_rpca_step(h, 2), serialised on the handle's stream:
  //   ev0 pre ev1 Gram ev2 eig ev3 [apply, T_pad > 64] ev4 prox ev5 fused pass ev6
  //   [Gram, T_pad > 64] ev7 eig ev8 apply ev9 prox ev10 post ev11
  constexpr int kEv = 12;
  cudaEvent_t ev[kEv] = {};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kEv && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
  const long long plane = h->G.plane;
  int rc = OT_OK;
  auto rec = [&](int k) {
    if (e == cudaSuccess && rc == OT_OK) e = cudaEventRecord(ev[k], h->stream);
  };
  auto gram = [&]() {
    if (e == cudaSuccess && rc == OT_OK)
      e = svt_launch_gram(h->P.LD, plane, plane, h->prm.T, h->gram_partials, h->Gm, h->prox->derr, h->stream);
  };
  auto eig = [&]() {
    if (e == cudaSuccess && rc == OT_OK) {
      e = svt_launch_eig(h->Gm, h->prm.T, h->warm, (float)(h->prm.gamma / h->prm.rho), h->prm.svt_max_sweeps,
                         svt_tolerance(h->prm.T), h->V, h->Wm, h->sig, h->sweeps, h->stream);
      h->warm = 1;
    }
  };
  auto apply = [&]() {
    if (e == cudaSuccess && rc == OT_OK)
      e = svt_launch_apply(h->P.LD, plane, plane, h->prm.T, h->Wm, h->P.Tn, plane, false, nullptr, h->prox->derr,
                           h->stream);
  };
  auto prox = [&]() {
    if (e == cudaSuccess && rc == OT_OK) rc = ot_prox_step(h->prox, h->prm.n_inner);
  };
  rec(0);
  if (e == cudaSuccess) e = rpca_launch_pre(h->G, h->C, h->P, pre_rows(h, h->tpar), h->stream);
  rec(1);
  gram();
  rec(2);
  eig();
  rec(3);
  if (!h->fgram) apply();
  rec(4);
  prox();
  rec(5);
  if (e == cudaSuccess && rc == OT_OK) {
    e = launch_between(h, true);
    swap_svt_planes(h);
  }
  rec(6);
  if (!h->fgram) gram();
  rec(7);
  eig();
  rec(8);
  apply();
  rec(9);
  prox();
  rec(10);
  if (e == cudaSuccess && rc == OT_OK) {
    e = rpca_launch_post(h->G, h->P, post_rows(h), h->stream);
    swap_svt_planes(h);
  }
  rec(11);
  if (e == cudaSuccess && rc == OT_OK) e = cudaEventSynchronize(ev[11]);
  // phases: pre, Gram, eig, apply (the second iteration's), prox, post, fused pass, second Gram
  const int from[8] = {0, 1, 2, 8, 4, 10, 5, 6}, to[8] = {1, 2, 3, 9, 5, 11, 6, 7};
  for (int k = 0; k < 8 && e == cudaSuccess && rc == OT_OK; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[from[k]], ev[to[k]]);
    phase_ms[k] = ms;
  }
  for (int k = 0; k < kEv; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  if (rc != OT_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "ot_rpca_step_profiled");
  return OT_OK;
}

int ot_rpca_get(ot_rpca_t h, int32_t var, float* out) {
  if (!h || !out) return fail(OT_EINVAL, "ot_rpca_get: NULL argument");
  const RpcaPlanes& P = h->P;
  const float* src = nullptr;
  int nf = h->prm.T;
  const bool minus = (var & OT_RPCA_MINUS) != 0;
  if (minus) {
    var &= ~OT_RPCA_MINUS;
    if (!h->prm.signed_fg || var < OT_RPCA_B || var > OT_RPCA_DUAL)
      return fail(OT_EINVAL, "ot_rpca_get: OT_RPCA_MINUS needs the signed foreground and a pair variable");
  }
  if ((var == OT_RPCA_SP || var == OT_RPCA_SM) && !h->prm.signed_fg)
    return fail(OT_EINVAL, "ot_rpca_get: S+ and S- exist only with signed_fg");
  switch (var) {
    case OT_RPCA_S: src = P.S; break;
    case OT_RPCA_L: src = P.L; break;
    case OT_RPCA_X: src = P.X; break;
    case OT_RPCA_T: src = P.Tm; break;
    case OT_RPCA_A: src = P.A; break;
    case OT_RPCA_D: src = P.D; break;
    case OT_RPCA_B: src = P.Bz; nf = h->prm.T - 1; break;
    case OT_RPCA_C: src = P.Cw; nf = h->prm.T - 1; break;
    case OT_RPCA_Z: src = P.z; nf = h->prm.T - 1; break;
    case OT_RPCA_W: src = P.w; nf = h->prm.T - 1; break;
    case OT_RPCA_MX: src = h->prox->Mx[h->prox->cur]; nf = h->prm.T - 1; break;
    case OT_RPCA_MY: src = h->prox->My[h->prox->cur]; nf = h->prm.T - 1; break;
    case OT_RPCA_R: src = h->prox->r; nf = h->prm.T - 1; break;
    case OT_RPCA_DUAL: src = h->prox->a[h->prox->cur]; nf = h->prm.T - 1; break;
    case OT_RPCA_SP: src = P.Sp; break;
    case OT_RPCA_SM: src = P.Sm; break;
    default: return fail(OT_EINVAL, "ot_rpca_get: unknown variable %d", var);
  }
  if (minus) src += P.sgn_off;     // the S- sign's pairs follow the S+ sign's
  const size_t wb = (size_t)h->G.W * sizeof(float);
  OT_CUDA(cudaMemcpy2DAsync(out, wb, src, (size_t)h->G.Wp * sizeof(float), wb, (size_t)nf * h->G.H,
                            cudaMemcpyDefault, h->stream),
          "ot_rpca_get: copy");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_rpca_get: sync");
  return OT_OK;
}

int ot_svt(const float* X, float* Y, int64_t N, int32_t T, double theta, void* cuda_stream) {
  if (!X || !Y) return fail(OT_EINVAL, "ot_svt: NULL argument");
  if (N < 1 || T < 1 || T > 128) return fail(OT_EINVAL, "ot_svt: need N >= 1 and 1 <= T <= 128");
  if (!(theta >= 0) || !isfinite(theta)) return fail(OT_EINVAL, "ot_svt: theta must be >= 0");
  if (X == Y) return fail(OT_EINVAL, "ot_svt: X and Y must not alias");
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int TP = svt_padded_T(T);
  const int ng = svt_gram_blocks(N);
  const size_t bytes = (size_t)ng * TP * TP * sizeof(double) + (size_t)TP * TP * sizeof(double) +
                       (size_t)3 * TP * TP * sizeof(float) + 64 + 16;
  OT_CUDA(svt_prepare(), "ot_svt: prepare");
  void* ws = nullptr;
  OT_CUDA(cudaMallocAsync(&ws, bytes, st), "ot_svt: cudaMallocAsync");
  double* part = static_cast<double*>(ws);
  double* Gm = part + (size_t)ng * TP * TP;
  float* V = reinterpret_cast<float*>(Gm + (size_t)TP * TP);
  float* Wm = V + (size_t)TP * TP;
  float* sig = Wm + (size_t)TP * TP;
  int* sweeps = reinterpret_cast<int*>(sig + (size_t)TP * TP);
  int* derr = sweeps + 4;
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(int), st);
  if (e == cudaSuccess) e = svt_launch_gram(X, N, N, T, part, Gm, derr, st);
  if (e == cudaSuccess) e = svt_launch_eig(Gm, T, 0, (float)theta, 60, svt_tolerance(T), V, Wm, sig, sweeps, st);
  if (e == cudaSuccess) e = svt_launch_apply(X, N, N, T, Wm, Y, N, false, nullptr, derr, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ot_svt");
  if (e2 != cudaSuccess) return cuda_fail(e2, "ot_svt: cudaFreeAsync");
  if (herr) return fail(OT_ETIMEOUT, "ot_svt: a bounded device wait expired in the Gram kernel");
  return OT_OK;
}

}  // extern "C"
