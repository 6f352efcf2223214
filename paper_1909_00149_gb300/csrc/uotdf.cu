// Algorithm 2 (UOT-DF ADMM, Sec. IV-A.1) with Phi = I, for B independent
// frames [B][H][W]: the dynamic-filtering problem
//   min_{s >= 0} 1/2 ||y - s||^2 + R(s) + kappa V_mu(s, s0),
// R = 0 (UOT-DF) or lambda ||s||_1 (BPDN+UOT-DF), with s0 the prediction.
//
// One ADMM iteration, in stream order:
//   uotdf_pre    line 4  s = prox_{R+}((x + a + z + b) / 2)   (weight 1/(2 rho))
//                line 5  x = (y + rho (s - a)) / (1 + rho)
//                        the prox centre s - b of line 6, and z kept for the
//                        dual residual
//   ot_prox_step line 6  n_inner warm-started Algorithm 1 iterations in the
//                        fixed-first form (x0 = s0 frozen, x1 = z free),
//                        prox weight kappa / rho
//   uotdf_post   lines 7-8  a += x - s,  b += z - s, and the residual sums
// Readings (see the oracle): s is the minimiser of both augmented terms
// (the printed line keeps only x + a); the BPDN threshold is lambda/(2 rho).
//
// Partial-sum slots (kNumSums per block): 0 ||dx||^2, 2 ||x - s||^2,
// 4 ||z - s||^2, 6 ||dz||^2, 7 non-finite count.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "../../include/otprox.h"
#include "device_util.cuh"
#include "otprox_internal.cuh"
#include "prox_handle.cuh"

using namespace otp;

namespace {

constexpr int kUThreads = 256;

struct UGeom {
  int B, H, W, Wp;
  long long n4;          // float4 groups of all B planes
};

struct UPlanes {
  float *Y, *S, *X, *A, *Bd, *zprev;   // this runtime's planes
  float *z, *p1;                        // the inner prox's x1 and prox centre
};

__global__ void __launch_bounds__(kUThreads)
uotdf_pre_kernel(const UGeom g, const UPlanes P, float rho, float thr, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const float inv1r = 1.f / (1.f + rho);
  for (long long q = blockIdx.x * (long long)kUThreads + threadIdx.x; q < g.n4; q += (long long)gridDim.x * kUThreads) {
    const long long o = 4 * q;
    const float4 x = ldg4(P.X + o), a = ldg4(P.A + o), z = ldg4(P.z + o), b = ldg4(P.Bd + o), y = ldg4(P.Y + o);
    float4 s4, x4, p4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float qv = 0.5f * ((f4c(x, e) + f4c(a, e)) + (f4c(z, e) + f4c(b, e)));
      const float s = fmaxf(qv - thr, 0.f);
      const float xv = (f4c(y, e) + rho * (s - f4c(a, e))) * inv1r;
      const float dx = xv - f4c(x, e);
      acc[0] = fmaf(dx, dx, acc[0]);
      f4(s4, e) = s;
      f4(x4, e) = xv;
      f4(p4, e) = s - f4c(b, e);
    }
    stg4v(P.S + o, s4);
    stg4v(P.X + o, x4);
    stg4v(P.p1 + o, p4);
    stg4v(P.zprev + o, z);
  }
  block_sums_to<kUThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

__global__ void __launch_bounds__(kUThreads)
uotdf_post_kernel(const UGeom g, const UPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  for (long long q = blockIdx.x * (long long)kUThreads + threadIdx.x; q < g.n4; q += (long long)gridDim.x * kUThreads) {
    const long long o = 4 * q;
    const float4 x = ldg4(P.X + o), s = ldg4(P.S + o), z = ldg4(P.z + o), zp = ldg4(P.zprev + o);
    float4 a = ldg4(P.A + o), b = ldg4(P.Bd + o);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float r1 = f4c(x, e) - f4c(s, e);
      const float r2 = f4c(z, e) - f4c(s, e);
      const float dz = f4c(z, e) - f4c(zp, e);
      f4(a, e) += r1;
      f4(b, e) += r2;
      acc[2] = fmaf(r1, r1, acc[2]);
      acc[4] = fmaf(r2, r2, acc[4]);
      acc[6] = fmaf(dz, dz, acc[6]);
      acc[7] += (!isfinite(f4c(a, e)) || !isfinite(f4c(b, e))) ? 1.f : 0.f;
    }
    stg4v(P.A + o, a);
    stg4v(P.Bd + o, b);
  }
  block_sums_to<kUThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// ||y||^2 into slot 0
__global__ void __launch_bounds__(kUThreads)
uotdf_sumsq_kernel(const float* __restrict__ Y, long long n4, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  for (long long q = blockIdx.x * (long long)kUThreads + threadIdx.x; q < n4; q += (long long)gridDim.x * kUThreads) {
    const float4 v = ldg4(Y + 4 * q);
    acc[0] += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  block_sums_to<kUThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

int u_num_blocks(const UGeom& g) {
  const long long nb = (g.n4 + kUThreads - 1) / kUThreads;
  return (int)(nb < 152 * 4 ? (nb < 1 ? 1 : nb) : 152 * 4);
}

}  // namespace

#define OT_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

struct ot_uotdf {
  ot_uotdf_params prm;
  cudaStream_t stream;
  UGeom G;
  UPlanes P;
  float* slab;
  ot_prox* prox;             // B problems, fixed-first, rho_prox = kappa / rho
  int nb;
  double* partials;          // [2 nb][kNumSums]
  double* dsums;             // [kNumSums]
  double* hsums;             // pinned [kNumSums]
  double y_norm;
  int have_input;
};

extern "C" {

void ot_uotdf_default_params(ot_uotdf_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->B = 1;
  p->H = p->W = 1;
  p->kappa = 0.5;
  p->mu = 3.0;
  p->rho = 1.0;
  p->lambda = 0.0;
  p->n_inner = 1;
  p->norm = OT_NORM_ISO;
  p->p_exp = 1;
  p->tol = 1e-5;
  p->max_iter = 20000;
  p->check_every = 10;
  p->prox_kernel = OT_KERNEL_AUTO;
}

int ot_uotdf_destroy(ot_uotdf_t h) {
  if (!h) return OT_OK;
  if (h->prox) ot_prox_destroy(h->prox);
  if (h->slab) cudaFree(h->slab);
  if (h->partials) cudaFree(h->partials);
  if (h->hsums) cudaFreeHost(h->hsums);
  free(h);
  return OT_OK;
}

int ot_uotdf_create(const ot_uotdf_params* params, void* cuda_stream, ot_uotdf_t* out) {
  if (!params || !out) return fail(OT_EINVAL, "ot_uotdf_create: params and out must be non-NULL");
  *out = nullptr;
  const ot_uotdf_params p = *params;
  if (p.B < 1 || p.H < 1 || p.W < 1) return fail(OT_EINVAL, "ot_uotdf_create: B, H, W must be >= 1");
  if (!(p.kappa > 0) || !(p.mu > 0) || !(p.rho > 0) || !(p.lambda >= 0) || !isfinite(p.kappa) ||
      !isfinite(p.mu) || !isfinite(p.rho) || !isfinite(p.lambda))
    return fail(OT_EINVAL, "ot_uotdf_create: kappa, mu, rho must be > 0 and lambda >= 0 (finite)");
  if (p.n_inner < 1 || p.max_iter < 0 || p.check_every < 1 || !(p.tol >= 0))
    return fail(OT_EINVAL, "ot_uotdf_create: n_inner >= 1, max_iter >= 0, check_every >= 1, tol >= 0 required");
  if (p.prox_kernel == OT_KERNEL_TEMPORAL)
    return fail(OT_EINVAL, "ot_uotdf_create: the inner prox cannot use OT_KERNEL_TEMPORAL (its x planes are shared)");
  ot_uotdf* h = (ot_uotdf*)calloc(1, sizeof(ot_uotdf));
  if (!h) return fail(OT_ENOMEM, "ot_uotdf_create: host allocation failed");
  h->prm = p;
  h->stream = (cudaStream_t)cuda_stream;

  ot_prox_params pp;
  ot_prox_default_params(&pp);
  pp.B = p.B;
  pp.H = p.H;
  pp.W = p.W;
  pp.mode = OT_MODE_FIXED_FIRST;
  pp.norm = p.norm;
  pp.p_exp = p.p_exp;
  pp.mu = p.mu;
  pp.rho = p.kappa / p.rho;
  pp.kernel = p.prox_kernel;
  pp.use_graph = 0;
  int rc = ot_prox_create(&pp, cuda_stream, &h->prox);
  if (rc != OT_OK) {
    ot_uotdf_destroy(h);
    return rc;
  }
  h->G.B = p.B;
  h->G.H = p.H;
  h->G.W = p.W;
  h->G.Wp = h->prox->G.Wp;
  const size_t np = (size_t)p.B * p.H * h->G.Wp;
  h->G.n4 = (long long)(np / 4);
  cudaError_t e = cudaMalloc(&h->slab, 6 * np * sizeof(float));
  if (e != cudaSuccess) {
    ot_uotdf_destroy(h);
    return cuda_fail(e, "ot_uotdf_create: cudaMalloc(state)");
  }
  float* q = h->slab;
  h->P.Y = q; q += np;
  h->P.S = q; q += np;
  h->P.X = q; q += np;
  h->P.A = q; q += np;
  h->P.Bd = q; q += np;
  h->P.zprev = q;
  h->P.z = h->prox->x1;
  h->P.p1 = h->prox->p1;
  h->nb = u_num_blocks(h->G);
  e = cudaMalloc(&h->partials, ((size_t)2 * h->nb * kNumSums + kNumSums) * sizeof(double));
  if (e == cudaSuccess) {
    h->dsums = h->partials + (size_t)2 * h->nb * kNumSums;
    e = cudaMallocHost(&h->hsums, kNumSums * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->slab, 0, 6 * np * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ot_uotdf_destroy(h);
    return cuda_fail(e, "ot_uotdf_create: workspace");
  }
  *out = h;
  return OT_OK;
}

int ot_uotdf_get_params(ot_uotdf_t h, ot_uotdf_params* out) {
  if (!h || !out) return fail(OT_EINVAL, "ot_uotdf_get_params: NULL argument");
  *out = h->prm;
  return OT_OK;
}

int ot_uotdf_reset(ot_uotdf_t h) {
  if (!h) return fail(OT_EINVAL, "ot_uotdf_reset: NULL handle");
  const size_t np = (size_t)h->G.B * h->G.H * h->G.Wp;
  // every plane but Y (line 2: s, x, z, a, b and the cached prox state are 0)
  OT_CUDA(cudaMemsetAsync(h->P.S, 0, 5 * np * sizeof(float), h->stream), "ot_uotdf_reset");
  return ot_prox_reset(h->prox);
}

int ot_uotdf_set_input(ot_uotdf_t h, const float* y, const float* s0) {
  if (!h || !y || !s0) return fail(OT_EINVAL, "ot_uotdf_set_input: NULL argument");
  const size_t wb = (size_t)h->G.W * sizeof(float), pitch = (size_t)h->G.Wp * sizeof(float);
  const size_t rows = (size_t)h->G.B * h->G.H;
  OT_CUDA(cudaMemcpy2DAsync(h->P.Y, pitch, y, wb, wb, rows, cudaMemcpyDefault, h->stream), "ot_uotdf_set_input: y");
  // the fixed argument of V_mu(., s0): the inner prox's p0 (its frozen x0)
  OT_CUDA(cudaMemcpy2DAsync(h->prox->p0, pitch, s0, wb, wb, rows, cudaMemcpyDefault, h->stream),
          "ot_uotdf_set_input: s0");
  uotdf_sumsq_kernel<<<h->nb, kUThreads, 0, h->stream>>>(h->P.Y, h->G.n4, h->partials);
  OT_CUDA(cudaGetLastError(), "ot_uotdf_set_input: ||y||");
  OT_CUDA(launch_finalize_sums(h->partials, h->nb, h->dsums, h->stream), "ot_uotdf_set_input: ||y||");
  OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
          "ot_uotdf_set_input");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_uotdf_set_input: sync");
  h->y_norm = sqrt(h->hsums[0]);
  if (!isfinite(h->y_norm)) return fail(OT_ENONFINITE, "ot_uotdf_set_input: y has non-finite values");
  h->have_input = 1;
  return OT_OK;
}

}  // extern "C"

static int enqueue_iteration(ot_uotdf* h, bool sums) {
  const float rho = (float)h->prm.rho;
  const float thr = (float)(h->prm.lambda / (2.0 * h->prm.rho));
  uotdf_pre_kernel<<<h->nb, kUThreads, 0, h->stream>>>(h->G, h->P, rho, thr, h->partials);
  OT_CUDA(cudaGetLastError(), "uotdf pre");
  const int rc = ot_prox_step(h->prox, h->prm.n_inner);
  if (rc != OT_OK) return rc;
  uotdf_post_kernel<<<h->nb, kUThreads, 0, h->stream>>>(h->G, h->P, h->partials + (size_t)h->nb * kNumSums);
  OT_CUDA(cudaGetLastError(), "uotdf post");
  if (sums) {
    OT_CUDA(launch_finalize_sums(h->partials, 2 * h->nb, h->dsums, h->stream), "uotdf finalize");
    OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, kNumSums * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
            "uotdf sums copy");
    OT_CUDA(cudaMemcpyAsync(h->prox->herr, h->prox->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
            "uotdf error flag copy");
  }
  return OT_OK;
}

extern "C" {

int ot_uotdf_step(ot_uotdf_t h, int32_t n) {
  if (!h) return fail(OT_EINVAL, "ot_uotdf_step: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_uotdf_step: no input (call ot_uotdf_set_input)");
  if (n < 0) return fail(OT_EINVAL, "ot_uotdf_step: n must be >= 0");
  for (int k = 0; k < n; ++k) {
    const int rc = enqueue_iteration(h, false);
    if (rc != OT_OK) return rc;
  }
  return OT_OK;
}

int ot_uotdf_iterate_checked(ot_uotdf_t h, int32_t n, ot_uotdf_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_uotdf_iterate_checked: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_uotdf_iterate_checked: no input (call ot_uotdf_set_input)");
  if (n < 1) return fail(OT_EINVAL, "ot_uotdf_iterate_checked: n must be >= 1");
  for (int k = 0; k < n; ++k) {
    const int rc = enqueue_iteration(h, k == n - 1);
    if (rc != OT_OK) return rc;
  }
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_uotdf_iterate_checked: sync");
  if (*h->prox->herr) return fail(OT_ETIMEOUT, "a bounded device wait expired in the prox kernel");
  const double* s = h->hsums;
  const double ny = fmax(h->y_norm, 1e-30);
  ot_uotdf_result r;
  memset(&r, 0, sizeof r);
  r.iters = n;
  r.res_pri = sqrt(s[2] + s[4]) / ny;
  r.res_dual = h->prm.rho * sqrt(s[0] + s[6]) / ny;
  bool bad = s[7] != 0.0;
  for (int k = 0; k < kNumSums; ++k) bad = bad || !isfinite(s[k]);
  r.status = bad ? OT_ENONFINITE : OT_OK;
  if (res) *res = r;
  if (bad) return fail(OT_ENONFINITE, "ot_uotdf_iterate_checked: non-finite values");
  return OT_OK;
}

int ot_uotdf_solve(ot_uotdf_t h, ot_uotdf_result* res) {
  if (!h) return fail(OT_EINVAL, "ot_uotdf_solve: NULL handle");
  if (!h->have_input) return fail(OT_EINVAL, "ot_uotdf_solve: no input (call ot_uotdf_set_input)");
  ot_uotdf_result r;
  memset(&r, 0, sizeof r);
  r.res_pri = r.res_dual = INFINITY;
  int status = OT_ENOTCONV, k = 0;
  while (k < h->prm.max_iter) {
    const int n = (h->prm.max_iter - k) < h->prm.check_every ? (h->prm.max_iter - k) : h->prm.check_every;
    ot_uotdf_result rr;
    const int rc = ot_uotdf_iterate_checked(h, n, &rr);
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
    fail(OT_ENOTCONV, "ot_uotdf_solve: max_iter = %d reached (res_pri %.3g, res_dual %.3g)", h->prm.max_iter,
         r.res_pri, r.res_dual);
  if (status == OT_ENONFINITE) fail(OT_ENONFINITE, "ot_uotdf_solve: non-finite values");
  return status;
}

int ot_uotdf_get(ot_uotdf_t h, int32_t var, float* out) {
  if (!h || !out) return fail(OT_EINVAL, "ot_uotdf_get: NULL argument");
  const float* src = nullptr;
  switch (var) {
    case OT_UOTDF_S: src = h->P.S; break;
    case OT_UOTDF_X: src = h->P.X; break;
    case OT_UOTDF_Z: src = h->P.z; break;
    case OT_UOTDF_A: src = h->P.A; break;
    case OT_UOTDF_B: src = h->P.Bd; break;
    default: return fail(OT_EINVAL, "ot_uotdf_get: unknown variable %d", var);
  }
  const size_t wb = (size_t)h->G.W * sizeof(float);
  OT_CUDA(cudaMemcpy2DAsync(out, wb, src, (size_t)h->G.Wp * sizeof(float), wb, (size_t)h->G.B * h->G.H,
                            cudaMemcpyDefault, h->stream),
          "ot_uotdf_get: copy");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_uotdf_get: sync");
  return OT_OK;
}

}  // extern "C"
