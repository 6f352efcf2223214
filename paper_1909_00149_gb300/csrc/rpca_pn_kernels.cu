// Elementwise passes of the signed-foreground RPCA+UOT-DF variant (eq.
// RPCA_UOTDF_PN, Sec. IV-B): S = S+ - S-, both non-negative, a transport
// term for each.  The paper gives only the objective; the iteration is
// Algorithm 3's ADMM with its splitting applied to each sign (X = S+ - S- + L,
// Tm = L, z+-_t = s+-_t, w+-_{t+1} = s+-_{t+1}, scaled duals A, D, b+-, c+-),
// the blocks in Algorithm 3's order with S+ before S-, each the exact
// minimiser of the augmented Lagrangian over its block.
//
// pre (lines 4-9 for both signs, and the inputs of lines 10-11):
//   k+_t = (x_t - l_t + a_t + s-_t) + w^z_t (z+_t + b+_t) + w^w_t (w+_t + c+_t)
//   s+_t = max(k+_t / sigma_t - lambda / (rho sigma_t), 0)
//   k-_t = (s+_t - x_t + l_t - a_t) + w^z_t (z-_t + b-_t) + w^w_t (w-_t + c-_t)
//   s-_t = max(k-_t / sigma_t - lambda / (rho sigma_t), 0)
//   S = S+ - S-,  L = 1/2 max(Tm - D + X - S + A, 0),
//   X = (Y + rho (S + L - A)) / (1 + rho),  LD = L + D
//   p0+-_t = s+-_t - b+-_t,  p1+-_t = s+-_{t+1} - c+-_{t+1}  (line 11 centres)
// with w^z_t = [t < T-1], w^w_t = [t > 0], sigma_t = 1 + w^z_t + w^w_t; z, w of
// this iteration are kept for the dual residual.
// post (lines 12-15): A += X - S - L, D += L - Tn, and for each sign
//   b+-_t += z+-_t - s+-_t,  c+-_{t+1} += w+-_{t+1} - s+-_{t+1},
// with the ADMM residual sums, both signs' terms in the same slots: 0 ||dX||^2
// (pre), 1 ||Tn - Tm||^2, 2 ||X-S-L||^2, 3 ||L-Tn||^2, 4 ||z-s_t||^2,
// 5 ||w-s_{t+1}||^2, 6 ||dz||^2, 7 ||dw||^2.
//
// Pair planes hold both signs: pair t of S+ at t * plane, of S- at
// (T - 1 + t) * plane (P.sgn_off further), so the inner Algorithm 1 handle
// runs both signs' T - 1 problems as one batch of 2 (T - 1).
#include <cuda_runtime.h>
#include <math.h>

#include "device_util.cuh"
#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kPnThreads = 256;

__global__ void __launch_bounds__(kPnThreads)
rpca_pn_pre_kernel(const RpcaGeom g, const RpcaCoeffs c, const RpcaPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per_frame = g.plane / 4;
  const long long total = per_frame * g.T;
  const float rho = c.rho, inv1r = 1.f / (1.f + c.rho);
  const long long so = P.sgn_off;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long q = blockIdx.x * (long long)kPnThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kPnThreads) {
    const int t = (int)(q / per_frame);
    const long long o = 4 * q;
    const long long op = o - (long long)t * g.plane;
    const bool hz = t < g.T - 1, hw = t > 0;
    const float sg = 1.f + (hz ? 1.f : 0.f) + (hw ? 1.f : 0.f);
    const float inv_sg = 1.f / sg, thr = c.lam / (c.rho * sg);
    const long long oz = (long long)t * g.plane + op;          // pair t (its z, b pair with s_t)
    const long long ow = (long long)(t - 1) * g.plane + op;    // pair t-1 (its w, c pair with s_t)
    const float4 x = ldg4(P.X + o), l = ldg4(P.L + o), a = ldg4(P.A + o), tm = ldg4(P.Tm + o),
                 d = ldg4(P.D + o), y = ldg4(P.Y + o), smo = ldg4(P.Sm + o);
    const float4 zp = hz ? ldg4(P.z + oz) : z4, bp = hz ? ldg4(P.Bz + oz) : z4;
    const float4 wp = hw ? ldg4(P.w + ow) : z4, cp = hw ? ldg4(P.Cw + ow) : z4;
    const float4 zm = hz ? ldg4(P.z + so + oz) : z4, bm = hz ? ldg4(P.Bz + so + oz) : z4;
    const float4 wm = hw ? ldg4(P.w + so + ow) : z4, cm = hw ? ldg4(P.Cw + so + ow) : z4;
    float4 sp4, sm4, s4, l4, x4, ld4, p0p, p1p, p0m, p1m;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xe = f4c(x, e), le = f4c(l, e), ae = f4c(a, e);
      const float kp = (xe - le + ae + f4c(smo, e)) + (f4c(zp, e) + f4c(bp, e)) + (f4c(wp, e) + f4c(cp, e));
      const float sp = fmaxf(fmaf(kp, inv_sg, -thr), 0.f);
      const float km = (sp - xe + le - ae) + (f4c(zm, e) + f4c(bm, e)) + (f4c(wm, e) + f4c(cm, e));
      const float sm = fmaxf(fmaf(km, inv_sg, -thr), 0.f);
      const float s = sp - sm;
      const float lv = 0.5f * fmaxf(f4c(tm, e) - f4c(d, e) + xe - s + ae, 0.f);
      const float xv = fmaf(rho, s + lv - ae, f4c(y, e)) * inv1r;
      const float dx = xv - xe;
      acc[0] = fmaf(dx, dx, acc[0]);
      f4(sp4, e) = sp;
      f4(sm4, e) = sm;
      f4(s4, e) = s;
      f4(l4, e) = lv;
      f4(x4, e) = xv;
      f4(ld4, e) = lv + f4c(d, e);
      f4(p0p, e) = sp - f4c(bp, e);
      f4(p1p, e) = sp - f4c(cp, e);
      f4(p0m, e) = sm - f4c(bm, e);
      f4(p1m, e) = sm - f4c(cm, e);
    }
    stg4v(P.Sp + o, sp4);
    stg4v(P.Sm + o, sm4);
    stg4v(P.S + o, s4);
    stg4v(P.L + o, l4);
    stg4v(P.X + o, x4);
    stg4v(P.LD + o, ld4);
    if (hz) {
      stg4v(P.p0 + oz, p0p);
      stg4v(P.p0 + so + oz, p0m);
      stg4v(P.zprev + oz, zp);
      stg4v(P.zprev + so + oz, zm);
    }
    if (hw) {
      stg4v(P.p1 + ow, p1p);
      stg4v(P.p1 + so + ow, p1m);
      stg4v(P.wprev + ow, wp);
      stg4v(P.wprev + so + ow, wm);
    }
  }
  block_sums_to<kPnThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// One sign's lines 14-15 at one pixel: b += z - s_t (pair t), c += w - s_t
// (pair t-1), with that sign's residual terms.
__device__ __forceinline__ void pn_pair_duals(float s, float z, float zp, float& b, float w, float wp, float& cc,
                                              bool hz, bool hw, float (&acc)[kNumSums]) {
  const float rz = z - s, rw = w - s;
  b += rz;
  cc += rw;
  const float dz = z - zp, dw = w - wp;
  if (hz) {
    acc[4] = fmaf(rz, rz, acc[4]);
    acc[6] = fmaf(dz, dz, acc[6]);
  }
  if (hw) {
    acc[5] = fmaf(rw, rw, acc[5]);
    acc[7] = fmaf(dw, dw, acc[7]);
  }
}

__global__ void __launch_bounds__(kPnThreads)
rpca_pn_post_kernel(const RpcaGeom g, const RpcaPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per_frame = g.plane / 4;
  const long long total = per_frame * g.T;
  const long long so = P.sgn_off;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long q = blockIdx.x * (long long)kPnThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kPnThreads) {
    const int t = (int)(q / per_frame);
    const long long o = 4 * q;
    const long long op = o - (long long)t * g.plane;
    const bool hz = t < g.T - 1, hw = t > 0;
    const long long oz = (long long)t * g.plane + op;
    const long long ow = (long long)(t - 1) * g.plane + op;
    // every load before any store (the planes are not marked restrict)
    const float4 x = ldg4(P.X + o), sp = ldg4(P.Sp + o), sm = ldg4(P.Sm + o), l = ldg4(P.L + o),
                 tn = ldg4(P.Tn + o), tm = ldg4(P.Tm + o);
    float4 a = ldg4(P.A + o), d = ldg4(P.D + o);
    const float4 zpl = hz ? ldg4(P.z + oz) : z4, zpp = hz ? ldg4(P.zprev + oz) : z4;
    const float4 zmi = hz ? ldg4(P.z + so + oz) : z4, zmp = hz ? ldg4(P.zprev + so + oz) : z4;
    float4 bpl = hz ? ldg4(P.Bz + oz) : z4, bmi = hz ? ldg4(P.Bz + so + oz) : z4;
    const float4 wpl = hw ? ldg4(P.w + ow) : z4, wpp = hw ? ldg4(P.wprev + ow) : z4;
    const float4 wmi = hw ? ldg4(P.w + so + ow) : z4, wmp = hw ? ldg4(P.wprev + so + ow) : z4;
    float4 cpl = hw ? ldg4(P.Cw + ow) : z4, cmi = hw ? ldg4(P.Cw + so + ow) : z4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float s = f4c(sp, e) - f4c(sm, e);
      const float r1 = f4c(x, e) - s - f4c(l, e);
      const float r2 = f4c(l, e) - f4c(tn, e);
      f4(a, e) += r1;
      f4(d, e) += r2;
      const float dt = f4c(tn, e) - f4c(tm, e);
      acc[1] = fmaf(dt, dt, acc[1]);
      acc[2] = fmaf(r1, r1, acc[2]);
      acc[3] = fmaf(r2, r2, acc[3]);
      pn_pair_duals(f4c(sp, e), f4c(zpl, e), f4c(zpp, e), f4(bpl, e), f4c(wpl, e), f4c(wpp, e), f4(cpl, e), hz, hw,
                    acc);
      pn_pair_duals(f4c(sm, e), f4c(zmi, e), f4c(zmp, e), f4(bmi, e), f4c(wmi, e), f4c(wmp, e), f4(cmi, e), hz, hw,
                    acc);
    }
    stg4v(P.A + o, a);
    stg4v(P.D + o, d);
    if (hz) {
      stg4v(P.Bz + oz, bpl);
      stg4v(P.Bz + so + oz, bmi);
    }
    if (hw) {
      stg4v(P.Cw + ow, cpl);
      stg4v(P.Cw + so + ow, cmi);
    }
  }
  block_sums_to<kPnThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

}  // namespace

cudaError_t rpca_launch_pn_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                               cudaStream_t st) {
  rpca_pn_pre_kernel<<<rpca_num_blocks(g), kPnThreads, 0, st>>>(g, c, P, partials);
  return cudaGetLastError();
}

cudaError_t rpca_launch_pn_post(const RpcaGeom& g, const RpcaPlanes& P, double* partials, cudaStream_t st) {
  rpca_pn_post_kernel<<<rpca_num_blocks(g), kPnThreads, 0, st>>>(g, P, partials);
  return cudaGetLastError();
}

}  // namespace otp
