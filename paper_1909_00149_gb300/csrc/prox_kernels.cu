// Algorithm 1 (Sec. III-B) of arXiv:1909.00149 on sm_103a.
//
// One iteration of Algorithm 1 (lines 3-7) is fused into a single pass over
// HBM: each CTA reads the state of its tile once, computes
//   M'  = shrink_{tau1}(M - tau1 D*(a))              (line 3, eq. Prox_UOT_M_prox)
//   x'  = Pi_+((tau1 p + rho x -/+ rho tau1 a) / (rho + tau1))   (line 4)
//   r'  = shrink^{l1}_{mu tau1}(r + tau1 a)          (line 5)
//   a'  = a + tau2 (2 K(z') - K(z))                  (lines 6-7)
// and writes the new state once.  K is linear, so 2K(z') - K(z) = K(2z' - z):
// the kernel forms Mbar = 2M' - M in shared memory and applies D to it once.
// D(Mbar) at a pixel needs Mbar one row up and one column left, so the CTA
// recomputes M' on a one-sided halo (top row, left column) from a's tile
// with a one-pixel ring.  Zero flux (Sec. III-A): Mx[H-1,:] = My[:,W-1] = 0.
//
// Layout: planes [B][H][Wp] float32, Wp = W rounded up to 4; padding
// columns are kept at zero by every writer.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "otprox_internal.cuh"
#include "prox_tile.cuh"

namespace otp {
namespace {
using namespace tile;

template <int NT>
__device__ void block_sum_store_d(double (&v)[kNumSums], double* out) {
  constexpr int NW = NT / 32;
  __shared__ double red[NW][kNumSums];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) red[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) {
      double t = lane < NW ? red[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) out[k] = t;
    }
  }
}

// ===================================================================== K1
template <int MODE, bool BAL, bool RED>
__global__ void __launch_bounds__(kTiledThreads, 2)
prox_tiled_kernel(const Geometry G, const IterCoeffs C, const StatePtrs S, double* __restrict__ partials) {
  prox_tile<MODE, BAL, RED, kTH>(G, C, S, blockIdx.x, RED ? partials + (size_t)blockIdx.x * kNumSums : nullptr);
}

// ===================================================================== K2
// Whole problem resident in shared memory, one CTA per problem, n_iter
// iterations per launch.  Shared planes (pitch Wp): Mx, My, Mbx, Mby, a, r,
// x0, x1, p0, p1 (frozen x and balanced r omitted).  Each iteration has two
// phases separated by a barrier: (A) line 3 per pixel, M updated in place
// and Mbar = 2M' - M stored; (B) lines 4-7 per pixel, a updated in place.
struct ResidentLayout {
  int nplanes;
  int oMx, oMy, oMbx, oMby, oA, oR, oX0, oX1, oP0, oP1;
};

__host__ __device__ inline ResidentLayout resident_layout(int mode, bool bal) {
  ResidentLayout L;
  int n = 0;
  L.oMx = n++;
  L.oMy = n++;
  L.oMbx = n++;
  L.oMby = n++;
  L.oA = n++;
  L.oP0 = n++;
  L.oP1 = n++;
  L.oR = bal ? -1 : n++;
  L.oX0 = mode == 0 ? n++ : -1;
  L.oX1 = mode != 2 ? n++ : -1;
  L.nplanes = n;
  return L;
}

template <int MODE, bool BAL>
__global__ void __launch_bounds__(kResidentThreads, 1)
prox_resident_kernel(const Geometry G, const IterCoeffs C, float* __restrict__ gMx, float* __restrict__ gMy,
                     float* __restrict__ ga, float* __restrict__ gx0, float* __restrict__ gx1,
                     float* __restrict__ gr, const float* __restrict__ gp0, const float* __restrict__ gp1,
                     int n_iter, int reduce_last, double* __restrict__ partials) {
  extern __shared__ __align__(16) float smem[];
  const ResidentLayout L = resident_layout(MODE, BAL);
  const int H = G.H, W = G.W, Wp = G.Wp;
  const int P = H * Wp;
  const int P4 = P / 4;
  const int W4 = Wp / 4;
  const long long base = (long long)blockIdx.x * G.plane;
  float* sMx = smem + (size_t)L.oMx * P;
  float* sMy = smem + (size_t)L.oMy * P;
  float* sMbx = smem + (size_t)L.oMbx * P;
  float* sMby = smem + (size_t)L.oMby * P;
  float* sA = smem + (size_t)L.oA * P;
  float* sP0 = smem + (size_t)L.oP0 * P;
  float* sP1 = smem + (size_t)L.oP1 * P;
  float* sR = BAL ? nullptr : smem + (size_t)L.oR * P;
  float* sX0 = MODE == 0 ? smem + (size_t)L.oX0 * P : sP0;
  float* sX1 = MODE != 2 ? smem + (size_t)L.oX1 * P : sP1;
  const int tid = threadIdx.x;

  for (int g = tid; g < P4; g += kResidentThreads) {
    const long long off = base + 4LL * g;
    st4(sMx + 4 * g, ld4(gMx + off));
    st4(sMy + 4 * g, ld4(gMy + off));
    st4(sA + 4 * g, ld4(ga + off));
    st4(sP0 + 4 * g, ld4(gp0 + off));
    st4(sP1 + 4 * g, ld4(gp1 + off));
    if (!BAL) st4(sR + 4 * g, ld4(gr + off));
    if (MODE == 0) st4(sX0 + 4 * g, ld4(gx0 + off));
    if (MODE != 2) st4(sX1 + 4 * g, ld4(gx1 + off));
  }
  __syncthreads();

  float acc[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) acc[k] = 0.f;

  for (int it = 0; it < n_iter; ++it) {
    const bool red = reduce_last && (it == n_iter - 1);
    // phase A: line 3
    for (int g = tid; g < P4; g += kResidentThreads) {
      const int i = g / W4, j = 4 * (g - i * W4);
      const int o = i * Wp + j;
      const float4 m4x = *reinterpret_cast<const float4*>(sMx + o);
      const float4 m4y = *reinterpret_cast<const float4*>(sMy + o);
      const float4 ac = *reinterpret_cast<const float4*>(sA + o);
      const float an = (j + 4 < Wp) ? sA[o + 4] : 0.f;
      const float4 ad = (i + 1 < H) ? *reinterpret_cast<const float4*>(sA + o + Wp) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 nx, ny, bx, by;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = j + e;
        const bool in = jj < W;
        const float a_r = e < 3 ? compc(ac, e + 1) : an;
        float ox, oy;
        flux_step(compc(m4x, e), compc(m4y, e), compc(ac, e), compc(ad, e), a_r, in && i < H - 1,
                  in && jj < W - 1, C, ox, oy);
        comp(nx, e) = ox;
        comp(ny, e) = oy;
        comp(bx, e) = 2.f * ox - compc(m4x, e);
        comp(by, e) = 2.f * oy - compc(m4y, e);
        if (red && in) {
          const float d0 = ox - compc(m4x, e), d1 = oy - compc(m4y, e);
          acc[1] += d0 * d0 + d1 * d1;
          acc[2] += ox * ox + oy * oy;
          acc[3] += norm_term(ox, oy, C.iso);
          acc[7] += (nonfinite(ox) || nonfinite(oy)) ? 1.f : 0.f;
        }
      }
      st4(sMx + o, nx);
      st4(sMy + o, ny);
      st4(sMbx + o, bx);
      st4(sMby + o, by);
    }
    __syncthreads();
    // phase B: lines 4-7
    for (int g = tid; g < P4; g += kResidentThreads) {
      const int i = g / W4, j = 4 * (g - i * W4);
      const int o = i * Wp + j;
      const float4 a4 = *reinterpret_cast<const float4*>(sA + o);
      const float4 p04 = *reinterpret_cast<const float4*>(sP0 + o);
      const float4 p14 = *reinterpret_cast<const float4*>(sP1 + o);
      const float4 x04 = *reinterpret_cast<const float4*>(sX0 + o);
      const float4 x14 = *reinterpret_cast<const float4*>(sX1 + o);
      const float4 r4 = BAL ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(sR + o);
      const float4 mbx = *reinterpret_cast<const float4*>(sMbx + o);
      const float4 mbx_up = i > 0 ? *reinterpret_cast<const float4*>(sMbx + o - Wp) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 mby = *reinterpret_cast<const float4*>(sMby + o);
      const float mby_l = j > 0 ? sMby[o - 1] : 0.f;
      float4 nx0, nx1, nr, na;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = j + e;
        const bool in = jj < W;
        const float a = compc(a4, e);
        float vx0 = compc(p04, e), vx1 = compc(p14, e);
        if (MODE == 0) vx0 = fmaxf(fmaf(C.cp, compc(p04, e), fmaf(C.cx, compc(x04, e), C.ca * a)), 0.f);
        if (MODE != 2) vx1 = fmaxf(fmaf(C.cp, compc(p14, e), fmaf(C.cx, compc(x14, e), -C.ca * a)), 0.f);
        const float vr = BAL ? 0.f : r_step(compc(r4, e), a, C);
        const float dmb = (compc(mbx, e) - compc(mbx_up, e)) +
                          (compc(mby, e) - (e == 0 ? mby_l : compc(mby, e - 1)));
        float bk = dmb - (2.f * vx0 - compc(x04, e)) + (2.f * vx1 - compc(x14, e));
        if (!BAL) bk -= 2.f * vr - compc(r4, e);
        const float va = fmaf(C.tau2, bk, a);
        comp(nx0, e) = in ? vx0 : 0.f;
        comp(nx1, e) = in ? vx1 : 0.f;
        comp(nr, e) = in ? vr : 0.f;
        comp(na, e) = in ? va : 0.f;
        if (red && in) {
          const float mxn = sMx[o + e], myn = sMy[o + e];
          const float mx_up = i > 0 ? sMx[o + e - Wp] : 0.f;
          const float my_l = (j + e) > 0 ? sMy[o + e - 1] : 0.f;
          const float kz = (mxn - mx_up) + (myn - my_l) - vx0 + vx1 - (BAL ? 0.f : vr);
          acc[0] = fmaf(kz, kz, acc[0]);
          const float d2 = vx0 - compc(x04, e), d3 = vx1 - compc(x14, e);
          const float d4 = vr - compc(r4, e), d5 = va - a;
          acc[1] += d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5;
          acc[2] += vx0 * vx0 + vx1 * vx1 + vr * vr + va * va;
          acc[4] += C.pexp == 1 ? fabsf(vr) : vr * vr;
          const float e0 = vx0 - compc(p04, e), e1 = vx1 - compc(p14, e);
          if (MODE == 0) acc[5] = fmaf(e0, e0, acc[5]);
          if (MODE != 2) acc[5] = fmaf(e1, e1, acc[5]);
          acc[6] += compc(p04, e) * compc(p04, e) + compc(p14, e) * compc(p14, e);
          acc[7] += (nonfinite(va) || nonfinite(vx0) || nonfinite(vx1) || nonfinite(vr) || nonfinite(compc(p04, e)) ||
                     nonfinite(compc(p14, e))) ? 1.f : 0.f;
        }
      }
      st4(sA + o, na);
      if (MODE == 0) st4(sX0 + o, nx0);
      if (MODE != 2) st4(sX1 + o, nx1);
      if (!BAL) st4(sR + o, nr);
    }
    __syncthreads();
  }

  for (int g = tid; g < P4; g += kResidentThreads) {
    const long long off = base + 4LL * g;
    st4(gMx + off, *reinterpret_cast<const float4*>(sMx + 4 * g));
    st4(gMy + off, *reinterpret_cast<const float4*>(sMy + 4 * g));
    st4(ga + off, *reinterpret_cast<const float4*>(sA + 4 * g));
    if (!BAL) st4(gr + off, *reinterpret_cast<const float4*>(sR + 4 * g));
    if (MODE == 0) st4(gx0 + off, *reinterpret_cast<const float4*>(sX0 + 4 * g));
    if (MODE != 2) st4(gx1 + off, *reinterpret_cast<const float4*>(sX1 + 4 * g));
  }
  if (reduce_last && n_iter > 0) {
    __syncthreads();
    block_sum_store<kResidentThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
  }
}

// ===================================================================== K3
// Fixed-order FP64 sum of per-CTA partials (deterministic: no atomics).
// partials[p][k], p < n, k < NQ (NQ a power of two).  One CTA of 1024
// threads reads the n * NQ values coalesced: thread t always meets quantity
// k = t % NQ and sums every 1024th value; lanes with equal k are then
// combined by shuffles, the 32 warp results in shared memory by warp 0.
// Quantities whose bit is set in max_mask are reduced by max instead of sum.
constexpr int kFinThreads = 1024;

template <int NQ>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const double* __restrict__ partials, int n,
                                                               unsigned max_mask, double* __restrict__ out) {
  static_assert(NQ >= 1 && NQ <= 32 && (NQ & (NQ - 1)) == 0, "NQ must be a power of two <= 32");
  __shared__ double red[kFinThreads / 32][NQ];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = tid & (NQ - 1);
  const bool is_max = (max_mask >> k) & 1u;
  const long long total = (long long)n * NQ;
  double v = 0.0;
  for (long long e = tid; e < total; e += kFinThreads) {
    const double x = __ldg(partials + e);
    v = is_max ? fmax(v, x) : v + x;
  }
#pragma unroll
  for (int o = 16; o >= NQ; o >>= 1) {
    const double y = __shfl_down_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, y) : v + y;
  }
  if (lane < NQ) red[warp][lane] = v;
  __syncthreads();
  if (warp == 0 && lane < NQ) {
    double t = red[0][lane];
    for (int w = 1; w < kFinThreads / 32; ++w) t = is_max ? fmax(t, red[w][lane]) : t + red[w][lane];
    out[lane] = t;
  }
}

// ===================================================================== evaluation
// Check sums and duality-gap certificate of a state (not on the hot loop).
// Pass 1: sums 0, 2..7 of the state itself and max_i ||(D* a)_i||.
// Pass 2: dual objective at a_bar = clip(a / max(1, max||D*a||), -mu, mu) and
// the objective of the feasible primal point r' = D(M) + A x.
constexpr int kCertThreads = 256;
constexpr int kCertQ = 4;

__device__ __forceinline__ float at(const float* p, long long base, int i, int j, int Wp) {
  return p[base + (long long)i * Wp + j];
}

__global__ void __launch_bounds__(kCertThreads)
eval_pass1_kernel(const Geometry G, const CertCoeffs cc, const float* __restrict__ Mx, const float* __restrict__ My,
                  const float* __restrict__ a, const float* __restrict__ x0, const float* __restrict__ x1,
                  const float* __restrict__ r, const float* __restrict__ p0, const float* __restrict__ p1,
                  double* __restrict__ partials, double* __restrict__ cpart) {
  const long long total = (long long)G.B * G.H * G.W;
  double acc[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) acc[k] = 0.0;
  double nmax = 0.0;
  const int H = G.H, W = G.W, Wp = G.Wp;
  for (long long idx = blockIdx.x * (long long)kCertThreads + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * kCertThreads) {
    const int jj = (int)(idx % W);
    const long long t = idx / W;
    const int i = (int)(t % H);
    const long long b = t / H;
    const long long base = b * G.plane;
    const double mx = at(Mx, base, i, jj, Wp), my = at(My, base, i, jj, Wp);
    const double mx_up = i > 0 ? at(Mx, base, i - 1, jj, Wp) : 0.0;
    const double my_l = jj > 0 ? at(My, base, i, jj - 1, Wp) : 0.0;
    const double vp0 = at(p0, base, i, jj, Wp), vp1 = at(p1, base, i, jj, Wp);
    const double vx0 = cc.mode == 0 ? at(x0, base, i, jj, Wp) : vp0;
    const double vx1 = cc.mode != 2 ? at(x1, base, i, jj, Wp) : vp1;
    const double vr = cc.balanced ? 0.0 : at(r, base, i, jj, Wp);
    const double va = at(a, base, i, jj, Wp);
    const double kz = (mx - mx_up) + (my - my_l) - vx0 + vx1 - vr;
    acc[0] += kz * kz;
    acc[2] += mx * mx + my * my + vx0 * vx0 + vx1 * vx1 + vr * vr + va * va;
    acc[3] += cc.iso ? sqrt(mx * mx + my * my) : fabs(mx) + fabs(my);
    acc[4] += cc.pexp == 1 ? fabs(vr) : vr * vr;
    if (cc.mode == 0) acc[5] += (vx0 - vp0) * (vx0 - vp0);
    if (cc.mode != 2) acc[5] += (vx1 - vp1) * (vx1 - vp1);
    acc[6] += vp0 * vp0 + vp1 * vp1;
    acc[7] += (isfinite(mx) && isfinite(my) && isfinite(va) && isfinite(vx0) && isfinite(vx1) && isfinite(vr)) ? 0.0 : 1.0;
    const double gx = i < H - 1 ? va - at(a, base, i + 1, jj, Wp) : 0.0;
    const double gy = jj < W - 1 ? va - at(a, base, i, jj + 1, Wp) : 0.0;
    const double n = cc.iso ? sqrt(gx * gx + gy * gy) : fmax(fabs(gx), fabs(gy));
    nmax = fmax(nmax, n);
  }
  block_sum_store_d<kCertThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
  // block max of nmax
  __shared__ double smax[kCertThreads / 32];
  for (int o = 16; o > 0; o >>= 1) nmax = fmax(nmax, __shfl_down_sync(0xffffffffu, nmax, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = nmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < kCertThreads / 32; ++w) m = fmax(m, smax[w]);
    cpart[(size_t)blockIdx.x * kCertQ + 0] = m;
  }
}

__global__ void __launch_bounds__(kCertThreads)
eval_pass2_kernel(const Geometry G, const CertCoeffs cc, const float* __restrict__ Mx, const float* __restrict__ My,
                  const float* __restrict__ a, const float* __restrict__ x0, const float* __restrict__ x1,
                  const float* __restrict__ p0, const float* __restrict__ p1, const double* __restrict__ cert_out,
                  double* __restrict__ cpart) {
  const long long total = (long long)G.B * G.H * G.W;
  const double scale = fmax(1.0, cert_out[0]);
  double dual = 0.0, primal = 0.0;
  const int H = G.H, W = G.W, Wp = G.Wp;
  for (long long idx = blockIdx.x * (long long)kCertThreads + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * kCertThreads) {
    const int jj = (int)(idx % W);
    const long long t = idx / W;
    const int i = (int)(t % H);
    const long long b = t / H;
    const long long base = b * G.plane;
    double ab = at(a, base, i, jj, Wp) / scale;
    if (!cc.balanced && cc.pexp == 1) ab = fmin(fmax(ab, -cc.mu), cc.mu);
    const double vp0 = at(p0, base, i, jj, Wp), vp1 = at(p1, base, i, jj, Wp);
    const double vx0 = cc.mode == 0 ? at(x0, base, i, jj, Wp) : vp0;
    const double vx1 = cc.mode != 2 ? at(x1, base, i, jj, Wp) : vp1;
    // dual: x0 enters K with -1, x1 with +1
    if (cc.mode == 0) {
      const double c = -ab, xs = fmax(vp0 - cc.rho * c, 0.0);
      dual += (xs - vp0) * (xs - vp0) / (2.0 * cc.rho) + c * xs;
    } else {
      dual += -ab * vp0;
    }
    if (cc.mode != 2) {
      const double c = ab, xs = fmax(vp1 - cc.rho * c, 0.0);
      dual += (xs - vp1) * (xs - vp1) / (2.0 * cc.rho) + c * xs;
    } else {
      dual += ab * vp1;
    }
    if (!cc.balanced && cc.pexp == 2) dual -= ab * ab / (4.0 * cc.mu);
    // feasible primal
    const double mx = at(Mx, base, i, jj, Wp), my = at(My, base, i, jj, Wp);
    const double mx_up = i > 0 ? at(Mx, base, i - 1, jj, Wp) : 0.0;
    const double my_l = jj > 0 ? at(My, base, i, jj - 1, Wp) : 0.0;
    const double rp = (mx - mx_up) + (my - my_l) - vx0 + vx1;
    primal += cc.iso ? sqrt(mx * mx + my * my) : fabs(mx) + fabs(my);
    if (!cc.balanced) primal += cc.mu * (cc.pexp == 1 ? fabs(rp) : rp * rp);
    if (cc.mode == 0) primal += (vx0 - vp0) * (vx0 - vp0) / (2.0 * cc.rho);
    if (cc.mode != 2) primal += (vx1 - vp1) * (vx1 - vp1) / (2.0 * cc.rho);
  }
  __shared__ double s[2][kCertThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    dual += __shfl_down_sync(0xffffffffu, dual, o);
    primal += __shfl_down_sync(0xffffffffu, primal, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s[0][threadIdx.x >> 5] = dual;
    s[1][threadIdx.x >> 5] = primal;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0, p = 0.0;
    for (int w = 0; w < kCertThreads / 32; ++w) {
      d += s[0][w];
      p += s[1][w];
    }
    cpart[(size_t)blockIdx.x * kCertQ + 1] = d;
    cpart[(size_t)blockIdx.x * kCertQ + 2] = p;
    cpart[(size_t)blockIdx.x * kCertQ + 3] = 0.0;
  }
}

template <int MODE, bool BAL, bool RED>
cudaError_t launch_tiled_t(const Geometry& g, const IterCoeffs& c, const StatePtrs& s, double* partials,
                           cudaStream_t st) {
  const dim3 block(kTX, kTY);
  prox_tiled_kernel<MODE, BAL, RED><<<tiled_num_ctas(g), block, 0, st>>>(g, c, s, partials);
  return cudaGetLastError();
}

// The attribute belongs to the kernel, not to a handle: raise it to the cap
// of every resident geometry, so that a handle created later with a smaller
// state cannot lower it under an earlier handle's launch size.
template <int MODE, bool BAL>
cudaError_t prepare_resident_t(const Geometry& g) {
  (void)g;
  return cudaFuncSetAttribute(prox_resident_kernel<MODE, BAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kResidentSmemCap);
}

template <int MODE, bool BAL>
cudaError_t launch_resident_t(const Geometry& g, const IterCoeffs& c, float* Mx, float* My, float* a, float* x0,
                              float* x1, float* r, const float* p0, const float* p1, int n_iter, bool reduce_last,
                              double* partials, cudaStream_t st) {
  const size_t smem = resident_smem_bytes(g, MODE, BAL);
  prox_resident_kernel<MODE, BAL><<<g.B, kResidentThreads, smem, st>>>(g, c, Mx, My, a, x0, x1, r, p0, p1, n_iter,
                                                                        reduce_last ? 1 : 0, partials);
  return cudaGetLastError();
}

}  // namespace

int tiled_num_ctas(const Geometry& g) { return g.B * g.tiles_x * g.tiles_y; }

cudaError_t launch_prox_tiled(int mode, bool balanced, bool reduce, const Geometry& g, const IterCoeffs& c,
                              const StatePtrs& s, double* partials, cudaStream_t st) {
#define OTP_TILED(M, BL)                                                                     \
  if (mode == M && balanced == BL)                                                           \
    return reduce ? launch_tiled_t<M, BL, true>(g, c, s, partials, st)                       \
                  : launch_tiled_t<M, BL, false>(g, c, s, partials, st);
  OTP_TILED(0, false)
  OTP_TILED(0, true)
  OTP_TILED(1, false)
  OTP_TILED(1, true)
  OTP_TILED(2, false)
  OTP_TILED(2, true)
#undef OTP_TILED
  return cudaErrorInvalidValue;
}

size_t resident_smem_bytes(const Geometry& g, int mode, bool balanced) {
  const ResidentLayout L = resident_layout(mode, balanced);
  return (size_t)L.nplanes * (size_t)g.H * (size_t)g.Wp * sizeof(float);
}

bool resident_fits(const Geometry& g, int mode, bool balanced) {
  return resident_smem_bytes(g, mode, balanced) <= kResidentSmemCap;
}

cudaError_t launch_prox_resident(int mode, bool balanced, const Geometry& g, const IterCoeffs& c, float* Mx,
                                 float* My, float* a, float* x0, float* x1, float* r, const float* p0,
                                 const float* p1, int n_iter, bool reduce_last, double* partials,
                                 cudaStream_t st) {
#define OTP_RES(M, BL) \
  if (mode == M && balanced == BL) return launch_resident_t<M, BL>(g, c, Mx, My, a, x0, x1, r, p0, p1, n_iter, reduce_last, partials, st);
  OTP_RES(0, false)
  OTP_RES(0, true)
  OTP_RES(1, false)
  OTP_RES(1, true)
  OTP_RES(2, false)
  OTP_RES(2, true)
#undef OTP_RES
  return cudaErrorInvalidValue;
}

cudaError_t prepare_prox_resident(int mode, bool balanced, const Geometry& g) {
#define OTP_PREP(M, BL) \
  if (mode == M && balanced == BL) return prepare_resident_t<M, BL>(g);
  OTP_PREP(0, false)
  OTP_PREP(0, true)
  OTP_PREP(1, false)
  OTP_PREP(1, true)
  OTP_PREP(2, false)
  OTP_PREP(2, true)
#undef OTP_PREP
  return cudaErrorInvalidValue;
}

cudaError_t launch_finalize_sums(const double* partials, int n, double* out, cudaStream_t st) {
  finalize_kernel<kNumSums><<<1, kFinThreads, 0, st>>>(partials, n, 0u, out);
  return cudaGetLastError();
}

int cert_num_blocks(const Geometry& g) {
  const long long total = (long long)g.B * g.H * g.W;
  long long nb = (total + kCertThreads - 1) / kCertThreads;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  return (int)nb;
}

cudaError_t launch_evaluate(const Geometry& g, const CertCoeffs& cc, const float* Mx, const float* My,
                            const float* a, const float* x0, const float* x1, const float* r, const float* p0,
                            const float* p1, double* partials, double* sums_out, double* cert_partials,
                            double* cert_out, cudaStream_t st) {
  const int nb = cert_num_blocks(g);
  eval_pass1_kernel<<<nb, kCertThreads, 0, st>>>(g, cc, Mx, My, a, x0, x1, r, p0, p1, partials, cert_partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<kNumSums><<<1, kFinThreads, 0, st>>>(partials, nb, 0u, sums_out);
  finalize_kernel<kCertQ><<<1, kFinThreads, 0, st>>>(cert_partials, nb, 1u, cert_out);
  eval_pass2_kernel<<<nb, kCertThreads, 0, st>>>(g, cc, Mx, My, a, x0, x1, p0, p1, cert_out, cert_partials);
  finalize_kernel<kCertQ><<<1, kFinThreads, 0, st>>>(cert_partials, nb, 1u, cert_out);
  return cudaGetLastError();
}

}  // namespace otp
