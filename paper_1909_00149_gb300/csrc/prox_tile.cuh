// The fused Algorithm 1 iteration (Sec. III-B, lines 3-7) on one tile: shared
// by the one-problem tiled kernel (prox_kernels.cu) and the multi-sequence
// batched kernel (prox_batch.cu).
//
// A CTA of 32 x 8 threads owns TH rows x kTW (128) columns of one problem,
// each thread a float4 column group on TH / 8 rows.  It reads the state of
// its tile once, computes
//   M'  = shrink_{tau1}(M - tau1 D*(a))              (line 3, eq. Prox_UOT_M_prox)
//   x'  = Pi_+((tau1 p + rho x -/+ rho tau1 a) / (rho + tau1))   (line 4)
//   r'  = shrink^{l1}_{mu tau1}(r + tau1 a)          (line 5)
//   a'  = a + tau2 (2 K(z') - K(z))                  (lines 6-7)
// and writes the new state once.  K is linear, so 2K(z') - K(z) = K(2z' - z):
// Mbar = 2M' - M is formed in shared memory and D applied to it once.  D(Mbar)
// at a pixel needs Mbar one row up and one column left, so M' is recomputed
// on a one-sided halo (top row, left column) from a's tile with a one-pixel
// ring.  Zero flux (Sec. III-A): Mx[H-1,:] = My[:,W-1] = 0.  The per-pixel
// arithmetic does not depend on TH.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "otprox_internal.cuh"

namespace otp {
namespace tile {

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& comp(float4& v, int e) { return (&v.x)[e]; }
__device__ __forceinline__ float compc(const float4& v, int e) { return (&v.x)[e]; }

// Line 3 for one pixel: q = m - tau1 D*(a); vector (or componentwise) soft
// shrinkage with threshold tau1.  ex / ey: the x / y edge exists here.
__device__ __forceinline__ void flux_step(float mx, float my, float a_c, float a_down, float a_right,
                                          bool ex, bool ey, const IterCoeffs& c, float& ox, float& oy) {
  const float qx = ex ? fmaf(-c.tau1, a_c - a_down, mx) : 0.f;
  const float qy = ey ? fmaf(-c.tau1, a_c - a_right, my) : 0.f;
  if (c.iso) {
    const float n2 = fmaf(qx, qx, qy * qy);
    const float s = (n2 > c.tau1 * c.tau1) ? (1.f - c.tau1 * rsqrtf(n2)) : 0.f;
    ox = qx * s;
    oy = qy * s;
  } else {
    ox = copysignf(fmaxf(fabsf(qx) - c.tau1, 0.f), qx);
    oy = copysignf(fmaxf(fabsf(qy) - c.tau1, 0.f), qy);
  }
}

__device__ __forceinline__ float r_step(float r, float a, const IterCoeffs& c) {
  const float q = fmaf(c.tau1, a, r);
  if (c.pexp == 1) return copysignf(fmaxf(fabsf(q) - c.mu_tau1, 0.f), q);
  return q * c.r2;
}

// Line 4 for one pixel, each marginal: x' = Pi_+((tau1 p + rho x +/- rho tau1 a) / (rho + tau1)),
// + for x0 (A = [-I, I] puts -x0 in K) and - for x1.
__device__ __forceinline__ float x0_step(float p, float x, float a, const IterCoeffs& c) {
  return fmaxf(fmaf(c.cp, p, fmaf(c.cx, x, c.ca * a)), 0.f);
}
__device__ __forceinline__ float x1_step(float p, float x, float a, const IterCoeffs& c) {
  return fmaxf(fmaf(c.cp, p, fmaf(c.cx, x, -c.ca * a)), 0.f);
}

// Lines 6-7 for one pixel: a' = a + tau2 K(2z' - z), with dmb = D(Mbar) at
// the pixel and K(z) = D(M) - x0 + x1 - r.
template <bool BAL>
__device__ __forceinline__ float dual_step(float dmb, float vx0, float x0, float vx1, float x1, float vr, float r,
                                           float a, const IterCoeffs& c) {
  float bk = dmb - (2.f * vx0 - x0) + (2.f * vx1 - x1);
  if (!BAL) bk -= 2.f * vr - r;
  return fmaf(c.tau2, bk, a);
}

__device__ __forceinline__ float norm_term(float mx, float my, int iso) {
  return iso ? sqrtf(fmaf(mx, mx, my * my)) : fabsf(mx) + fabsf(my);
}

__device__ __forceinline__ bool nonfinite(float v) { return !isfinite(v); }

// One pixel's terms of the stopping-check sums (kNumSums) after an
// iteration: new flux (nmx, nmy) with its up / left neighbours' new flux,
// the old flux (mx, my), new and old x0, x1, r, a, and the inputs p0, p1.
template <int MODE, bool BAL>
__device__ __forceinline__ void check_terms(float nmxe, float nmye, float nmx_up, float nmy_l, float mx, float my,
                                            float vx0, float x0, float vx1, float x1, float vr, float r, float va,
                                            float a, float p0, float p1, const IterCoeffs& C,
                                            float (&acc)[kNumSums]) {
  const float kz = (nmxe - nmx_up) + (nmye - nmy_l) - vx0 + vx1 - (BAL ? 0.f : vr);
  acc[0] = fmaf(kz, kz, acc[0]);
  const float d0 = nmxe - mx, d1 = nmye - my;
  const float d2 = vx0 - x0, d3 = vx1 - x1;
  const float d4 = vr - r, d5 = va - a;
  acc[1] += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5;
  acc[2] += nmxe * nmxe + nmye * nmye + vx0 * vx0 + vx1 * vx1 + vr * vr + va * va;
  acc[3] += norm_term(nmxe, nmye, C.iso);
  acc[4] += C.pexp == 1 ? fabsf(vr) : vr * vr;
  const float e0 = vx0 - p0, e1 = vx1 - p1;
  if (MODE == 0) acc[5] = fmaf(e0, e0, acc[5]);
  if (MODE != 2) acc[5] = fmaf(e1, e1, acc[5]);
  acc[6] += p0 * p0 + p1 * p1;
  acc[7] += (nonfinite(va) || nonfinite(nmxe) || nonfinite(nmye) || nonfinite(vx0) || nonfinite(vx1) ||
             nonfinite(vr) || nonfinite(p0) || nonfinite(p1)) ? 1.f : 0.f;
}

// Sum kNumSums values over the block in FP64; thread 0 writes them to out.
// Each thread's own partial sums (a handful of pixels) are FP32: FP64
// arithmetic is scarce on this GPU, so it is used only across threads.
template <int NT>
__device__ void block_sum_store(float (&v)[kNumSums], double* out) {
  constexpr int NW = NT / 32;
  __shared__ double red[NW][kNumSums];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  // within a warp in FP32 (32 partials), across warps and blocks in FP64
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) red[warp][k] = (double)v[k];
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

template <int MODE, bool BAL, bool RED, int TH>
__device__ __forceinline__ void prox_tile(const Geometry& G, const IterCoeffs& C, const StatePtrs& S, int tile,
                                          double* partial_out) {
  constexpr int A4 = kTW / 4 + 2;
  constexpr int RPT = TH / kTY;                 // a tile: columns j0-4 .. j0+kTW+3
  __shared__ __align__(16) float4 s_a[TH + 2][A4];
  __shared__ __align__(16) float s_mbx[TH + 1][kTW];       // rows i0-1 .. i0+TH-1
  __shared__ __align__(16) float s_mby[TH][kTW + 4];       // cols j0-4 .. j0+kTW-1
  __shared__ __align__(16) float s_mnx[RED ? TH + 1 : 1][RED ? kTW : 4];
  __shared__ __align__(16) float s_mny[RED ? TH : 1][RED ? kTW + 4 : 4];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  int t = tile;
  const int bx = t % G.tiles_x;
  t /= G.tiles_x;
  const int by = t % G.tiles_y;
  const int b = t / G.tiles_y;
  const int i0 = by * TH, j0 = bx * kTW;
  const int H = G.H, W = G.W, Wp = G.Wp;
  const long long base = (long long)b * G.plane;

  // ---- stage a^k on the tile plus a one-pixel ring (float4-aligned: 4 extra columns each side)
  for (int idx = tid; idx < (TH + 2) * A4; idx += kTiledThreads) {
    const int rr = idx / A4, c4 = idx - rr * A4;
    const int gi = i0 - 1 + rr, gj = j0 - 4 + 4 * c4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gi >= 0 && gi < H && gj >= 0 && gj < Wp) v = ld4(S.a_in + base + (long long)gi * Wp + gj);
    s_a[rr][c4] = v;
  }

  // ---- own state
  const int j = j0 + 4 * tx;
  const bool colok = j < Wp;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 mx[RPT], my[RPT], x0[RPT], x1[RPT], rv[RPT], p0[RPT], p1[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int i = i0 + ty + kTY * q;
    const bool ok = colok && i < H;
    const long long off = base + (long long)i * Wp + j;
    mx[q] = ok ? ld4(S.Mx_in + off) : z4;
    my[q] = ok ? ld4(S.My_in + off) : z4;
    p0[q] = ok ? ld4(S.p0 + off) : z4;
    p1[q] = ok ? ld4(S.p1 + off) : z4;
    x0[q] = (ok && MODE == 0) ? ld4(S.x0 + off) : p0[q];
    x1[q] = (ok && MODE != 2) ? ld4(S.x1 + off) : p1[q];
    rv[q] = (ok && !BAL) ? ld4(S.r + off) : z4;
  }
  // ---- halo flux M^k: row i0-1 (threads ty == 0), column j0-1 (threads tx == 0)
  float4 hmx = z4, hmy = z4;
  if (ty == 0 && i0 >= 1 && colok) {
    const long long off = base + (long long)(i0 - 1) * Wp + j;
    hmx = ld4(S.Mx_in + off);
    hmy = ld4(S.My_in + off);
  }
  float lmx[RPT], lmy[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int i = i0 + ty + kTY * q;
    lmx[q] = lmy[q] = 0.f;
    if (tx == 0 && j0 >= 1 && i < H) {
      const long long off = base + (long long)i * Wp + (j0 - 1);
      lmx[q] = __ldg(S.Mx_in + off);
      lmy[q] = __ldg(S.My_in + off);
    }
  }
  __syncthreads();

  // ---- line 3 on own pixels
  float4 nmx[RPT], nmy[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int rr = ty + kTY * q + 1;
    const int i = i0 + rr - 1;
    const float4 ac = s_a[rr][tx + 1];
    const float an = s_a[rr][tx + 2].x;
    const float4 ad = s_a[rr + 1][tx + 1];
    float4 bx4, by4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j + e;
      const bool in = (i < H) && (jj < W);
      const float a_r = e < 3 ? compc(ac, e + 1) : an;
      float ox, oy;
      flux_step(compc(mx[q], e), compc(my[q], e), compc(ac, e), compc(ad, e), a_r,
                in && i < H - 1, in && jj < W - 1, C, ox, oy);
      comp(nmx[q], e) = ox;
      comp(nmy[q], e) = oy;
      comp(bx4, e) = 2.f * ox - compc(mx[q], e);
      comp(by4, e) = 2.f * oy - compc(my[q], e);
    }
    *reinterpret_cast<float4*>(&s_mbx[rr][4 * tx]) = bx4;
    *reinterpret_cast<float4*>(&s_mby[rr - 1][4 * tx + 4]) = by4;
    if (RED) {
      *reinterpret_cast<float4*>(&s_mnx[rr][4 * tx]) = nmx[q];
      *reinterpret_cast<float4*>(&s_mny[rr - 1][4 * tx + 4]) = nmy[q];
    }
  }
  // ---- halo row i0-1: only Mbar_x is consumed, both components enter the shrink
  if (ty == 0) {
    float4 bx4 = z4, nx4 = z4;
    if (i0 >= 1) {
      const int i = i0 - 1;
      const float4 ac = s_a[0][tx + 1];
      const float an = s_a[0][tx + 2].x;
      const float4 ad = s_a[1][tx + 1];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = j + e;
        const bool in = jj < W;
        const float a_r = e < 3 ? compc(ac, e + 1) : an;
        float ox, oy;
        flux_step(compc(hmx, e), compc(hmy, e), compc(ac, e), compc(ad, e), a_r, in && i < H - 1,
                  in && jj < W - 1, C, ox, oy);
        comp(bx4, e) = 2.f * ox - compc(hmx, e);
        comp(nx4, e) = ox;
      }
    }
    *reinterpret_cast<float4*>(&s_mbx[0][4 * tx]) = bx4;
    if (RED) *reinterpret_cast<float4*>(&s_mnx[0][4 * tx]) = nx4;
  }
  // ---- halo column j0-1: only Mbar_y is consumed
  if (tx == 0) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int rr = ty + kTY * q + 1;
      const int i = i0 + rr - 1;
      float by = 0.f, ny = 0.f;
      if (j0 >= 1 && i < H) {
        const float a_c = s_a[rr][0].w, a_r = s_a[rr][1].x, a_d = s_a[rr + 1][0].w;
        float ox, oy;
        flux_step(lmx[q], lmy[q], a_c, a_d, a_r, i < H - 1, true, C, ox, oy);
        by = 2.f * oy - lmy[q];
        ny = oy;
      }
      s_mby[rr - 1][3] = by;
      if (RED) s_mny[rr - 1][3] = ny;
    }
  }
  __syncthreads();

  // ---- lines 4-7 on own pixels
  float acc[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) acc[k] = 0.f;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int rr = ty + kTY * q + 1;
    const int i = i0 + rr - 1;
    if (!(colok && i < H)) continue;
    const float4 a4 = s_a[rr][tx + 1];
    const float4 mbx = *reinterpret_cast<const float4*>(&s_mbx[rr][4 * tx]);
    const float4 mbx_up = *reinterpret_cast<const float4*>(&s_mbx[rr - 1][4 * tx]);
    const float4 mby = *reinterpret_cast<const float4*>(&s_mby[rr - 1][4 * tx + 4]);
    const float mby_l = s_mby[rr - 1][4 * tx + 3];
    float4 nx0, nx1, nr, na;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j + e;
      const bool in = jj < W;
      const float a = compc(a4, e);
      float vx0 = compc(p0[q], e), vx1 = compc(p1[q], e);
      if (MODE == 0) vx0 = x0_step(compc(p0[q], e), compc(x0[q], e), a, C);
      if (MODE != 2) vx1 = x1_step(compc(p1[q], e), compc(x1[q], e), a, C);
      const float vr = BAL ? 0.f : r_step(compc(rv[q], e), a, C);
      const float dmb = (compc(mbx, e) - compc(mbx_up, e)) +
                        (compc(mby, e) - (e == 0 ? mby_l : compc(mby, e - 1)));
      const float va = dual_step<BAL>(dmb, vx0, compc(x0[q], e), vx1, compc(x1[q], e), vr, compc(rv[q], e), a, C);
      comp(nx0, e) = in ? vx0 : 0.f;
      comp(nx1, e) = in ? vx1 : 0.f;
      comp(nr, e) = in ? vr : 0.f;
      comp(na, e) = in ? va : 0.f;
      if (RED && in)
        check_terms<MODE, BAL>(compc(nmx[q], e), compc(nmy[q], e), s_mnx[rr - 1][4 * tx + e],
                               s_mny[rr - 1][4 * tx + 3 + e], compc(mx[q], e), compc(my[q], e), vx0,
                               compc(x0[q], e), vx1, compc(x1[q], e), vr, compc(rv[q], e), va, a, compc(p0[q], e),
                               compc(p1[q], e), C, acc);
    }
    const long long off = base + (long long)i * Wp + j;
    st4(S.Mx_out + off, nmx[q]);
    st4(S.My_out + off, nmy[q]);
    st4(S.a_out + off, na);
    if (MODE == 0) st4(S.x0 + off, nx0);
    if (MODE != 2) st4(S.x1 + off, nx1);
    if (!BAL) st4(S.r + off, nr);
  }
  if (RED) block_sum_store<kTiledThreads>(acc, partial_out);
}

}  // namespace tile
}  // namespace otp
