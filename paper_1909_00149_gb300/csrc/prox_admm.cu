// The prox of eq. (Prox_UOT) by ADMM with an exact projection onto the
// constraint set (the "projection form"; the paper itself uses the explicit
// Algorithm 1).  Variables z = (M, free x, r), copies w, scaled duals u:
//   z <- prox_{f/beta}(w - u)                         (admm_z_kernel)
//   k <- K(z + u) - k0                                (admm_rhs_kernel)
//   y <- (D D* + n_id I)^{-1} k                       (DCT-II solve)
//   w <- (z + u) - K^T y,  u <- u + z - w,  a = beta y  (admm_w_kernel)
// with K w = D(M) - x0 + x1 - r (A = [-I, I], Sec. III-B) over the free
// variables and k0 = p0 (x0 frozen) - p1 (x1 frozen).  K K^T = D D* + n_id I,
// the identity of Theorem 1's proof.  a = beta y is the multiplier of
// K z = k0 at the fixed point (K^T a = beta u there).
// Check sums use the slots of the Algorithm 1 kernels: 0 ||K z - k0||^2,
// 1 ||d(z, w, u)||^2, 2 ||(z, w, u)||^2, 3 ||M||_{2,1}, 4 sum|r| (r^2),
// 5 sum (x - p)^2, 6 ||p||^2, 7 non-finite count.
#include <cuda_runtime.h>
#include <math.h>

#include "device_util.cuh"
#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kAdmmThreads = 256;

__device__ __forceinline__ float ld(const float* p, long long o) { return __ldg(p + o); }

// z = prox_{f/beta}(w - u), one float4 group per thread.
__global__ void __launch_bounds__(kAdmmThreads)
admm_z_kernel(const Geometry G, const AdmmCoeffs C, const AdmmPlanes P, int reduce, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per = G.plane / 4;
  const long long total = per * G.B;
  const int W4 = G.Wp / 4;
  for (long long q = blockIdx.x * (long long)kAdmmThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kAdmmThreads) {
    const long long o = 4 * q;
    const long long inb = q % per;
    const int i = (int)(inb / W4), j = (int)(4 * (inb % W4));
    const float4 wmx = ldg4(P.w[0] + o), wmy = ldg4(P.w[1] + o), umx = ldg4(P.u[0] + o), umy = ldg4(P.u[1] + o);
    float4 zmx, zmy, zx0, zx1, zr;
    const float4 p0 = ldg4(P.p0 + o), p1 = ldg4(P.p1 + o);
    float4 wx0 = p0, wx1 = p1, ux0 = make_float4(0.f, 0.f, 0.f, 0.f), ux1 = ux0, wr = ux0, ur = ux0;
    if (C.free0) { wx0 = ldg4(P.w[2] + o); ux0 = ldg4(P.u[2] + o); }
    if (C.free1) { wx1 = ldg4(P.w[3] + o); ux1 = ldg4(P.u[3] + o); }
    if (!C.balanced) { wr = ldg4(P.w[4] + o); ur = ldg4(P.u[4] + o); }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j + e;
      const bool in = jj < G.W;
      const bool ex = in && i < G.H - 1, ey = in && jj < G.W - 1;
      const float vx = ex ? f4c(wmx, e) - f4c(umx, e) : 0.f;
      const float vy = ey ? f4c(wmy, e) - f4c(umy, e) : 0.f;
      float ox, oy;
      if (C.iso) {
        const float n2 = fmaf(vx, vx, vy * vy);
        const float s = (n2 > C.inv_beta * C.inv_beta) ? (1.f - C.inv_beta * rsqrtf(n2)) : 0.f;
        ox = vx * s;
        oy = vy * s;
      } else {
        ox = copysignf(fmaxf(fabsf(vx) - C.inv_beta, 0.f), vx);
        oy = copysignf(fmaxf(fabsf(vy) - C.inv_beta, 0.f), vy);
      }
      f4(zmx, e) = ox;
      f4(zmy, e) = oy;
      float a0 = f4c(p0, e), a1 = f4c(p1, e);
      if (C.free0) a0 = in ? fmaxf((f4c(p0, e) + C.rb * (f4c(wx0, e) - f4c(ux0, e))) * C.inv_1rb, 0.f) : 0.f;
      if (C.free1) a1 = in ? fmaxf((f4c(p1, e) + C.rb * (f4c(wx1, e) - f4c(ux1, e))) * C.inv_1rb, 0.f) : 0.f;
      f4(zx0, e) = a0;
      f4(zx1, e) = a1;
      float rv = 0.f;
      if (!C.balanced && in) {
        const float v = f4c(wr, e) - f4c(ur, e);
        rv = C.pexp == 1 ? copysignf(fmaxf(fabsf(v) - C.mu_over_beta, 0.f), v) : v * C.r2;
      }
      f4(zr, e) = rv;
      if (reduce && in) {
        acc[3] += C.iso ? sqrtf(fmaf(ox, ox, oy * oy)) : fabsf(ox) + fabsf(oy);
        acc[4] += C.pexp == 1 ? fabsf(rv) : rv * rv;
        const float e0 = a0 - f4c(p0, e), e1 = a1 - f4c(p1, e);
        if (C.free0) acc[5] = fmaf(e0, e0, acc[5]);
        if (C.free1) acc[5] = fmaf(e1, e1, acc[5]);
        acc[6] += f4c(p0, e) * f4c(p0, e) + f4c(p1, e) * f4c(p1, e);
        const float4 ozx = ldg4(P.z[0] + o), ozy = ldg4(P.z[1] + o);
        const float d0 = ox - f4c(ozx, e), d1 = oy - f4c(ozy, e);
        float dd = d0 * d0 + d1 * d1, zz = ox * ox + oy * oy;
        if (C.free0) { const float d = a0 - P.z[2][o + e]; dd += d * d; zz += a0 * a0; }
        if (C.free1) { const float d = a1 - P.z[3][o + e]; dd += d * d; zz += a1 * a1; }
        if (!C.balanced) { const float d = rv - P.z[4][o + e]; dd += d * d; zz += rv * rv; }
        acc[1] += dd;
        acc[2] += zz;
        acc[7] += (!isfinite(ox) || !isfinite(oy) || !isfinite(a0) || !isfinite(a1) || !isfinite(rv) ||
                   !isfinite(f4c(p0, e)) || !isfinite(f4c(p1, e))) ? 1.f : 0.f;
      }
    }
    (void)i;
    stg4v(P.z[0] + o, zmx);
    stg4v(P.z[1] + o, zmy);
    if (C.free0) stg4v(P.z[2] + o, zx0);
    if (C.free1) stg4v(P.z[3] + o, zx1);
    if (!C.balanced) stg4v(P.z[4] + o, zr);
  }
  if (reduce) block_sums_to<kAdmmThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// k = K(z + u) - k0; on check iterations also ||K z - k0||^2.
__global__ void __launch_bounds__(kAdmmThreads)
admm_rhs_kernel(const Geometry G, const AdmmCoeffs C, const AdmmPlanes P, int reduce, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per = G.plane / 4;
  const long long total = per * G.B;
  const int W4 = G.Wp / 4, Wp = G.Wp;
  for (long long q = blockIdx.x * (long long)kAdmmThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kAdmmThreads) {
    const long long o = 4 * q;
    const long long inb = q % per;
    const int i = (int)(inb / W4), j = (int)(4 * (inb % W4));
    const float4 zx = ldg4(P.z[0] + o), zy = ldg4(P.z[1] + o), ux = ldg4(P.u[0] + o), uy = ldg4(P.u[1] + o);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 zxu = i > 0 ? ldg4(P.z[0] + o - Wp) : z4, uxu = i > 0 ? ldg4(P.u[0] + o - Wp) : z4;
    const float zyl = j > 0 ? ld(P.z[1], o - 1) : 0.f, uyl = j > 0 ? ld(P.u[1], o - 1) : 0.f;
    const float4 p0 = ldg4(P.p0 + o), p1 = ldg4(P.p1 + o);
    float4 s0 = z4, s1 = z4, sr = z4, t0 = z4, t1 = z4, tr = z4;   // z and u parts of x0, x1, r
    if (C.free0) { s0 = ldg4(P.z[2] + o); t0 = ldg4(P.u[2] + o); }
    if (C.free1) { s1 = ldg4(P.z[3] + o); t1 = ldg4(P.u[3] + o); }
    if (!C.balanced) { sr = ldg4(P.z[4] + o); tr = ldg4(P.u[4] + o); }
    float4 kout;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j + e;
      const bool in = jj < G.W;
      const float vx = f4c(zx, e) + f4c(ux, e), vxu = f4c(zxu, e) + f4c(uxu, e);
      const float vy = f4c(zy, e) + f4c(uy, e);
      const float vyl = e == 0 ? zyl + uyl : f4c(zy, e - 1) + f4c(uy, e - 1);
      const float k0 = (C.free0 ? 0.f : f4c(p0, e)) - (C.free1 ? 0.f : f4c(p1, e));
      float kv = (vx - vxu) + (vy - vyl) - k0;
      if (C.free0) kv -= f4c(s0, e) + f4c(t0, e);
      if (C.free1) kv += f4c(s1, e) + f4c(t1, e);
      if (!C.balanced) kv -= f4c(sr, e) + f4c(tr, e);
      f4(kout, e) = in ? kv : 0.f;
      if (reduce && in) {
        const float zxl = f4c(zx, e), zxup = f4c(zxu, e), zyv = f4c(zy, e);
        const float zyle = e == 0 ? zyl : f4c(zy, e - 1);
        float kz = (zxl - zxup) + (zyv - zyle) - k0;
        if (C.free0) kz -= f4c(s0, e);
        if (C.free1) kz += f4c(s1, e);
        if (!C.balanced) kz -= f4c(sr, e);
        acc[0] = fmaf(kz, kz, acc[0]);
      }
    }
    stg4v(P.k + o, kout);
  }
  if (reduce) block_sums_to<kAdmmThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// w = (z + u) - K^T y, u = u + z - w, a = beta y.
__global__ void __launch_bounds__(kAdmmThreads)
admm_w_kernel(const Geometry G, const AdmmCoeffs C, const AdmmPlanes P, int reduce, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per = G.plane / 4;
  const long long total = per * G.B;
  const int W4 = G.Wp / 4, Wp = G.Wp;
  for (long long q = blockIdx.x * (long long)kAdmmThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kAdmmThreads) {
    const long long o = 4 * q;
    const long long inb = q % per;
    const int i = (int)(inb / W4), j = (int)(4 * (inb % W4));
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 y = ldg4(P.y + o);
    const float4 yd = (i + 1 < G.H) ? ldg4(P.y + o + Wp) : z4;
    const float yr = (j + 4 < Wp) ? ld(P.y, o + 4) : 0.f;
    float4 na;
#pragma unroll
    for (int e = 0; e < 4; ++e) f4(na, e) = (j + e < G.W) ? C.beta * f4c(y, e) : 0.f;
    stg4v(P.a + o, na);
    // M components: (K^T y)_M = D* y
    for (int comp = 0; comp < 2; ++comp) {
      const float4 z = ldg4(P.z[comp] + o), u = ldg4(P.u[comp] + o), wo = ldg4(P.w[comp] + o);
      float4 nw, nu;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = j + e;
        const bool in = jj < G.W;
        float g = 0.f;
        if (comp == 0 && in && i < G.H - 1) g = f4c(y, e) - f4c(yd, e);
        if (comp == 1 && in && jj < G.W - 1) g = f4c(y, e) - (e < 3 ? f4c(y, e + 1) : yr);
        const bool edge = in && (comp == 0 ? i < G.H - 1 : jj < G.W - 1);
        const float v = f4c(z, e) + f4c(u, e);
        const float wv = edge ? v - g : 0.f;
        const float uv = edge ? f4c(u, e) + f4c(z, e) - wv : 0.f;
        f4(nw, e) = wv;
        f4(nu, e) = uv;
        if (reduce && in) {
          const float dw = wv - f4c(wo, e), du = uv - f4c(u, e);
          acc[1] += dw * dw + du * du;
          acc[2] += wv * wv + uv * uv;
        }
      }
      stg4v(P.w[comp] + o, nw);
      stg4v(P.u[comp] + o, nu);
    }
    // x0 (K coefficient -1), x1 (+1), r (-1)
    for (int comp = 2; comp < 5; ++comp) {
      if (comp == 2 && !C.free0) continue;
      if (comp == 3 && !C.free1) continue;
      if (comp == 4 && C.balanced) continue;
      const float sgn = comp == 3 ? 1.f : -1.f;
      const float4 z = ldg4(P.z[comp] + o), u = ldg4(P.u[comp] + o), wo = ldg4(P.w[comp] + o);
      float4 nw, nu;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool in = (j + e) < G.W;
        const float v = f4c(z, e) + f4c(u, e);
        const float wv = in ? v - sgn * f4c(y, e) : 0.f;
        const float uv = in ? f4c(u, e) + f4c(z, e) - wv : 0.f;
        f4(nw, e) = wv;
        f4(nu, e) = uv;
        if (reduce && in) {
          const float dw = wv - f4c(wo, e), du = uv - f4c(u, e);
          acc[1] += dw * dw + du * du;
          acc[2] += wv * wv + uv * uv;
        }
      }
      stg4v(P.w[comp] + o, nw);
      stg4v(P.u[comp] + o, nu);
    }
  }
  if (reduce) block_sums_to<kAdmmThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

}  // namespace

int admm_num_blocks(const Geometry& g) {
  const long long n4 = g.plane / 4 * g.B;
  const long long nb = (n4 + kAdmmThreads - 1) / kAdmmThreads;
  return (int)(nb < 152 * 4 ? (nb < 1 ? 1 : nb) : 152 * 4);
}

cudaError_t admm_launch_z(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce, double* partials,
                          cudaStream_t st) {
  admm_z_kernel<<<admm_num_blocks(g), kAdmmThreads, 0, st>>>(g, c, P, reduce ? 1 : 0, partials);
  return cudaGetLastError();
}

cudaError_t admm_launch_rhs(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce,
                            double* partials, cudaStream_t st) {
  admm_rhs_kernel<<<admm_num_blocks(g), kAdmmThreads, 0, st>>>(g, c, P, reduce ? 1 : 0, partials);
  return cudaGetLastError();
}

cudaError_t admm_launch_w(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce, double* partials,
                          cudaStream_t st) {
  admm_w_kernel<<<admm_num_blocks(g), kAdmmThreads, 0, st>>>(g, c, P, reduce ? 1 : 0, partials);
  return cudaGetLastError();
}

}  // namespace otp
