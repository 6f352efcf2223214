// Elementwise passes of Algorithm 3 (RPCA+UOT-DF ADMM, Sec. IV-B.1) with
// Phi_t = I, fused into two HBM passes over the frame planes [T][H][Wp]
// (pre, post), and between consecutive outer iterations into one (post of
// iteration k with pre of iteration k + 1).
//
// pre  (lines 4-9, and the inputs of lines 10-11):
//   k_t = (x_t - l_t + a_t) + w^z_t (z_t + b_t) + w^w_t (w_t + c_t),
//   sigma_t = 1 + w^z_t + w^w_t,  w^z_t = [t < T-1],  w^w_t = [t > 0]
//   s_t = max(k_t / sigma_t - lambda / (rho sigma_t), 0)
//   L   = 1/2 max(Tm - D + X - S + A, 0)
//   X   = (Y + rho (S + L - A)) / (1 + rho)
//   LD  = L + D                                   (the SVT input, line 10)
//   p0_t = s_t - b_t,  p1_t = s_{t+1} - c_{t+1}   (the prox centres, line 11)
// and keeps z, w of this iteration for the dual residual.
// post (lines 12-15), with Tn the SVT output of this iteration and Tm the
// previous one:
//   A += X - S - L,  D += L - Tn,  b_t += z_t - s_t,  c_{t+1} += w_{t+1} - s_{t+1}
// with the ADMM residual sums.  Readings (see the oracle): the sign of the
// A-update follows the augmented Lagrangian; the x-update keeps rho; S >= 0.
//
// Partial-sum slots (kNumSums per block): 0 ||dX||^2, 1 ||Tn - Tm||^2,
// 2 ||X-S-L||^2, 3 ||L-Tn||^2, 4 ||z-s_t||^2, 5 ||w-s_{t+1}||^2,
// 6 ||dz||^2, 7 ||dw||^2.
#include <cuda_runtime.h>
#include <math.h>

#include "device_util.cuh"
#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kRpcaThreads = 256;

// Lines 4-9 for one pixel of frame t (x, l, a, tm, d, y: frame values; zt, bt:
// pair t's z and b, wt, ct: pair t-1's w and c, zero where the pair does not
// exist).  The explicit fmaf fixes the rounding, so every kernel that calls
// this computes the same bits.
struct PreOut {
  float s, l, x, ld, p0, p1, dx;
};
__device__ __forceinline__ PreOut pre_elem(float x, float l, float a, float tm, float d, float y, float zt, float bt,
                                           float wt, float ct, float inv_sg, float thr, float rho, float inv1r) {
  const float k = (x - l + a) + (zt + bt) + (wt + ct);
  const float s = fmaxf(fmaf(k, inv_sg, -thr), 0.f);
  const float lv = 0.5f * fmaxf(tm - d + x - s + a, 0.f);
  const float xv = fmaf(rho, s + lv - a, y) * inv1r;
  return {s, lv, xv, lv + d, s - bt, s - ct, xv - x};
}

struct PreConst {
  float inv_sg, thr;
};
__device__ __forceinline__ PreConst pre_const(const RpcaGeom& g, const RpcaCoeffs& c, int t) {
  const float sg = 1.f + (t < g.T - 1 ? 1.f : 0.f) + (t > 0 ? 1.f : 0.f);
  return {1.f / sg, c.lam / (c.rho * sg)};
}

__global__ void __launch_bounds__(kRpcaThreads)
rpca_pre_kernel(const RpcaGeom g, const RpcaCoeffs c, const RpcaPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per_frame = g.plane / 4;             // float4 groups per frame
  const long long total = per_frame * g.T;
  const float rho = c.rho, inv1r = 1.f / (1.f + c.rho);
  for (long long q = blockIdx.x * (long long)kRpcaThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kRpcaThreads) {
    const int t = (int)(q / per_frame);
    const long long o = 4 * q;                          // offset in [T][plane]
    const long long op = o - (long long)t * g.plane;   // offset inside the frame
    const bool hz = t < g.T - 1, hw = t > 0;
    const PreConst k = pre_const(g, c, t);
    const float4 x = ldg4(P.X + o), l = ldg4(P.L + o), a = ldg4(P.A + o), tm = ldg4(P.Tm + o), d = ldg4(P.D + o),
                 y = ldg4(P.Y + o);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long oz = (long long)t * g.plane + op;          // pair t
    const long long ow = (long long)(t - 1) * g.plane + op;    // pair t-1
    const float4 zt = hz ? ldg4(P.z + oz) : z4, bt = hz ? ldg4(P.Bz + oz) : z4;
    const float4 wt = hw ? ldg4(P.w + ow) : z4, ct = hw ? ldg4(P.Cw + ow) : z4;
    float4 s4, l4, x4, ld4, p04, p14;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const PreOut r = pre_elem(f4c(x, e), f4c(l, e), f4c(a, e), f4c(tm, e), f4c(d, e), f4c(y, e), f4c(zt, e),
                                f4c(bt, e), f4c(wt, e), f4c(ct, e), k.inv_sg, k.thr, rho, inv1r);
      acc[0] = fmaf(r.dx, r.dx, acc[0]);
      f4(s4, e) = r.s;
      f4(l4, e) = r.l;
      f4(x4, e) = r.x;
      f4(ld4, e) = r.ld;
      f4(p04, e) = r.p0;
      f4(p14, e) = r.p1;
    }
    stg4v(P.S + o, s4);
    stg4v(P.L + o, l4);
    stg4v(P.X + o, x4);
    stg4v(P.LD + o, ld4);
    if (hz) {
      stg4v(P.p0 + oz, p04);
      stg4v(P.zprev + oz, zt);
    }
    if (hw) {
      stg4v(P.p1 + ow, p14);
      stg4v(P.wprev + ow, wt);
    }
  }
  block_sums_to<kRpcaThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// Lines 12-15 for one pixel (a, d, b, cc updated in place); the residual
// terms go to acc when SUMS.
template <bool SUMS>
__device__ __forceinline__ void post_elem(float x, float s, float l, float tn, float tm, float& a, float& d, float z,
                                          float zp, float& b, float w, float wp, float& cc, bool hz, bool hw,
                                          float (&acc)[kNumSums]) {
  const float r1 = x - s - l;
  const float r2 = l - tn;
  a += r1;
  d += r2;
  const float rz = z - s, rw = w - s;
  b += rz;
  cc += rw;
  if (SUMS) {
    const float dt = tn - tm;
    acc[1] = fmaf(dt, dt, acc[1]);
    acc[2] = fmaf(r1, r1, acc[2]);
    acc[3] = fmaf(r2, r2, acc[3]);
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
}

__global__ void __launch_bounds__(kRpcaThreads)
rpca_post_kernel(const RpcaGeom g, const RpcaPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per_frame = g.plane / 4;
  const long long total = per_frame * g.T;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long q = blockIdx.x * (long long)kRpcaThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kRpcaThreads) {
    const int t = (int)(q / per_frame);
    const long long o = 4 * q;
    const long long op = o - (long long)t * g.plane;
    const bool hz = t < g.T - 1, hw = t > 0;
    const long long oz = (long long)t * g.plane + op;         // pair t: z_t pairs with s_t
    const long long ow = (long long)(t - 1) * g.plane + op;   // pair t-1: w_{t} pairs with s_t
    // every load before any store (the planes are not marked restrict)
    const float4 x = ldg4(P.X + o), s = ldg4(P.S + o), l = ldg4(P.L + o), tn = ldg4(P.Tn + o), tm = ldg4(P.Tm + o);
    float4 a = ldg4(P.A + o), d = ldg4(P.D + o);
    const float4 z = hz ? ldg4(P.z + oz) : z4, zp = hz ? ldg4(P.zprev + oz) : z4;
    float4 b = hz ? ldg4(P.Bz + oz) : z4;
    const float4 w = hw ? ldg4(P.w + ow) : z4, wp = hw ? ldg4(P.wprev + ow) : z4;
    float4 cc = hw ? ldg4(P.Cw + ow) : z4;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      post_elem<true>(f4c(x, e), f4c(s, e), f4c(l, e), f4c(tn, e), f4c(tm, e), f4(a, e), f4(d, e), f4c(z, e),
                      f4c(zp, e), f4(b, e), f4c(w, e), f4c(wp, e), f4(cc, e), hz, hw, acc);
    stg4v(P.A + o, a);
    stg4v(P.D + o, d);
    if (hz) stg4v(P.Bz + oz, b);
    if (hw) stg4v(P.Cw + ow, cc);
  }
  block_sums_to<kRpcaThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// Lines 12-15 of outer iteration k fused with lines 4-9 of iteration k + 1
// (one pass instead of two): the SVT output Tn of iteration k is the
// previous output of iteration k + 1, the duals a, d, b, c just updated feed
// its s-, l- and x-updates.  Same per-pixel arithmetic as the two kernels in
// turn (pre_elem, post_elem), so the iterates are bit-identical; only the
// sum of iteration k + 1's lines 4-9 (slot 0) is produced.
__global__ void __launch_bounds__(kRpcaThreads)
rpca_post_pre_kernel(const RpcaGeom g, const RpcaCoeffs c, const RpcaPlanes P, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const long long per_frame = g.plane / 4;
  const long long total = per_frame * g.T;
  const float rho = c.rho, inv1r = 1.f / (1.f + c.rho);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long q = blockIdx.x * (long long)kRpcaThreads + threadIdx.x; q < total;
       q += (long long)gridDim.x * kRpcaThreads) {
    const int t = (int)(q / per_frame);
    const long long o = 4 * q;
    const long long op = o - (long long)t * g.plane;
    const bool hz = t < g.T - 1, hw = t > 0;
    const long long oz = (long long)t * g.plane + op;
    const long long ow = (long long)(t - 1) * g.plane + op;
    const PreConst k = pre_const(g, c, t);
    const float4 x = ldg4(P.X + o), s = ldg4(P.S + o), l = ldg4(P.L + o), tn = ldg4(P.Tn + o), y = ldg4(P.Y + o);
    float4 a = ldg4(P.A + o), d = ldg4(P.D + o);
    const float4 z = hz ? ldg4(P.z + oz) : z4;
    float4 b = hz ? ldg4(P.Bz + oz) : z4;
    const float4 w = hw ? ldg4(P.w + ow) : z4;
    float4 cc = hw ? ldg4(P.Cw + ow) : z4;
    float4 s4, l4, x4, ld4, p04, p14;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      post_elem<false>(f4c(x, e), f4c(s, e), f4c(l, e), f4c(tn, e), 0.f, f4(a, e), f4(d, e), f4c(z, e), 0.f, f4(b, e),
                       f4c(w, e), 0.f, f4(cc, e), hz, hw, acc);
      // a zero pair slot (hz or hw false) keeps b, cc at 0, as in rpca_pre_kernel
      const PreOut r = pre_elem(f4c(x, e), f4c(l, e), f4c(a, e), f4c(tn, e), f4c(d, e), f4c(y, e), f4c(z, e),
                                hz ? f4c(b, e) : 0.f, f4c(w, e), hw ? f4c(cc, e) : 0.f, k.inv_sg, k.thr, rho, inv1r);
      acc[0] = fmaf(r.dx, r.dx, acc[0]);
      f4(s4, e) = r.s;
      f4(l4, e) = r.l;
      f4(x4, e) = r.x;
      f4(ld4, e) = r.ld;
      f4(p04, e) = r.p0;
      f4(p14, e) = r.p1;
    }
    stg4v(P.A + o, a);
    stg4v(P.D + o, d);
    stg4v(P.S + o, s4);
    stg4v(P.L + o, l4);
    stg4v(P.X + o, x4);
    stg4v(P.LD + o, ld4);
    if (hz) {
      stg4v(P.Bz + oz, b);
      stg4v(P.p0 + oz, p04);
      stg4v(P.zprev + oz, z);
    }
    if (hw) {
      stg4v(P.Cw + ow, cc);
      stg4v(P.p1 + ow, p14);
      stg4v(P.wprev + ow, w);
    }
  }
  block_sums_to<kRpcaThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// The fused pass of rpca_post_pre_kernel that also accumulates the SVT Gram
// matrix of the LD = L + D it writes (Alg. 3 line 10 of iteration k + 1):
// a CTA owns chunks of kGC consecutive pixels of a frame plane across all T
// frames, stages their LD values in shared memory, and adds
// LD_chunk^T LD_chunk to a TP x TP FP32 accumulator (a 16 x 16 grid of
// threads, each a TP/16 x TP/16 block); every CTA writes its partial Gram to
// gpart[blockIdx.x], and the FP64 reduction of the partials follows.  Per
// (frame, pixel) the arithmetic is that of rpca_post_pre_kernel.  The slot-0
// rows blockIdx.x + k gridDim.x < nrows of partials are written (zero beyond
// the CTA's own), so the residual finalisation sees nrows rows as before.
constexpr int kGC = 64;             // pixels per Gram chunk
constexpr int kFGThreads = 512;   // one CTA per SM: 152 partial Grams

template <int TP>
__global__ void __launch_bounds__(kFGThreads, 1)
rpca_post_pre_gram_kernel(const RpcaGeom g, const RpcaCoeffs c, const RpcaPlanes P, double* __restrict__ partials,
                          int nrows, float* __restrict__ gpart) {
  // Gram blocks of RB x CB entries on an (TP / RB) x (TP / CB) thread grid
  constexpr int RB = TP >= 64 ? 2 : 1, CB = TP >= 32 ? 4 : 1;
  constexpr int NCB = TP / CB;
  constexpr int LDS = TP + 4;       // padded row of the staged tile (16-byte aligned)
  __shared__ __align__(16) float sLD[kGC][LDS];
  float acc[kNumSums] = {};
  float gacc[RB][CB];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int q = 0; q < CB; ++q) gacc[r][q] = 0.f;
  const int tid = threadIdx.x, bi = tid / NCB, bj = tid % NCB;
  const bool gown = bi < TP / RB;   // the whole grid for TP >= 32; half the threads for TP = 16
  for (int e = tid; e < kGC * LDS; e += kFGThreads) (&sLD[0][0])[e] = 0.f;   // frames T..TP-1 stay zero
  __syncthreads();
  const float rho = c.rho, inv1r = 1.f / (1.f + c.rho);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long nch = (g.plane + kGC - 1) / kGC;
  const int items = g.T * (kGC / 4);
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long p0 = ch * kGC;
#pragma unroll 2
    for (int it = tid; it < items; it += kFGThreads) {
      const int t = it / (kGC / 4), j = it % (kGC / 4);
      const long long op = p0 + 4 * j;            // offset inside the frame (plane is a multiple of 4)
      if (op >= g.plane) {
#pragma unroll
        for (int e = 0; e < 4; ++e) sLD[4 * j + e][t] = 0.f;
        continue;
      }
      const long long o = (long long)t * g.plane + op;
      const bool hz = t < g.T - 1, hw = t > 0;
      const long long oz = (long long)t * g.plane + op;
      const long long ow = (long long)(t - 1) * g.plane + op;
      const PreConst k = pre_const(g, c, t);
      const float4 x = ldg4(P.X + o), s = ldg4(P.S + o), l = ldg4(P.L + o), tn = ldg4(P.Tn + o), y = ldg4(P.Y + o);
      float4 a = ldg4(P.A + o), d = ldg4(P.D + o);
      const float4 z = hz ? ldg4(P.z + oz) : z4;
      float4 b = hz ? ldg4(P.Bz + oz) : z4;
      const float4 w = hw ? ldg4(P.w + ow) : z4;
      float4 cc = hw ? ldg4(P.Cw + ow) : z4;
      float4 s4, l4, x4, ld4, p04, p14;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        post_elem<false>(f4c(x, e), f4c(s, e), f4c(l, e), f4c(tn, e), 0.f, f4(a, e), f4(d, e), f4c(z, e), 0.f,
                         f4(b, e), f4c(w, e), 0.f, f4(cc, e), hz, hw, acc);
        const PreOut r = pre_elem(f4c(x, e), f4c(l, e), f4c(a, e), f4c(tn, e), f4c(d, e), f4c(y, e), f4c(z, e),
                                  hz ? f4c(b, e) : 0.f, f4c(w, e), hw ? f4c(cc, e) : 0.f, k.inv_sg, k.thr, rho, inv1r);
        acc[0] = fmaf(r.dx, r.dx, acc[0]);
        f4(s4, e) = r.s;
        f4(l4, e) = r.l;
        f4(x4, e) = r.x;
        f4(ld4, e) = r.ld;
        f4(p04, e) = r.p0;
        f4(p14, e) = r.p1;
        sLD[4 * j + e][t] = r.ld;
      }
      stg4v(P.A + o, a);
      stg4v(P.D + o, d);
      stg4v(P.S + o, s4);
      stg4v(P.L + o, l4);
      stg4v(P.X + o, x4);
      stg4v(P.LD + o, ld4);
      if (hz) {
        stg4v(P.Bz + oz, b);
        stg4v(P.p0 + oz, p04);
        stg4v(P.zprev + oz, z);
      }
      if (hw) {
        stg4v(P.Cw + ow, cc);
        stg4v(P.p1 + ow, p14);
        stg4v(P.wprev + ow, w);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int p = 0; p < kGC; ++p) {
      float av[RB], bv[CB];
#pragma unroll
      for (int r = 0; r < RB; ++r) av[r] = sLD[p][gown ? RB * bi + r : 0];
#pragma unroll
      for (int q = 0; q < CB; ++q) bv[q] = sLD[p][CB * bj + q];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int q = 0; q < CB; ++q) gacc[r][q] = fmaf(av[r], bv[q], gacc[r][q]);
    }
    __syncthreads();
  }
  float* out = gpart + (size_t)blockIdx.x * TP * TP;
  if (gown) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int q = 0; q < CB; ++q) out[(RB * bi + r) * TP + CB * bj + q] = gacc[r][q];
  }
  block_sums_to<kFGThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
  for (int row = blockIdx.x + gridDim.x; row < nrows; row += gridDim.x)
    if (tid < kNumSums) partials[(size_t)row * kNumSums + tid] = 0.0;
}

// ||Y||^2 (once per input) into partials[block][0].
__global__ void __launch_bounds__(kRpcaThreads)
sumsq_kernel(const float* __restrict__ Y, long long n4, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  for (long long q = blockIdx.x * (long long)kRpcaThreads + threadIdx.x; q < n4; q += (long long)gridDim.x * kRpcaThreads) {
    const float4 v = ldg4(Y + 4 * q);
    acc[0] += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  block_sums_to<kRpcaThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

}  // namespace

int rpca_num_blocks(const RpcaGeom& g) {
  const long long n4 = g.plane / 4 * g.T;
  const long long nb = (n4 + kRpcaThreads - 1) / kRpcaThreads;
  return (int)(nb < 152 * 4 ? (nb < 1 ? 1 : nb) : 152 * 4);
}

cudaError_t rpca_launch_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                            cudaStream_t st) {
  rpca_pre_kernel<<<rpca_num_blocks(g), kRpcaThreads, 0, st>>>(g, c, P, partials);
  return cudaGetLastError();
}

cudaError_t rpca_launch_post(const RpcaGeom& g, const RpcaPlanes& P, double* partials, cudaStream_t st) {
  rpca_post_kernel<<<rpca_num_blocks(g), kRpcaThreads, 0, st>>>(g, P, partials);
  return cudaGetLastError();
}

cudaError_t rpca_launch_post_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                                 cudaStream_t st) {
  rpca_post_pre_kernel<<<rpca_num_blocks(g), kRpcaThreads, 0, st>>>(g, c, P, partials);
  return cudaGetLastError();
}

// CTAs of the Gram-fused pass = its partial Grams: at most one per SM, one
// per chunk, and no more than the residual rows it writes (rpca_num_blocks).
int rpca_gram_parts(const RpcaGeom& g) {
  long long n = (g.plane + kGC - 1) / kGC;
  if (n > 152) n = 152;
  const int nr = rpca_num_blocks(g);
  if (n > nr) n = nr;
  return (int)(n < 1 ? 1 : n);
}

cudaError_t rpca_launch_post_pre_gram(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, int TP,
                                      double* partials, int nrows, float* gpart, cudaStream_t st) {
  const int grid = rpca_gram_parts(g);
  switch (TP) {
    case 16: rpca_post_pre_gram_kernel<16><<<grid, kFGThreads, 0, st>>>(g, c, P, partials, nrows, gpart); break;
    case 32: rpca_post_pre_gram_kernel<32><<<grid, kFGThreads, 0, st>>>(g, c, P, partials, nrows, gpart); break;
    case 64: rpca_post_pre_gram_kernel<64><<<grid, kFGThreads, 0, st>>>(g, c, P, partials, nrows, gpart); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t rpca_launch_sumsq(const RpcaGeom& g, const float* Y, double* partials, cudaStream_t st) {
  sumsq_kernel<<<rpca_num_blocks(g), kRpcaThreads, 0, st>>>(Y, g.plane / 4 * g.T, partials);
  return cudaGetLastError();
}

}  // namespace otp
