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

// The pass between outer iterations k and k + 1 for T_pad <= 64: the SVT
// apply of iteration k (Alg. 3 line 10, T^k = LD^k Wm), its lines 12-15,
// lines 4-9 of iteration k + 1 and the Gram matrix of the LD^{k+1} they
// write (line 10 of k + 1), in one cooperative launch.  A CTA owns chunks of
// kGC consecutive pixels of a frame plane across all T frames, taken in the
// order blockIdx.x, blockIdx.x + gridDim.x, ...  Its warps are split by role
// so that the contractions overlap the memory traffic:
//   * kFGGram warps (the contraction warps) copy chunk j + 2 of LD^k into
//     shared memory (cp.async) while they form T^k of chunk j = Wm applied
//     to its LD^k columns (FP32 FMAs, s in order) into a shared tile, then
//     add LD^{k+1}_chunk^T LD^{k+1}_chunk of chunk j - 1 to a TP x TP FP32
//     accumulator held in registers (RB x CB entries a thread), pixel by
//     pixel in chunk order;
//   * kFGUpd updating warps run the per-(frame, pixel) arithmetic of
//     rpca_post_pre_kernel on chunk j with T^k from the shared tile and
//     leave its LD^{k+1} values in another shared tile (LD is updated in
//     place: a chunk's LD^k is copied before its LD^{k+1} is stored).
// Double-buffered tiles, handed over through mbarriers (every producing
// thread arrives, every consuming thread waits for the phase of the tile's
// use; every thread of a role runs the same number of chunks).  With
// store_tn the updating warps also store T^k (needed only before the last
// outer iteration of a call, whose lines 12-15 form ||T^{k+1} - T^k||),
// and the z, w it read (that iteration's dual residual ||z^{k+1} - z^k||).
// Every CTA writes its partial Gram to gpart[blockIdx.x]; the CTAs then meet
// at a grid barrier (all resident: the launch is cooperative) and each sums
// its slice of the TP x TP entries over the partials, in partial order and
// FP64, into G.  The slot-0 rows blockIdx.x + k gridDim.x < nrows of
// partials are written (zero beyond the CTA's own), so the residual
// finalisation sees nrows rows as before.
constexpr int kGC = 64;                          // pixels per chunk
constexpr int kFGUpd = 512;                      // updating threads (16 warps)
constexpr int kFGGram = 128;                     // contraction threads (4 warps)
constexpr int kFGThreads = kFGUpd + kFGGram;     // one CTA per SM: 152 partial Grams
// named barriers (0 is __syncthreads): tile b of T^k full / free, tile b of
// LD^{k+1} full / free, and one among the contraction warps alone
constexpr int kBarMma = 9;   // named barrier among the contraction warps alone
// mbarriers of the tile hand-over, two tiles each: T^k full (arrivals: the
// kFGGram contraction threads), T^k free and LD^{k+1} full (the kFGUpd
// updating threads), LD^{k+1} free (the contraction threads)
enum { kMbTnFull = 0, kMbTnFree = 2, kMbLdFull = 4, kMbLdFree = 6, kMbCount = 8 };

template <int TP>
constexpr size_t between_smem() {   // Wm^T, 2 x LD^k chunk, 2 x T^k chunk, 2 x LD^{k+1} chunk
  return sizeof(float) * ((size_t)TP * (TP + 4) + 4 * (size_t)TP * (kGC + 4) + 2 * (size_t)kGC * TP);
}

// Column of frame t in pixel row p of an LD^{k+1} tile (rows of TP floats):
// groups of 4 frames are permuted by an XOR with p / 4, so that the
// updating warps' stores (lanes on pixels 4 apart) spread over the banks
// while every 4-frame group stays contiguous for the Gram's vector reads.
template <int TP>
__device__ __forceinline__ int ld_col(int p, int t) {
  constexpr int mask = (TP / 4 < 8 ? TP / 4 : 8) - 1;
  return 4 * ((t >> 2) ^ ((p >> 2) & mask)) + (t & 3);
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Tile hand-over between the warp roles by mbarriers: a producing thread
// arrives (release) once its part of a tile is written or read, a consuming
// thread waits (acquire) for the phase of the tile's use.  Unlike a named
// barrier, a waiting warp is held only by the producers, not by the other
// consumers.  Waits are bounded; on expiry the error flag is set and the
// thread goes on (the host reports OT_ETIMEOUT).
__device__ __forceinline__ void mb_init(uint64_t* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(n)
               : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((unsigned)__cvta_generic_to_shared(b)) : "memory");
}
__device__ __forceinline__ void mb_wait(uint64_t* b, unsigned parity, int* err) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(b);
  for (unsigned it = 0; it < (1u << 22); ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return;
  }
  atomicExch(err, 1);
}

constexpr unsigned kBarSpin = 1u << 20;         // polls (about 1 s) before the grid barrier gives up

// Grid barrier over the gridDim.x resident CTAs of one launch: bar[0] counts
// arrivals, bar[1] is a generation number that the last arriver advances
// (after resetting the count, so the next launch starts from zero).  The
// wait is bounded: on expiry *err is set and false returned.
__device__ bool grid_barrier(unsigned* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      for (unsigned it = 0; *gen == g0; ++it) {
        if (it >= kBarSpin) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// CTA b's slice [b E / nb, (b + 1) E / nb) of G = sum of the nb = gridDim.x
// FP32 partials gpart[q][E] (E = TP^2): warp w sums partials w, w + NW, ...
// in FP64, then warp 0 adds the NW warp sums in warp order.  Partials are
// read through L2 (written by other CTAs of this launch).
template <int TP>
__device__ void gram_slice_reduce(const float* gpart, double* G) {
  constexpr int E = TP * TP, NW = kFGThreads / 32, U = 8;
  __shared__ double s[NW][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nparts = gridDim.x;
  const int e0 = (int)((long long)blockIdx.x * E / nparts), e1 = (int)((long long)(blockIdx.x + 1) * E / nparts);
  for (int eb = e0; eb < e1; eb += 32) {
    const int e = eb + lane;
    double v = 0.0;
    if (e < e1) {
      for (int qb = warp; qb < nparts; qb += U * NW) {
        float x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = qb + u * NW;
          x[u] = q < nparts ? __ldcg(gpart + (size_t)q * E + e) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (qb + u * NW < nparts) v += (double)x[u];
      }
    }
    s[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && e < e1) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += s[w][lane];
      G[e] = t;
    }
    __syncthreads();
  }
}

// The grid barrier alone (for the diagnostic entry point).
__global__ void __launch_bounds__(32) grid_barrier_probe_kernel(unsigned* bar, int* err) { grid_barrier(bar, err); }

// n consecutive floats of a 16-byte aligned shared-memory row into v.
template <int n>
__device__ __forceinline__ void lds_row(const float* p, float (&v)[n]) {
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int k = 0; k < n / 4; ++k) {
      const float4 t = reinterpret_cast<const float4*>(p)[k];
      v[4 * k] = t.x;
      v[4 * k + 1] = t.y;
      v[4 * k + 2] = t.z;
      v[4 * k + 3] = t.w;
    }
  } else if constexpr (n == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) v[k] = p[k];
  }
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros
// (the source address must still be valid).
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int TP>
__global__ void __launch_bounds__(kFGThreads, 1)
rpca_apply_post_pre_gram_kernel(const RpcaGeom g, const RpcaCoeffs c, const RpcaPlanes P,
                                const float* __restrict__ Wm, int store_tn, double* __restrict__ partials, int nrows,
                                float* __restrict__ gpart, double* __restrict__ G, unsigned* __restrict__ bar,
                                int* __restrict__ err) {
  constexpr int CB = TP / 8, RB = TP / 16;   // Gram block of a contraction thread (16 x 8 grid)
  constexpr int AT = TP / 8;                 // apply block: 4 pixels x AT frames (16 x 8 grid)
  constexpr int AH = AT < 4 ? AT : 4;
  static_assert(16 * 8 == kFGGram && RB >= 1 && 16 * 4 == kGC, "contraction thread grid");
  constexpr int LDS = TP + 4, LDP = kGC + 4;   // padded rows (16-byte aligned)
  extern __shared__ __align__(16) float smf[];
  float* sW = smf;                       // [TP][LDS]: sW[s][t] = Wm[t][s]
  float* sIn = sW + TP * LDS;            // [2][TP][LDP]: LD^k of a chunk, frame rows
  float* sTn = sIn + 2 * TP * LDP;       // [2][TP][LDP]: T^k of a chunk, frame rows
  float* sLD = sTn + 2 * TP * LDP;       // [2][kGC][TP]: LD^{k+1} of a chunk, pixel rows (ld_col)
  __shared__ __align__(8) uint64_t mb[kMbCount];
  float acc[kNumSums] = {};
  const int tid = threadIdx.x;
  const int nsm = (int)(between_smem<TP>() / sizeof(float));
  for (int e = tid; e < nsm; e += kFGThreads) smf[e] = 0.f;   // frames T..TP-1 stay zero
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      mb_init(&mb[kMbTnFull + q], kFGGram);
      mb_init(&mb[kMbTnFree + q], kFGUpd);
      mb_init(&mb[kMbLdFull + q], kFGUpd);
      mb_init(&mb[kMbLdFree + q], kFGGram);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long nch = (g.plane + kGC - 1) / kGC;
  const int nk = blockIdx.x < nch ? (int)((nch - 1 - blockIdx.x) / gridDim.x + 1) : 0;   // chunks of this CTA
  for (int e = tid; e < g.T * g.T; e += kFGThreads) sW[(e % g.T) * LDS + e / g.T] = Wm[(e / g.T) * TP + e % g.T];
  __syncthreads();
  if (tid < kFGUpd) {
    const float rho = c.rho, inv1r = 1.f / (1.f + c.rho);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int items = g.T * (kGC / 4);
    for (int k = 0; k < nk; ++k) {
      const int b = k & 1;
      mb_wait(&mb[kMbTnFull + b], (k >> 1) & 1, err);
      if (k >= 2) mb_wait(&mb[kMbLdFree + b], ((k >> 1) - 1) & 1, err);
      const long long p0 = (blockIdx.x + (long long)k * gridDim.x) * kGC;
      const float* tnb = sTn + b * TP * LDP;
      float* ldb = sLD + b * kGC * TP;
#pragma unroll 2
      for (int it = tid; it < items; it += kFGUpd) {
        const int t = it / (kGC / 4), j = it % (kGC / 4);
        const long long op = p0 + 4 * j;            // offset inside the frame (plane is a multiple of 4)
        if (op >= g.plane) {
#pragma unroll
          for (int e = 0; e < 4; ++e) ldb[(4 * j + e) * TP + ld_col<TP>(4 * j + e, t)] = 0.f;
          continue;
        }
        const long long o = (long long)t * g.plane + op;
        const bool hz = t < g.T - 1, hw = t > 0;
        const long long oz = (long long)t * g.plane + op;
        const long long ow = (long long)(t - 1) * g.plane + op;
        const PreConst kc = pre_const(g, c, t);
        const float4 tn = *reinterpret_cast<const float4*>(tnb + t * LDP + 4 * j);
        const float4 x = ldg4(P.X + o), s = ldg4(P.S + o), l = ldg4(P.L + o), y = ldg4(P.Y + o);
        float4 a = ldg4(P.A + o), d = ldg4(P.D + o);
        const float4 z = hz ? ldg4(P.z + oz) : z4;
        float4 bz = hz ? ldg4(P.Bz + oz) : z4;
        const float4 w = hw ? ldg4(P.w + ow) : z4;
        float4 cc = hw ? ldg4(P.Cw + ow) : z4;
        float4 s4, l4, x4, ld4, p04, p14;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          post_elem<false>(f4c(x, e), f4c(s, e), f4c(l, e), f4c(tn, e), 0.f, f4(a, e), f4(d, e), f4c(z, e), 0.f,
                           f4(bz, e), f4c(w, e), 0.f, f4(cc, e), hz, hw, acc);
          const PreOut r = pre_elem(f4c(x, e), f4c(l, e), f4c(a, e), f4c(tn, e), f4c(d, e), f4c(y, e), f4c(z, e),
                                    hz ? f4c(bz, e) : 0.f, f4c(w, e), hw ? f4c(cc, e) : 0.f, kc.inv_sg, kc.thr, rho,
                                    inv1r);
          acc[0] = fmaf(r.dx, r.dx, acc[0]);
          f4(s4, e) = r.s;
          f4(l4, e) = r.l;
          f4(x4, e) = r.x;
          f4(ld4, e) = r.ld;
          f4(p04, e) = r.p0;
          f4(p14, e) = r.p1;
          ldb[(4 * j + e) * TP + ld_col<TP>(4 * j + e, t)] = r.ld;
        }
        if (store_tn) stg4v(P.Tn + o, tn);
        stg4v(P.A + o, a);
        stg4v(P.D + o, d);
        stg4v(P.S + o, s4);
        stg4v(P.L + o, l4);
        stg4v(P.X + o, x4);
        stg4v(P.LD + o, ld4);
        // z^k and w^k enter only the dual residual of the next outer
        // iteration's lines 12-15, which run in a pass of their own after
        // the last iteration of a call: the pass before it (store_tn) keeps them
        if (hz) {
          stg4v(P.Bz + oz, bz);
          stg4v(P.p0 + oz, p04);
          if (store_tn) stg4v(P.zprev + oz, z);
        }
        if (hw) {
          stg4v(P.Cw + ow, cc);
          stg4v(P.p1 + ow, p14);
          if (store_tn) stg4v(P.wprev + ow, w);
        }
      }
      mb_arrive(&mb[kMbTnFree + b]);
      mb_arrive(&mb[kMbLdFull + b]);
    }
  } else {
    const int gt = tid - kFGUpd, bi = gt / 8, bj = gt % 8;
    // LD^k of chunk k into tile k & 1 (one commit group per chunk, empty
    // beyond the last, so that wait_group 1 always means "chunk k is in")
    auto prefetch = [&](int k) {
      if (k < nk) {
        const long long p0 = (blockIdx.x + (long long)k * gridDim.x) * kGC;
        float* dst = sIn + (k & 1) * TP * LDP;
        for (int e = gt; e < g.T * (kGC / 4); e += kFGGram) {
          const int s = e / (kGC / 4), q = e % (kGC / 4);
          const long long op = p0 + 4 * q;
          const bool in = op < g.plane;
          cp_async16(dst + s * LDP + 4 * q, in ? P.LD + (long long)s * g.plane + op : P.LD, in ? 16 : 0);
        }
      }
      cp_async_commit();
    };
    float gacc[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int q = 0; q < CB; ++q) gacc[r][q] = 0.f;
    // Gram of chunk j from LD^{k+1} tile j & 1
    auto gram_chunk = [&](int j) {
      const int b = j & 1;
      mb_wait(&mb[kMbLdFull + b], (j >> 1) & 1, err);
      const float* ldb = sLD + b * kGC * TP;
#pragma unroll 4
      for (int p = 0; p < kGC; ++p) {
        float av[RB], bv[CB];
        lds_row<RB>(ldb + p * TP + ld_col<TP>(p, RB * bi), av);   // RB <= 4: inside one group
        if constexpr (CB == 8) {
          float b0[4], b1[4];
          lds_row<4>(ldb + p * TP + ld_col<TP>(p, 8 * bj), b0);
          lds_row<4>(ldb + p * TP + ld_col<TP>(p, 8 * bj + 4), b1);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            bv[q] = b0[q];
            bv[4 + q] = b1[q];
          }
        } else {
          lds_row<CB>(ldb + p * TP + ld_col<TP>(p, CB * bj), bv);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int q = 0; q < CB; ++q) gacc[r][q] = fmaf(av[r], bv[q], gacc[r][q]);
      }
      mb_arrive(&mb[kMbLdFree + b]);
    };
    prefetch(0);
    prefetch(1);
    for (int k = 0; k < nk; ++k) {
      const int b = k & 1;
      cp_async_wait<1>();                      // this thread's copies of chunk k are in
      named_sync(kBarMma, kFGGram);            // ... and every contraction thread's
      if (k >= 2) mb_wait(&mb[kMbTnFree + b], ((k >> 1) - 1) & 1, err);
      // T^k of chunk k, pixels 4 bi .. 4 bi + 3: AT rows t in runs of AH,
      // the run starting at h = 0, AH, ... covering t = 8 h + AH bj .. + AH - 1
      // (the 8 threads of a pixel group read consecutive Wm runs), one run at
      // a time to bound the registers beside the Gram accumulator
      const float* in = sIn + b * TP * LDP;
      float* tnb = sTn + b * TP * LDP;
#pragma unroll
      for (int h = 0; h < AT; h += AH) {
        float o[AH][4];
#pragma unroll
        for (int r = 0; r < AH; ++r) o[r][0] = o[r][1] = o[r][2] = o[r][3] = 0.f;
#pragma unroll 4
        for (int s = 0; s < TP; ++s) {
          const float4 xv = *reinterpret_cast<const float4*>(in + s * LDP + 4 * bi);
          float wv[AH];
          lds_row<AH>(sW + s * LDS + 8 * h + AH * bj, wv);
#pragma unroll
          for (int r = 0; r < AH; ++r) {
            o[r][0] = fmaf(wv[r], xv.x, o[r][0]);
            o[r][1] = fmaf(wv[r], xv.y, o[r][1]);
            o[r][2] = fmaf(wv[r], xv.z, o[r][2]);
            o[r][3] = fmaf(wv[r], xv.w, o[r][3]);
          }
        }
#pragma unroll
        for (int r = 0; r < AH; ++r)
          *reinterpret_cast<float4*>(tnb + (8 * h + AH * bj + r) * LDP + 4 * bi) =
              make_float4(o[r][0], o[r][1], o[r][2], o[r][3]);
      }
      mb_arrive(&mb[kMbTnFull + b]);
      named_sync(kBarMma, kFGGram);            // every contraction thread is done with tile b of LD^k
      prefetch(k + 2);
      if (k >= 1) gram_chunk(k - 1);
    }
    if (nk >= 1) gram_chunk(nk - 1);
    cp_async_wait<0>();
    float* out = gpart + (size_t)blockIdx.x * TP * TP;
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int q = 0; q < CB; ++q) out[(RB * bi + r) * TP + CB * bj + q] = gacc[r][q];
  }
  block_sums_to<kFGThreads>(acc, partials + (size_t)blockIdx.x * kNumSums);
  for (int row = blockIdx.x + gridDim.x; row < nrows; row += gridDim.x)
    if (tid < kNumSums) partials[(size_t)row * kNumSums + tid] = 0.0;
  if (grid_barrier(bar, err)) gram_slice_reduce<TP>(gpart, G);
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
static int device_sms() {
  int dev = 0, n_sm = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n_sm = 152;
  return n_sm;
}

int rpca_gram_parts(const RpcaGeom& g) {
  long long n = (g.plane + kGC - 1) / kGC;
  const int n_sm = device_sms();
  if (n > n_sm) n = n_sm;
  const int nr = rpca_num_blocks(g);
  if (n > nr) n = nr;
  return (int)(n < 1 ? 1 : n);
}

cudaError_t rpca_launch_apply_post_pre_gram(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, int TP,
                                            const float* Wm, int store_tn, double* partials, int nrows, float* gpart,
                                            double* G, unsigned* bar, int* err, cudaStream_t st) {
  static unsigned long long attr_set = 0;   // raised once to the largest (TP = 64) size
  if (needs_setup(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(rpca_apply_post_pre_gram_kernel<16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)between_smem<16>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(rpca_apply_post_pre_gram_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)between_smem<32>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(rpca_apply_post_pre_gram_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)between_smem<64>());
    if (e != cudaSuccess) return e;
    mark_setup(attr_set);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(rpca_gram_parts(g));
  cfg.blockDim = dim3(kFGThreads);
  cfg.stream = st;
  cudaLaunchAttribute coop[1];
  coop[0].id = cudaLaunchAttributeCooperative;   // the CTAs meet at a grid barrier
  coop[0].val.cooperative = 1;
  cfg.attrs = coop;
  cfg.numAttrs = 1;
  switch (TP) {
    case 16:
      cfg.dynamicSmemBytes = between_smem<16>();
      return cudaLaunchKernelEx(&cfg, rpca_apply_post_pre_gram_kernel<16>, g, c, P, Wm, store_tn, partials, nrows,
                                gpart, G, bar, err);
    case 32:
      cfg.dynamicSmemBytes = between_smem<32>();
      return cudaLaunchKernelEx(&cfg, rpca_apply_post_pre_gram_kernel<32>, g, c, P, Wm, store_tn, partials, nrows,
                                gpart, G, bar, err);
    case 64:
      cfg.dynamicSmemBytes = between_smem<64>();
      return cudaLaunchKernelEx(&cfg, rpca_apply_post_pre_gram_kernel<64>, g, c, P, Wm, store_tn, partials, nrows,
                                gpart, G, bar, err);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t grid_barrier_probe(int ctas, unsigned preset, int* err, unsigned* generation) {
  if (ctas < 1 || ctas > device_sms()) return cudaErrorInvalidValue;
  unsigned* bar = nullptr;   // bar[0] count, bar[1] generation, bar[2] error flag
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&bar, 4 * sizeof(unsigned));
  const unsigned init[4] = {preset, 0u, 0u, 0u};
  unsigned out[4] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(bar, init, sizeof init, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute coop[1];
    coop[0].id = cudaLaunchAttributeCooperative;
    coop[0].val.cooperative = 1;
    cfg.attrs = coop;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, grid_barrier_probe_kernel, bar, reinterpret_cast<int*>(bar + 2));
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, bar, sizeof out, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    *err = (int)out[2];
    *generation = out[1];
  }
  if (bar) cudaFree(bar);
  if (st) cudaStreamDestroy(st);
  return e;
}

cudaError_t rpca_launch_sumsq(const RpcaGeom& g, const float* Y, double* partials, cudaStream_t st) {
  sumsq_kernel<<<rpca_num_blocks(g), kRpcaThreads, 0, st>>>(Y, g.plane / 4 * g.T, partials);
  return cudaGetLastError();
}

}  // namespace otp
