// Algorithm 1 iteration (Sec. III-B, lines 3-7) as a persistent, TMA-fed
// pipeline on sm_103a.
//
// The same fused update as the tiled kernel in prox_kernels.cu (one HBM pass
// per iteration; Mbar = 2M' - M staged in shared memory so that
// 2K(z') - K(z) = K(2z' - z) needs D applied once), but the inputs of each
// 16 x 128 tile are staged by the tensor-memory accelerator:
//   a      rows i0-1 .. i0+16, cols j0-4 .. j0+131  (one-pixel ring)
//   Mx, My rows i0-1 .. i0+15, cols j0-4 .. j0+127  (top/left halo)
//   x0 x1 r p0 p1   rows i0 .. i0+15, cols j0 .. j0+127
// into NS shared-memory stages.  One CTA per SM loops over the tiles; while
// it computes one tile the next NS-1 tiles are in flight, so HBM stays busy
// through the compute phases.  Coordinates outside the image (including the
// negative ones of the first tile row/column) are zero-filled by the TMA
// unit, which is exactly the zero-flux boundary for M and a harmless value
// for a (the flux on the outer slots is forced to zero anyway).
// Every mbarrier wait is bounded: on expiry the CTA records an error flag
// (reported as OT_ETIMEOUT by the host) and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kTmaTY = 16;                      // 32 x 16 threads, one row each
constexpr int kTmaThreads = 32 * kTmaTY;
constexpr int kAW = kTW + 8, kAH = kTH + 2;     // a box
constexpr int kMW = kTW + 4, kMH = kTH + 1;     // Mx, My box
constexpr int kPW = kTW, kPH = kTH;             // pointwise planes
constexpr uint32_t kSpinLimit = 1u << 22;

constexpr int align128(int b) { return (b + 127) / 128 * 128; }
constexpr int kABytes = kAW * kAH * 4;
constexpr int kMBytes = kMW * kMH * 4;
constexpr int kPBytes = kPW * kPH * 4;

template <int MODE, bool BAL>
struct StageLayout {
  static constexpr int nP = 2 + (MODE == 0 ? 1 : 0) + (MODE != 2 ? 1 : 0) + (BAL ? 0 : 1);
  static constexpr int oA = 0;
  static constexpr int oMx = align128(kABytes);
  static constexpr int oMy = oMx + align128(kMBytes);
  static constexpr int oP = oMy + align128(kMBytes);   // p0, p1, [x0], [x1], [r]
  static constexpr int bytes = oP + nP * kPBytes;
  static constexpr uint32_t tx_bytes = kABytes + 2 * kMBytes + nP * kPBytes;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within kSpinLimit tries.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void stg4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& cmp(float4& v, int e) { return (&v.x)[e]; }
__device__ __forceinline__ float cmpc(const float4& v, int e) { return (&v.x)[e]; }

__device__ __forceinline__ void flux_step(float mx, float my, float a_c, float a_down, float a_right, bool ex,
                                          bool ey, const IterCoeffs& c, float& ox, float& oy) {
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

// Issue the TMA copies of tile (b, i0, j0) into stage st, completing on bar.
template <int MODE, bool BAL>
__device__ __forceinline__ void tma_issue_tile(unsigned char* st, uint32_t bar, const TmaMaps* maps, int b, int i0,
                                               int j0) {
  using L = StageLayout<MODE, BAL>;
  mbar_expect_tx(bar, L::tx_bytes);
  tma_load_3d(smem_u32(st + L::oA), &maps->a, j0 - 4, i0 - 1, b, bar);
  tma_load_3d(smem_u32(st + L::oMx), &maps->Mx, j0 - 4, i0 - 1, b, bar);
  tma_load_3d(smem_u32(st + L::oMy), &maps->My, j0 - 4, i0 - 1, b, bar);
  int k = 0;
  tma_load_3d(smem_u32(st + L::oP + (k++) * kPBytes), &maps->p0, j0, i0, b, bar);
  tma_load_3d(smem_u32(st + L::oP + (k++) * kPBytes), &maps->p1, j0, i0, b, bar);
  if (MODE == 0) tma_load_3d(smem_u32(st + L::oP + (k++) * kPBytes), &maps->x0, j0, i0, b, bar);
  if (MODE != 2) tma_load_3d(smem_u32(st + L::oP + (k++) * kPBytes), &maps->x1, j0, i0, b, bar);
  if (!BAL) tma_load_3d(smem_u32(st + L::oP + (k++) * kPBytes), &maps->r, j0, i0, b, bar);
}

// Lines 3-7 of Algorithm 1 on tile (b, i0, j0) whose inputs sit in stage st;
// writes the new state to S and adds the check sums (RED) to accs.
template <int MODE, bool BAL, bool RED>
__device__ __forceinline__ void tma_compute_tile(const unsigned char* st, const Geometry& G, const IterCoeffs& C,
                                                 const StatePtrs& S, int b, int i0, int j0, float* s_mbx,
                                                 float* s_mby, float* s_mnx, float* s_mny,
                                                 float (&accs)[kNumSums]) {
  using L = StageLayout<MODE, BAL>;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int H = G.H, W = G.W, Wp = G.Wp;
    const float* sA = reinterpret_cast<const float*>(st + L::oA);
  const float* sMx = reinterpret_cast<const float*>(st + L::oMx);
  const float* sMy = reinterpret_cast<const float*>(st + L::oMy);
  const float* sP0 = reinterpret_cast<const float*>(st + L::oP);
  const float* sP1 = sP0 + kPW * kPH;
  const float* sX0 = MODE == 0 ? sP1 + kPW * kPH : sP0;
  const float* sX1 = MODE != 2 ? sP1 + (MODE == 0 ? 2 : 1) * kPW * kPH : sP1;
  const float* sR = sP1 + ((MODE == 0 ? 1 : 0) + (MODE != 2 ? 1 : 0) + 1) * kPW * kPH;

  // ---- line 3 on own pixels: row rr = ty + 1 of the halo'd boxes
  const int rr = ty + 1;
  const int i = i0 + ty;
  const int j = j0 + 4 * tx;
  const float4 mx4 = lds4(sMx + rr * kMW + 4 + 4 * tx);
  const float4 my4 = lds4(sMy + rr * kMW + 4 + 4 * tx);
  const float4 ac = lds4(sA + rr * kAW + 4 + 4 * tx);
  const float an = sA[rr * kAW + 8 + 4 * tx];
  const float4 ad = lds4(sA + (rr + 1) * kAW + 4 + 4 * tx);
  float4 nmx, nmy, bx4, by4;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int jj = j + e;
    const bool in = (i < H) && (jj < W);
    const float a_r = e < 3 ? cmpc(ac, e + 1) : an;
    float ox, oy;
    flux_step(cmpc(mx4, e), cmpc(my4, e), cmpc(ac, e), cmpc(ad, e), a_r, in && i < H - 1, in && jj < W - 1, C,
              ox, oy);
    cmp(nmx, e) = ox;
    cmp(nmy, e) = oy;
    cmp(bx4, e) = 2.f * ox - cmpc(mx4, e);
    cmp(by4, e) = 2.f * oy - cmpc(my4, e);
  }
  stg4(s_mbx + rr * kTW + 4 * tx, bx4);
  stg4(s_mby + ty * (kTW + 4) + 4 + 4 * tx, by4);
  if (RED) {
    stg4(s_mnx + rr * kTW + 4 * tx, nmx);
    stg4(s_mny + ty * (kTW + 4) + 4 + 4 * tx, nmy);
  }
  // halo row i0-1 (only Mbar_x is consumed)
  if (ty == 0) {
    float4 hb = make_float4(0.f, 0.f, 0.f, 0.f), hn = hb;
    if (i0 >= 1) {
      const float4 hmx = lds4(sMx + 4 + 4 * tx);
      const float4 hmy = lds4(sMy + 4 + 4 * tx);
      const float4 hac = lds4(sA + 4 + 4 * tx);
      const float han = sA[8 + 4 * tx];
      const float4 had = lds4(sA + kAW + 4 + 4 * tx);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int jj = j + e;
        const bool in = jj < W;
        const float a_r = e < 3 ? cmpc(hac, e + 1) : han;
        float ox, oy;
        flux_step(cmpc(hmx, e), cmpc(hmy, e), cmpc(hac, e), cmpc(had, e), a_r, in, in && jj < W - 1, C, ox, oy);
        cmp(hb, e) = 2.f * ox - cmpc(hmx, e);
        cmp(hn, e) = ox;
      }
    }
    stg4(s_mbx + 4 * tx, hb);
    if (RED) stg4(s_mnx + 4 * tx, hn);
  }
  // halo column j0-1 (only Mbar_y is consumed)
  if (tx == 0) {
    float hb = 0.f, hn = 0.f;
    if (j0 >= 1 && i < H) {
      const float lmx = sMx[rr * kMW + 3], lmy = sMy[rr * kMW + 3];
      const float a_c = sA[rr * kAW + 3], a_r = sA[rr * kAW + 4], a_d = sA[(rr + 1) * kAW + 3];
      float ox, oy;
      flux_step(lmx, lmy, a_c, a_d, a_r, i < H - 1, true, C, ox, oy);
      hb = 2.f * oy - lmy;
      hn = oy;
    }
    s_mby[ty * (kTW + 4) + 3] = hb;
    if (RED) s_mny[ty * (kTW + 4) + 3] = hn;
  }
  __syncthreads();

  // ---- lines 4-7 on own pixels
  float* acc = accs;
  if (i < H && j < Wp) {
    const int po = ty * kPW + 4 * tx;
    const float4 a4 = ac;
    const float4 p04 = lds4(sP0 + po), p14 = lds4(sP1 + po);
    const float4 x04 = MODE == 0 ? lds4(sX0 + po) : p04;
    const float4 x14 = MODE != 2 ? lds4(sX1 + po) : p14;
    const float4 r4 = BAL ? make_float4(0.f, 0.f, 0.f, 0.f) : lds4(sR + po);
    const float4 mbx = lds4(s_mbx + rr * kTW + 4 * tx);
    const float4 mbx_up = lds4(s_mbx + ty * kTW + 4 * tx);
    const float4 mby = lds4(s_mby + ty * (kTW + 4) + 4 + 4 * tx);
    const float mby_l = s_mby[ty * (kTW + 4) + 3 + 4 * tx];
    float4 nx0, nx1, nr, na;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool in = (j + e) < W;
      const float a = cmpc(a4, e);
      float vx0 = cmpc(p04, e), vx1 = cmpc(p14, e);
      if (MODE == 0) vx0 = fmaxf(fmaf(C.cp, cmpc(p04, e), fmaf(C.cx, cmpc(x04, e), C.ca * a)), 0.f);
      if (MODE != 2) vx1 = fmaxf(fmaf(C.cp, cmpc(p14, e), fmaf(C.cx, cmpc(x14, e), -C.ca * a)), 0.f);
      const float vr = BAL ? 0.f : r_step(cmpc(r4, e), a, C);
      const float dmb = (cmpc(mbx, e) - cmpc(mbx_up, e)) + (cmpc(mby, e) - (e == 0 ? mby_l : cmpc(mby, e - 1)));
      float bk = dmb - (2.f * vx0 - cmpc(x04, e)) + (2.f * vx1 - cmpc(x14, e));
      if (!BAL) bk -= 2.f * vr - cmpc(r4, e);
      const float va = fmaf(C.tau2, bk, a);
      cmp(nx0, e) = in ? vx0 : 0.f;
      cmp(nx1, e) = in ? vx1 : 0.f;
      cmp(nr, e) = in ? vr : 0.f;
      cmp(na, e) = in ? va : 0.f;
      if (RED && in) {
        const float nmxe = cmpc(nmx, e), nmye = cmpc(nmy, e);
        const float nmx_up = s_mnx[ty * kTW + 4 * tx + e];
        const float nmy_l = s_mny[ty * (kTW + 4) + 3 + 4 * tx + e];
        const float kz = (nmxe - nmx_up) + (nmye - nmy_l) - vx0 + vx1 - (BAL ? 0.f : vr);
        acc[0] = fmaf(kz, kz, acc[0]);
        const float d0 = nmxe - cmpc(mx4, e), d1 = nmye - cmpc(my4, e);
        const float d2 = vx0 - cmpc(x04, e), d3 = vx1 - cmpc(x14, e);
        const float d4 = vr - cmpc(r4, e), d5 = va - a;
        acc[1] += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5;
        acc[2] += nmxe * nmxe + nmye * nmye + vx0 * vx0 + vx1 * vx1 + vr * vr + va * va;
        acc[3] += C.iso ? sqrtf(fmaf(nmxe, nmxe, nmye * nmye)) : fabsf(nmxe) + fabsf(nmye);
        acc[4] += C.pexp == 1 ? fabsf(vr) : vr * vr;
        const float e0 = vx0 - cmpc(p04, e), e1 = vx1 - cmpc(p14, e);
        if (MODE == 0) acc[5] = fmaf(e0, e0, acc[5]);
        if (MODE != 2) acc[5] = fmaf(e1, e1, acc[5]);
        acc[6] += cmpc(p04, e) * cmpc(p04, e) + cmpc(p14, e) * cmpc(p14, e);
        acc[7] += (!isfinite(va) || !isfinite(nmxe) || !isfinite(nmye) || !isfinite(vx0) || !isfinite(vx1) ||
                   !isfinite(vr) || !isfinite(cmpc(p04, e)) || !isfinite(cmpc(p14, e)))
                      ? 1.f
                      : 0.f;
      }
    }
    const long long off = (long long)b * G.plane + (long long)i * Wp + j;
    stg4(S.Mx_out + off, nmx);
    stg4(S.My_out + off, nmy);
    stg4(S.a_out + off, na);
    if (MODE == 0) stg4(S.x0 + off, nx0);
    if (MODE != 2) stg4(S.x1 + off, nx1);
    if (!BAL) stg4(S.r + off, nr);
  }
}

template <int MODE, bool BAL, bool RED, int NS>
__global__ void __launch_bounds__(kTmaThreads, 1)
prox_tma_kernel(const __grid_constant__ TmaMaps maps, const Geometry G, const IterCoeffs C, const StatePtrs S,
                double* __restrict__ partials, int* __restrict__ err) {
  using L = StageLayout<MODE, BAL>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA tile destinations want 128-byte alignment: align the base by hand
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* s_mbx = reinterpret_cast<float*>(smem + NS * L::bytes);            // [kTH+1][kTW]
  float* s_mby = s_mbx + (kTH + 1) * kTW;                                    // [kTH][kTW+4]
  float* s_mnx = s_mby + kTH * (kTW + 4);                                    // RED only
  float* s_mny = s_mnx + (RED ? (kTH + 1) * kTW : 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_mny + (RED ? kTH * (kTW + 4) : 0));
  double* red = reinterpret_cast<double*>(bars + NS);                       // [warps][kNumSums]

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ntiles = G.B * G.tiles_x * G.tiles_y;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue = [&](int tile, int s) {
    int t = tile;
    const int bx = t % G.tiles_x;
    t /= G.tiles_x;
    const int by = t % G.tiles_y;
    const int b = t / G.tiles_y;
    tma_issue_tile<MODE, BAL>(smem + s * L::bytes, smem_u32(&bars[s]), &maps, b, by * kTH, bx * kTW);
  };


  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile < ntiles) issue(tile, s);
    }
  }

  // Per-thread sums stay FP32 (a few dozen pixels per thread); FP64, which
  // is scarce on this GPU, is used only across warps and CTAs.
  float accs[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) accs[k] = 0.f;

  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int s = k % NS;
    const uint32_t parity = (uint32_t)((k / NS) & 1);
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), parity);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      // bounded wait for the copies still in flight, then leave
      for (int s2 = 0; s2 < NS; ++s2) (void)mbar_wait_bounded(smem_u32(&bars[s2]), parity);
      return;
    }
    int t = tile;
    const int bx = t % G.tiles_x;
    t /= G.tiles_x;
    const int by = t % G.tiles_y;
    const int b = t / G.tiles_y;
    const int i0 = by * kTH, j0 = bx * kTW;
    tma_compute_tile<MODE, BAL, RED>(smem + s * L::bytes, G, C, S, b, i0, j0, s_mbx, s_mby, s_mnx, s_mny, accs);
    // every thread is done with stage s and with the Mbar arrays of this tile
    __syncthreads();
    if (tid == 0) {
      const int next = tile + NS * gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(next, s);
      }
    }
  }

  if (RED) {
    // block reduction in FP64 of the per-thread sums
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) accs[q] += __shfl_down_sync(0xffffffffu, accs[q], o);
      if (lane == 0) red[warp * kNumSums + q] = (double)accs[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) {
        double v = lane < kTmaThreads / 32 ? red[lane * kNumSums + q] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) partials[(size_t)blockIdx.x * kNumSums + q] = v;
      }
    }
  }
}

// The same pipeline over the tiles of many sequences (the batched runtime in
// prox_batch.cu): a device-side work list (act[0] = n, act[1..n] = sequence
// ids, act[1+n..1+2n] = tile prefix sums) is walked with a grid stride; each
// tile uses its sequence's tensor maps (device memory), geometry and step
// sizes, so every pixel's arithmetic is that of the one-problem kernel.
// Check iterations write one partial-sum row per tile.
template <int MODE, bool BAL, bool RED, int NS>
__global__ void __launch_bounds__(kTmaThreads, 1)
prox_tma_batch_kernel(const BatchSeq* __restrict__ seqs, const int* __restrict__ act, int parity, const BatchPlanes P,
                      double* __restrict__ partials, int* __restrict__ err) {
  using L = StageLayout<MODE, BAL>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* s_mbx = reinterpret_cast<float*>(smem + NS * L::bytes);
  float* s_mby = s_mbx + (kTH + 1) * kTW;
  float* s_mnx = s_mby + kTH * (kTW + 4);
  float* s_mny = s_mnx + (RED ? (kTH + 1) * kTW : 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_mny + (RED ? kTH * (kTW + 4) : 0));
  double* red = reinterpret_cast<double*>(bars + NS);
  __shared__ int s_seq[kBatchMaxSeq];
  __shared__ int s_pre[kBatchMaxSeq + 1];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int n_act = act[0];
  for (int k = tid; k < n_act; k += kTmaThreads) s_seq[k] = act[1 + k];
  for (int k = tid; k <= n_act; k += kTmaThreads) s_pre[k] = act[1 + n_act + k];
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int total = s_pre[n_act];

  // work item w -> (sequence, tile of that sequence)
  auto locate = [&](int w, int& seq, int& t) {
    int lo = 0, hi = n_act - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    seq = s_seq[lo];
    t = w - s_pre[lo];
  };
  auto issue = [&](int w, int s) {
    int seq, t;
    locate(w, seq, t);
    const BatchSeq& d = seqs[seq];
    const int bx = t % d.G.tiles_x;
    const int rest = t / d.G.tiles_x;
    const int by = rest % d.G.tiles_y;
    const int b = rest / d.G.tiles_y;
    tma_issue_tile<MODE, BAL>(smem + s * L::bytes, smem_u32(&bars[s]), parity ? &d.maps[1] : &d.maps[0], b, by * kTH,
                              bx * kTW);
  };

  // a contiguous range of work items per CTA: consecutive tiles mostly share
  // a sequence, so its descriptors and coefficients stay in cache
  const int w0 = (int)((long long)total * blockIdx.x / gridDim.x);
  const int w1 = (int)((long long)total * (blockIdx.x + 1) / gridDim.x);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      const int w = w0 + s;
      if (w < w1) issue(w, s);
    }
  }

  float accs[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) accs[k] = 0.f;

  int k = 0;
  for (int w = w0; w < w1; ++w, ++k) {
    const int s = k % NS;
    const uint32_t ph = (uint32_t)((k / NS) & 1);
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), ph);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicExch(err, 1);
      for (int s2 = 0; s2 < NS; ++s2) (void)mbar_wait_bounded(smem_u32(&bars[s2]), ph);
      return;
    }
    int seq, t;
    locate(w, seq, t);
    const BatchSeq& d = seqs[seq];
    const int bx = t % d.G.tiles_x;
    const int rest = t / d.G.tiles_x;
    const int by = rest % d.G.tiles_y;
    const int b = rest / d.G.tiles_y;
    StatePtrs S;
    // selects, not P.Mx[parity]: a runtime index into a kernel parameter would go through local memory
    S.Mx_in = (parity ? P.Mx[1] : P.Mx[0]) + d.off;
    S.My_in = (parity ? P.My[1] : P.My[0]) + d.off;
    S.a_in = (parity ? P.a[1] : P.a[0]) + d.off;
    S.Mx_out = (parity ? P.Mx[0] : P.Mx[1]) + d.off;
    S.My_out = (parity ? P.My[0] : P.My[1]) + d.off;
    S.a_out = (parity ? P.a[0] : P.a[1]) + d.off;
    S.x0 = P.x0 + d.off;
    S.x1 = P.x1 + d.off;
    S.r = P.r + d.off;
    S.p0 = P.p0 + d.off;
    S.p1 = P.p1 + d.off;
    tma_compute_tile<MODE, BAL, RED>(smem + s * L::bytes, d.G, d.C, S, b, by * kTH, bx * kTW, s_mbx, s_mby, s_mnx,
                                     s_mny, accs);
    if (RED) {   // this tile's check sums: FP32 within the warp, FP64 across warps
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int q = 0; q < kNumSums; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) accs[q] += __shfl_down_sync(0xffffffffu, accs[q], o);
        if (lane == 0) red[warp * kNumSums + q] = (double)accs[q];
        accs[q] = 0.f;
      }
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kNumSums; ++q) {
          double v = lane < kTmaThreads / 32 ? red[lane * kNumSums + q] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if (lane == 0) partials[(size_t)(d.tile0 + t) * kNumSums + q] = v;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      const int next = w + NS;
      if (next < w1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(next, s);
      }
    }
  }
}

template <int MODE, bool BAL, bool RED, int NS>
constexpr size_t tma_smem_bytes() {
  return 128 /* base alignment slack */ + (size_t)NS * StageLayout<MODE, BAL>::bytes +
         (size_t)(RED ? 2 : 1) * ((kTH + 1) * kTW + kTH * (kTW + 4)) * 4 + NS * sizeof(uint64_t) +
         (RED ? (kTmaThreads / 32) * kNumSums * sizeof(double) : 0);
}

// Stages: 3 without the reduction, 2 with it (its two extra shared arrays
// would not fit beside a third stage).
template <int MODE, bool BAL, bool RED>
constexpr int tma_stages() {
  return (!RED && tma_smem_bytes<MODE, BAL, false, 3>() <= 227 * 1024) ? 3 : 2;
}
// the batched kernel also holds its work list (2 KB) in static shared memory
constexpr size_t kBatchListBytes = (2 * kBatchMaxSeq + 1) * sizeof(int);
template <int MODE, bool BAL, bool RED>
constexpr int tma_batch_stages() {
  return (!RED && tma_smem_bytes<MODE, BAL, false, 3>() + kBatchListBytes <= 227 * 1024) ? 3 : 2;
}

template <int MODE, bool BAL, bool RED>
cudaError_t prepare_batch_t() {
  constexpr int NS = tma_batch_stages<MODE, BAL, RED>();
  return cudaFuncSetAttribute(prox_tma_batch_kernel<MODE, BAL, RED, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tma_smem_bytes<MODE, BAL, RED, NS>());
}

template <int MODE, bool BAL, bool RED>
cudaError_t launch_batch_t(const BatchSeq* seqs, const int* act, int parity, const BatchPlanes& P, double* partials,
                           int* err, int grid, cudaStream_t st) {
  constexpr int NS = tma_batch_stages<MODE, BAL, RED>();
  prox_tma_batch_kernel<MODE, BAL, RED, NS><<<grid, dim3(32, kTmaTY), tma_smem_bytes<MODE, BAL, RED, NS>(), st>>>(
      seqs, act, parity, P, partials, err);
  return cudaGetLastError();
}

template <int MODE, bool BAL, bool RED>
cudaError_t prepare_t() {
  constexpr int NS = tma_stages<MODE, BAL, RED>();
  return cudaFuncSetAttribute(prox_tma_kernel<MODE, BAL, RED, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tma_smem_bytes<MODE, BAL, RED, NS>());
}

template <int MODE, bool BAL, bool RED>
cudaError_t launch_t(const TmaMaps& maps, const Geometry& g, const IterCoeffs& c, const StatePtrs& s,
                     double* partials, int* err, int grid, cudaStream_t st) {
  constexpr int NS = tma_stages<MODE, BAL, RED>();
  prox_tma_kernel<MODE, BAL, RED, NS><<<grid, dim3(32, kTmaTY), tma_smem_bytes<MODE, BAL, RED, NS>(), st>>>(
      maps, g, c, s, partials, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_prox_tma(int mode, bool balanced) {
  cudaError_t e = cudaSuccess;
#define OTP_PREP(M, BL)                                        \
  if (mode == M && balanced == BL) {                           \
    e = prepare_t<M, BL, false>();                             \
    if (e == cudaSuccess) e = prepare_t<M, BL, true>();        \
    return e;                                                  \
  }
  OTP_PREP(0, false)
  OTP_PREP(0, true)
  OTP_PREP(1, false)
  OTP_PREP(1, true)
  OTP_PREP(2, false)
  OTP_PREP(2, true)
#undef OTP_PREP
  return cudaErrorInvalidValue;
}

cudaError_t prepare_prox_tma_batch(int mode, bool balanced) {
  cudaError_t e = cudaSuccess;
#define OTP_PREP(M, BL)                                        \
  if (mode == M && balanced == BL) {                           \
    e = prepare_batch_t<M, BL, false>();                       \
    if (e == cudaSuccess) e = prepare_batch_t<M, BL, true>();  \
    return e;                                                  \
  }
  OTP_PREP(0, false)
  OTP_PREP(0, true)
  OTP_PREP(1, false)
  OTP_PREP(1, true)
  OTP_PREP(2, false)
  OTP_PREP(2, true)
#undef OTP_PREP
  return cudaErrorInvalidValue;
}

cudaError_t launch_prox_tma_batch(int mode, bool balanced, bool reduce, const BatchSeq* seqs, const int* act,
                                  int parity, const BatchPlanes& P, double* partials, int* err, int grid,
                                  cudaStream_t st) {
#define OTP_L(M, BL)                                                                              \
  if (mode == M && balanced == BL)                                                                \
    return reduce ? launch_batch_t<M, BL, true>(seqs, act, parity, P, partials, err, grid, st)    \
                  : launch_batch_t<M, BL, false>(seqs, act, parity, P, partials, err, grid, st);
  OTP_L(0, false)
  OTP_L(0, true)
  OTP_L(1, false)
  OTP_L(1, true)
  OTP_L(2, false)
  OTP_L(2, true)
#undef OTP_L
  return cudaErrorInvalidValue;
}

cudaError_t launch_prox_tma(int mode, bool balanced, bool reduce, const TmaMaps& maps, const Geometry& g,
                            const IterCoeffs& c, const StatePtrs& s, double* partials, int* err, int grid,
                            cudaStream_t st) {
#define OTP_L(M, BL)                                                                      \
  if (mode == M && balanced == BL)                                                        \
    return reduce ? launch_t<M, BL, true>(maps, g, c, s, partials, err, grid, st)         \
                  : launch_t<M, BL, false>(maps, g, c, s, partials, err, grid, st);
  OTP_L(0, false)
  OTP_L(0, true)
  OTP_L(1, false)
  OTP_L(1, true)
  OTP_L(2, false)
  OTP_L(2, true)
#undef OTP_L
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ tensor maps
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
}  // namespace

// A [B][H][Wp] float32 plane seen as a 3-D tensor of extent (W, H, B):
// columns W..Wp-1 and everything outside read as zero.
int encode_plane_map(CUtensorMap* map, const float* base, const Geometry& g, int box_w, int box_h) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const cuuint64_t dims[3] = {(cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.B};
  const cuuint64_t strides[2] = {(cuuint64_t)g.Wp * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

int tma_box(int which, int* w, int* h) {
  switch (which) {
    case 0: *w = kAW; *h = kAH; return 0;   // a
    case 1: *w = kMW; *h = kMH; return 0;   // Mx, My
    default: *w = kPW; *h = kPH; return 0;  // pointwise planes
  }
}

}  // namespace otp
