// Temporal blocking of Algorithm 1 (Sec. III-B, lines 3-7): up to KD
// iterations per pass over HBM.
//
// One iteration at a pixel reads a on the pixel's 3 x 3 neighbourhood and M
// on the pixel and its up / left neighbours (the divergence D of the
// extrapolated flux), so k iterations of a tile depend on the state of the
// tile grown by k pixels on every side.  A CTA stages that grown tile (KD
// rows above and below, 4 columns left and right: the float4 group), runs
// n <= KD iterations on all of it, and after iteration s the values are exact
// on the tile grown by KD - s; only the tile itself is written back.  The
// arithmetic of a pixel is the same sequence of operations as the one-pass
// kernels' (the line 3-7 helpers of prox_tile.cuh), so the result is
// bit-identical to n single iterations.
//
// Layout: 512 threads; thread t < 510 owns float4 column group t % 34 on the
// rows t / 34 + 15 q (q < 3) of the 45-row extended tile; M, x, r live in its
// registers, a, Mbar = 2M' - M and the inputs p in shared memory.  Pixels
// outside the image are zero at every iteration (zero flux, zero densities),
// as in the one-pass kernels.  Each CTA writes the rows and columns it owns
// only, so x and r are ping-ponged like M and a (a neighbouring tile reads
// them on its halo).
#include <cuda_runtime.h>
#include <math.h>

#include "otprox_internal.cuh"
#include "prox_tile.cuh"

namespace otp {
namespace {

using tile::comp;
using tile::compc;
using tile::ld4;
using tile::st4;

constexpr int kGX = kTbGroups;           // float4 groups of an extended row (4 + 128 + 4 columns)
constexpr int kGY = kTbThreadRows;       // thread rows
constexpr int kRPT = kTbRowsPerThread;   // rows per thread
constexpr int kEH = kTbExtRows;          // rows of the extended tile
constexpr int kNT = kTbThreads;          // 512 (the last two threads own no pixel)

template <bool RED>
constexpr size_t tb_smem_bytes() {
  return (size_t)(RED ? 7 : 5) * kEH * kGX * sizeof(float4);
}

template <int MODE, bool BAL, bool RED, int KD>
__global__ void __launch_bounds__(kNT, 1)
prox_temporal_kernel(const Geometry G, const IterCoeffs C, const TbPtrs S, int n_sub, int pf_stride,
                     double* __restrict__ partials) {
  constexpr int TH = kEH - 2 * KD;
  extern __shared__ float4 tb_smem[];
  float4(*s_a)[kGX] = reinterpret_cast<float4(*)[kGX]>(tb_smem);
  float4(*s_mbx)[kGX] = s_a + kEH;
  float4(*s_mby)[kGX] = s_mbx + kEH;
  float4(*s_p0)[kGX] = s_mby + kEH;
  float4(*s_p1)[kGX] = s_p0 + kEH;
  float4(*s_mnx)[kGX] = s_p1 + kEH;     // RED: the last iteration's M'
  float4(*s_mny)[kGX] = s_mnx + kEH;

  const int tid = threadIdx.x;
  const bool owner = tid < kGX * kGY;
  const int tx = owner ? tid % kGX : 0, ty = owner ? tid / kGX : 0;
  const int H = G.H, W = G.W, Wp = G.Wp;
  const int ntiles = G.B * G.tiles_x * G.tiles_y;
  // tile t -> problem b, tile row by, tile column bx; rows from i0 - KD, columns from j0 - 4
  auto tile_origin = [&](int t, long long& base, int& i0, int& j0) {
    const int bx = t % G.tiles_x;
    t /= G.tiles_x;
    const int by = t % G.tiles_y;
    base = (long long)(t / G.tiles_y) * G.plane;
    i0 = by * TH;
    j0 = bx * kTW;
  };
  long long base;
  int i0, j0;
  tile_origin(blockIdx.x, base, i0, j0);
  const int j = j0 - 4 + 4 * tx;
  const bool colok = owner && j >= 0 && j < Wp;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

  // ---- stage the extended tile: M, x, r in registers; a, p in shared memory
  float4 mx[kRPT], my[kRPT], x0[kRPT], x1[kRPT], rv[kRPT];
#pragma unroll
  for (int q = 0; q < kRPT; ++q) {
    const int u = ty + kGY * q;
    const int i = i0 - KD + u;
    const bool ok = colok && i >= 0 && i < H;
    const long long off = base + (long long)i * Wp + j;
    mx[q] = ok ? ld4(S.Mx_in + off) : z4;
    my[q] = ok ? ld4(S.My_in + off) : z4;
    x0[q] = (ok && MODE == 0) ? ld4(S.x0_in + off) : z4;
    x1[q] = (ok && MODE != 2) ? ld4(S.x1_in + off) : z4;
    rv[q] = (ok && !BAL) ? ld4(S.r_in + off) : z4;
    if (owner) {
      s_a[u][tx] = ok ? ld4(S.a_in + off) : z4;
      s_p0[u][tx] = ok ? ld4(S.p0 + off) : z4;
      s_p1[u][tx] = ok ? ld4(S.p1 + off) : z4;
    }
  }
  // ---- L2 prefetch of the tile the next wave runs here (one CTA per SM:
  // block + pf_stride), one row of one plane per thread, once this block's
  // own loads are in flight
  if (pf_stride > 0 && blockIdx.x + pf_stride < ntiles && tid < 8 * kEH) {
    long long nb;
    int ni0, nj0;
    tile_origin(blockIdx.x + pf_stride, nb, ni0, nj0);
    const int pl = tid / kEH, i = ni0 - KD + tid % kEH;
    const float* src = pl == 0 ? S.Mx_in : pl == 1 ? S.My_in : pl == 2 ? S.a_in : pl == 3 ? S.p0 : pl == 4 ? S.p1
                     : pl == 5 ? (MODE == 0 ? S.x0_in : nullptr) : pl == 6 ? (MODE != 2 ? S.x1_in : nullptr)
                     : (!BAL ? S.r_in : nullptr);
    const int c0 = nj0 - 4 > 0 ? nj0 - 4 : 0, c1 = nj0 + kTW + 4 < Wp ? nj0 + kTW + 4 : Wp;
    if (src && i >= 0 && i < H && c1 > c0) {
      const float* row = src + nb + (long long)i * Wp + c0;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row), "r"((c1 - c0) * 4) : "memory");
    }
  }
  __syncthreads();

  float acc[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) acc[k] = 0.f;

  for (int s = 1; s <= n_sub; ++s) {
    const bool chk = RED && s == n_sub;
    // the region later iterations still read: rows [lo, kEH - lo) for a, x, r
    // (the halo shrinks by one row per iteration), one row more above for M;
    // the halo column groups only before the last iteration
    const int lo = KD - (n_sub - s);
    const bool edge_groups = s < n_sub;
    // ---- line 3; Mbar = 2M' - M to shared memory
    if (owner && (edge_groups || tx < kGX - 1)) {
#pragma unroll
      for (int q = 0; q < kRPT; ++q) {
        const int u = ty + kGY * q;
        if (u < lo - 1 || u >= kEH - lo) continue;
        const int i = i0 - KD + u;
        const bool rowin = i >= 0 && i < H && j >= 0;
        const float4 ac = s_a[u][tx];
        const float an = tx + 1 < kGX ? s_a[u][tx + 1].x : 0.f;
        const float4 ad = u + 1 < kEH ? s_a[u + 1][tx] : z4;
        float4 nx4, ny4, bx4, by4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int jj = j + e;
          const bool in = rowin && jj < W;
          const float a_r = e < 3 ? compc(ac, e + 1) : an;
          float ox, oy;
          tile::flux_step(compc(mx[q], e), compc(my[q], e), compc(ac, e), compc(ad, e), a_r, in && i < H - 1,
                          in && jj < W - 1, C, ox, oy);
          comp(nx4, e) = ox;
          comp(ny4, e) = oy;
          comp(bx4, e) = 2.f * ox - compc(mx[q], e);
          comp(by4, e) = 2.f * oy - compc(my[q], e);
        }
        s_mbx[u][tx] = bx4;
        s_mby[u][tx] = by4;
        if (chk) {
          // keep M (the old flux) for the check terms; M' goes to shared memory
          s_mnx[u][tx] = nx4;
          s_mny[u][tx] = ny4;
        } else {
          mx[q] = nx4;
          my[q] = ny4;
        }
      }
    }
    __syncthreads();
    // ---- lines 4-7; a' in place (only the own pixel's a is read here)
    if (owner && (edge_groups || (tx >= 1 && tx < kGX - 1))) {
#pragma unroll
      for (int q = 0; q < kRPT; ++q) {
        const int u = ty + kGY * q;
        if (u < lo || u >= kEH - lo) continue;
        const int i = i0 - KD + u;
        const bool rowin = i >= 0 && i < H && j >= 0;
        const bool own = chk && u >= KD && u < KD + TH && i < H && tx >= 1 && tx < kGX - 1;
        const float4 a4 = s_a[u][tx];
        const float4 mbx = s_mbx[u][tx];
        const float4 mbx_up = s_mbx[u - 1][tx];
        const float4 mby = s_mby[u][tx];
        const float mby_l = tx > 0 ? s_mby[u][tx - 1].w : 0.f;
        const float4 p04 = s_p0[u][tx], p14 = s_p1[u][tx];
        float4 nx0, nx1, nr, na;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int jj = j + e;
          const bool in = rowin && jj < W;
          const float a = compc(a4, e);
          const float x0e = MODE == 0 ? compc(x0[q], e) : compc(p04, e);
          const float x1e = MODE != 2 ? compc(x1[q], e) : compc(p14, e);
          const float re = BAL ? 0.f : compc(rv[q], e);
          float vx0 = compc(p04, e), vx1 = compc(p14, e);
          if (MODE == 0) vx0 = tile::x0_step(compc(p04, e), x0e, a, C);
          if (MODE != 2) vx1 = tile::x1_step(compc(p14, e), x1e, a, C);
          const float vr = BAL ? 0.f : tile::r_step(re, a, C);
          const float dmb = (compc(mbx, e) - compc(mbx_up, e)) +
                            (compc(mby, e) - (e == 0 ? mby_l : compc(mby, e - 1)));
          const float va = tile::dual_step<BAL>(dmb, vx0, x0e, vx1, x1e, vr, re, a, C);
          comp(nx0, e) = in ? vx0 : 0.f;
          comp(nx1, e) = in ? vx1 : 0.f;
          comp(nr, e) = in ? vr : 0.f;
          comp(na, e) = in ? va : 0.f;
          if (RED && own && in) {
            const float4 nmx4 = s_mnx[u][tx], nmx_up4 = s_mnx[u - 1][tx], nmy4 = s_mny[u][tx];
            const float nmy_l = e == 0 ? s_mny[u][tx - 1].w : compc(nmy4, e - 1);
            tile::check_terms<MODE, BAL>(compc(nmx4, e), compc(nmy4, e), compc(nmx_up4, e), nmy_l, compc(mx[q], e),
                                         compc(my[q], e), vx0, x0e, vx1, x1e, vr, re, va, a, compc(p04, e),
                                         compc(p14, e), C, acc);
          }
        }
        s_a[u][tx] = na;
        if (MODE == 0) x0[q] = nx0;
        if (MODE != 2) x1[q] = nx1;
        if (!BAL) rv[q] = nr;
        if (chk) {
          mx[q] = s_mnx[u][tx];
          my[q] = s_mny[u][tx];
        }
      }
    }
    __syncthreads();
  }

  // ---- write the tile's own rows and columns
  if (owner && tx >= 1 && tx < kGX - 1 && j < Wp) {
#pragma unroll
    for (int q = 0; q < kRPT; ++q) {
      const int u = ty + kGY * q;
      const int i = i0 - KD + u;
      if (u < KD || u >= KD + TH || i >= H) continue;
      const long long off = base + (long long)i * Wp + j;
      st4(S.Mx_out + off, mx[q]);
      st4(S.My_out + off, my[q]);
      st4(S.a_out + off, s_a[u][tx]);
      if (MODE == 0) st4(S.x0_out + off, x0[q]);
      if (MODE != 2) st4(S.x1_out + off, x1[q]);
      if (!BAL) st4(S.r_out + off, rv[q]);
    }
  }
  if (RED) tile::block_sum_store<kNT>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

template <int MODE, bool BAL, bool RED, int KD>
cudaError_t launch_t(const Geometry& g, const IterCoeffs& c, const TbPtrs& s, int n_sub, double* partials,
                     cudaStream_t st) {
  // one CTA per SM: the block pf_stride further runs on this SM in the next wave
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
      n_sm = 152;
  }
  prox_temporal_kernel<MODE, BAL, RED, KD>
      <<<temporal_num_ctas(g, KD), kNT, tb_smem_bytes<RED>(), st>>>(g, c, s, n_sub, n_sm, partials);
  return cudaGetLastError();
}

template <int MODE, bool BAL, int KD>
cudaError_t prepare_t() {
  cudaError_t e = cudaFuncSetAttribute(prox_temporal_kernel<MODE, BAL, false, KD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb_smem_bytes<false>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(prox_temporal_kernel<MODE, BAL, true, KD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tb_smem_bytes<true>());
  return e;
}

}  // namespace

int temporal_halo(int depth) { return depth <= 2 ? 2 : 4; }

int temporal_tile_rows(int depth) { return kEH - 2 * temporal_halo(depth); }

int temporal_num_ctas(const Geometry& g, int depth) {
  const int th = temporal_tile_rows(depth);
  const int ty = (g.H + th - 1) / th;
  const int tx = (g.Wp + kTW - 1) / kTW;
  return g.B * tx * ty;
}

cudaError_t prepare_prox_temporal(int mode, bool balanced, int depth) {
#define OTP_TBP(M, BL)                                                            \
  if (mode == M && balanced == BL)                                                \
    return temporal_halo(depth) == 2 ? prepare_t<M, BL, 2>() : prepare_t<M, BL, 4>();
  OTP_TBP(0, false)
  OTP_TBP(0, true)
  OTP_TBP(1, false)
  OTP_TBP(1, true)
  OTP_TBP(2, false)
  OTP_TBP(2, true)
#undef OTP_TBP
  return cudaErrorInvalidValue;
}

cudaError_t launch_prox_temporal(int mode, bool balanced, bool reduce, int depth, int n_sub, const Geometry& g,
                                 const IterCoeffs& c, const TbPtrs& s, double* partials, cudaStream_t st) {
  if (n_sub < 1 || n_sub > temporal_halo(depth)) return cudaErrorInvalidValue;
  Geometry gt = g;
  gt.tiles_x = (g.Wp + kTW - 1) / kTW;
  gt.tiles_y = (g.H + temporal_tile_rows(depth) - 1) / temporal_tile_rows(depth);
#define OTP_TB(M, BL, KD)                                                                                    \
  if (mode == M && balanced == BL && temporal_halo(depth) == KD)                                             \
    return reduce ? launch_t<M, BL, true, KD>(gt, c, s, n_sub, partials, st)                                 \
                  : launch_t<M, BL, false, KD>(gt, c, s, n_sub, partials, st);
  OTP_TB(0, false, 2)
  OTP_TB(0, false, 4)
  OTP_TB(0, true, 2)
  OTP_TB(0, true, 4)
  OTP_TB(1, false, 2)
  OTP_TB(1, false, 4)
  OTP_TB(1, true, 2)
  OTP_TB(1, true, 4)
  OTP_TB(2, false, 2)
  OTP_TB(2, false, 4)
  OTP_TB(2, true, 2)
  OTP_TB(2, true, 4)
#undef OTP_TB
  return cudaErrorInvalidValue;
}

}  // namespace otp
