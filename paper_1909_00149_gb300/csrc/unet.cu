// The learned warm start: a 4-level convolutional U-Net that maps a frame
// pair (p0, p1) to the fields of a converged Algorithm 1 state (Mx, My, r, a),
// used to warm-start the solver (Sec. III-B warm-starts the iterates from a
// cache; the network predicts that cache for a new pair).  The plain
// iterations then always run to the stopping rule.
//
// Architecture, C = 32 base channels (3x3 convolutions zero-padded, each
// followed by ReLU; 2x2 average pooling down, nearest-neighbour 2x
// upsampling up, each skip concatenated after the upsampled channels):
//   enc0 2->C->C | enc1 C->2C->2C | enc2 2C->4C->4C | bott 4C->8C->8C
//   dec2 [up(8C), s2]->4C->4C | dec1 [up(4C), s1]->2C->2C | dec0 [up(2C), s0]->C->C
//   head C->4 (1x1, no ReLU)
//
// Precision: weights BF16 (FP32 master copy for Adam), every product
// accumulated in FP32, every stored activation and activation gradient
// rounded to BF16 (round to nearest even), stored NHWC.  The network input,
// its output, the loss gradient and the weight gradients stay FP32.
//
// The thirteen inner 3x3 convolutions, forward and data gradient, run on the
// tensor cores as implicit GEMMs (M = 128 pixels of a 16 x 8 tile, N = the
// CTA's output channels, K = 9 offsets x input channels):
//   warp 0 (one lane): TMA loads, per K step, one 18 x 8-pixel halo box of
//     32 input channels (64-byte rows, 64-byte swizzle) and the three weight
//     boxes of the offsets (u, v) sharing its column shift v; the row shift u
//     is a start-address offset of u x 8 rows (one 512-byte swizzle atom);
//   warp 1 (one lane): tcgen05.mma into one FP32 accumulator in tensor memory;
//   warps 2-5: bias, ReLU or the ReLU mask of the gradient, BF16 rounding and
//     TMA tile stores (the concatenated output of a data gradient is split
//     between two tensors by channel).
// The data gradient is the same kernel with the weights transposed and
// flipped.  enc0a (2 input channels), the 1x1 head and the weight gradients
// are CUDA-core kernels; the weight gradients sum over pixel ranges in a
// fixed order (no atomics), so training is deterministic.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/otprox.h"
#include "device_util.cuh"
#include "otprox_internal.cuh"
#include "tc_util.cuh"

using namespace otp;
using bf16 = __nv_bfloat16;

namespace {
using namespace otp::tc;

constexpr int kBase = 32;                                 // base channels C
constexpr int kTH = 16, kTW = 8;                          // tensor-core output tile: 128 pixels
constexpr int kKC = 32;                                   // input channels per K step (64-byte rows)
constexpr uint32_t kABytes = (kTH + 2) * kTW * kKC * 2;   // halo box, 18 x 8 pixels x 32 channels
constexpr int kConvThreads = 192;
constexpr uint32_t kStgBytes = 32 * kKC * 2;              // a warp's store box: 4 x 8 pixels x 32 channels
constexpr int kMaxStages = 8;

struct ConvMaps {
  CUtensorMap inA, inB, w, outA, outB;
};

struct ConvArgs {
  int ca, cb;            // channels of the two input tensors (cb = 0: one input)
  int co_total;          // output channels of the convolution (weight rows per offset)
  int n_out;             // output channels per CTA (multiple of 32, <= 256)
  int split;             // output channels [0, split) -> outA, [split, co_total) -> outB
  int H, W, tiles_x, tiles_y, n_img;
  int relu, nstages;
  uint32_t tmem_cols;
  const float* bias;     // may be null
  const bf16* maskA;     // zero output channel c < split where maskA[pixel][c] <= 0 (may be null)
  int mca;
  const bf16* maskB;     // the same for c >= split against maskB[pixel][c - split]
  int mcb;
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ void unpack8(uint4 u, float (&f)[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    f[2 * e] = bf_lo(w[e]);
    f[2 * e + 1] = bf_hi(w[e]);
  }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  return make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
}

// ---------------------------------------------------------------- tensor-core 3x3 convolution
// Persistent: CTA x walks the tiles x, x + gridDim.x, ...; the stage ring runs
// on across tiles, and two TMEM accumulators let the epilogue of one tile
// overlap the MMAs of the next.
__global__ void __launch_bounds__(kConvThreads, 1)
conv3x3_tc_kernel(const __grid_constant__ ConvMaps M, const ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (s_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t bbytes = (uint32_t)a.n_out * (kKC * 2);
  const uint32_t sb = kABytes + 3 * bbytes;
  const int NS = a.nstages;
  unsigned char* stg = smem + (size_t)NS * sb;               // 4 warps x 2 store boxes
  __shared__ __align__(8) uint64_t full[kMaxStages], freef[kMaxStages], tfull[2], tfree[2], drain;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = a.n_img * a.tiles_x * a.tiles_y;
  const int nmine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int co0 = (int)blockIdx.y * a.n_out;
  const int nsteps = 3 * ((a.ca + a.cb) / kKC);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      bar_init(s_u32(&full[s]), 1);
      bar_init(s_u32(&freef[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(s_u32(&tfull[b]), 1);
      bar_init(s_u32(&tfree[b]), 4);
    }
    bar_init(s_u32(&drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(s_u32(&s_tmem), a.tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {   // producer: per tile, step t = (32-channel chunk t / 3, column shift v = t % 3)
      long long issued = 0;
      for (int i = 0; i < nmine && ok; ++i) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        const int txi = tile % a.tiles_x, rest = tile / a.tiles_x;
        const int x0 = txi * kTW, y0 = (rest % a.tiles_y) * kTH, img = rest / a.tiles_y;
        for (int t = 0; t < nsteps; ++t) {
          const long long gs = (long long)i * nsteps + t;
          const int s = (int)(gs % NS);
          if (gs >= NS && !bar_wait(s_u32(&freef[s]), (uint32_t)((gs / NS - 1) & 1))) { ok = false; break; }
          const int c = (t / 3) * kKC, v = t % 3;
          const uint32_t base = s_u32(smem + (size_t)s * sb), fb = s_u32(&full[s]);
          bar_expect(fb, sb);
          if (c < a.ca) tma4d(base, &M.inA, c, x0 + v - 1, y0 - 1, img, fb);
          else tma4d(base, &M.inB, c - a.ca, x0 + v - 1, y0 - 1, img, fb);
#pragma unroll
          for (int u = 0; u < 3; ++u)
            tma2d(base + kABytes + u * bbytes, &M.w, c, (u * 3 + v) * a.co_total + co0, fb);
          issued = gs + 1;
        }
      }
      // copies still in flight land before the CTA's shared memory goes away
      for (long long gs = issued - NS < 0 ? 0 : issued - NS; gs < issued; ++gs)
        (void)bar_wait(s_u32(&full[gs % NS]), (uint32_t)((gs / NS) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      const uint32_t idesc = bf16_idesc(128, a.n_out);
      for (int i = 0; i < nmine && ok; ++i) {
        const int b = i & 1;
        // the epilogue of tile i - 2 has read accumulator b
        if (i >= 2 && !bar_wait(s_u32(&tfree[b]), (uint32_t)(((i >> 1) - 1) & 1))) { ok = false; break; }
        fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)b * (a.tmem_cols / 2);
        for (int t = 0; t < nsteps; ++t) {
          const long long gs = (long long)i * nsteps + t;
          const int s = (int)(gs % NS);
          if (!bar_wait(s_u32(&full[s]), (uint32_t)((gs / NS) & 1))) { ok = false; break; }
          fence_after_sync();
          const uint32_t base = s_u32(smem + (size_t)s * sb);
#pragma unroll
          for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)   // K = 16 per instruction: 32 bytes along the row
              mma_bf16(acc, sw64_desc(base + u * 512 + kk * 32), sw64_desc(base + kABytes + u * bbytes + kk * 32),
                       idesc, (t > 0 || u > 0 || kk > 0) ? 1u : 0u);
          mma_commit(s_u32(&freef[s]));
        }
        if (ok) mma_commit(s_u32(&tfull[b]));
      }
      // every MMA issued above completes before the tensor memory is released
      mma_commit(s_u32(&drain));
      (void)bar_wait(s_u32(&drain), 0);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 q ... + 31 (q = w % 4) = pixel rows 4q ... 4q + 3 of the tile
    const int q = warp & 3;
    unsigned char* my = stg + (size_t)q * 2 * kStgBytes;
    int buf = 0;
    for (int i = 0; i < nmine && ok; ++i) {
      const int b = i & 1;
      if (!bar_wait(s_u32(&tfull[b]), (uint32_t)((i >> 1) & 1))) { ok = false; break; }
      fence_after_sync();
      const int tile = (int)blockIdx.x + i * (int)gridDim.x;
      const int txi = tile % a.tiles_x, rest = tile / a.tiles_x;
      const int x0 = txi * kTW, y0 = (rest % a.tiles_y) * kTH, img = rest / a.tiles_y;
      const int ty = 4 * q + (lane >> 3), tx = lane & 7;
      const int py = y0 + ty, px = x0 + tx;
      const bool inside = py < a.H && px < a.W;
      const long long pix = ((long long)img * a.H + py) * a.W + px;
      const bool box_live = y0 + 4 * q < a.H;   // warp-uniform
#pragma unroll 1
      for (int g = 0; g < a.n_out / 32; ++g) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * (a.tmem_cols / 2) + (uint32_t)(32 * g), v);
        const int c = co0 + 32 * g;
        if (a.bias) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += __ldg(a.bias + c + j);
        }
        if (a.relu) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
        }
        const bf16* mk = nullptr;
        if (c < a.split) {
          if (a.maskA) mk = a.maskA + pix * a.mca + c;
        } else if (a.maskB) {
          mk = a.maskB + pix * a.mcb + (c - a.split);
        }
        if (mk && inside) {
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            float f[8];
            unpack8(__ldg(reinterpret_cast<const uint4*>(mk) + c4), f);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (!(f[e] > 0.f)) v[8 * c4 + e] = 0.f;
          }
        }
        unsigned char* box = my + buf * kStgBytes;
        if (lane == 0) bulk_wait_read<1>();   // the store that last used this box has read it
        __syncwarp();
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {      // row lane, 16-byte chunk c4, 64-byte swizzle
          const uint4 w4 = make_uint4(pack_bf16(v[8 * c4], v[8 * c4 + 1]), pack_bf16(v[8 * c4 + 2], v[8 * c4 + 3]),
                                      pack_bf16(v[8 * c4 + 4], v[8 * c4 + 5]), pack_bf16(v[8 * c4 + 6], v[8 * c4 + 7]));
          *reinterpret_cast<uint4*>(box + lane * 64 + ((c4 ^ ((lane >> 1) & 3)) << 4)) = w4;
        }
        fence_async_shared();
        __syncwarp();
        if (lane == 0 && box_live) {   // pixels beyond the image are clipped by the store
          if (c < a.split) tma_store4d(&M.outA, s_u32(box), c, x0, y0 + 4 * q, img);
          else tma_store4d(&M.outB, s_u32(box), c - a.split, x0, y0 + 4 * q, img);
          bulk_commit();
        }
        buf ^= 1;
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) bar_arrive(s_u32(&tfree[b]));   // accumulator b may be overwritten
    }
    if (lane == 0) bulk_wait_all();   // the stores complete before the CTA exits
  }
  if (!ok) atomicExch(a.err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---------------------------------------------------------------- CUDA-core layers
// enc0a: x FP32 [n][2][H][W] -> y = bf16(ReLU(conv + b)) NHWC [n][H][W][C];
// w [C][2][3][3] BF16.  One thread per pixel.
__global__ void __launch_bounds__(256) conv_in_kernel(const float* __restrict__ x, long long total, int H, int W,
                                                      const bf16* __restrict__ w, const float* __restrict__ bias,
                                                      bf16* __restrict__ y) {
  __shared__ float s_w[18][kBase];
  __shared__ float s_b[kBase];
  for (int e = threadIdx.x; e < 18 * kBase; e += blockDim.x) s_w[e % 18][e / 18] = __bfloat162float(w[e]);
  if (threadIdx.x < kBase) s_b[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const long long hw = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / hw;
    const int r = (int)((i / W) % H), q = (int)(i % W);
    float in[18];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const int yy = r + u - 1, xx = q + v - 1;
          in[c * 9 + u * 3 + v] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? x[(n * 2 + c) * hw + (long long)yy * W + xx] : 0.f;
        }
    uint4* dst = reinterpret_cast<uint4*>(y + i * kBase);
#pragma unroll
    for (int g = 0; g < kBase / 8; ++g) {
      float o8[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float acc = s_b[8 * g + e];
#pragma unroll
        for (int ck = 0; ck < 18; ++ck) acc = fmaf(s_w[ck][8 * g + e], in[ck], acc);
        o8[e] = fmaxf(acc, 0.f);
      }
      dst[g] = pack8(o8);
    }
  }
}

// head: out FP32 [n][4][H][W] = b + w [4][C] . d0 (NHWC BF16).
__global__ void __launch_bounds__(256) head_fwd_kernel(const bf16* __restrict__ d0, long long total, long long hw,
                                                       const bf16* __restrict__ w, const float* __restrict__ bias,
                                                       float* __restrict__ out) {
  __shared__ float s_w[4][kBase];
  for (int e = threadIdx.x; e < 4 * kBase; e += blockDim.x) s_w[e / kBase][e % kBase] = __bfloat162float(w[e]);
  __syncthreads();
  const float b0 = bias[0], b1 = bias[1], b2 = bias[2], b3 = bias[3];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / hw, p = i % hw;
    float acc[4] = {b0, b1, b2, b3};
    const uint4* src = reinterpret_cast<const uint4*>(d0 + i * kBase);
#pragma unroll
    for (int g = 0; g < kBase / 8; ++g) {
      float f[8];
      unpack8(__ldg(src + g), f);
#pragma unroll
      for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[o] = fmaf(s_w[o][8 * g + e], f[e], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) out[(n * 4 + o) * hw + p] = acc[o];
  }
}

// head data gradient: g_d0 = bf16(1[d0 > 0] w^T g_out), NHWC.
__global__ void __launch_bounds__(256) head_dgrad_kernel(const float* __restrict__ gout, const bf16* __restrict__ d0,
                                                         long long total, long long hw, const bf16* __restrict__ w,
                                                         bf16* __restrict__ gd0) {
  __shared__ float s_w[4][kBase];
  for (int e = threadIdx.x; e < 4 * kBase; e += blockDim.x) s_w[e / kBase][e % kBase] = __bfloat162float(w[e]);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / hw, p = i % hw;
    float g[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) g[o] = gout[(n * 4 + o) * hw + p];
    const uint4* m = reinterpret_cast<const uint4*>(d0 + i * kBase);
    uint4* dst = reinterpret_cast<uint4*>(gd0 + i * kBase);
#pragma unroll
    for (int gg = 0; gg < kBase / 8; ++gg) {
      float f[8], o8[8];
      unpack8(__ldg(m + gg), f);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = 8 * gg + e;
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < 4; ++o) acc = fmaf(s_w[o][c], g[o], acc);
        o8[e] = f[e] > 0.f ? acc : 0.f;
      }
      dst[gg] = pack8(o8);
    }
  }
}

// Weight and bias gradients of one convolution:
//   gw[o][c][u][v] = sum_{n, p} gy[n][p][o] x[n][p + (u, v) - P][c],  gb[o] = sum gy[n][p][o].
// x: FP32 NCHW (XF32, the network input) or BF16 NHWC, the channel
// concatenation of xa (ca) and xb (cb); gy: FP32 NCHW (GF32, the head) or
// BF16 NHWC.  A CTA owns 16 output and 8 input channels and the contiguous
// range [z U / S, (z + 1) U / S) of the U = N x tiles 16 x 16-pixel tiles
// (z = blockIdx.z of S) and writes its partial sums to
// ws[z][co * ci * KS^2 + co] (biases by the CTAs with blockIdx.y == 0);
// wgrad_reduce_kernel adds the S partials in order.
constexpr int kCT = 16;    // pixel tile edge of the weight gradient
constexpr int kCO = 16;    // output channels per CTA
constexpr int kCI = 8;     // input channels per CTA
constexpr int kMaxSplits = 256;

template <int KS, bool XF32, bool GF32>
__global__ void __launch_bounds__(kCT* kCT)
wgrad_kernel(const void* __restrict__ xa, int ca, const void* __restrict__ xb, int cb, int N, int H, int W,
             const void* __restrict__ gy, int co, float* __restrict__ ws) {
  constexpr int P = (KS - 1) / 2;
  constexpr int TE = kCT + 2 * P;
  constexpr int NOUT = kCO * kCI * KS * KS;
  constexpr int PER = (NOUT + kCT * kCT - 1) / (kCT * kCT);
  __shared__ float s_x[kCI][TE][TE + 1];
  __shared__ float s_g[kCO][kCT * kCT + 1];
  const int o0 = blockIdx.x * kCO, c0 = blockIdx.y * kCI;
  const int ci_total = ca + cb;
  const long long hw = (long long)H * W;
  const int tiles_x = (W + kCT - 1) / kCT, tiles = tiles_x * ((H + kCT - 1) / kCT);
  const long long units = (long long)N * tiles;
  const long long u_begin = units * blockIdx.z / gridDim.z, u_end = units * (blockIdx.z + 1) / gridDim.z;
  float acc[PER];
  float accb = 0.f;
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  for (long long unit = u_begin; unit < u_end; ++unit) {
    const int n = (int)(unit / tiles), t = (int)(unit % tiles);
    const int x0 = (t % tiles_x) * kCT, y0 = (t / tiles_x) * kCT;
    for (int e = threadIdx.x; e < kCI * TE * TE; e += kCT * kCT) {   // channel fastest: NHWC rows
      const int c = e % kCI, pp = e / kCI, r = pp / TE, q = pp % TE;
      const int gc = c0 + c, yy = y0 + r - P, xx = x0 + q - P;
      float v = 0.f;
      if (gc < ci_total && yy >= 0 && yy < H && xx >= 0 && xx < W) {
        const long long pix = ((long long)n * H + yy) * W + xx;
        if (XF32) v = static_cast<const float*>(xa)[((long long)n * ca + gc) * hw + (long long)yy * W + xx];
        else if (gc < ca) v = __bfloat162float(static_cast<const bf16*>(xa)[pix * ca + gc]);
        else v = __bfloat162float(static_cast<const bf16*>(xb)[pix * cb + gc - ca]);
      }
      s_x[c][r][q] = v;
    }
    for (int e = threadIdx.x; e < kCO * kCT * kCT; e += kCT * kCT) {
      const int o = e % kCO, p = e / kCO;
      const int go = o0 + o, yy = y0 + p / kCT, xx = x0 + p % kCT;
      float v = 0.f;
      if (go < co && yy < H && xx < W) {
        if (GF32) v = static_cast<const float*>(gy)[((long long)n * co + go) * hw + (long long)yy * W + xx];
        else v = __bfloat162float(static_cast<const bf16*>(gy)[(((long long)n * H + yy) * W + xx) * co + go]);
      }
      s_g[o][p] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * kCT * kCT;
      if (idx < NOUT) {
        const int o = idx / (kCI * KS * KS), r = idx % (kCI * KS * KS);
        const int c = r / (KS * KS), u = (r % (KS * KS)) / KS, v = r % KS;
        float s = 0.f;
        for (int p = 0; p < kCT * kCT; ++p) s = fmaf(s_g[o][p], s_x[c][p / kCT + u][p % kCT + v], s);
        acc[q] += s;
      }
    }
    if (blockIdx.y == 0 && threadIdx.x < kCO) {
      float s = 0.f;
      for (int p = 0; p < kCT * kCT; ++p) s += s_g[threadIdx.x][p];
      accb += s;
    }
    __syncthreads();
  }
  const long long stride = (long long)co * ci_total * KS * KS + co;
  float* out = ws + blockIdx.z * stride;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * kCT * kCT;
    if (idx < NOUT) {
      const int o = idx / (kCI * KS * KS), r = idx % (kCI * KS * KS);
      const int c = r / (KS * KS), k = r % (KS * KS);
      if (o0 + o < co && c0 + c < ci_total) out[((long long)(o0 + o) * ci_total + c0 + c) * KS * KS + k] = acc[q];
    }
  }
  if (blockIdx.y == 0 && threadIdx.x < kCO && o0 + threadIdx.x < co)
    out[(long long)co * ci_total * KS * KS + o0 + threadIdx.x] = accb;
}

// g[i] = sum_{z < S} ws[z][i] in order of z (a layer's weights and biases
// are contiguous in the flat parameter layout, as in ws); the bias entries
// (i >= nweights) are reported as 0 when the network is trained bias-free.
__global__ void wgrad_reduce_kernel(const float* __restrict__ ws, int S, long long stride, long long nweights,
                                    int bias_free, float* __restrict__ g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += ws[z * stride + i];
    g[i] = (bias_free && i >= nweights) ? 0.f : s;
  }
}

// ---------------------------------------------------------------- pooling, upsampling (NHWC BF16, 8 channels a thread)
// y[n][r][q] = bf16(average of x's 2 x 2 block); x [n][2h][2w][C].
__global__ void pool_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, long long n_img, int h, int w, int C) {
  const int cv = C / 8;
  const long long total = n_img * h * w * cv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % cv);
    const long long pix = i / cv;
    const long long n = pix / ((long long)h * w);
    const int r = (int)((pix / w) % h), q = (int)(pix % w);
    const uint4* s = reinterpret_cast<const uint4*>(x + ((n * 2 * h + 2 * r) * 2 * w + 2 * q) * C) + g;
    const long long row = (long long)2 * w * cv;
    float a[8], b[8], c[8], d[8], o[8];
    unpack8(__ldg(s), a);
    unpack8(__ldg(s + cv), b);
    unpack8(__ldg(s + row), c);
    unpack8(__ldg(s + row + cv), d);
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = 0.25f * ((a[e] + b[e]) + (c[e] + d[e]));
    reinterpret_cast<uint4*>(y)[i] = pack8(o);
  }
}

// g_s[n][R][Q] = bf16(g_s + 1[s > 0] g_p[n][R/2][Q/2] / 4): the pooled
// path's gradient added to the skip's (both masked by the ReLU of s).
__global__ void pool_grad_kernel(const bf16* __restrict__ gp, const bf16* __restrict__ s, bf16* __restrict__ gs,
                                 long long n_img, int H, int W, int C) {
  const int cv = C / 8;
  const long long total = n_img * H * W * cv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % cv);
    const long long pix = i / cv;
    const long long n = pix / ((long long)H * W);
    const int r = (int)((pix / W) % H), q = (int)(pix % W);
    float p[8], m[8], a[8], o[8];
    unpack8(__ldg(reinterpret_cast<const uint4*>(gp + ((n * (H / 2) + r / 2) * (W / 2) + q / 2) * C) + g), p);
    unpack8(__ldg(reinterpret_cast<const uint4*>(s) + i), m);
    unpack8(reinterpret_cast<const uint4*>(gs)[i], a);
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = m[e] > 0.f ? a[e] + 0.25f * p[e] : 0.f;
    reinterpret_cast<uint4*>(gs)[i] = pack8(o);
  }
}

// y [n][2h][2w][C] = x [n][h][w][C] at the parent pixel.
__global__ void up_kernel(const bf16* __restrict__ x, bf16* __restrict__ y, long long n_img, int h, int w, int C) {
  const int cv = C / 8;
  const long long total = n_img * 4 * h * w * cv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % cv);
    const long long pix = i / cv;
    const long long n = pix / (4LL * h * w);
    const int r = (int)((pix / (2 * w)) % (2 * h)), q = (int)(pix % (2 * w));
    reinterpret_cast<uint4*>(y)[i] = __ldg(reinterpret_cast<const uint4*>(x + ((n * h + r / 2) * w + q / 2) * C) + g);
  }
}

// its gradient: g_x [n][h][w] = bf16(sum of g_y's 2 x 2 block).
__global__ void up_grad_kernel(const bf16* __restrict__ gy, bf16* __restrict__ gx, long long n_img, int h, int w, int C) {
  const int cv = C / 8;
  const long long total = n_img * h * w * cv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i % cv);
    const long long pix = i / cv;
    const long long n = pix / ((long long)h * w);
    const int r = (int)((pix / w) % h), q = (int)(pix % w);
    const uint4* s = reinterpret_cast<const uint4*>(gy + ((n * 2 * h + 2 * r) * 2 * w + 2 * q) * C) + g;
    const long long row = (long long)2 * w * cv;
    float a[8], b[8], c[8], d[8], o[8];
    unpack8(__ldg(s), a);
    unpack8(__ldg(s + cv), b);
    unpack8(__ldg(s + row), c);
    unpack8(__ldg(s + row + cv), d);
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = (a[e] + b[e]) + (c[e] + d[e]);
    reinterpret_cast<uint4*>(gx)[i] = pack8(o);
  }
}

// ---------------------------------------------------------------- loss, optimiser
// MSE: g = 2 (y - t) / n, partial sums of (y - t)^2 in slot 0.
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                  float* __restrict__ g, long long n, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const float s = 2.f / (float)n;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float d = y[i] - t[i];
    acc[0] = fmaf(d, d, acc[0]);
    g[i] = s * d;
  }
  block_sums_to<256>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

struct LayerDev {
  long long w_off, b_off;   // into the flat parameter array
  long long wb_off;         // into the BF16 weight arrays
  int ci, co, ks;
};

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 copies of the FP32 master weights w [co][ci][k]: wb as stored (the
// CUDA-core layers), wf [k][co][ci] (the tensor-core forward) and
// wd [8 - k][ci][co] (transposed and flipped: the data gradient).
__global__ void bf16_refresh_kernel(const float* __restrict__ p, const LayerDev* __restrict__ L,
                                    bf16* __restrict__ wb, bf16* __restrict__ wf, bf16* __restrict__ wd) {
  const LayerDev d = L[blockIdx.y];
  const int kk = d.ks * d.ks;
  const long long n = (long long)d.co * d.ci * kk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const bf16 v = __float2bfloat16_rn(p[d.w_off + i]);
    const long long o = i / ((long long)d.ci * kk), c = (i / kk) % d.ci, k = i % kk;
    wb[d.wb_off + i] = v;
    wf[d.wb_off + (k * d.co + o) * d.ci + c] = v;
    wd[d.wb_off + ((kk - 1 - k) * d.ci + c) * d.co + o] = v;
  }
}

int grid_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

}  // namespace

#define OT_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

namespace {

// BF16 NHWC activation buffers and their gradients (level l: H >> l x W >> l)
enum Buf {
  E0A, S0, P0, E1A, S1, P1, E2A, S2, P2, BTA, BT, U2, D2A, D2, U1, D1A, D1, U0, D0A, D0,
  G_D0, G_D0A, G_U0, G_S0, G_D1, G_D1A, G_U1, G_S1, G_D2, G_D2A, G_U2, G_S2, G_BT, G_BTA, G_P2, G_E2A, G_P1,
  G_E1A, G_P0, G_E0A, NBUF
};
// channels (in units of C) and level of each buffer
constexpr int kBufC[NBUF] = {1, 1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1,
                             1, 1, 2, 1, 2, 2, 4, 2, 4, 4, 8, 4, 8, 8, 4, 4, 2, 2, 1, 1};
constexpr int kBufL[NBUF] = {0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0,
                             0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 2, 2, 1, 1, 0};
// FP32 NCHW buffers
enum FBuf { X_IN, OUT, G_OUT, TARGET, NFBUF };

struct Act {
  bf16* p;
  int C, level;
  CUtensorMap ld, st;   // TMA maps: 18 x 8-pixel halo loads, 4 x 8-pixel stores
};

}  // namespace

struct ot_unet {
  int H, W, maxN, C;
  cudaStream_t stream;
  std::vector<LayerDev> L;      // 15 convolutions in forward order
  long long nparams, nw;
  float *p, *g, *m, *v;         // flat FP32 parameters, gradients, Adam moments
  bf16 *wb, *wf, *wd;           // BF16 weights in the three layouts
  LayerDev* dL;
  CUtensorMap wf_map[15], wd_map[15];
  int nf_out[15], nd_out[15];
  bf16* act_slab;              // forward activations
  float* f_slab;                // input, output
  bf16* grad_slab;              // activation gradients (allocated by the first gradient call)
  float* gf_slab;               // loss gradient, target
  bool bwd;
  int bias_free;                // 1: bias gradients are 0 (biases keep their values)
  Act A[NBUF];
  float* F[NFBUF];
  float* ws;                    // weight-gradient partials
  double* partials;
  double* dsums;
  double* hsums;
  int* derr;
  int* herr;
  int nb_loss;
  long long step;
};

namespace {

int level_h(const ot_unet* h, int l) { return h->H >> l; }
int level_w(const ot_unet* h, int l) { return h->W >> l; }

int encode_bf16(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int encode_act(Act& a, int maxN, int Hl, int Wl) {
  const cuuint64_t dims[4] = {(cuuint64_t)a.C, (cuuint64_t)Wl, (cuuint64_t)Hl, (cuuint64_t)maxN};
  const cuuint64_t strides[3] = {(cuuint64_t)a.C * 2, (cuuint64_t)Wl * a.C * 2, (cuuint64_t)Hl * Wl * a.C * 2};
  const cuuint32_t box_ld[4] = {(cuuint32_t)kKC, (cuuint32_t)kTW, (cuuint32_t)(kTH + 2), 1};
  const cuuint32_t box_st[4] = {(cuuint32_t)kKC, (cuuint32_t)kTW, 4, 1};
  if (encode_bf16(&a.ld, a.p, 4, dims, strides, box_ld)) return -1;
  return encode_bf16(&a.st, a.p, 4, dims, strides, box_st);
}

// weights [9 * rows][cols] BF16, box 32 columns x n_out rows
int encode_weights(CUtensorMap* m, const bf16* base, int rows, int cols, int n_out) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)9 * rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)n_out};
  return encode_bf16(m, base, 2, dims, strides, box);
}

// output channels per CTA for a convolution with co output channels
int n_out_for(int co) { return co <= 256 ? co : co / 2; }

uint32_t conv_smem(int n_out, int* stages) {
  const uint32_t sb = kABytes + 3u * (uint32_t)n_out * kKC * 2;
  const uint32_t stg = 4 * 2 * kStgBytes;
  const uint32_t budget = n_out <= 64 ? 112u * 1024 : 220u * 1024;   // two CTAs per SM for the narrow layers
  int ns = (int)((budget - stg - 1024) / sb);
  ns = ns < 2 ? 2 : (ns > kMaxStages ? kMaxStages : ns);
  *stages = ns;
  return 1024 + (uint32_t)ns * sb + stg;
}

// a tensor-core 3x3 convolution over n images at the inputs' level
cudaError_t conv_tc(ot_unet* h, const Act& inA, const Act* inB, const CUtensorMap& wmap, int co_total, int n_out,
                    const Act& outA, const Act* outB, int split, int n, const float* bias, bool relu, const Act* maskA,
                    const Act* maskB) {
  static unsigned long long attr = 0;
  if (needs_setup(attr)) {
    const cudaError_t e =
        cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
    if (e != cudaSuccess) return e;
    mark_setup(attr);
  }
  ConvMaps M;
  M.inA = inA.ld;
  M.inB = inB ? inB->ld : inA.ld;
  M.w = wmap;
  M.outA = outA.st;
  M.outB = outB ? outB->st : outA.st;
  ConvArgs a;
  a.ca = inA.C;
  a.cb = inB ? inB->C : 0;
  a.co_total = co_total;
  a.n_out = n_out;
  a.split = split;
  a.H = level_h(h, inA.level);
  a.W = level_w(h, inA.level);
  a.tiles_x = (a.W + kTW - 1) / kTW;
  a.tiles_y = (a.H + kTH - 1) / kTH;
  a.relu = relu ? 1 : 0;
  const uint32_t smem = conv_smem(n_out, &a.nstages);
  // two accumulators, each at a power-of-two column offset of at least n_out
  a.tmem_cols = n_out <= 16 ? 32u : n_out <= 32 ? 64u : n_out <= 64 ? 128u : n_out <= 128 ? 256u : 512u;
  a.n_img = n;
  a.bias = bias;
  a.maskA = maskA ? maskA->p : nullptr;
  a.mca = maskA ? maskA->C : 0;
  a.maskB = maskB ? maskB->p : nullptr;
  a.mcb = maskB ? maskB->C : 0;
  a.err = h->derr;
  // persistent: as many CTAs as fit at once (two per SM for the narrow layers)
  const int gy = co_total / n_out, ntiles = n * a.tiles_x * a.tiles_y;
  int gx = (n_out <= 64 ? 2 * 152 : 152) / gy;
  gx = gx < 1 ? 1 : (gx > ntiles ? ntiles : gx);
  conv3x3_tc_kernel<<<dim3((unsigned)gx, (unsigned)gy), kConvThreads, smem, h->stream>>>(M, a);
  return cudaGetLastError();
}

const float* bias_of(const ot_unet* h, int l) { return h->p + h->L[l].b_off; }

// forward of inner layer l: inputs inA (+ inB concatenated), output out
cudaError_t fwd(ot_unet* h, int l, int inA, int inB, int out, int n) {
  return conv_tc(h, h->A[inA], inB >= 0 ? &h->A[inB] : nullptr, h->wf_map[l], h->L[l].co, h->nf_out[l], h->A[out],
                 nullptr, h->L[l].co, n, bias_of(h, l), true, nullptr, nullptr);
}

// data gradient of inner layer l from gy: outputs outA (+ outB for a
// concatenated input), masked by the ReLU of the layer's inputs mA / mB (-1: none)
cudaError_t dgrad(ot_unet* h, int l, int gy, int outA, int outB, int mA, int mB, int n) {
  const int split = h->A[outA].C;
  return conv_tc(h, h->A[gy], nullptr, h->wd_map[l], h->L[l].ci, h->nd_out[l], h->A[outA],
                 outB >= 0 ? &h->A[outB] : nullptr, split, n, nullptr, false, mA >= 0 ? &h->A[mA] : nullptr,
                 mB >= 0 ? &h->A[mB] : nullptr);
}

int wgrad_splits(const LayerDev& d, int n, int Hh, int Ww) {
  const long long units = (long long)n * ((Ww + kCT - 1) / kCT) * ((Hh + kCT - 1) / kCT);
  const long long ctas = (long long)((d.co + kCO - 1) / kCO) * ((d.ci + kCI - 1) / kCI);
  long long s = (2 * 152 + ctas - 1) / ctas;
  if (s > units) s = units;
  if (s > kMaxSplits) s = kMaxSplits;
  return (int)(s < 1 ? 1 : s);
}

// weight gradient of layer l; x / gy given as raw pointers with their layouts
template <int KS, bool XF32, bool GF32>
cudaError_t wgrad_raw(ot_unet* h, int l, const void* xa, int ca, const void* xb, int cb, const void* gy, int n,
                      int level) {
  const LayerDev& d = h->L[l];
  const int Hh = level_h(h, level), Ww = level_w(h, level);
  const int S = wgrad_splits(d, n, Hh, Ww);
  const dim3 grid((d.co + kCO - 1) / kCO, (d.ci + kCI - 1) / kCI, S);
  wgrad_kernel<KS, XF32, GF32><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, n, Hh, Ww, gy, d.co, h->ws);
  const long long nweights = (long long)d.co * d.ci * d.ks * d.ks;
  wgrad_reduce_kernel<<<grid_for(nweights + d.co), 256, 0, h->stream>>>(h->ws, S, nweights + d.co, nweights,
                                                                        h->bias_free, h->g + d.w_off);
  return cudaGetLastError();
}

cudaError_t wgrad(ot_unet* h, int l, int xA, int xB, int gy, int n) {
  const Act& a = h->A[xA];
  return wgrad_raw<3, false, false>(h, l, a.p, a.C, xB >= 0 ? h->A[xB].p : nullptr, xB >= 0 ? h->A[xB].C : 0,
                                    h->A[gy].p, n, a.level);
}

#define UCHK(x)                         \
  do {                                  \
    cudaError_t e__ = (x);              \
    if (e__ != cudaSuccess) return e__; \
  } while (0)

cudaError_t pool(ot_unet* h, int src, int dst, int n) {
  const Act& d = h->A[dst];
  const int hh = level_h(h, d.level), ww = level_w(h, d.level);
  pool_kernel<<<grid_for((long long)n * hh * ww * d.C / 8), 256, 0, h->stream>>>(h->A[src].p, d.p, n, hh, ww, d.C);
  return cudaGetLastError();
}
cudaError_t up(ot_unet* h, int src, int dst, int n) {
  const Act& s = h->A[src];
  const int hh = level_h(h, s.level), ww = level_w(h, s.level);
  up_kernel<<<grid_for((long long)n * 4 * hh * ww * s.C / 8), 256, 0, h->stream>>>(s.p, h->A[dst].p, n, hh, ww, s.C);
  return cudaGetLastError();
}
cudaError_t up_grad(ot_unet* h, int src, int dst, int n) {
  const Act& d = h->A[dst];
  const int hh = level_h(h, d.level), ww = level_w(h, d.level);
  up_grad_kernel<<<grid_for((long long)n * hh * ww * d.C / 8), 256, 0, h->stream>>>(h->A[src].p, d.p, n, hh, ww, d.C);
  return cudaGetLastError();
}
cudaError_t pool_grad(ot_unet* h, int gp, int s, int gs, int n) {
  const Act& d = h->A[gs];
  const int H = level_h(h, d.level), W = level_w(h, d.level);
  pool_grad_kernel<<<grid_for((long long)n * H * W * d.C / 8), 256, 0, h->stream>>>(h->A[gp].p, h->A[s].p, d.p, n, H,
                                                                                    W, d.C);
  return cudaGetLastError();
}

cudaError_t forward(ot_unet* h, int n) {
  const long long hw = (long long)h->H * h->W;
  conv_in_kernel<<<grid_for(n * hw), 256, 0, h->stream>>>(h->F[X_IN], n * hw, h->H, h->W, h->wb + h->L[0].wb_off,
                                                          bias_of(h, 0), h->A[E0A].p);
  UCHK(cudaGetLastError());
  UCHK(fwd(h, 1, E0A, -1, S0, n));
  UCHK(pool(h, S0, P0, n));
  UCHK(fwd(h, 2, P0, -1, E1A, n));
  UCHK(fwd(h, 3, E1A, -1, S1, n));
  UCHK(pool(h, S1, P1, n));
  UCHK(fwd(h, 4, P1, -1, E2A, n));
  UCHK(fwd(h, 5, E2A, -1, S2, n));
  UCHK(pool(h, S2, P2, n));
  UCHK(fwd(h, 6, P2, -1, BTA, n));
  UCHK(fwd(h, 7, BTA, -1, BT, n));
  UCHK(up(h, BT, U2, n));
  UCHK(fwd(h, 8, U2, S2, D2A, n));
  UCHK(fwd(h, 9, D2A, -1, D2, n));
  UCHK(up(h, D2, U1, n));
  UCHK(fwd(h, 10, U1, S1, D1A, n));
  UCHK(fwd(h, 11, D1A, -1, D1, n));
  UCHK(up(h, D1, U0, n));
  UCHK(fwd(h, 12, U0, S0, D0A, n));
  UCHK(fwd(h, 13, D0A, -1, D0, n));
  head_fwd_kernel<<<grid_for(n * hw), 256, 0, h->stream>>>(h->A[D0].p, n * hw, hw, h->wb + h->L[14].wb_off,
                                                           bias_of(h, 14), h->F[OUT]);
  return cudaGetLastError();
}

// gradients of the MSE loss for the current batch into h->g (loss sums into partials)
cudaError_t backward(ot_unet* h, int n) {
  const long long hw = (long long)h->H * h->W;
  const long long nout = n * 4 * hw;
  h->nb_loss = grid_for(nout);
  mse_kernel<<<h->nb_loss, 256, 0, h->stream>>>(h->F[OUT], h->F[TARGET], h->F[G_OUT], nout, h->partials);
  // head (1 x 1)
  UCHK((wgrad_raw<1, false, true>(h, 14, h->A[D0].p, h->C, nullptr, 0, h->F[G_OUT], n, 0)));
  head_dgrad_kernel<<<grid_for(n * hw), 256, 0, h->stream>>>(h->F[G_OUT], h->A[D0].p, n * hw, hw,
                                                             h->wb + h->L[14].wb_off, h->A[G_D0].p);
  // decoder
  UCHK(wgrad(h, 13, D0A, -1, G_D0, n));
  UCHK(dgrad(h, 13, G_D0, G_D0A, -1, D0A, -1, n));
  UCHK(wgrad(h, 12, U0, S0, G_D0A, n));
  UCHK(dgrad(h, 12, G_D0A, G_U0, G_S0, U0, S0, n));
  UCHK(up_grad(h, G_U0, G_D1, n));
  UCHK(wgrad(h, 11, D1A, -1, G_D1, n));
  UCHK(dgrad(h, 11, G_D1, G_D1A, -1, D1A, -1, n));
  UCHK(wgrad(h, 10, U1, S1, G_D1A, n));
  UCHK(dgrad(h, 10, G_D1A, G_U1, G_S1, U1, S1, n));
  UCHK(up_grad(h, G_U1, G_D2, n));
  UCHK(wgrad(h, 9, D2A, -1, G_D2, n));
  UCHK(dgrad(h, 9, G_D2, G_D2A, -1, D2A, -1, n));
  UCHK(wgrad(h, 8, U2, S2, G_D2A, n));
  UCHK(dgrad(h, 8, G_D2A, G_U2, G_S2, U2, S2, n));
  UCHK(up_grad(h, G_U2, G_BT, n));
  // bottleneck
  UCHK(wgrad(h, 7, BTA, -1, G_BT, n));
  UCHK(dgrad(h, 7, G_BT, G_BTA, -1, BTA, -1, n));
  UCHK(wgrad(h, 6, P2, -1, G_BTA, n));
  UCHK(dgrad(h, 6, G_BTA, G_P2, -1, -1, -1, n));
  // encoder: the skip's gradient gains the pooled path's
  UCHK(pool_grad(h, G_P2, S2, G_S2, n));
  UCHK(wgrad(h, 5, E2A, -1, G_S2, n));
  UCHK(dgrad(h, 5, G_S2, G_E2A, -1, E2A, -1, n));
  UCHK(wgrad(h, 4, P1, -1, G_E2A, n));
  UCHK(dgrad(h, 4, G_E2A, G_P1, -1, -1, -1, n));
  UCHK(pool_grad(h, G_P1, S1, G_S1, n));
  UCHK(wgrad(h, 3, E1A, -1, G_S1, n));
  UCHK(dgrad(h, 3, G_S1, G_E1A, -1, E1A, -1, n));
  UCHK(wgrad(h, 2, P0, -1, G_E1A, n));
  UCHK(dgrad(h, 2, G_E1A, G_P0, -1, -1, -1, n));
  UCHK(pool_grad(h, G_P0, S0, G_S0, n));
  UCHK(wgrad(h, 1, E0A, -1, G_S0, n));
  UCHK(dgrad(h, 1, G_S0, G_E0A, -1, E0A, -1, n));
  UCHK((wgrad_raw<3, true, false>(h, 0, h->F[X_IN], 2, nullptr, 0, h->A[G_E0A].p, n, 0)));
  return cudaGetLastError();
}

cudaError_t refresh_bf16(ot_unet* h) {
  const dim3 grid(64, (unsigned)h->L.size());
  bf16_refresh_kernel<<<grid, 256, 0, h->stream>>>(h->p, h->dL, h->wb, h->wf, h->wd);
  return cudaGetLastError();
}

// a bounded wait inside a tensor-core kernel gave up: OT_ETIMEOUT (flag cleared)
int check_err(ot_unet* h, const char* what) {
  OT_CUDA(cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), what);
  OT_CUDA(cudaStreamSynchronize(h->stream), what);
  if (*h->herr) {
    *h->herr = 0;
    OT_CUDA(cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream), what);
    return fail(OT_ETIMEOUT, "%s: a bounded wait in the tensor-core convolution expired", what);
  }
  return OT_OK;
}

int read_loss(ot_unet* h, double* loss, long long count) {
  OT_CUDA(launch_finalize_sums(h->partials, h->nb_loss, h->dsums, h->stream), "unet: loss");
  OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "unet: loss copy");
  const int rc = check_err(h, "unet: gradients");
  if (rc != OT_OK) return rc;
  if (loss) *loss = h->hsums[0] / (double)count;
  if (!isfinite(h->hsums[0])) return fail(OT_ENONFINITE, "unet: non-finite loss");
  return OT_OK;
}

// Allocate (zeroed) and map the BF16 buffers [b0, b1) and the FP32 buffers
// [f0, f1) for max_batch images, one slab each.
int alloc_buffers(ot_unet* h, int b0, int b1, int f0, int f1, bf16** slab, float** fslab) {
  const long long hw = (long long)h->H * h->W;
  const int fch[NFBUF] = {2, 4, 4, 4};
  long long act = 0, fl = 0;
  for (int b = b0; b < b1; ++b)
    act += ((long long)h->maxN * (h->H >> kBufL[b]) * (h->W >> kBufL[b]) * kBufC[b] * h->C + 63) / 64 * 64;
  for (int b = f0; b < f1; ++b) fl += ((long long)h->maxN * fch[b] * hw + 63) / 64 * 64;
  cudaError_t e = cudaMalloc(slab, (size_t)act * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(fslab, (size_t)fl * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(*slab, 0, (size_t)act * sizeof(bf16), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(*fslab, 0, (size_t)fl * sizeof(float), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "unet: activation buffers");
  bf16* q = *slab;
  for (int b = b0; b < b1; ++b) {
    Act& a = h->A[b];
    a.p = q;
    a.C = kBufC[b] * h->C;
    a.level = kBufL[b];
    q += ((long long)h->maxN * (h->H >> a.level) * (h->W >> a.level) * a.C + 63) / 64 * 64;
    if (encode_act(a, h->maxN, h->H >> a.level, h->W >> a.level))
      return fail(OT_ECUDA, "unet: tensor map of an activation buffer");
  }
  float* fq = *fslab;
  for (int b = f0; b < f1; ++b) {
    h->F[b] = fq;
    fq += ((long long)h->maxN * fch[b] * hw + 63) / 64 * 64;
  }
  return OT_OK;
}

// The gradient buffers and the weight-gradient workspace, on first use.
int ensure_backward(ot_unet* h) {
  if (h->bwd) return OT_OK;
  int rc = alloc_buffers(h, G_D0, NBUF, G_OUT, NFBUF, &h->grad_slab, &h->gf_slab);
  if (rc != OT_OK) return rc;
  long long ws = 0;   // the largest split count any layer can take times that layer's size
  for (const LayerDev& d : h->L) {
    const long long ctas = (long long)((d.co + kCO - 1) / kCO) * ((d.ci + kCI - 1) / kCI);
    long long sp = (2 * 152 + ctas - 1) / ctas;
    if (sp > kMaxSplits) sp = kMaxSplits;
    const long long need = sp * ((long long)d.co * d.ci * d.ks * d.ks + d.co);
    if (need > ws) ws = need;
  }
  const cudaError_t e = cudaMalloc(&h->ws, (size_t)ws * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "unet: weight-gradient workspace");
  h->bwd = true;
  return OT_OK;
}

}  // namespace

extern "C" {

int ot_unet_destroy(ot_unet_t h) {
  if (!h) return OT_OK;
  cudaFree(h->p);
  cudaFree(h->wb);
  cudaFree(h->dL);
  cudaFree(h->act_slab);
  cudaFree(h->f_slab);
  cudaFree(h->grad_slab);
  cudaFree(h->gf_slab);
  cudaFree(h->partials);
  cudaFree(h->ws);
  cudaFree(h->derr);
  if (h->hsums) cudaFreeHost(h->hsums);
  if (h->herr) cudaFreeHost(h->herr);
  delete h;
  return OT_OK;
}

int ot_unet_create(int32_t H, int32_t W, int32_t max_batch, int32_t base_channels, void* cuda_stream, ot_unet_t* out) {
  if (!out) return fail(OT_EINVAL, "ot_unet_create: NULL out");
  *out = nullptr;
  if (H < 8 || W < 8 || H % 8 || W % 8) return fail(OT_EINVAL, "ot_unet_create: H and W must be multiples of 8");
  if (max_batch < 1) return fail(OT_EINVAL, "ot_unet_create: max_batch must be >= 1");
  if (base_channels != kBase) return fail(OT_EINVAL, "ot_unet_create: base_channels must be %d", kBase);
  ot_unet* h = new ot_unet();
  h->H = H;
  h->W = W;
  h->maxN = max_batch;
  h->C = base_channels;
  h->stream = (cudaStream_t)cuda_stream;
  const int C = base_channels;
  const int spec[15][3] = {{2, C, 3},          {C, C, 3},         {C, 2 * C, 3},     {2 * C, 2 * C, 3},
                           {2 * C, 4 * C, 3},  {4 * C, 4 * C, 3}, {4 * C, 8 * C, 3}, {8 * C, 8 * C, 3},
                           {12 * C, 4 * C, 3}, {4 * C, 4 * C, 3}, {6 * C, 2 * C, 3}, {2 * C, 2 * C, 3},
                           {3 * C, C, 3},      {C, C, 3},         {C, 4, 1}};
  long long off = 0, wboff = 0;
  for (auto& sp : spec) {
    LayerDev d;
    d.ci = sp[0];
    d.co = sp[1];
    d.ks = sp[2];
    d.w_off = off;
    off += (long long)d.co * d.ci * d.ks * d.ks;
    d.b_off = off;
    off += d.co;
    d.wb_off = wboff;
    wboff += (long long)d.co * d.ci * d.ks * d.ks;
    h->L.push_back(d);
  }
  h->nparams = off;
  h->nw = wboff;
  cudaError_t e = cudaMalloc(&h->p, 4 * (size_t)off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->wb, 3 * (size_t)wboff * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&h->dL, h->L.size() * sizeof(LayerDev));
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, ((size_t)152 * 8 + 1) * kNumSums * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hsums, kNumSums * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&h->herr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, 4 * (size_t)off * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->wb, 0, 3 * (size_t)wboff * sizeof(bf16), h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->dL, h->L.data(), h->L.size() * sizeof(LayerDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) {
    ot_unet_destroy(h);
    return cuda_fail(e, "ot_unet_create: allocation");
  }
  *h->herr = 0;
  h->g = h->p + off;
  h->m = h->g + off;
  h->v = h->m + off;
  h->wf = h->wb + wboff;
  h->wd = h->wf + wboff;
  h->dsums = h->partials + (size_t)152 * 8 * kNumSums;
  const int rc = alloc_buffers(h, 0, G_D0, X_IN, G_OUT, &h->act_slab, &h->f_slab);
  if (rc != OT_OK) {
    ot_unet_destroy(h);
    return rc;
  }
  for (int l = 1; l <= 13; ++l) {
    const LayerDev& d = h->L[l];
    h->nf_out[l] = n_out_for(d.co);
    h->nd_out[l] = n_out_for(d.ci);
    if (encode_weights(&h->wf_map[l], h->wf + d.wb_off, d.co, d.ci, h->nf_out[l]) ||
        encode_weights(&h->wd_map[l], h->wd + d.wb_off, d.ci, d.co, h->nd_out[l])) {
      ot_unet_destroy(h);
      return fail(OT_ECUDA, "ot_unet_create: tensor map of a weight array");
    }
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ot_unet_destroy(h);
    return cuda_fail(e, "ot_unet_create: sync");
  }
  *out = h;
  return OT_OK;
}

int64_t ot_unet_param_count(ot_unet_t h) {
  if (!h) return fail(OT_EINVAL, "ot_unet_param_count: NULL handle");
  return h->nparams;
}

int ot_unet_set_params(ot_unet_t h, const float* params) {
  if (!h || !params) return fail(OT_EINVAL, "ot_unet_set_params: NULL argument");
  OT_CUDA(cudaMemcpyAsync(h->p, params, (size_t)h->nparams * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_set_params");
  OT_CUDA(cudaMemsetAsync(h->m, 0, 2 * (size_t)h->nparams * sizeof(float), h->stream), "ot_unet_set_params");
  h->step = 0;
  OT_CUDA(refresh_bf16(h), "ot_unet_set_params: BF16 weights");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_unet_set_params: sync");
  return OT_OK;
}

int ot_unet_get_params(ot_unet_t h, float* params) {
  if (!h || !params) return fail(OT_EINVAL, "ot_unet_get_params: NULL argument");
  OT_CUDA(cudaMemcpyAsync(params, h->p, (size_t)h->nparams * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_get_params");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_unet_get_params: sync");
  return OT_OK;
}

int ot_unet_set_bias_free(ot_unet_t h, int32_t bias_free) {
  if (!h) return fail(OT_EINVAL, "ot_unet_set_bias_free: NULL handle");
  h->bias_free = bias_free ? 1 : 0;
  return OT_OK;
}

int ot_unet_forward(ot_unet_t h, const float* x, float* y, int32_t n) {
  if (!h || !x || !y) return fail(OT_EINVAL, "ot_unet_forward: NULL argument");
  if (n < 1 || n > h->maxN) return fail(OT_EINVAL, "ot_unet_forward: batch must be in [1, %d]", h->maxN);
  const long long hw = (long long)h->H * h->W;
  OT_CUDA(cudaMemcpyAsync(h->F[X_IN], x, (size_t)n * 2 * hw * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_forward: input");
  OT_CUDA(forward(h, n), "ot_unet_forward");
  OT_CUDA(cudaMemcpyAsync(y, h->F[OUT], (size_t)n * 4 * hw * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_forward: output");
  return check_err(h, "ot_unet_forward");
}

int ot_unet_gradients(ot_unet_t h, const float* x, const float* target, int32_t n, float* grads, double* loss) {
  if (!h || !x || !target) return fail(OT_EINVAL, "ot_unet_gradients: NULL argument");
  if (n < 1 || n > h->maxN) return fail(OT_EINVAL, "ot_unet_gradients: batch must be in [1, %d]", h->maxN);
  const int rc = ensure_backward(h);
  if (rc != OT_OK) return rc;
  const long long hw = (long long)h->H * h->W;
  OT_CUDA(cudaMemcpyAsync(h->F[X_IN], x, (size_t)n * 2 * hw * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_gradients: input");
  OT_CUDA(cudaMemcpyAsync(h->F[TARGET], target, (size_t)n * 4 * hw * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_gradients: target");
  OT_CUDA(forward(h, n), "ot_unet_gradients: forward");
  OT_CUDA(backward(h, n), "ot_unet_gradients: backward");
  if (grads)
    OT_CUDA(cudaMemcpyAsync(grads, h->g, (size_t)h->nparams * sizeof(float), cudaMemcpyDefault, h->stream),
            "ot_unet_gradients: copy");
  return read_loss(h, loss, (long long)n * 4 * hw);
}

int ot_unet_train_step(ot_unet_t h, const float* x, const float* target, int32_t n, float lr, double* loss) {
  int rc = ot_unet_gradients(h, x, target, n, nullptr, loss);
  if (rc != OT_OK) return rc;
  h->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)h->step)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)h->step)));
  adam_kernel<<<grid_for(h->nparams), 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->nparams, lr, b1, b2, 1e-8f, c1, c2);
  OT_CUDA(cudaGetLastError(), "ot_unet_train_step: Adam");
  OT_CUDA(refresh_bf16(h), "ot_unet_train_step: BF16 weights");
  return OT_OK;
}

}  // extern "C"
