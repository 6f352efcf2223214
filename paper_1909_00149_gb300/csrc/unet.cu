// The learned warm start: a 4-level convolutional U-Net (base C channels)
// that maps a frame pair (p0, p1) to the fields of a converged Algorithm 1
// state (Mx, My, r, a), used to warm-start the solver (Sec. III-B caches and
// warm-starts the iterates; the network predicts that cache for a new pair).
// The plain iterations then always run to the stopping rule.
//
// Architecture (3x3 convolutions zero-padded, each followed by ReLU; 2x2
// average pooling down, nearest-neighbour 2x upsampling up, each skip
// concatenated after the upsampled tensor's channels):
//   enc0 2->C->C | enc1 C->2C->2C | enc2 2C->4C->4C | bott 4C->8C->8C
//   dec2 [up(8C), s2]->4C->4C | dec1 [up(4C), s1]->2C->2C | dec0 [up(2C), s0]->C->C
//   head C->4 (1x1, no ReLU)
// Tensors are [N][C][H][W] FP32; weights are BF16 (an FP32 master copy is
// kept for the optimiser), every product is accumulated in FP32.
//
// Kernels: one direct convolution (a CTA computes 16 x 16 pixels x 16
// output channels of one image, input channels staged 8 at a time with
// their halo in shared memory) serves the forward pass and the data
// gradient (the latter with the weights transposed and flipped); a second
// kernel computes weight and bias gradients (a CTA owns 16 output x 8 input
// channels and sums over every pixel and image in a fixed order: no atomics,
// deterministic); plus pooling, upsampling, the ReLU mask, the MSE loss and
// Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/otprox.h"
#include "device_util.cuh"
#include "otprox_internal.cuh"

using namespace otp;

namespace {

constexpr int kCT = 16;    // pixel tile edge
constexpr int kCO = 16;    // output channels per CTA
constexpr int kCI = 8;     // input channels staged per step
constexpr int kMaxSplits = 256;  // pixel-range splits of a weight-gradient launch

// y = conv(x, w) (+ b) (, ReLU).  x is the channel concatenation of xa (ca
// channels) and xb (cb channels, may be null); y's channels [0, split) go to
// ya and [split, co) to yb (data gradients of a concatenation).  w:
// [co][ca + cb][KS][KS] BF16.
template <int KS, bool RELU>
__global__ void __launch_bounds__(kCT* kCT)
conv_kernel(const float* __restrict__ xa, int ca, const float* __restrict__ xb, int cb, int H, int W,
            const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias, float* __restrict__ ya,
            float* __restrict__ yb, int co, int split) {
  constexpr int P = (KS - 1) / 2;
  constexpr int TE = kCT + 2 * P;
  __shared__ float s_x[kCI][TE][TE + 1];
  __shared__ __align__(16) float s_w[kCI * KS * KS][kCO];
  const int tx = threadIdx.x % kCT, ty = threadIdx.x / kCT;
  const int tiles_x = (W + kCT - 1) / kCT;
  const int x0 = (blockIdx.x % tiles_x) * kCT, y0 = (blockIdx.x / tiles_x) * kCT;
  const int o0 = blockIdx.y * kCO, n = blockIdx.z;
  const int ci_total = ca + cb;
  const long long hw = (long long)H * W;
  float acc[kCO];
#pragma unroll
  for (int o = 0; o < kCO; ++o) acc[o] = 0.f;
  for (int c0 = 0; c0 < ci_total; c0 += kCI) {
    for (int e = threadIdx.x; e < kCI * TE * TE; e += kCT * kCT) {
      const int c = e / (TE * TE), r = (e / TE) % TE, q = e % TE;
      const int gc = c0 + c, gy = y0 + r - P, gx = x0 + q - P;
      float v = 0.f;
      if (gc < ci_total && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        const float* src = gc < ca ? xa + ((long long)n * ca + gc) * hw : xb + ((long long)n * cb + (gc - ca)) * hw;
        v = src[(long long)gy * W + gx];
      }
      s_x[c][r][q] = v;
    }
    for (int e = threadIdx.x; e < kCI * KS * KS * kCO; e += kCT * kCT) {
      const int o = e % kCO, ck = e / kCO;               // ck = c * KS*KS + k
      const int c = ck / (KS * KS), k = ck % (KS * KS);
      const int go = o0 + o, gc = c0 + c;
      s_w[ck][o] = (go < co && gc < ci_total) ? __bfloat162float(w[((long long)go * ci_total + gc) * KS * KS + k]) : 0.f;
    }
    __syncthreads();
#pragma unroll 2
    for (int c = 0; c < kCI; ++c) {
#pragma unroll
      for (int u = 0; u < KS; ++u)
#pragma unroll
        for (int v = 0; v < KS; ++v) {
          const float xv = s_x[c][ty + u][tx + v];
          const float* wr = &s_w[c * KS * KS + u * KS + v][0];
#pragma unroll
          for (int o = 0; o < kCO; o += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wr + o);
            acc[o] = fmaf(w4.x, xv, acc[o]);
            acc[o + 1] = fmaf(w4.y, xv, acc[o + 1]);
            acc[o + 2] = fmaf(w4.z, xv, acc[o + 2]);
            acc[o + 3] = fmaf(w4.w, xv, acc[o + 3]);
          }
        }
    }
    __syncthreads();
  }
  const int gy = y0 + ty, gx = x0 + tx;
  if (gy >= H || gx >= W) return;
#pragma unroll
  for (int o = 0; o < kCO; ++o) {
    const int go = o0 + o;
    if (go >= co) break;
    float v = acc[o] + (bias ? bias[go] : 0.f);
    if (RELU) v = fmaxf(v, 0.f);
    float* dst = go < split ? ya + ((long long)n * split + go) * hw : yb + ((long long)n * (co - split) + (go - split)) * hw;
    dst[(long long)gy * W + gx] = v;
  }
}

// gw[o][c][u][v] = sum_{n, pixels} gy[n][o][p] x[n][c][p + (u, v) - P] and
// gb[o] = sum gy[n][o][p].  A CTA owns 16 output and 8 input channels and
// the contiguous range [z U / S, (z + 1) U / S) of the U = N x tiles pixel
// tiles (z = blockIdx.z of S); it writes its partial sums to
// ws[z][co * ci * KS^2 + co] (biases by the CTAs with blockIdx.y == 0), and
// wgrad_reduce_kernel adds the S partials in order: deterministic.
template <int KS>
__global__ void __launch_bounds__(kCT* kCT)
conv_wgrad_kernel(const float* __restrict__ xa, int ca, const float* __restrict__ xb, int cb, int N, int H, int W,
                  const float* __restrict__ gy, int co, float* __restrict__ ws) {
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
    for (int e = threadIdx.x; e < kCI * TE * TE; e += kCT * kCT) {
      const int c = e / (TE * TE), r = (e / TE) % TE, q = e % TE;
      const int gc = c0 + c, yy = y0 + r - P, xx = x0 + q - P;
      float v = 0.f;
      if (gc < ci_total && yy >= 0 && yy < H && xx >= 0 && xx < W) {
        const float* src = gc < ca ? xa + ((long long)n * ca + gc) * hw : xb + ((long long)n * cb + (gc - ca)) * hw;
        v = src[(long long)yy * W + xx];
      }
      s_x[c][r][q] = v;
    }
    for (int e = threadIdx.x; e < kCO * kCT * kCT; e += kCT * kCT) {
      const int o = e / (kCT * kCT), p = e % (kCT * kCT);
      const int go = o0 + o, yy = y0 + p / kCT, xx = x0 + p % kCT;
      s_g[o][p] = (go < co && yy < H && xx < W) ? gy[((long long)n * co + go) * hw + (long long)yy * W + xx] : 0.f;
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

// g[i] = sum_{z < S} ws[z][i] in order of z; the weights and the biases of a
// layer are contiguous in the flat parameter layout, as in ws.
__global__ void wgrad_reduce_kernel(const float* __restrict__ ws, int S, long long stride, float* __restrict__ g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < stride; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += ws[z * stride + i];
    g[i] = s;
  }
}

__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(y[i] > 0.f)) g[i] = 0.f;
}

// [NC][H][W] -> [NC][H/2][W/2] average
__global__ void pool_kernel(const float* __restrict__ x, float* __restrict__ y, long long nc, int H, int W) {
  const int h = H / 2, w = W / 2;
  const long long total = nc * h * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / ((long long)h * w);
    const int r = (int)((i / w) % h), q = (int)(i % w);
    const float* s = x + c * H * W + (long long)(2 * r) * W + 2 * q;
    y[i] = 0.25f * ((s[0] + s[1]) + (s[W] + s[W + 1]));
  }
}

// gradient of the average pool: g_x[2r+a][2q+b] (+)= g_y[r][q] / 4
__global__ void pool_grad_kernel(const float* __restrict__ gy, float* __restrict__ gx, long long nc, int H, int W,
                                 int accumulate) {
  const long long total = nc * H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / ((long long)H * W);
    const int r = (int)((i / W) % H), q = (int)(i % W);
    const float v = 0.25f * gy[c * (H / 2) * (W / 2) + (long long)(r / 2) * (W / 2) + q / 2];
    gx[i] = accumulate ? gx[i] + v : v;
  }
}

// nearest-neighbour 2x upsampling [NC][h][w] -> [NC][2h][2w]
__global__ void up_kernel(const float* __restrict__ x, float* __restrict__ y, long long nc, int h, int w) {
  const long long total = nc * 4 * h * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / (4LL * h * w);
    const int r = (int)((i / (2 * w)) % (2 * h)), q = (int)(i % (2 * w));
    y[i] = x[c * h * w + (long long)(r / 2) * w + q / 2];
  }
}

// its gradient: g_x[r][q] = sum of the 2x2 block of g_y
__global__ void up_grad_kernel(const float* __restrict__ gy, float* __restrict__ gx, long long nc, int h, int w) {
  const long long total = nc * h * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / ((long long)h * w);
    const int r = (int)((i / w) % h), q = (int)(i % w);
    const float* s = gy + c * 4 * h * w + (long long)(2 * r) * (2 * w) + 2 * q;
    gx[i] = (s[0] + s[1]) + (s[2 * w] + s[2 * w + 1]);
  }
}

// MSE: g = 2 (y - t) / n, partial sums of (y - t)^2 in slot 0
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ g,
                                                  long long n, double* __restrict__ partials) {
  float acc[kNumSums] = {};
  const float s = 2.f / (float)n;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float d = y[i] - t[i];
    acc[0] = fmaf(d, d, acc[0]);
    g[i] = s * d;
  }
  block_sums_to<256>(acc, partials + (size_t)blockIdx.x * kNumSums);
}

// Adam on the FP32 master weights; refreshes the BF16 copies (w as stored,
// and wT = transposed and spatially flipped, for the data gradient).
struct LayerDev {
  long long w_off, b_off;   // into the flat parameter array
  long long wb_off;         // into the BF16 arrays
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

__global__ void bf16_refresh_kernel(const float* __restrict__ p, const LayerDev* __restrict__ L, int nl,
                                    __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wtb) {
  const LayerDev d = L[blockIdx.y];
  const long long n = (long long)d.co * d.ci * d.ks * d.ks;
  const int kk = d.ks * d.ks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const __nv_bfloat16 v = __float2bfloat16_rn(p[d.w_off + i]);
    wb[d.wb_off + i] = v;
    const long long o = i / ((long long)d.ci * kk), c = (i / kk) % d.ci, k = i % kk;
    wtb[d.wb_off + (c * d.co + o) * kk + (kk - 1 - k)] = v;   // [ci][co][flipped k]
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

struct ot_unet {
  int H, W, maxN, C;
  cudaStream_t stream;
  std::vector<LayerDev> L;      // 15 convolutions in forward order
  long long nparams, nweights_bf;
  float *p, *g, *m, *v;         // flat FP32 parameters, gradients, Adam moments
  __nv_bfloat16 *wb, *wtb;      // BF16 weights and their transposed flipped copy
  LayerDev* dL;
  float* act;                   // activations and gradients (one slab)
  std::vector<float*> A;        // named buffers, see make_buffers
  float* ws;                    // weight-gradient partials [splits][layer weights + biases]
  double* partials;
  double* dsums;
  double* hsums;
  int nb_loss;
  long long step;
};

namespace {

enum Buf {
  X_IN, E0A, S0, P0, E1A, S1, P1, E2A, S2, P2, BTA, BT, U2, D2A, D2, U1, D1A, D1, U0, D0A, D0, OUT,
  G_OUT, G_D0, G_D0A, G_U0, G_S0, G_D1, G_D1A, G_U1, G_S1, G_D2, G_D2A, G_U2, G_S2, G_BT, G_BTA, G_P2, G_E2A,
  G_P1, G_E1A, G_P0, G_E0A, TARGET, NBUF
};

long long buf_elems(const ot_unet* h, int b) {
  const long long N = h->maxN, H = h->H, W = h->W, C = h->C;
  const long long l0 = H * W, l1 = l0 / 4, l2 = l1 / 4, l3 = l2 / 4;
  switch (b) {
    case X_IN: return N * 2 * l0;
    case E0A: case S0: case D0A: case D0: case G_D0: case G_D0A: case G_S0: case G_E0A: return N * C * l0;
    case P0: case G_P0: return N * C * l1;
    case E1A: case S1: case D1A: case D1: case G_D1: case G_D1A: case G_S1: case G_E1A: return N * 2 * C * l1;
    case P1: case G_P1: return N * 2 * C * l2;
    case E2A: case S2: case D2A: case D2: case G_D2: case G_D2A: case G_S2: case G_E2A: return N * 4 * C * l2;
    case P2: case G_P2: return N * 4 * C * l3;
    case BTA: case BT: case G_BT: case G_BTA: return N * 8 * C * l3;
    case U2: case G_U2: return N * 8 * C * l2;
    case U1: case G_U1: return N * 4 * C * l1;
    case U0: case G_U0: return N * 2 * C * l0;
    case OUT: case G_OUT: case TARGET: return N * 4 * l0;
  }
  return 0;
}

const __nv_bfloat16* wl(const ot_unet* h, int l) { return h->wb + h->L[l].wb_off; }
const __nv_bfloat16* wtl(const ot_unet* h, int l) { return h->wtb + h->L[l].wb_off; }
const float* bl(const ot_unet* h, int l) { return h->p + h->L[l].b_off; }

cudaError_t conv(const ot_unet* h, int l, const float* xa, int ca, const float* xb, int cb, int n, int Hh, int Ww,
                 float* y, bool relu) {
  const LayerDev& d = h->L[l];
  const dim3 grid(((Ww + kCT - 1) / kCT) * ((Hh + kCT - 1) / kCT), (d.co + kCO - 1) / kCO, n);
  if (d.ks == 3) {
    if (relu) conv_kernel<3, true><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, Hh, Ww, wl(h, l), bl(h, l), y, nullptr, d.co, d.co);
    else conv_kernel<3, false><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, Hh, Ww, wl(h, l), bl(h, l), y, nullptr, d.co, d.co);
  } else {
    conv_kernel<1, false><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, Hh, Ww, wl(h, l), bl(h, l), y, nullptr, d.co, d.co);
  }
  return cudaGetLastError();
}

// data gradient of layer l: gy (co channels) -> gx split into (ga: split, gb: rest)
cudaError_t conv_dgrad(const ot_unet* h, int l, const float* gy, int n, int Hh, int Ww, float* ga, float* gb, int split) {
  const LayerDev& d = h->L[l];
  const dim3 grid(((Ww + kCT - 1) / kCT) * ((Hh + kCT - 1) / kCT), (d.ci + kCO - 1) / kCO, n);
  if (d.ks == 3)
    conv_kernel<3, false><<<grid, kCT * kCT, 0, h->stream>>>(gy, d.co, nullptr, 0, Hh, Ww, wtl(h, l), nullptr, ga, gb, d.ci, split);
  else
    conv_kernel<1, false><<<grid, kCT * kCT, 0, h->stream>>>(gy, d.co, nullptr, 0, Hh, Ww, wtl(h, l), nullptr, ga, gb, d.ci, split);
  return cudaGetLastError();
}

// pixel-range splits of a weight-gradient launch: about two waves of CTAs
int wgrad_splits(const LayerDev& d, int n, int Hh, int Ww) {
  const long long units = (long long)n * ((Ww + kCT - 1) / kCT) * ((Hh + kCT - 1) / kCT);
  const long long ctas = (long long)((d.co + kCO - 1) / kCO) * ((d.ci + kCI - 1) / kCI);
  long long s = (2 * 152 + ctas - 1) / ctas;
  if (s > units) s = units;
  if (s > kMaxSplits) s = kMaxSplits;
  return (int)(s < 1 ? 1 : s);
}

cudaError_t conv_wgrad(const ot_unet* h, int l, const float* xa, int ca, const float* xb, int cb, const float* gy, int n,
                       int Hh, int Ww) {
  const LayerDev& d = h->L[l];
  const int S = wgrad_splits(d, n, Hh, Ww);
  const dim3 grid((d.co + kCO - 1) / kCO, (d.ci + kCI - 1) / kCI, S);
  if (d.ks == 3) conv_wgrad_kernel<3><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, n, Hh, Ww, gy, d.co, h->ws);
  else conv_wgrad_kernel<1><<<grid, kCT * kCT, 0, h->stream>>>(xa, ca, xb, cb, n, Hh, Ww, gy, d.co, h->ws);
  const long long stride = (long long)d.co * d.ci * d.ks * d.ks + d.co;
  wgrad_reduce_kernel<<<grid_for(stride), 256, 0, h->stream>>>(h->ws, S, stride, h->g + d.w_off);
  return cudaGetLastError();
}

cudaError_t relu_mask(const ot_unet* h, float* g, const float* y, long long n) {
  relu_mask_kernel<<<grid_for(n), 256, 0, h->stream>>>(g, y, n);
  return cudaGetLastError();
}

#define UCHK(x)                                \
  do {                                         \
    cudaError_t e__ = (x);                     \
    if (e__ != cudaSuccess) return e__;        \
  } while (0)

cudaError_t forward(ot_unet* h, int n) {
  auto& A = h->A;
  const int C = h->C, H0 = h->H, W0 = h->W, H1 = H0 / 2, W1 = W0 / 2, H2 = H1 / 2, W2 = W1 / 2, H3 = H2 / 2,
            W3 = W2 / 2;
  UCHK(conv(h, 0, A[X_IN], 2, nullptr, 0, n, H0, W0, A[E0A], true));
  UCHK(conv(h, 1, A[E0A], C, nullptr, 0, n, H0, W0, A[S0], true));
  pool_kernel<<<grid_for((long long)n * C * H1 * W1), 256, 0, h->stream>>>(A[S0], A[P0], (long long)n * C, H0, W0);
  UCHK(conv(h, 2, A[P0], C, nullptr, 0, n, H1, W1, A[E1A], true));
  UCHK(conv(h, 3, A[E1A], 2 * C, nullptr, 0, n, H1, W1, A[S1], true));
  pool_kernel<<<grid_for((long long)n * 2 * C * H2 * W2), 256, 0, h->stream>>>(A[S1], A[P1], (long long)n * 2 * C, H1, W1);
  UCHK(conv(h, 4, A[P1], 2 * C, nullptr, 0, n, H2, W2, A[E2A], true));
  UCHK(conv(h, 5, A[E2A], 4 * C, nullptr, 0, n, H2, W2, A[S2], true));
  pool_kernel<<<grid_for((long long)n * 4 * C * H3 * W3), 256, 0, h->stream>>>(A[S2], A[P2], (long long)n * 4 * C, H2, W2);
  UCHK(conv(h, 6, A[P2], 4 * C, nullptr, 0, n, H3, W3, A[BTA], true));
  UCHK(conv(h, 7, A[BTA], 8 * C, nullptr, 0, n, H3, W3, A[BT], true));
  up_kernel<<<grid_for((long long)n * 8 * C * H2 * W2), 256, 0, h->stream>>>(A[BT], A[U2], (long long)n * 8 * C, H3, W3);
  UCHK(conv(h, 8, A[U2], 8 * C, A[S2], 4 * C, n, H2, W2, A[D2A], true));
  UCHK(conv(h, 9, A[D2A], 4 * C, nullptr, 0, n, H2, W2, A[D2], true));
  up_kernel<<<grid_for((long long)n * 4 * C * H1 * W1), 256, 0, h->stream>>>(A[D2], A[U1], (long long)n * 4 * C, H2, W2);
  UCHK(conv(h, 10, A[U1], 4 * C, A[S1], 2 * C, n, H1, W1, A[D1A], true));
  UCHK(conv(h, 11, A[D1A], 2 * C, nullptr, 0, n, H1, W1, A[D1], true));
  up_kernel<<<grid_for((long long)n * 2 * C * H0 * W0), 256, 0, h->stream>>>(A[D1], A[U0], (long long)n * 2 * C, H1, W1);
  UCHK(conv(h, 12, A[U0], 2 * C, A[S0], C, n, H0, W0, A[D0A], true));
  UCHK(conv(h, 13, A[D0A], C, nullptr, 0, n, H0, W0, A[D0], true));
  UCHK(conv(h, 14, A[D0], C, nullptr, 0, n, H0, W0, A[OUT], false));
  return cudaGetLastError();
}

// gradients of the MSE loss for the current batch into h->g (loss sums into partials)
cudaError_t backward(ot_unet* h, int n) {
  auto& A = h->A;
  const int C = h->C, H0 = h->H, W0 = h->W, H1 = H0 / 2, W1 = W0 / 2, H2 = H1 / 2, W2 = W1 / 2, H3 = H2 / 2,
            W3 = W2 / 2;
  const long long nout = (long long)n * 4 * H0 * W0;
  h->nb_loss = grid_for(nout);
  mse_kernel<<<h->nb_loss, 256, 0, h->stream>>>(A[OUT], A[TARGET], A[G_OUT], nout, h->partials);
  // head
  UCHK(conv_wgrad(h, 14, A[D0], C, nullptr, 0, A[G_OUT], n, H0, W0));
  UCHK(conv_dgrad(h, 14, A[G_OUT], n, H0, W0, A[G_D0], nullptr, C));
  // dec0
  UCHK(relu_mask(h, A[G_D0], A[D0], (long long)n * C * H0 * W0));
  UCHK(conv_wgrad(h, 13, A[D0A], C, nullptr, 0, A[G_D0], n, H0, W0));
  UCHK(conv_dgrad(h, 13, A[G_D0], n, H0, W0, A[G_D0A], nullptr, C));
  UCHK(relu_mask(h, A[G_D0A], A[D0A], (long long)n * C * H0 * W0));
  UCHK(conv_wgrad(h, 12, A[U0], 2 * C, A[S0], C, A[G_D0A], n, H0, W0));
  UCHK(conv_dgrad(h, 12, A[G_D0A], n, H0, W0, A[G_U0], A[G_S0], 2 * C));
  up_grad_kernel<<<grid_for((long long)n * 2 * C * H1 * W1), 256, 0, h->stream>>>(A[G_U0], A[G_D1], (long long)n * 2 * C, H1, W1);
  // dec1
  UCHK(relu_mask(h, A[G_D1], A[D1], (long long)n * 2 * C * H1 * W1));
  UCHK(conv_wgrad(h, 11, A[D1A], 2 * C, nullptr, 0, A[G_D1], n, H1, W1));
  UCHK(conv_dgrad(h, 11, A[G_D1], n, H1, W1, A[G_D1A], nullptr, 2 * C));
  UCHK(relu_mask(h, A[G_D1A], A[D1A], (long long)n * 2 * C * H1 * W1));
  UCHK(conv_wgrad(h, 10, A[U1], 4 * C, A[S1], 2 * C, A[G_D1A], n, H1, W1));
  UCHK(conv_dgrad(h, 10, A[G_D1A], n, H1, W1, A[G_U1], A[G_S1], 4 * C));
  up_grad_kernel<<<grid_for((long long)n * 4 * C * H2 * W2), 256, 0, h->stream>>>(A[G_U1], A[G_D2], (long long)n * 4 * C, H2, W2);
  // dec2
  UCHK(relu_mask(h, A[G_D2], A[D2], (long long)n * 4 * C * H2 * W2));
  UCHK(conv_wgrad(h, 9, A[D2A], 4 * C, nullptr, 0, A[G_D2], n, H2, W2));
  UCHK(conv_dgrad(h, 9, A[G_D2], n, H2, W2, A[G_D2A], nullptr, 4 * C));
  UCHK(relu_mask(h, A[G_D2A], A[D2A], (long long)n * 4 * C * H2 * W2));
  UCHK(conv_wgrad(h, 8, A[U2], 8 * C, A[S2], 4 * C, A[G_D2A], n, H2, W2));
  UCHK(conv_dgrad(h, 8, A[G_D2A], n, H2, W2, A[G_U2], A[G_S2], 8 * C));
  up_grad_kernel<<<grid_for((long long)n * 8 * C * H3 * W3), 256, 0, h->stream>>>(A[G_U2], A[G_BT], (long long)n * 8 * C, H3, W3);
  // bottleneck
  UCHK(relu_mask(h, A[G_BT], A[BT], (long long)n * 8 * C * H3 * W3));
  UCHK(conv_wgrad(h, 7, A[BTA], 8 * C, nullptr, 0, A[G_BT], n, H3, W3));
  UCHK(conv_dgrad(h, 7, A[G_BT], n, H3, W3, A[G_BTA], nullptr, 8 * C));
  UCHK(relu_mask(h, A[G_BTA], A[BTA], (long long)n * 8 * C * H3 * W3));
  UCHK(conv_wgrad(h, 6, A[P2], 4 * C, nullptr, 0, A[G_BTA], n, H3, W3));
  UCHK(conv_dgrad(h, 6, A[G_BTA], n, H3, W3, A[G_P2], nullptr, 4 * C));
  // enc2: gradient of s2 = skip part + pooled path
  pool_grad_kernel<<<grid_for((long long)n * 4 * C * H2 * W2), 256, 0, h->stream>>>(A[G_P2], A[G_S2], (long long)n * 4 * C, H2, W2, 1);
  UCHK(relu_mask(h, A[G_S2], A[S2], (long long)n * 4 * C * H2 * W2));
  UCHK(conv_wgrad(h, 5, A[E2A], 4 * C, nullptr, 0, A[G_S2], n, H2, W2));
  UCHK(conv_dgrad(h, 5, A[G_S2], n, H2, W2, A[G_E2A], nullptr, 4 * C));
  UCHK(relu_mask(h, A[G_E2A], A[E2A], (long long)n * 4 * C * H2 * W2));
  UCHK(conv_wgrad(h, 4, A[P1], 2 * C, nullptr, 0, A[G_E2A], n, H2, W2));
  UCHK(conv_dgrad(h, 4, A[G_E2A], n, H2, W2, A[G_P1], nullptr, 2 * C));
  // enc1
  pool_grad_kernel<<<grid_for((long long)n * 2 * C * H1 * W1), 256, 0, h->stream>>>(A[G_P1], A[G_S1], (long long)n * 2 * C, H1, W1, 1);
  UCHK(relu_mask(h, A[G_S1], A[S1], (long long)n * 2 * C * H1 * W1));
  UCHK(conv_wgrad(h, 3, A[E1A], 2 * C, nullptr, 0, A[G_S1], n, H1, W1));
  UCHK(conv_dgrad(h, 3, A[G_S1], n, H1, W1, A[G_E1A], nullptr, 2 * C));
  UCHK(relu_mask(h, A[G_E1A], A[E1A], (long long)n * 2 * C * H1 * W1));
  UCHK(conv_wgrad(h, 2, A[P0], C, nullptr, 0, A[G_E1A], n, H1, W1));
  UCHK(conv_dgrad(h, 2, A[G_E1A], n, H1, W1, A[G_P0], nullptr, C));
  // enc0
  pool_grad_kernel<<<grid_for((long long)n * C * H0 * W0), 256, 0, h->stream>>>(A[G_P0], A[G_S0], (long long)n * C, H0, W0, 1);
  UCHK(relu_mask(h, A[G_S0], A[S0], (long long)n * C * H0 * W0));
  UCHK(conv_wgrad(h, 1, A[E0A], C, nullptr, 0, A[G_S0], n, H0, W0));
  UCHK(conv_dgrad(h, 1, A[G_S0], n, H0, W0, A[G_E0A], nullptr, C));
  UCHK(relu_mask(h, A[G_E0A], A[E0A], (long long)n * C * H0 * W0));
  UCHK(conv_wgrad(h, 0, A[X_IN], 2, nullptr, 0, A[G_E0A], n, H0, W0));
  return cudaGetLastError();
}

cudaError_t refresh_bf16(ot_unet* h) {
  const dim3 grid(64, (unsigned)h->L.size());
  bf16_refresh_kernel<<<grid, 256, 0, h->stream>>>(h->p, h->dL, (int)h->L.size(), h->wb, h->wtb);
  return cudaGetLastError();
}

int copy_batch(ot_unet* h, float* dst, const float* src, long long elems) {
  OT_CUDA(cudaMemcpyAsync(dst, src, elems * sizeof(float), cudaMemcpyDefault, h->stream), "unet: input copy");
  return OT_OK;
}

int read_loss(ot_unet* h, double* loss, long long count) {
  OT_CUDA(launch_finalize_sums(h->partials, h->nb_loss, h->dsums, h->stream), "unet: loss");
  OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "unet: loss copy");
  OT_CUDA(cudaStreamSynchronize(h->stream), "unet: sync");
  if (loss) *loss = h->hsums[0] / (double)count;
  if (!isfinite(h->hsums[0])) return fail(OT_ENONFINITE, "unet: non-finite loss");
  return OT_OK;
}

}  // namespace

extern "C" {

int ot_unet_destroy(ot_unet_t h) {
  if (!h) return OT_OK;
  cudaFree(h->p);
  cudaFree(h->wb);
  cudaFree(h->dL);
  cudaFree(h->act);
  cudaFree(h->partials);
  cudaFree(h->ws);
  if (h->hsums) cudaFreeHost(h->hsums);
  delete h;
  return OT_OK;
}

int ot_unet_create(int32_t H, int32_t W, int32_t max_batch, int32_t base_channels, void* cuda_stream, ot_unet_t* out) {
  if (!out) return fail(OT_EINVAL, "ot_unet_create: NULL out");
  *out = nullptr;
  if (H < 8 || W < 8 || H % 8 || W % 8) return fail(OT_EINVAL, "ot_unet_create: H and W must be multiples of 8");
  if (max_batch < 1 || base_channels < 1 || base_channels > 256)
    return fail(OT_EINVAL, "ot_unet_create: max_batch >= 1, base_channels in [1, 256]");
  ot_unet* h = new ot_unet();
  h->H = H;
  h->W = W;
  h->maxN = max_batch;
  h->C = base_channels;
  h->stream = (cudaStream_t)cuda_stream;
  const int C = base_channels;
  const int spec[15][3] = {{2, C, 3},      {C, C, 3},         {C, 2 * C, 3},     {2 * C, 2 * C, 3},
                           {2 * C, 4 * C, 3}, {4 * C, 4 * C, 3}, {4 * C, 8 * C, 3}, {8 * C, 8 * C, 3},
                           {12 * C, 4 * C, 3}, {4 * C, 4 * C, 3}, {6 * C, 2 * C, 3}, {2 * C, 2 * C, 3},
                           {3 * C, C, 3},     {C, C, 3},         {C, 4, 1}};
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
  h->nweights_bf = wboff;
  long long act = 0;
  for (int b = 0; b < NBUF; ++b) act += (buf_elems(h, b) + 63) / 64 * 64;
  cudaError_t e = cudaMalloc(&h->p, 4 * (size_t)off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->wb, 2 * (size_t)wboff * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&h->dL, h->L.size() * sizeof(LayerDev));
  if (e == cudaSuccess) e = cudaMalloc(&h->act, (size_t)act * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, ((size_t)152 * 8 + 1) * kNumSums * sizeof(double));
  // the largest split count any layer can take times that layer's size
  long long ws = 0;
  for (const LayerDev& d : h->L) {
    const long long ctas = (long long)((d.co + kCO - 1) / kCO) * ((d.ci + kCI - 1) / kCI);
    long long sp = (2 * 152 + ctas - 1) / ctas;
    if (sp > kMaxSplits) sp = kMaxSplits;
    const long long need = sp * ((long long)d.co * d.ci * d.ks * d.ks + d.co);
    if (need > ws) ws = need;
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->ws, (size_t)ws * sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hsums, kNumSums * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, 4 * (size_t)off * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->dL, h->L.data(), h->L.size() * sizeof(LayerDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->act, 0, (size_t)act * sizeof(float), h->stream);
  if (e != cudaSuccess) {
    ot_unet_destroy(h);
    return cuda_fail(e, "ot_unet_create: allocation");
  }
  h->g = h->p + off;
  h->m = h->g + off;
  h->v = h->m + off;
  h->wtb = h->wb + wboff;
  h->dsums = h->partials + (size_t)152 * 8 * kNumSums;
  float* q = h->act;
  h->A.resize(NBUF);
  for (int b = 0; b < NBUF; ++b) {
    h->A[b] = q;
    q += (buf_elems(h, b) + 63) / 64 * 64;
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ot_unet_destroy(h);
    return cuda_fail(e, "ot_unet_create: sync");
  }
  *out = h;
  return OT_OK;
}

int64_t ot_unet_param_count(ot_unet_t h) { return h ? h->nparams : -1; }

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

int ot_unet_forward(ot_unet_t h, const float* x, float* y, int32_t n) {
  if (!h || !x || !y) return fail(OT_EINVAL, "ot_unet_forward: NULL argument");
  if (n < 1 || n > h->maxN) return fail(OT_EINVAL, "ot_unet_forward: batch must be in [1, %d]", h->maxN);
  const long long hw = (long long)h->H * h->W;
  int rc = copy_batch(h, h->A[X_IN], x, (long long)n * 2 * hw);
  if (rc != OT_OK) return rc;
  OT_CUDA(forward(h, n), "ot_unet_forward");
  OT_CUDA(cudaMemcpyAsync(y, h->A[OUT], (size_t)n * 4 * hw * sizeof(float), cudaMemcpyDefault, h->stream),
          "ot_unet_forward: output");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_unet_forward: sync");
  return OT_OK;
}

int ot_unet_gradients(ot_unet_t h, const float* x, const float* target, int32_t n, float* grads, double* loss) {
  if (!h || !x || !target) return fail(OT_EINVAL, "ot_unet_gradients: NULL argument");
  if (n < 1 || n > h->maxN) return fail(OT_EINVAL, "ot_unet_gradients: batch must be in [1, %d]", h->maxN);
  const long long hw = (long long)h->H * h->W;
  int rc = copy_batch(h, h->A[X_IN], x, (long long)n * 2 * hw);
  if (rc == OT_OK) rc = copy_batch(h, h->A[TARGET], target, (long long)n * 4 * hw);
  if (rc != OT_OK) return rc;
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
