// Singular-value thresholding through a T x T Gram matrix (Algorithm 3
// line 10, Sec. IV-B.1): shrink*_theta(X) = U shrink_theta(Sigma) V^T.
//
// For a tall X (N x T, frames as columns, N >> T):
//   G = X^T X = V Sigma^2 V^T            (Gram: one pass over X)
//   shrink*_theta(X) = X V diag(max(sigma - theta, 0) / sigma) V^T = X Wm
// so the only passes over the N x T data are the Gram and the final X Wm; the
// T x T eigenproblem is solved in one CTA by cyclic (round-robin) Jacobi in
// FP32, warm-started from the previous call's eigenvectors (the ADMM
// iterates change slowly, so one or two sweeps usually suffice).  FP32
// because FP64 throughput on this GPU is a small fraction of FP32; the Gram
// is summed in FP64 across CTAs.
//
// X layout: column t at X + t * ld, rows 0..N-1 (frame planes, ld = plane).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "device_util.cuh"
#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kGramChunk = 128;      // pixels staged per step

// Per-CTA partial Gram over a strided set of pixel chunks.  Thread (ty, tx)
// of a (Tp/4) x (Tp/4) block owns the 4 x 4 output tile rows 4ty.., cols 4tx..
template <int TP>
__global__ void __launch_bounds__((TP / 4) * (TP / 4))
gram_partial_kernel(const float* __restrict__ X, long long ld, long long N, int T, double* __restrict__ partials) {
  constexpr int NT = (TP / 4) * (TP / 4);
  __shared__ __align__(16) float sx[TP][kGramChunk];
  const int tid = threadIdx.x;
  const int ty = tid / (TP / 4), tx = tid % (TP / 4);
  float acc[4][4] = {};
  const long long nchunks = (N + kGramChunk - 1) / kGramChunk;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long i0 = ch * kGramChunk;
    for (int e = tid; e < TP * kGramChunk; e += NT) {
      const int t = e / kGramChunk, i = e % kGramChunk;
      const long long gi = i0 + i;
      sx[t][i] = (t < T && gi < N) ? __ldg(X + (long long)t * ld + gi) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < kGramChunk; i += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = *reinterpret_cast<const float4*>(&sx[4 * ty + r][i]);
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = *reinterpret_cast<const float4*>(&sx[4 * tx + c][i]);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          acc[r][c] = fmaf(a[r].x, b[c].x, fmaf(a[r].y, b[c].y, fmaf(a[r].z, b[c].z, fmaf(a[r].w, b[c].w, acc[r][c]))));
    }
    __syncthreads();
  }
  double* out = partials + (size_t)blockIdx.x * TP * TP;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) out[(4 * ty + r) * TP + 4 * tx + c] = (double)acc[r][c];
}

// G[e] = sum over CTAs of partials[b][e], fixed order, FP64.
__global__ void gram_reduce_kernel(const double* __restrict__ partials, int nparts, int n, double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += partials[(size_t)b * n + e];
  G[e] = s;
}

// One-CTA cyclic Jacobi on the symmetric G (TP x TP, zero beyond T), then
// Wm = V diag(f) V^T with f_i = max(sigma_i - theta, 0) / sigma_i,
// sigma_i = sqrt(max(lambda_i, 0)).  V_io: warm-start eigenvectors in (when
// warm) and the new ones out.  sig_out: sigma_i (diagnostics), sweeps_out:
// sweeps used.
template <int TP>
__global__ void __launch_bounds__(1024)
jacobi_svt_kernel(const double* __restrict__ G, int warm, float theta, int max_sweeps, float tol,
                  float* __restrict__ V_io, float* __restrict__ Wm, float* __restrict__ sig_out,
                  int* __restrict__ sweeps_out) {
  constexpr int LDA = TP + 1;
  extern __shared__ float sm[];
  float* A = sm;                 // [TP][LDA]
  float* V = A + TP * LDA;       // [TP][LDA]
  float* Tmp = V + TP * LDA;     // [TP][LDA]
  float* cs = Tmp + TP * LDA;    // [TP/2] c, [TP/2] s
  int* pq = reinterpret_cast<int*>(cs + TP);   // [TP/2] p, [TP/2] q
  __shared__ float red[32];
  __shared__ float s_off, s_diag;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < TP * TP; e += nt) {
    const int i = e / TP, j = e % TP;
    A[i * LDA + j] = (float)G[e];
    V[i * LDA + j] = warm ? V_io[e] : (i == j ? 1.f : 0.f);
  }
  __syncthreads();
  if (warm) {   // A <- V^T G V
    for (int e = tid; e < TP * TP; e += nt) {
      const int i = e / TP, j = e % TP;
      float s = 0.f;
      for (int k = 0; k < TP; ++k) s = fmaf(A[i * LDA + k], V[k * LDA + j], s);
      Tmp[i * LDA + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < TP * TP; e += nt) {
      const int i = e / TP, j = e % TP;
      float s = 0.f;
      for (int k = 0; k < TP; ++k) s = fmaf(V[k * LDA + i], Tmp[k * LDA + j], s);
      A[i * LDA + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < TP * TP; e += nt) {   // symmetrise the rounding
      const int i = e / TP, j = e % TP;
      if (i < j) {
        const float m = 0.5f * (A[i * LDA + j] + A[j * LDA + i]);
        A[i * LDA + j] = m;
        A[j * LDA + i] = m;
      }
    }
    __syncthreads();
  }

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal mass vs diagonal mass
    float off = 0.f, dg = 0.f;
    for (int e = tid; e < TP * TP; e += nt) {
      const int i = e / TP, j = e % TP;
      const float v = A[i * LDA + j];
      if (i == j) dg += v * v; else off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dg += __shfl_down_sync(0xffffffffu, dg, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int w = 0; w < nt / 32; ++w) s += red[w];
      s_off = s;
    }
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dg;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int w = 0; w < nt / 32; ++w) s += red[w];
      s_diag = s;
    }
    __syncthreads();
    if (!(s_off > tol * tol * s_diag)) break;

    for (int r = 0; r < TP - 1; ++r) {
      // round-robin pairing of 0..TP-1 (TP-1 fixed)
      if (tid < TP / 2) {
        const int k = tid;
        int p = (r + k) % (TP - 1);
        int q = k == 0 ? TP - 1 : (r - k + TP - 1) % (TP - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        const float app = A[p * LDA + p], aqq = A[q * LDA + q], apq = A[p * LDA + q];
        float c = 1.f, s = 0.f;
        if (apq != 0.f && fabsf(apq) > 1e-30f * sqrtf(fabsf(app * aqq))) {
          const float tau = (aqq - app) / (2.f * apq);
          const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = 1.f / sqrtf(1.f + t * t);
          s = t * c;
        }
        cs[k] = c;
        cs[TP / 2 + k] = s;
        pq[k] = p;
        pq[TP / 2 + k] = q;
      }
      __syncthreads();
      // rows p, q of A  (A <- J^T A)
      for (int e = tid; e < (TP / 2) * TP; e += nt) {
        const int k = e / TP, j = e % TP;
        const int p = pq[k], q = pq[TP / 2 + k];
        const float c = cs[k], s = cs[TP / 2 + k];
        const float ap = A[p * LDA + j], aq = A[q * LDA + j];
        A[p * LDA + j] = c * ap - s * aq;
        A[q * LDA + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and V  (A <- A J, V <- V J)
      for (int e = tid; e < (TP / 2) * TP; e += nt) {
        const int k = e / TP, i = e % TP;
        const int p = pq[k], q = pq[TP / 2 + k];
        const float c = cs[k], s = cs[TP / 2 + k];
        const float ap = A[i * LDA + p], aq = A[i * LDA + q];
        A[i * LDA + p] = c * ap - s * aq;
        A[i * LDA + q] = s * ap + c * aq;
        const float vp = V[i * LDA + p], vq = V[i * LDA + q];
        V[i * LDA + p] = c * vp - s * vq;
        V[i * LDA + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // f_i into cs-sized scratch (reuse Tmp row 0)
  float* f = Tmp;
  for (int i = tid; i < TP; i += nt) {
    const float lam = A[i * LDA + i];
    const float sg = sqrtf(fmaxf(lam, 0.f));
    f[i] = (sg > theta) ? (sg - theta) / sg : 0.f;
    sig_out[i] = sg;
  }
  __syncthreads();
  for (int e = tid; e < TP * TP; e += nt) {
    const int s = e / TP, t = e % TP;
    float w = 0.f;
    for (int i = 0; i < TP; ++i) w = fmaf(V[s * LDA + i] * f[i], V[t * LDA + i], w);
    Wm[e] = w;
    V_io[e] = V[s * LDA + t];
  }
  if (tid == 0) *sweeps_out = sweep;
}

// Y[:, t] = sum_s Wm[s][t] X[:, s] for t in [t0, t0 + 64); optional
// accumulation of ||Y - Y_old||^2 (dual residual of Algorithm 3) into
// partials[block][1].  One thread per row (pixel).
template <int TP>
__global__ void __launch_bounds__(256)
svt_apply_kernel(const float* __restrict__ X, long long ld, long long N, int T, const float* __restrict__ Wm,
                 float* __restrict__ Y, long long ldy, int reduce, double* __restrict__ partials) {
  constexpr int TB = 64;
  __shared__ __align__(16) float sW[TP][TB];
  const int t0 = blockIdx.y * TB;
  for (int e = threadIdx.x; e < TP * TB; e += blockDim.x) {
    const int s = e / TB, t = e % TB;
    sW[s][t] = (t0 + t < TP) ? Wm[s * TP + t0 + t] : 0.f;
  }
  __syncthreads();
  float acc[kNumSums] = {};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float y[TB];
#pragma unroll
    for (int t = 0; t < TB; ++t) y[t] = 0.f;
    for (int s = 0; s < T; ++s) {
      const float x = __ldg(X + (long long)s * ld + i);
#pragma unroll
      for (int t = 0; t < TB; t += 4) {
        const float4 w = *reinterpret_cast<const float4*>(&sW[s][t]);
        y[t] = fmaf(w.x, x, y[t]);
        y[t + 1] = fmaf(w.y, x, y[t + 1]);
        y[t + 2] = fmaf(w.z, x, y[t + 2]);
        y[t + 3] = fmaf(w.w, x, y[t + 3]);
      }
    }
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      if (t0 + t < T) {
        float* dst = Y + (long long)(t0 + t) * ldy + i;
        if (reduce) {
          const float d = y[t] - *dst;
          acc[1] = fmaf(d, d, acc[1]);
        }
        *dst = y[t];
      }
    }
  }
  if (reduce) {
    block_sums_to<256>(acc, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNumSums);
  }
}

template <int TP>
size_t jacobi_smem() {
  return (size_t)(3 * TP * (TP + 1) + TP) * sizeof(float) + TP * sizeof(int);
}

}  // namespace

int svt_padded_T(int T) { return T <= 16 ? 16 : (T <= 32 ? 32 : (T <= 64 ? 64 : 128)); }

int svt_gram_blocks(long long N) {
  const long long nch = (N + kGramChunk - 1) / kGramChunk;
  return (int)(nch < 152 ? nch : 152);
}

int svt_apply_blocks(long long N, int T, int* gy) {
  *gy = (svt_padded_T(T) + 63) / 64;
  const long long nb = (N + 255) / 256;
  return (int)(nb < 152 * 8 ? nb : 152 * 8);
}

cudaError_t svt_prepare() {
  cudaError_t e = cudaFuncSetAttribute(jacobi_svt_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_smem<128>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jacobi_svt_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jacobi_smem<64>());
  return e;
}

// partials: >= svt_gram_blocks(N) * TP * TP doubles; G: TP * TP doubles.
cudaError_t svt_launch_gram(const float* X, long long ld, long long N, int T, double* partials, double* G,
                            cudaStream_t st) {
  const int TP = svt_padded_T(T);
  const int nb = svt_gram_blocks(N);
  switch (TP) {
    case 16: gram_partial_kernel<16><<<nb, 16, 0, st>>>(X, ld, N, T, partials); break;
    case 32: gram_partial_kernel<32><<<nb, 64, 0, st>>>(X, ld, N, T, partials); break;
    case 64: gram_partial_kernel<64><<<nb, 256, 0, st>>>(X, ld, N, T, partials); break;
    default: gram_partial_kernel<128><<<nb, 1024, 0, st>>>(X, ld, N, T, partials); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = TP * TP;
  gram_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(partials, nb, n, G);
  return cudaGetLastError();
}

cudaError_t svt_launch_eig(const double* G, int T, int warm, float theta, int max_sweeps, float tol, float* V_io,
                           float* Wm, float* sig, int* sweeps, cudaStream_t st) {
  const int TP = svt_padded_T(T);
  switch (TP) {
    case 16: jacobi_svt_kernel<16><<<1, 256, jacobi_smem<16>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    case 32: jacobi_svt_kernel<32><<<1, 512, jacobi_smem<32>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    case 64: jacobi_svt_kernel<64><<<1, 1024, jacobi_smem<64>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    default: jacobi_svt_kernel<128><<<1, 1024, jacobi_smem<128>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
  }
  return cudaGetLastError();
}

cudaError_t svt_launch_apply(const float* X, long long ld, long long N, int T, const float* Wm, float* Y,
                             long long ldy, bool reduce, double* partials, cudaStream_t st) {
  const int TP = svt_padded_T(T);
  int gy = 1;
  const int nb = svt_apply_blocks(N, T, &gy);
  const dim3 grid(nb, gy);
  switch (TP) {
    case 16: svt_apply_kernel<16><<<grid, 256, 0, st>>>(X, ld, N, T, Wm, Y, ldy, reduce, partials); break;
    case 32: svt_apply_kernel<32><<<grid, 256, 0, st>>>(X, ld, N, T, Wm, Y, ldy, reduce, partials); break;
    case 64: svt_apply_kernel<64><<<grid, 256, 0, st>>>(X, ld, N, T, Wm, Y, ldy, reduce, partials); break;
    default: svt_apply_kernel<128><<<grid, 256, 0, st>>>(X, ld, N, T, Wm, Y, ldy, reduce, partials); break;
  }
  return cudaGetLastError();
}

}  // namespace otp
