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
constexpr int kGramThreads = 256;

// Per-CTA partial Gram over a strided set of pixel chunks.  The chunk is
// staged pixel-major (sx[pixel][t]).  Every thread owns an 8 x 8 tile of the
// TP x TP output; the (TP/8)^2 threads covering the output form a group, and
// the 256 / (TP/8)^2 groups split the chunk's pixels.  Two float4 reads per
// operand per pixel feed 64 FMAs.  The groups are summed in shared memory at
// the end and the CTA's total is written in FP64.
template <int TP>
constexpr int gram_groups() { return kGramThreads / ((TP / 8) * (TP / 8)); }

template <int TP>
constexpr size_t gram_smem() {
  const size_t stage = (size_t)kGramChunk * (TP + 4) * sizeof(float);
  const size_t red = (size_t)gram_groups<TP>() * TP * TP * sizeof(float);
  return stage > red ? stage : red;
}

template <int TP>
__global__ void __launch_bounds__(kGramThreads)
gram_partial_kernel(const float* __restrict__ X, long long ld, long long N, int T, double* __restrict__ partials) {
  constexpr int R = 8;
  constexpr int TPG = (TP / 8) * (TP / 8);        // threads per group
  constexpr int NG = gram_groups<TP>();
  constexpr int PPG = kGramChunk / NG;            // pixels per group and chunk
  constexpr int LDS = TP + 4;                     // padded pixel row
  extern __shared__ __align__(16) float sx[];
  const int tid = threadIdx.x;
  const int grp = tid / TPG, gt = tid % TPG;
  const int ty = gt / (TP / 8), tx = gt % (TP / 8);
  float acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.f;
  const long long nchunks = (N + kGramChunk - 1) / kGramChunk;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long i0 = ch * kGramChunk;
    for (int e = tid; e < TP * kGramChunk; e += kGramThreads) {
      const int t = e / kGramChunk, p = e % kGramChunk;
      const long long gi = i0 + p;
      sx[p * LDS + t] = (t < T && gi < N) ? __ldg(X + (long long)t * ld + gi) : 0.f;
    }
    __syncthreads();
    const float* base = sx + grp * PPG * LDS;
#pragma unroll 2
    for (int p = 0; p < PPG; ++p) {
      float a[R], b[R];
#pragma unroll
      for (int r = 0; r < R; r += 4) {
        const float4 va = *reinterpret_cast<const float4*>(base + p * LDS + R * ty + r);
        const float4 vb = *reinterpret_cast<const float4*>(base + p * LDS + R * tx + r);
        a[r] = va.x; a[r + 1] = va.y; a[r + 2] = va.z; a[r + 3] = va.w;
        b[r] = vb.x; b[r + 1] = vb.y; b[r + 2] = vb.z; b[r + 3] = vb.w;
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  // sum the groups through shared memory (reusing the staging buffer)
  float* red = sx;   // [NG][TP][TP]
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) red[((size_t)grp * TP + R * ty + r) * TP + R * tx + c] = acc[r][c];
  __syncthreads();
  double* out = partials + (size_t)blockIdx.x * TP * TP;
  for (int e = tid; e < TP * TP; e += kGramThreads) {
    double v = 0.0;
    for (int g = 0; g < NG; ++g) v += (double)red[(size_t)g * TP * TP + e];
    out[e] = v;
  }
}

// G[e] = sum over CTAs of partials[b][e] in FP64, fixed order: a block owns
// 32 consecutive entries (one per lane); its 32 warps take every 32nd
// partial and are summed in warp order.
constexpr int kRedWarps = 32;

template <typename P>
__global__ void __launch_bounds__(32 * kRedWarps) gram_reduce_kernel(const P* __restrict__ partials, int nparts,
                                                                   int n, double* __restrict__ G) {
  __shared__ double s[kRedWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double v = 0.0;
  if (e < n) {
    int b = warp;
    for (; b + 3 * kRedWarps < nparts; b += 4 * kRedWarps) {   // four loads in flight, summed in order
      const double x0 = (double)__ldg(partials + (size_t)b * n + e);
      const double x1 = (double)__ldg(partials + (size_t)(b + kRedWarps) * n + e);
      const double x2 = (double)__ldg(partials + (size_t)(b + 2 * kRedWarps) * n + e);
      const double x3 = (double)__ldg(partials + (size_t)(b + 3 * kRedWarps) * n + e);
      v += x0;
      v += x1;
      v += x2;
      v += x3;
    }
    for (; b < nparts; b += kRedWarps) v += (double)__ldg(partials + (size_t)b * n + e);
  }
  s[warp][lane] = v;
  __syncthreads();
  if (warp == 0 && e < n) {
    double t = 0.0;
    for (int w = 0; w < kRedWarps; ++w) t += s[w][lane];
    G[e] = t;
  }
}

// C = op(A) * diag(d) * B for TP x TP shared matrices (leading dimension
// LDA).  Threads take 4 x 4 output blocks in turn.  transA: use A^T.
// RB x 4 output blocks (RB = 4 by default; 2 spreads a 64 x 64 product over
// 512 threads).
template <int TP, int LDA, int RB = 4>
__device__ __forceinline__ void small_gemm(const float* A, const float* B, float* C, bool transA, const float* diag) {
  constexpr int NBR = TP / RB, NBC = TP / 4;   // blocks per column, per row
  for (int blk = threadIdx.x; blk < NBR * NBC; blk += blockDim.x) {
    const int by = blk / NBC, bx = blk % NBC;
    float acc[RB][4] = {};
    for (int k = 0; k < TP; ++k) {
      float a[RB], b[4];
      const float dk = diag ? diag[k] : 1.f;
#pragma unroll
      for (int r = 0; r < RB; ++r) a[r] = transA ? A[k * LDA + RB * by + r] : A[(RB * by + r) * LDA + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = dk * B[k * LDA + 4 * bx + c];
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) C[(RB * by + r) * LDA + 4 * bx + c] = acc[r][c];
  }
}

// One Newton-Schulz step towards the orthogonal polar factor of V (TP x TP,
// row-major in shared memory): V <- V (3 I - V^T V) / 2.  The eigenvectors
// are carried from one outer iteration's eigensolve to the next and every
// FP32 rotation perturbs their orthonormality by about u; without this the
// drift accumulates over the outer iterations and Wm = V diag(f) V^T (a
// near-projector onto the dominant subspace) drifts with it.  One step maps
// a deviation e of V^T V from I to about 3 e^2 / 4 (plus the rounding of the
// two products).  Tmp, Out: TP x TP scratch.  Every thread must reach it.
template <int TP, int LDA, int RB>
__device__ __forceinline__ void reorthonormalize(float* V, float* Tmp, float* Out) {
  small_gemm<TP, LDA, RB>(V, V, Tmp, true, nullptr);   // V^T V
  __syncthreads();
  for (int e = threadIdx.x; e < TP * TP; e += blockDim.x) {
    const int i = e / TP, j = e % TP;
    Tmp[i * LDA + j] = (i == j ? 1.5f : 0.f) - 0.5f * Tmp[i * LDA + j];
  }
  __syncthreads();
  small_gemm<TP, LDA, RB>(V, Tmp, Out, false, nullptr);
  __syncthreads();
  for (int e = threadIdx.x; e < TP * TP; e += blockDim.x) {
    const int i = e / TP, j = e % TP;
    V[i * LDA + j] = Out[i * LDA + j];
  }
  __syncthreads();
}

// One-CTA cyclic Jacobi on the symmetric G (TP x TP, zero beyond T), then
// Wm = V diag(f) V^T with f_i = max(sigma_i - theta, 0) / sigma_i,
// sigma_i = sqrt(max(lambda_i, 0)).  V_io: warm-start eigenvectors in (when
// warm) and the new ones out.  sig_out: sigma_i (diagnostics), sweeps_out:
// Jacobi rounds used (TP - 1 per sweep).
// Round-robin ordering: each round rotates the TP/2 disjoint pairs of a
// precomputed schedule.  Phase 1: warp k forms the rotation J_k of pair k
// from its 2 x 2 diagonal block.  Phase 2: each thread owns 2 x 2 blocks
// (pair kb rows x pair kc columns) and applies both rotations at once,
// B <- J_kb^T B J_kc, and rotates two rows of V.  The rotation need only be
// orthogonal (c^2 + s^2 = 1 to rounding), not correctly rounded, so the
// approximate reciprocal and reciprocal square root are used.
constexpr int kJacobiThreads = 1024;
// at most this many dominant eigenpairs are deflated from the warm start
// (the SVT's data are low rank: a few dominant singular values)
constexpr int kMaxDeflate = 4;

__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float& c, float& s, float& t) {
  c = 1.f;
  s = 0.f;
  t = 0.f;
  if (apq != 0.f) {
    float tau = (aqq - app) * __fdividef(0.5f, apq);
    tau = fminf(fmaxf(tau, -1e18f), 1e18f);
    const float h2 = fmaf(tau, tau, 1.f);
    const float h = h2 * rsqrtf(h2);                      // sqrt(1 + tau^2)
    t = copysignf(__fdividef(1.f, fabsf(tau) + h), tau);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = t * c;
  }
}

template <int TP>
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_svt_kernel(const double* __restrict__ G, int warm, float theta, int max_sweeps, float tol,
                  float* __restrict__ V_io, float* __restrict__ Wm, float* __restrict__ sig_out,
                  int* __restrict__ sweeps_out) {
  constexpr int LDA = TP + 1;
  constexpr int NP = TP / 2;
  constexpr int NW = kJacobiThreads / 32;
  extern __shared__ float sm[];
  float* A = sm;                 // [TP][LDA]
  float* V = A + TP * LDA;       // [TP][LDA]
  float* Tmp = V + TP * LDA;     // [TP][LDA]
  float* f = Tmp + TP * LDA;     // [TP]
  __shared__ float s_c[NP], s_s[NP], s_t[NP];
  __shared__ unsigned char s_sched[(TP - 1) * NP * 2];   // (p, q) of pair k in round r
  __shared__ float red[2][NW];
  __shared__ int s_go;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int e = tid; e < (TP - 1) * NP; e += kJacobiThreads) {
    const int r = e / NP, k = e % NP;
    int p = (r + k) % (TP - 1);
    int q = k == 0 ? TP - 1 : (r - k + TP - 1) % (TP - 1);
    if (p > q) { const int t = p; p = q; q = t; }
    s_sched[2 * e] = (unsigned char)p;
    s_sched[2 * e + 1] = (unsigned char)q;
  }
  __shared__ float s_lam_big[TP];
  __shared__ unsigned char s_big[TP];
  __shared__ int s_nbig;
  __shared__ double s_wbig[kMaxDeflate][TP];
  if (tid == 0) {
    // warm start: the previous solve's dominant eigenpairs (sigma > 8 theta),
    // deflated from G in FP64 before G is rounded to FP32 (as in
    // jacobi_reg_kernel: A = V^T G' V + diag(lam_big))
    int nb = 0;
    for (int j = 0; j < TP; ++j) {
      const float sg = warm && theta > 0.f ? sig_out[j] : 0.f;
      const bool big = sg > 8.f * theta && nb < kMaxDeflate;
      if (big) s_big[nb++] = (unsigned char)j;
      s_lam_big[j] = big ? sg * sg : 0.f;
    }
    s_nbig = nb;
  }
  for (int e = tid; e < TP * TP; e += kJacobiThreads) {
    const int i = e / TP, j = e % TP;
    V[i * LDA + j] = warm ? V_io[e] : (i == j ? 1.f : 0.f);
  }
  __syncthreads();
  for (int e = tid; e < s_nbig * TP; e += kJacobiThreads) {
    const int b = e / TP, k = e % TP, c = s_big[b];
    s_wbig[b][k] = sqrt((double)s_lam_big[c]) * (double)V[k * LDA + c];
  }
  __syncthreads();
  for (int e = tid; e < TP * TP; e += kJacobiThreads) {
    const int i = e / TP, j = e % TP;
    double gd = G[e];
    for (int b = 0; b < s_nbig; ++b) gd = fma(-s_wbig[b][i], s_wbig[b][j], gd);
    A[i * LDA + j] = (float)gd;
  }
  __syncthreads();
  if (warm) {   // A <- V^T G' V + diag(lam_big)
    small_gemm<TP, LDA>(A, V, Tmp, false, nullptr);   // Tmp = G' V
    __syncthreads();
    small_gemm<TP, LDA>(V, Tmp, A, true, nullptr);    // A = V^T Tmp
    __syncthreads();
    if (tid < TP) A[tid * LDA + tid] += s_lam_big[tid];
    __syncthreads();
    for (int e = tid; e < TP * TP; e += kJacobiThreads) {   // symmetrise the rounding
      const int i = e / TP, j = e % TP;
      if (i < j) {
        const float m = 0.5f * (A[i * LDA + j] + A[j * LDA + i]);
        A[i * LDA + j] = m;
        A[j * LDA + i] = m;
      }
    }
    __syncthreads();
  }

  // Convergence, once per sweep.  With theta > 0: each off-diagonal entry
  // against sqrt(d_i d_j), the diagonal floored at theta^2 / 4 (below that
  // f is 0 and the eigenvalue's own accuracy does not matter), so that the
  // eigenvalues near theta^2, far below the largest, are resolved to tol
  // relative to themselves; the solver also stops when a sweep has not
  // halved that measure (FP32 rounding floor).  With theta <= 0: the plain
  // relative off-diagonal Frobenius norm.
  const float dfloor = 0.25f * theta * theta;
  float prev = 3.0e38f;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float off = 0.f, dg = 0.f;
    for (int e = tid; e < TP * TP; e += kJacobiThreads) {
      const int i = e / TP, j = e % TP;
      const float v = A[i * LDA + j];
      if (i == j) {
        dg = fmaf(v, v, dg);
      } else if (theta > 0.f) {
        const float di = fmaxf(fabsf(A[i * LDA + i]), dfloor), dj = fmaxf(fabsf(A[j * LDA + j]), dfloor);
        off = fmaf(v, v * __frcp_rn(di * dj), off);
      } else {
        off = fmaf(v, v, off);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dg += __shfl_down_sync(0xffffffffu, dg, o);
    }
    if (lane == 0) {
      red[0][warp] = off;
      red[1][warp] = dg;
    }
    __syncthreads();
    if (tid == 0) {
      float so = 0.f, sd = 0.f;
      for (int w = 0; w < NW; ++w) {
        so += red[0][w];
        sd += red[1][w];
      }
      s_go = theta > 0.f ? (so > tol * tol && so < 0.25f * prev) : so > tol * tol * sd;
      prev = so;
    }
    __syncthreads();
    if (!s_go) break;

    for (int r = 0; r < TP - 1; ++r) {
      const unsigned char* sch = s_sched + 2 * r * NP;
      // phase 1: rotations
      for (int k = warp; k < NP; k += NW) {
        const int p = sch[2 * k], q = sch[2 * k + 1];
        float c, sn, tn;
        jacobi_rotation(A[p * LDA + p], A[q * LDA + q], A[p * LDA + q], c, sn, tn);
        if (lane == 0) {
          s_c[k] = c;
          s_s[k] = sn;
          s_t[k] = tn;
        }
      }
      __syncthreads();
      // phase 2: 2 x 2 blocks of A, and rows of V
      for (int e = tid; e < NP * NP; e += kJacobiThreads) {
        const int kb = e / NP, kc = e % NP;
        const int p = sch[2 * kb], q = sch[2 * kb + 1], pc = sch[2 * kc], qc = sch[2 * kc + 1];
        const float c = s_c[kb], sn = s_s[kb], c2 = s_c[kc], s2 = s_s[kc];
        const float a00 = A[p * LDA + pc], a01 = A[p * LDA + qc], a10 = A[q * LDA + pc], a11 = A[q * LDA + qc];
        if (kb == kc) {
          // the pair's own block: the rotation zeroes a_pq exactly and moves
          // -/+ t a_pq onto the diagonal (the accurate classical update)
          const float tn = s_t[kb];
          A[p * LDA + p] = a00 - tn * a01;
          A[q * LDA + q] = a11 + tn * a01;
          A[p * LDA + q] = 0.f;
          A[q * LDA + p] = 0.f;
          continue;
        }
        // rows: J^T B
        const float r00 = c * a00 - sn * a10, r01 = c * a01 - sn * a11;
        const float r10 = sn * a00 + c * a10, r11 = sn * a01 + c * a11;
        // columns: (J^T B) J'
        A[p * LDA + pc] = c2 * r00 - s2 * r01;
        A[p * LDA + qc] = s2 * r00 + c2 * r01;
        A[q * LDA + pc] = c2 * r10 - s2 * r11;
        A[q * LDA + qc] = s2 * r10 + c2 * r11;
      }
      for (int e = tid; e < NP * TP; e += kJacobiThreads) {
        const int k = e / TP, i = e % TP;
        const int p = sch[2 * k], q = sch[2 * k + 1];
        const float c = s_c[k], sn = s_s[k];
        const float vp = V[i * LDA + p], vq = V[i * LDA + q];
        V[i * LDA + p] = c * vp - sn * vq;
        V[i * LDA + q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // f_i, then Wm = V diag(f) V^T
  for (int i = tid; i < TP; i += kJacobiThreads) {
    const float lam = A[i * LDA + i];
    const float sg = sqrtf(fmaxf(lam, 0.f));
    f[i] = (sg > theta) ? (sg - theta) / sg : 0.f;
    sig_out[i] = sg;
  }
  __syncthreads();
  if (sweep > 0) reorthonormalize<TP, LDA, 4>(V, Tmp, A);
  // Tmp <- V^T (small_gemm reads B row-major)
  for (int e = tid; e < TP * TP; e += kJacobiThreads) {
    const int i = e / TP, j = e % TP;
    Tmp[i * LDA + j] = V[j * LDA + i];
  }
  __syncthreads();
  small_gemm<TP, LDA>(V, Tmp, A, false, f);    // A = V diag(f) V^T
  __syncthreads();
  for (int e = tid; e < TP * TP; e += kJacobiThreads) {
    const int i = e / TP, j = e % TP;
    Wm[e] = A[i * LDA + j];
    V_io[e] = V[i * LDA + j];
  }
  if (tid == 0) *sweeps_out = sweep * (TP - 1);   // rounds
}

// The same eigensolve for TP <= 64, pipelined with fixed addressing.
// Pairing by the circle method: slots top k = k and bottom k = TP/2 + k form
// pair k; between rounds slot 0 stays and the other TP - 1 slots advance one
// step along the ring top 1 -> ... -> top TP/2-1 -> bottom TP/2-1 -> ... ->
// bottom 0 -> top 1, so each index meets every other once per sweep of TP - 1
// rounds.  A is stored in slot order (A_slot[s][s'] = A[index at s][index at
// s']), upper triangle, double-buffered: a round reads the pair blocks of the
// current buffer and writes the rotated entries straight to their shifted
// slots in the other, so every shared-memory address a thread touches is the
// same in every round.  The rows of V live in registers in slot order: thread
// (row i, segment g) holds the kJregM pairs g*kJregM..., rotates them in place
// and passes one value to each ring neighbour segment by a warp shuffle.
// One barrier per round: while warps 1.. apply the rotations of round r,
// lane k of warp 0 forms the rotation of round r + 1's pair k from the three
// entries that round r produces for it (recomputed with the same operations,
// so they are bit-identical to the stored ones).
//
// Stopping.  Only Wm = F(A) = V f(Lambda) V^T is needed, f(lam) =
// max(1 - theta / sqrt(lam), 0).  Writing A = D + E (E off-diagonal), the
// first-order change of F is dd_ij e_ij with dd_ij the divided difference of
// f between lam_i and lam_j, so rotations inside the subspace that f maps to
// zero do not change Wm.  What the SVT returns is X Wm = U Sigma f(Sigma)
// V^T, so that change reaches the output as U Sigma (dd o E) V^T, whose
// squared Frobenius norm is sum_{i<j} (lam_i + lam_j) (dd_ij e_ij)^2.  With
// theta > 0 the solver stops, every kJregCheck rounds, when that is at most
// tol^2 ||shrink*(X)||_F^2 = tol^2 sum_i max(sigma_i - theta, 0)^2: the
// output's error relative to the output (couplings among the small
// eigenvalues near theta^2 weigh with their own sigma, not with the
// largest one; lam_i from the diagonal, plus eps).  By Weyl's
// inequality every eigenvalue lies within eps = ||E||_F of the diagonal, so
// dd_ij is bounded by the largest slope of f on [min(d_i, d_j) - eps,
// max(d_i, d_j) + eps] (a pair whose interval stays below theta^2 cannot
// contribute) and, since 0 <= f < 1, by 1 / (|d_i - d_j| - 2 eps): the
// second bound is the tight one for well separated pairs, whose coupling
// keeps a rounding floor of about u times the larger eigenvalue.  The test
// is weighted per pair, not relative to ||diag||: the eigenvalues near
// theta^2 that decide Wm are far below the largest one, so an off-diagonal
// mass that is small against ||diag|| can still move them by much more than
// tol.  The solver also stops when a whole sweep has not halved the
// weighted measure once the plain off-diagonal norm is within 2 tol of
// ||diag|| (the FP32 rounding floor: the rotations leave about u times the
// largest eigenvalue in each coupling of its row).  With theta <= 0, f is 1 on every positive
// eigenvalue and the plain test ||E||_F <= tol ||diag||_2 is used.
constexpr int kJregThreads = 512;
constexpr int kJregCheck = 16;  // rounds between stopping tests
constexpr int kJregM = 4;       // pairs per register segment of a V row

// C[i][j] = sum_k X[k][i] d_k Y[k][j] for TP x TP matrices in shared memory
// with 16-byte aligned rows of LDA floats (d_k = 1 when diag is null): both
// operands are read along k as float4 rows.  Thread t owns the 4 x 4 output
// block t % NB (NB = (TP/4)^2) over half of the k range; the second half's
// partials pass through C to the first half's threads, which add them.
// Every thread of the block must reach it; C may not alias X or Y.
template <int TP, int LDA>
__device__ __forceinline__ void kgemm(const float* X, const float* Y, float* C, const float* diag) {
  static_assert(LDA % 4 == 0 && TP % 4 == 0, "float4 rows");
  constexpr int NBS = TP / 4, NB = NBS * NBS;
  constexpr int KS = 2 * NB <= kJregThreads ? 2 : 1;
  static_assert(NB * KS <= kJregThreads, "one output block per thread");
  const int t = threadIdx.x;
  const int blk = t % NB, part = t / NB;
  const int bi = blk / NBS, bj = blk % NBS;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  if (part < KS) {
    const int k0 = part * (TP / KS);
#pragma unroll 4
    for (int k = k0; k < k0 + TP / KS; ++k) {
      const float4 x = *reinterpret_cast<const float4*>(X + k * LDA + 4 * bi);
      float4 y = *reinterpret_cast<const float4*>(Y + k * LDA + 4 * bj);
      if (diag) {
        const float dk = diag[k];
        y.x *= dk;
        y.y *= dk;
        y.z *= dk;
        y.w *= dk;
      }
      const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xv[r], yv[c], acc[r][c]);
    }
  }
  if (KS == 2 && part == 1) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      *reinterpret_cast<float4*>(C + (4 * bi + r) * LDA + 4 * bj) =
          make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
  }
  __syncthreads();
  if (part == 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float4 o = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
      if (KS == 2) {
        const float4 h = *reinterpret_cast<const float4*>(C + (4 * bi + r) * LDA + 4 * bj);
        o.x += h.x;
        o.y += h.y;
        o.z += h.z;
        o.w += h.w;
      }
      *reinterpret_cast<float4*>(C + (4 * bi + r) * LDA + 4 * bj) = o;
    }
  }
}

// The Newton-Schulz step V <- V (3 I - V^T V) / 2 of reorthonormalize, in
// k-major products: M = V^T V, then V = (V^T)^T M with V^T staged in Out.
template <int TP, int LDA>
__device__ __forceinline__ void reorthonormalize_k(float* V, float* Tmp, float* Out) {
  kgemm<TP, LDA>(V, V, Tmp, nullptr);   // V^T V
  __syncthreads();
  for (int e = threadIdx.x; e < TP * TP; e += blockDim.x) {
    const int i = e / TP, j = e % TP;
    Tmp[i * LDA + j] = (i == j ? 1.5f : 0.f) - 0.5f * Tmp[i * LDA + j];
    Out[i * LDA + j] = V[j * LDA + i];
  }
  __syncthreads();
  kgemm<TP, LDA>(Out, Tmp, V, nullptr);   // V M (M symmetric)
  __syncthreads();
}

__host__ __device__ constexpr int upper_idx(int i, int j, int ld) { return i < j ? i * ld + j : j * ld + i; }

// slot that the value at slot s moves to between rounds, and its inverse
template <int NP>
__device__ __forceinline__ int ring_next(int s) {
  return s == 0 ? 0 : s < NP - 1 ? s + 1 : s == NP - 1 ? 2 * NP - 1 : s == NP ? 1 : s - 1;
}
template <int NP>
__device__ __forceinline__ int ring_prev(int s) {
  return s == 0 ? 0 : s == 1 ? NP : s < NP ? s - 1 : s == 2 * NP - 1 ? NP - 1 : s + 1;
}

// c x - s y and s x + c y with a fixed operation order (no contraction
// choices), so that two threads computing the same entry agree bit for bit
__device__ __forceinline__ float rot_lo(float c, float s, float x, float y) { return fmaf(c, x, __fmul_rn(-s, y)); }
__device__ __forceinline__ float rot_hi(float c, float s, float x, float y) { return fmaf(s, x, __fmul_rn(c, y)); }

template <int TP>
constexpr size_t jreg_smem() {
  return (size_t)(4 * TP * (TP + 4) + TP) * sizeof(float);
}

template <int TP>
__global__ void __launch_bounds__(kJregThreads, 1)
jacobi_reg_kernel(const double* __restrict__ G, int warm, float theta, int max_sweeps, float tol,
                  float* __restrict__ V_io, float* __restrict__ Wm, float* __restrict__ sig_out,
                  int* __restrict__ rounds_out) {
  constexpr int LDA = TP + 4;            // 16-byte aligned rows for the float4 products
  constexpr int NP = TP / 2;
  constexpr int S = NP / kJregM;           // register segments per V row
  constexpr int NOFF = NP * (NP - 1) / 2;  // off-diagonal pair blocks kb < kc
  constexpr int NB = NOFF + NP;
  constexpr int NAPP = kJregThreads - 32;  // block-applying threads (warps 1..)
  constexpr int NBT = (NB + NAPP - 1) / NAPP;
  constexpr int R = TP - 1;                // rounds per sweep
  constexpr int NW = kJregThreads / 32;
  static_assert(NP <= 32, "one rotation per lane of warp 0");
  static_assert(S >= 2 && S <= 32 && (S & (S - 1)) == 0, "segments must be a power of two within a warp");
  static_assert((TP * S) % 32 == 0 && TP * S <= kJregThreads, "V rows must fill whole warps");
  static_assert(NBT <= 2, "at most two pair blocks per thread");
  extern __shared__ float sm[];
  // sm: two slot-ordered copies of A (upper triangle, ping-pong), then V, Tmp, f
  float* V = sm + 2 * TP * LDA;           // [TP][LDA]
  float* Tmp = V + TP * LDA;              // [TP][LDA]
  float* f = Tmp + TP * LDA;              // [TP]
  __shared__ float s_rot[2][3][NP];       // (c, s, t) of each pair, by round parity
  __shared__ unsigned char s_pl[TP];      // index held by each slot after the last round
  __shared__ float s_slope[TP];
  __shared__ float s_dg[TP];
  __shared__ unsigned char s_act[TP];
  __shared__ float red[2][NW];
  __shared__ int s_go;
  __shared__ float s_eps;
  __shared__ float s_best;                // smallest weighted measure, halved at least once per sweep
  __shared__ int s_best_at;               // round at which s_best was last halved
  __shared__ float s_lam_big[TP];         // warm start: deflated eigenvalues (0: not deflated)
  __shared__ unsigned char s_big[TP];
  __shared__ int s_nbig;
  __shared__ double s_wbig[kMaxDeflate][TP];   // sqrt(lam) v of the deflated pairs, FP64
  __shared__ int s_floor;                 // the plain off-diagonal norm is at its FP32 floor
  __shared__ float s_sig[TP];
  __shared__ double s_sq[kMaxDeflate];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_best = 3.0e38f;
    s_best_at = 0;
  }

  // applier threads: their pair blocks (read offsets in the current buffer,
  // write offsets at the shifted slots in the next); kind 0 none, 1 off-diagonal, 2 own pair
  int rd[NBT][4], wr[NBT][4], bkb[NBT], bkc[NBT], kind[NBT];
#pragma unroll
  for (int u = 0; u < NBT; ++u) {
    const int e = tid - 32 + u * NAPP;
    kind[u] = 0;
    bkb[u] = bkc[u] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) rd[u][q] = wr[u][q] = 0;
    if (warp > 0 && e < NB) {
      int kb, kc;
      if (e < NOFF) {
        int rem = e;
        kb = 0;
        while (rem >= NP - 1 - kb) { rem -= NP - 1 - kb; ++kb; }
        kc = kb + 1 + rem;
        kind[u] = 1;
      } else {
        kb = kc = e - NOFF;
        kind[u] = 2;
      }
      bkb[u] = kb;
      bkc[u] = kc;
      const int rs[2] = {kb, NP + kb};
      const int cs[2] = {kc, NP + kc};
      if (kind[u] == 1) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            rd[u][2 * a + b] = upper_idx(rs[a], cs[b], LDA);
            wr[u][2 * a + b] = upper_idx(ring_next<NP>(rs[a]), ring_next<NP>(cs[b]), LDA);
          }
      } else {
        rd[u][0] = rs[0] * LDA + rs[0];
        rd[u][1] = rs[1] * LDA + rs[1];
        rd[u][2] = upper_idx(rs[0], rs[1], LDA);
        const int n0 = ring_next<NP>(rs[0]), n1 = ring_next<NP>(rs[1]);
        wr[u][0] = n0 * LDA + n0;
        wr[u][1] = n1 * LDA + n1;
        wr[u][2] = upper_idx(n0, n1, LDA);
      }
    }
  }
  // rotation lanes (warp 0, lane k < NP): where next round's pair k comes from.
  // Its top is now at slot P, its bottom at slot Q, in pairs kP != kQ.
  int pP = 0, pQ = 0, pPdg = 0, pQdg = 0, pPpq = 0, pQpq = 0, pB[4] = {0, 0, 0, 0};
  int pkP = 0, pkQ = 0, pkb = 0, pkc = 0;
  bool pPbot = false, pQbot = false, pa = false, pb = false;
  if (warp == 0 && lane < NP) {
    const int P = ring_prev<NP>(lane), Q = ring_prev<NP>(NP + lane);
    pP = P;
    pQ = Q;
    pPbot = P >= NP;
    pQbot = Q >= NP;
    pkP = pPbot ? P - NP : P;
    pkQ = pQbot ? Q - NP : Q;
    pPdg = P * LDA + P;
    pQdg = Q * LDA + Q;
    pPpq = pkP * LDA + NP + pkP;
    pQpq = pkQ * LDA + NP + pkQ;
    pkb = pkP < pkQ ? pkP : pkQ;
    pkc = pkP < pkQ ? pkQ : pkP;
    pa = pkP < pkQ ? pPbot : pQbot;         // row slot (in pair kb) is a bottom slot
    pb = pkP < pkQ ? pQbot : pPbot;         // column slot (in pair kc) is a bottom slot
    pB[0] = upper_idx(pkb, pkc, LDA);
    pB[1] = upper_idx(pkb, NP + pkc, LDA);
    pB[2] = upper_idx(NP + pkb, pkc, LDA);
    pB[3] = upper_idx(NP + pkb, NP + pkc, LDA);
  }
  (void)pP;
  (void)pQ;

  float* A = sm;
  {   // all global loads first, so that they are in flight together
    constexpr int NL = (TP * TP + kJregThreads - 1) / kJregThreads;
    double g[NL];
    float v[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int e = tid + u * kJregThreads;
      g[u] = e < TP * TP ? __ldg(G + e) : 0.0;
      v[u] = (e < TP * TP && warm) ? V_io[e] : 0.f;
    }
    // warm start: the previous solve's dominant eigenpairs (sigma > 8 theta),
    // the first kMaxDeflate of them in index order, are deflated from G in
    // FP64 before G is rounded to FP32, see below
    if (tid < TP) s_sig[tid] = warm && theta > 0.f ? sig_out[tid] : 0.f;
    __syncthreads();
    if (warp == 0) {
      int base = 0;
#pragma unroll
      for (int h = 0; h < TP; h += 32) {
        const int j = h + lane;
        const float sg = j < TP ? s_sig[j] : 0.f;
        const bool over = j < TP && sg > 8.f * theta;
        const unsigned m = __ballot_sync(0xffffffffu, over);
        const int rank = base + __popc(m & ((1u << lane) - 1u));
        const bool big = over && rank < kMaxDeflate;
        if (big) s_big[rank] = (unsigned char)j;
        if (j < TP) s_lam_big[j] = big ? sg * sg : 0.f;
        base += __popc(m);
      }
      if (lane == 0) s_nbig = base < kMaxDeflate ? base : kMaxDeflate;
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int e = tid + u * kJregThreads;
      if (e < TP * TP) {
        const int i = e / TP, j = e % TP;
        V[i * LDA + j] = warm ? v[u] : (i == j ? 1.f : 0.f);
      }
    }
    __syncthreads();
    // Warm start A = V^T G V.  Formed in FP32 from G as it stands, its
    // rounding (about u ||G||) would move the eigenvalues near theta^2, far
    // below ||G||, by more than the tolerance.  So the dominant part is
    // taken out first, in FP64: G' = G - sum_j lam_j v_j v_j^T over the
    // previous solve's dominant eigenpairs (an exact identity whatever the
    // pairs), then A = V^T G' V in FP32 (its rounding is now relative to
    // ||G'||) and lam_j is added back on the diagonal (V^T v_j = e_j up to
    // the FP32 orthogonality of V, whose error only touches the couplings
    // of the dominant eigenvalues, harmlessly).
    const int nb = s_nbig;
    // w_b = sqrt(lam_c) v_c in FP64, once, so that each entry costs one FP64
    // FMA per deflated pair (FP64 throughput is a small fraction of FP32
    // here); one square root per pair
    if (tid < nb) s_sq[tid] = sqrt((double)s_lam_big[s_big[tid]]);
    __syncthreads();
    for (int e = tid; e < nb * TP; e += kJregThreads) {
      const int b = e / TP, k = e % TP, c = s_big[b];
      s_wbig[b][k] = s_sq[b] * (double)V[k * LDA + c];
    }
    __syncthreads();
    // G' on the upper triangle (G is symmetric), mirrored: A is exactly symmetric
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int e = tid + u * kJregThreads;
      if (e < TP * TP) {
        const int i = e / TP, j = e % TP;
        if (i <= j) {
          double gd = g[u];
          for (int b = 0; b < nb; ++b) gd = fma(-s_wbig[b][i], s_wbig[b][j], gd);
          A[i * LDA + j] = A[j * LDA + i] = (float)gd;
        }
      }
    }
  }
  __syncthreads();
  if (warm) {   // A <- V^T G' V + diag(lam_big)
    kgemm<TP, LDA>(A, V, Tmp, nullptr);   // G' V (G' symmetric)
    __syncthreads();
    kgemm<TP, LDA>(V, Tmp, A, nullptr);   // V^T (G' V)
    __syncthreads();
    if (tid < TP) A[tid * LDA + tid] += s_lam_big[tid];
    __syncthreads();
  }
  for (int e = tid; e < TP * TP; e += kJregThreads) {   // symmetric part into the upper triangle
    const int i = e / TP, j = e % TP;
    if (i < j) A[i * LDA + j] = 0.5f * (A[i * LDA + j] + A[j * LDA + i]);
  }
  const bool vown = tid < TP * S;          // warp-uniform
  const int vi = tid / S, vg = tid % S;
  float vt[kJregM], vb[kJregM];
  if (vown) {
#pragma unroll
    for (int j = 0; j < kJregM; ++j) {
      vt[j] = V[vi * LDA + vg * kJregM + j];
      vb[j] = V[vi * LDA + NP + vg * kJregM + j];
    }
  }
  __syncthreads();
  if (tid < NP) {   // rotations of the first round
    float c, sn, tn;
    jacobi_rotation(A[tid * LDA + tid], A[(NP + tid) * LDA + NP + tid], A[tid * LDA + NP + tid], c, sn, tn);
    s_rot[0][0][tid] = c;
    s_rot[0][1][tid] = sn;
    s_rot[0][2][tid] = tn;
  }
  __syncthreads();

  const float th2 = theta * theta;
  const int max_rounds = max_sweeps * R;
  int done = 0, r = 0, cur = 0;    // rounds done; round within the sweep; current buffer
  for (;; ++done, r = (r + 1 == R) ? 0 : r + 1) {
    A = sm + cur * (TP * LDA);
    if (done % kJregCheck == 0 || done == max_rounds) {
      float off = 0.f, dg = 0.f;
      for (int e = tid; e < TP * TP; e += kJregThreads) {
        const int i = e / TP, j = e % TP;
        const float v = A[i * LDA + j];
        if (i == j) dg = fmaf(v, v, dg);
        else if (i < j) off = fmaf(2.f * v, v, off);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_down_sync(0xffffffffu, off, o);
        dg += __shfl_down_sync(0xffffffffu, dg, o);
      }
      if (lane == 0) {
        red[0][warp] = off;
        red[1][warp] = dg;
      }
      __syncthreads();
      if (warp == 0) {
        float so = lane < NW ? red[0][lane] : 0.f, sd = lane < NW ? red[1][lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          so += __shfl_down_sync(0xffffffffu, so, o);
          sd += __shfl_down_sync(0xffffffffu, sd, o);
        }
        if (lane == 0) {
          s_go = theta > 0.f || so > tol * tol * sd;
          s_floor = so <= 4.f * tol * tol * sd;   // ||E||_F <= 2 tol ||diag|| = 64 u ||diag|| (TP = 64)
          s_eps = sqrtf(so);
        }
      }
      __syncthreads();
      if (theta > 0.f) {   // the weighted test
        const float eps = s_eps;
        float out2 = 0.f;   // ||shrink*(X)||_F^2 = sum_i max(sigma_i - theta, 0)^2
        if (tid < TP) {
          const float li = A[tid * LDA + tid];
          const float x = fmaxf(li - eps, th2);
          s_slope[tid] = theta * 0.5f / (x * sqrtf(x));   // largest slope of f on [li - eps, inf)
          s_act[tid] = li + eps > th2;
          s_dg[tid] = li;
          const float sg = sqrtf(fmaxf(li, 0.f));
          out2 = sg > theta ? (sg - theta) * (sg - theta) : 0.f;
        }
        __syncthreads();
        float wsum = 0.f;
        for (int e = tid; e < TP * TP; e += kJregThreads) {
          const int i = e / TP, j = e % TP;
          if (i < j && (s_act[i] | s_act[j])) {
            const float gap = fabsf(s_dg[i] - s_dg[j]) - 2.f * eps;
            const float dd = gap > 0.f ? fminf(fmaxf(s_slope[i], s_slope[j]), __fdividef(1.f, gap))
                                       : fmaxf(s_slope[i], s_slope[j]);
            const float t = A[i * LDA + j] * dd;
            // (i, j) and (j, i) of the change of Wm, seen through X: sigma_i^2 + sigma_j^2
            const float w = fmaxf(s_dg[i], 0.f) + fmaxf(s_dg[j], 0.f) + 2.f * eps;
            wsum = fmaf(w * t, t, wsum);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          wsum += __shfl_down_sync(0xffffffffu, wsum, o);
          out2 += __shfl_down_sync(0xffffffffu, out2, o);
        }
        if (lane == 0) {
          red[0][warp] = wsum;
          red[1][warp] = out2;
        }
        __syncthreads();
        if (warp == 0) {
          float sw = lane < NW ? red[0][lane] : 0.f, fm = lane < NW ? red[1][lane] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_down_sync(0xffffffffu, sw, o);
            fm += __shfl_down_sync(0xffffffffu, fm, o);
          }
          if (lane == 0) {
            if (sw < 0.25f * s_best) {      // the measure (a square) halved
              s_best = sw;
              s_best_at = done;
            }
            // stagnation counts only once the plain measure is at its FP32
            // floor (far from it, after a poor warm start, a sweep may reduce
            // the weighted bound slowly while the rotations still make
            // progress) and only over a whole sweep: a pair is rotated once
            // per sweep, so the measure may stay flat for most of one
            if (sw <= tol * tol * fm || (s_floor && done - s_best_at >= R)) s_go = 0;
          }
        }
        __syncthreads();
      }
      if (!s_go || done == max_rounds) break;
    }
    const float* rc = &s_rot[done & 1][0][0];
    float* rn = &s_rot[(done + 1) & 1][0][0];
    float* An = sm + (cur ^ 1) * (TP * LDA);
    if (warp == 0) {
      if (lane < NP) {
        // the three entries of next round's pair, as this round leaves them
        const float tP = rc[2 * NP + pkP], tQ = rc[2 * NP + pkQ];
        const float aPP = A[pPdg], aQQ = A[pQdg], aPpq = A[pPpq], aQpq = A[pQpq];
        const float app = pPbot ? fmaf(tP, aPpq, aPP) : fmaf(-tP, aPpq, aPP);
        const float aqq = pQbot ? fmaf(tQ, aQpq, aQQ) : fmaf(-tQ, aQpq, aQQ);
        const float c = rc[pkb], sn = rc[NP + pkb], c2 = rc[pkc], s2 = rc[NP + pkc];
        const float a00 = A[pB[0]], a01 = A[pB[1]], a10 = A[pB[2]], a11 = A[pB[3]];
        const float r0 = pa ? rot_hi(c, sn, a00, a10) : rot_lo(c, sn, a00, a10);
        const float r1 = pa ? rot_hi(c, sn, a01, a11) : rot_lo(c, sn, a01, a11);
        const float apq = pb ? rot_hi(c2, s2, r0, r1) : rot_lo(c2, s2, r0, r1);
        float cn, snn, tnn;
        jacobi_rotation(app, aqq, apq, cn, snn, tnn);
        rn[lane] = cn;
        rn[NP + lane] = snn;
        rn[2 * NP + lane] = tnn;
      }
    } else {
#pragma unroll
      for (int u = 0; u < NBT; ++u) {
        if (kind[u] == 1) {
          const float c = rc[bkb[u]], sn = rc[NP + bkb[u]], c2 = rc[bkc[u]], s2 = rc[NP + bkc[u]];
          const float a00 = A[rd[u][0]], a01 = A[rd[u][1]], a10 = A[rd[u][2]], a11 = A[rd[u][3]];
          const float r00 = rot_lo(c, sn, a00, a10), r01 = rot_lo(c, sn, a01, a11);
          const float r10 = rot_hi(c, sn, a00, a10), r11 = rot_hi(c, sn, a01, a11);
          An[wr[u][0]] = rot_lo(c2, s2, r00, r01);
          An[wr[u][1]] = rot_hi(c2, s2, r00, r01);
          An[wr[u][2]] = rot_lo(c2, s2, r10, r11);
          An[wr[u][3]] = rot_hi(c2, s2, r10, r11);
        } else if (kind[u] == 2) {
          // the pair's own block: a_pq is zeroed exactly and -/+ t a_pq moves
          // onto the diagonal (the accurate classical update)
          const float apq = A[rd[u][2]], tn = rc[2 * NP + bkb[u]];
          An[wr[u][0]] = fmaf(-tn, apq, A[rd[u][0]]);
          An[wr[u][1]] = fmaf(tn, apq, A[rd[u][1]]);
          An[wr[u][2]] = 0.f;
        }
      }
    }
    if (vown) {
#pragma unroll
      for (int j = 0; j < kJregM; ++j) {
        const int k = vg * kJregM + j;
        const float c = rc[k], sn = rc[NP + k];
        const float vp = vt[j], vq = vb[j];
        vt[j] = rot_lo(c, sn, vp, vq);
        vb[j] = rot_hi(c, sn, vp, vq);
      }
      // one step along the ring
      const float recv_top = __shfl_up_sync(0xffffffffu, vt[kJregM - 1], 1, S);
      const float recv_bot = __shfl_down_sync(0xffffffffu, vb[0], 1, S);
      float nt[kJregM], nb[kJregM];
      if (vg == 0) {
        nt[0] = vt[0];
        nt[1] = vb[0];
#pragma unroll
        for (int j = 2; j < kJregM; ++j) nt[j] = vt[j - 1];
      } else {
        nt[0] = recv_top;
#pragma unroll
        for (int j = 1; j < kJregM; ++j) nt[j] = vt[j - 1];
      }
#pragma unroll
      for (int j = 0; j < kJregM - 1; ++j) nb[j] = vb[j + 1];
      nb[kJregM - 1] = (vg == S - 1) ? vt[kJregM - 1] : recv_bot;
#pragma unroll
      for (int j = 0; j < kJregM; ++j) {
        vt[j] = nt[j];
        vb[j] = nb[j];
      }
    }
    cur ^= 1;
    __syncthreads();
  }
  // slot s holds index pl[s] after round r of the sweep
  for (int slot = tid; slot < TP; slot += kJregThreads) {
    int idx = 0;
    if (slot != 0) {
      const int ring = slot < NP ? slot - 1 : TP - 2 - (slot - NP);
      const int j = ((ring - r) % R + R) % R;       // ring position this slot's index started from
      idx = j <= NP - 2 ? j + 1 : NP + TP - 2 - j;
    }
    s_pl[slot] = (unsigned char)idx;
  }
  __syncthreads();
  const unsigned char* pl = s_pl;
  if (vown) {
#pragma unroll
    for (int j = 0; j < kJregM; ++j) {
      V[vi * LDA + pl[vg * kJregM + j]] = vt[j];
      V[vi * LDA + pl[NP + vg * kJregM + j]] = vb[j];
    }
  }
  for (int sl = tid; sl < TP; sl += kJregThreads) {
    const float lam = A[sl * LDA + sl];
    const float sg = sqrtf(fmaxf(lam, 0.f));
    f[pl[sl]] = (sg > theta) ? (sg - theta) / sg : 0.f;
    sig_out[pl[sl]] = sg;
  }
  __syncthreads();
  float* Out = sm + (cur ^ 1) * (TP * LDA);
  // a solve that rotated nothing leaves V as the previous solve left it,
  // already re-orthonormalised
  if (done > 0) reorthonormalize_k<TP, LDA>(V, Tmp, Out);
  for (int e = tid; e < TP * TP; e += kJregThreads) {
    const int i = e / TP, j = e % TP;
    Tmp[i * LDA + j] = V[j * LDA + i];
  }
  __syncthreads();
  kgemm<TP, LDA>(Tmp, Tmp, Out, f);    // V diag(f) V^T = (V^T)^T diag(f) V^T
  __syncthreads();
  for (int e = tid; e < TP * TP; e += kJregThreads) {
    const int i = e / TP, j = e % TP;
    Wm[e] = Out[i * LDA + j];
    V_io[e] = V[i * LDA + j];
  }
  if (tid == 0) *rounds_out = done;
}

// Y[:, t] = sum_s Wm[s][t] X[:, s]: an (N x TP) x (TP x 64) product per
// block column t0..t0+63.  A CTA computes 128 rows (pixels) x 64 outputs with
// 256 threads, each 4 pixels x 8 outputs; X and Wm are staged in shared
// memory.  Optionally accumulates ||Y - Y_old||^2 (the dual residual term of
// Algorithm 3) into slot 1 of partials[block].
constexpr int kApplyRows = 128;

template <int TP>
__global__ void __launch_bounds__(256)
svt_apply_kernel(const float* __restrict__ X, long long ld, long long N, int T, const float* __restrict__ Wm,
                 float* __restrict__ Y, long long ldy, int reduce, int vec, double* __restrict__ partials) {
  constexpr int TB = 64;
  extern __shared__ __align__(16) float sm_apply[];
  float (*sW)[TB] = reinterpret_cast<float (*)[TB]>(sm_apply);                       // [TP][TB]
  float (*sx)[kApplyRows] = reinterpret_cast<float (*)[kApplyRows]>(sm_apply + TP * TB);   // [TP][rows]
  const int tid = threadIdx.x;
  const int t0 = blockIdx.y * TB;
  const int tp = tid & 31;          // pixel group: rows 4tp .. 4tp+3
  const int tt = tid >> 5;          // output group: cols 8tt .. 8tt+7
  for (int e = tid; e < TP * TB; e += 256) {
    const int s = e / TB, t = e % TB;
    sW[s][t] = (t0 + t < TP) ? Wm[s * TP + t0 + t] : 0.f;
  }
  float acc[kNumSums] = {};
  const long long nblk = (N + kApplyRows - 1) / kApplyRows;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const long long i0 = blk * kApplyRows;
    __syncthreads();
    for (int e = tid; e < TP * (kApplyRows / 4); e += 256) {
      const int s = e / (kApplyRows / 4), q = e % (kApplyRows / 4);
      const long long gi = i0 + 4 * q;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s < T) {
        const float* src = X + (long long)s * ld + gi;
        if (vec && gi + 3 < N) {
          v = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          if (gi < N) v.x = __ldg(src);
          if (gi + 1 < N) v.y = __ldg(src + 1);
          if (gi + 2 < N) v.z = __ldg(src + 2);
          if (gi + 3 < N) v.w = __ldg(src + 3);
        }
      }
      *reinterpret_cast<float4*>(&sx[s][4 * q]) = v;
    }
    __syncthreads();
    float y[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) y[a][b] = 0.f;
#pragma unroll 4
    for (int s = 0; s < TP; ++s) {
      const float4 x4 = *reinterpret_cast<const float4*>(&sx[s][4 * tp]);
      const float4 w0 = *reinterpret_cast<const float4*>(&sW[s][8 * tt]);
      const float4 w1 = *reinterpret_cast<const float4*>(&sW[s][8 * tt + 4]);
      const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
      const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) y[a][b] = fmaf(wv[b], xv[a], y[a][b]);
    }
    const long long gi = i0 + 4 * tp;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int t = t0 + 8 * tt + b;
      if (t >= T) continue;
      float* dst = Y + (long long)t * ldy + gi;
      if (vec && gi + 3 < N) {
        const float4 nv = make_float4(y[0][b], y[1][b], y[2][b], y[3][b]);
        if (reduce) {
          const float4 ov = *reinterpret_cast<const float4*>(dst);
          const float d0 = nv.x - ov.x, d1 = nv.y - ov.y, d2 = nv.z - ov.z, d3 = nv.w - ov.w;
          acc[1] += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
        }
        *reinterpret_cast<float4*>(dst) = nv;
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (gi + a < N) {
            if (reduce) {
              const float d = y[a][b] - dst[a];
              acc[1] = fmaf(d, d, acc[1]);
            }
            dst[a] = y[a][b];
          }
        }
      }
    }
  }
  if (reduce) block_sums_to<256>(acc, partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kNumSums);
}

template <int TP>
constexpr size_t apply_smem() {
  return (size_t)TP * (64 + kApplyRows) * sizeof(float);
}

template <int TP>
size_t jacobi_smem() {
  return (size_t)(3 * TP * (TP + 1) + TP) * sizeof(float);
}

}  // namespace

// Stopping tolerance of the FP32 Jacobi: 8 u sqrt(TP) (3.8e-6 at TP = 64).
// The register solver (TP <= 64) applies it to the first-order change of
// the SVT output relative to the output, and leaves earlier if FP32 rounding
// stalls that measure; the TP = 128 solver to the off-diagonal entries
// relative to their diagonal.  Near the ADMM's convergence the warm start of
// each outer iteration already meets it, so the solve takes few rounds.
float svt_tolerance(int T) { return 8.f * 5.96e-8f * sqrtf((float)svt_padded_T(T)); }

int svt_padded_T(int T) { return T <= 16 ? 16 : (T <= 32 ? 32 : (T <= 64 ? 64 : 128)); }

static int gram_simt_blocks(long long N) {
  const long long nch = (N + kGramChunk - 1) / kGramChunk;
  return (int)(nch < 152 * 2 ? nch : 152 * 2);
}

// Partial-Gram slots to allocate: enough for either Gram kernel.
int svt_gram_blocks(long long N) {
  const int a = gram_simt_blocks(N), b = svt_gram_tc_blocks(N);
  return a > b ? a : b;
}

int svt_apply_blocks(long long N, int T, int* gy) {
  *gy = (svt_padded_T(T) + 63) / 64;
  const long long nb = (N + kApplyRows - 1) / kApplyRows;
  return (int)(nb < 152 * 8 ? nb : 152 * 8);
}

cudaError_t svt_prepare() {
  cudaError_t e = cudaFuncSetAttribute(jacobi_svt_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_smem<128>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jacobi_reg_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jreg_smem<64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_partial_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<128>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_partial_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<64>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_partial_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<32>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_partial_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<16>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(svt_apply_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem<128>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(svt_apply_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem<64>());
  return e;
}

// partials: >= svt_gram_blocks(N) * TP * TP doubles; G: TP * TP doubles.
// With an error flag (err != NULL) and T > 16 the tensor-core kernel runs
// (gram_tcgen05.cu); it sets *err if a bounded wait expires.
cudaError_t svt_launch_gram(const float* X, long long ld, long long N, int T, double* partials, double* G, int* err,
                            cudaStream_t st) {
  const int TP = svt_padded_T(T);
  const int n = TP * TP;
  if (err && TP >= 32 && (ld * 4) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    float* fpart = reinterpret_cast<float*>(partials);   // FP32 partials in the same buffer
    cudaError_t e = svt_launch_gram_tc(X, ld, N, T, fpart, err, st);
    if (e != cudaSuccess) return e;
    gram_reduce_kernel<float><<<(n + 31) / 32, 32 * kRedWarps, 0, st>>>(fpart, svt_gram_tc_blocks(N), n, G);
    return cudaGetLastError();
  }
  const int nb = gram_simt_blocks(N);
  switch (TP) {
    case 16: gram_partial_kernel<16><<<nb, kGramThreads, gram_smem<16>(), st>>>(X, ld, N, T, partials); break;
    case 32: gram_partial_kernel<32><<<nb, kGramThreads, gram_smem<32>(), st>>>(X, ld, N, T, partials); break;
    case 64: gram_partial_kernel<64><<<nb, kGramThreads, gram_smem<64>(), st>>>(X, ld, N, T, partials); break;
    default: gram_partial_kernel<128><<<nb, kGramThreads, gram_smem<128>(), st>>>(X, ld, N, T, partials); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gram_reduce_kernel<double><<<(n + 31) / 32, 32 * kRedWarps, 0, st>>>(partials, nb, n, G);
  return cudaGetLastError();
}

cudaError_t svt_launch_eig(const double* G, int T, int warm, float theta, int max_sweeps, float tol, float* V_io,
                           float* Wm, float* sig, int* sweeps, cudaStream_t st) {
  const int TP = svt_padded_T(T);
  switch (TP) {
    case 16: jacobi_reg_kernel<16><<<1, kJregThreads, jreg_smem<16>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    case 32: jacobi_reg_kernel<32><<<1, kJregThreads, jreg_smem<32>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    case 64: jacobi_reg_kernel<64><<<1, kJregThreads, jreg_smem<64>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
    default: jacobi_svt_kernel<128><<<1, kJacobiThreads, jacobi_smem<128>(), st>>>(G, warm, theta, max_sweeps, tol, V_io, Wm, sig, sweeps); break;
  }
  return cudaGetLastError();
}

// With an error flag (err != NULL), no residual sum, T_pad = 32 or 64 and a
// TMA-compatible X the tensor-core kernel runs (svt_tcgen05.cu); it sets
// *err if a bounded wait expires.  partials (when reduce):
// svt_apply_blocks(N, T) * gy slots, ||Y - Y_old||^2 in slot 1.
cudaError_t svt_launch_apply(const float* X, long long ld, long long N, int T, const float* Wm, float* Y,
                             long long ldy, bool reduce, double* partials, int* err, cudaStream_t st) {
  const int TP = svt_padded_T(T);
  int gy = 1;
  const int nb = svt_apply_blocks(N, T, &gy);
  if (err && !reduce && (TP == 32 || TP == 64) && ld % 4 == 0 && ldy % 4 == 0 &&
      (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0)
    return svt_launch_apply_tc(X, ld, N, T, Wm, Y, ldy, err, st);
  const dim3 grid(nb, gy);
  const int vec = ((ld % 4) == 0 && (ldy % 4) == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(Y) % 16) == 0) ? 1 : 0;
  switch (TP) {
    case 16: svt_apply_kernel<16><<<grid, 256, apply_smem<16>(), st>>>(X, ld, N, T, Wm, Y, ldy, reduce, vec, partials); break;
    case 32: svt_apply_kernel<32><<<grid, 256, apply_smem<32>(), st>>>(X, ld, N, T, Wm, Y, ldy, reduce, vec, partials); break;
    case 64: svt_apply_kernel<64><<<grid, 256, apply_smem<64>(), st>>>(X, ld, N, T, Wm, Y, ldy, reduce, vec, partials); break;
    default: svt_apply_kernel<128><<<grid, 256, apply_smem<128>(), st>>>(X, ld, N, T, Wm, Y, ldy, reduce, vec, partials); break;
  }
  return cudaGetLastError();
}

}  // namespace otp
