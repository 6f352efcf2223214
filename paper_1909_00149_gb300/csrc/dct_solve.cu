// Neumann grid-Laplacian solve (D D* + c I)^{-1} X by the orthonormal DCT-II.
//
// D D* is the graph Laplacian of the H x W grid with zero-flux boundary (the
// operator behind Theorem 1's step bound).  It is a Kronecker sum of two path
// Laplacians whose eigenvectors are the DCT-II basis C[k][m] = s_k cos(pi
// (m + 1/2) k / n), eigenvalues 4 sin^2(pi k / 2n), so
//   Y = C_H^T [ (C_H X C_W^T) / (lam_H[k] + lam_W[l] + c) ] C_W,
// the zero mode dropped when c = 0.
//
// Each transform is one large GEMM Z = A B^T with the whole batch folded into
// the rows of A (M = B * rows), and the epilogue writes Z transposed so that
// the next transform is again a row transform:
//   G1: U^T    = (X C_W^T)^T        rows (b, i) -> stored [B][W][H]
//   G2: Xhat^T = U^T C_H^T, / lam   rows (b, l) -> stored [B][W][H]  (scaled)
//   G3: P      = Xhat'^T C_H        rows (b, l) -> stored transposed [B][H][W]
//   G4: Y      = P^T C_W            rows (b, i) -> stored [B][H][W]
// Precision OT_PREC_FP32: FP32 CUDA-core tiles.  OT_PREC_SPLIT_BF16 and
// OT_PREC_SPLIT_BF16_3: tcgen05 tensor-core GEMMs on a 2- or 3-piece BF16
// split of every operand (dct_tcgen05.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"
#include "dct_plan.cuh"

namespace otp {
namespace {

constexpr int kGT = 64;        // output tile (rows x cols)
constexpr int kGK = 16;        // K chunk

// Z = A B^T: A [M][K] (row pitch lda), B [N][K] (row pitch ldb), FP32.
// Epilogue: scale by inv_lam[col][row-in-problem] (mode & 1), and write
// transposed per problem (mode & 2): row m = (b, i) of a problem with
// `rows_per_prob` rows -> out[b][col][i] (pitch out_ld), else out[m][col].
__global__ void __launch_bounds__(256)
gemm_f32_kernel(const float* __restrict__ A, int lda, const float* __restrict__ Bm, int ldb, int M, int N, int K,
                int mode, int rows_per_prob, const float* __restrict__ inv_lam, int lam_ld, float* __restrict__ out,
                long long out_ld, long long out_prob_stride) {
  __shared__ __align__(16) float sA[kGK][kGT + 4];
  __shared__ __align__(16) float sB[kGK][kGT + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int e = tid; e < kGT * kGK; e += 256) {
      const int r = e / kGK, kk = e % kGK;
      const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
      sA[kk][r] = (gm < M && gk < K) ? __ldg(A + (long long)gm * lda + gk) : 0.f;
      sB[kk][r] = (gn < N && gk < K) ? __ldg(Bm + (long long)gn * ldb + gk) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&sA[kk][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&sB[kk][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int m = m0 + 4 * ty + r;
    if (m >= M) continue;
    const int b = m / rows_per_prob, i = m % rows_per_prob;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = n0 + 4 * tx + c;
      if (n >= N) continue;
      float v = acc[r][c];
      if (mode & 1) v *= inv_lam[(long long)i * lam_ld + n];
      if (mode & 2)
        out[(long long)b * out_prob_stride + (long long)n * out_ld + i] = v;
      else
        out[(long long)m * out_ld + n] = v;
    }
  }
}

}  // namespace

std::vector<double> dct_matrix(int n) {
  std::vector<double> C((size_t)n * n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double s = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
    for (int m = 0; m < n; ++m) C[(size_t)k * n + m] = s * cos(pi * (m + 0.5) * k / n);
  }
  return C;
}

std::vector<double> path_laplacian_eigs(int n) {
  std::vector<double> lam(n);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double s = sin(pi * k / (2.0 * n));
    lam[k] = 4.0 * s * s;
  }
  return lam;
}

namespace {

cudaError_t upload(float** dst, const std::vector<float>& v) {
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

void dct_plan_destroy(DctPlan* p) {
  if (!p) return;
  if (p->tc) dct_tc_destroy(p);
  cudaFree(p->CH);
  cudaFree(p->CHt);
  cudaFree(p->CW);
  cudaFree(p->CWt);
  cudaFree(p->inv_lam);
  cudaFree(p->work);
  free(p);
}

int dct_plan_create(int B, int H, int W, double c, int precision, DctPlan** out) {
  *out = nullptr;
  DctPlan* p = (DctPlan*)calloc(1, sizeof(DctPlan));
  if (!p) return fail(OT_ENOMEM, "dct plan: host allocation");
  p->B = B;
  p->H = H;
  p->W = W;
  p->c = c;
  p->precision = precision;
  auto as_f32 = [](const std::vector<double>& v, bool transpose, int n) {
    std::vector<float> f(v.size());
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) f[(size_t)i * n + j] = (float)(transpose ? v[(size_t)j * n + i] : v[(size_t)i * n + j]);
    return f;
  };
  const std::vector<double> CH = dct_matrix(H), CW = dct_matrix(W);
  cudaError_t e = upload(&p->CH, as_f32(CH, false, H));
  if (e == cudaSuccess) e = upload(&p->CHt, as_f32(CH, true, H));
  if (e == cudaSuccess) e = upload(&p->CW, as_f32(CW, false, W));
  if (e == cudaSuccess) e = upload(&p->CWt, as_f32(CW, true, W));
  const std::vector<double> lH = path_laplacian_eigs(H), lW = path_laplacian_eigs(W);
  std::vector<float> il((size_t)W * H);
  for (int l = 0; l < W; ++l)
    for (int k = 0; k < H; ++k) {
      const double d = lW[l] + lH[k] + c;
      il[(size_t)l * H + k] = d > 1e-12 ? (float)(1.0 / d) : 0.f;
    }
  if (e == cudaSuccess) e = upload(&p->inv_lam, il);
  const int mx = H > W ? H : W;
  if (e == cudaSuccess) e = cudaMalloc(&p->work, (size_t)B * mx * mx * sizeof(float));
  if (e != cudaSuccess) {
    dct_plan_destroy(p);
    return cuda_fail(e, "dct plan: device tables");
  }
  if (precision == OT_PREC_SPLIT_BF16 || precision == OT_PREC_SPLIT_BF16_3) {
    const int rc = dct_tc_create(p);
    if (rc != OT_OK) {
      dct_plan_destroy(p);
      return rc;
    }
  }
  *out = p;
  return OT_OK;
}

void dct_plan_set_error_flag(DctPlan* p, int* derr) {
  if (p && derr) p->err = derr;
}

// Y = (D D* + c I)^{-1} X for B problems; X, Y device [B][H][*] with row
// pitch x_ld / y_ld floats (problem stride H * ld).  X and Y may alias.
cudaError_t dct_plan_solve(DctPlan* p, const float* X, long long x_ld, float* Y, long long y_ld, cudaStream_t st) {
  if (p->precision != OT_PREC_FP32) return dct_tc_solve(p, X, x_ld, Y, y_ld, st);
  const int B = p->B, H = p->H, W = p->W;
  float* U = p->work;
  const dim3 blk(256);
  // G1: U^T = (X C_W^T)^T, rows (b, i); X rows have pitch x_ld (problem stride H*x_ld = contiguous rows)
  {
    const dim3 grid((B * H + kGT - 1) / kGT, (W + kGT - 1) / kGT);
    gemm_f32_kernel<<<grid, blk, 0, st>>>(X, (int)x_ld, p->CW, W, B * H, W, W, 2, H, nullptr, 0, U, H,
                                          (long long)W * H);
  }
  // G2: Xhat^T scaled (in place is not possible: write into Y as scratch when it does not alias X)
  // Use a second region: Y (size >= B*H*y_ld >= B*H*W) as the scaled spectrum [B][W][H].
  float* V = Y;
  {
    const dim3 grid((B * W + kGT - 1) / kGT, (H + kGT - 1) / kGT);
    gemm_f32_kernel<<<grid, blk, 0, st>>>(U, H, p->CH, H, B * W, H, H, 1, W, p->inv_lam, H, V, H, 0);
  }
  // G3: P = Xhat'^T C_H -> stored transposed [B][H][W] into U
  {
    const dim3 grid((B * W + kGT - 1) / kGT, (H + kGT - 1) / kGT);
    gemm_f32_kernel<<<grid, blk, 0, st>>>(V, H, p->CHt, H, B * W, H, H, 2, W, nullptr, 0, U, W, (long long)H * W);
  }
  // G4: Y = P^T C_W, rows (b, i), out pitch y_ld
  {
    const dim3 grid((B * H + kGT - 1) / kGT, (W + kGT - 1) / kGT);
    gemm_f32_kernel<<<grid, blk, 0, st>>>(U, W, p->CWt, W, B * H, W, W, 0, H, nullptr, 0, Y, y_ld, 0);
  }
  return cudaGetLastError();
}

}  // namespace otp

using namespace otp;

extern "C" int ot_neumann_solve(const float* X, float* Y, int32_t B, int32_t H, int32_t W, double c,
                                int32_t precision, void* cuda_stream) {
  if (!X || !Y) return fail(OT_EINVAL, "ot_neumann_solve: NULL argument");
  if (B < 1 || H < 1 || W < 1) return fail(OT_EINVAL, "ot_neumann_solve: B, H, W must be >= 1");
  if (!(c >= 0) || !isfinite(c)) return fail(OT_EINVAL, "ot_neumann_solve: c must be >= 0");
  if (precision != OT_PREC_FP32 && precision != OT_PREC_SPLIT_BF16 && precision != OT_PREC_SPLIT_BF16_3)
    return fail(OT_EINVAL, "ot_neumann_solve: unknown precision %d", precision);
  if ((double)B * H * W > 2.0e9) return fail(OT_EINVAL, "ot_neumann_solve: problem too large");
  DctPlan* p = nullptr;
  int rc = dct_plan_create(B, H, W, c, precision, &p);
  if (rc != OT_OK) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  // X is read by G1 before Y is first written (G2), so X and Y may alias.
  cudaError_t e = dct_plan_solve(p, X, W, Y, W, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int flag = 0;
  if (e == cudaSuccess && p->err) e = cudaMemcpy(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost);
  dct_plan_destroy(p);
  if (e != cudaSuccess) return cuda_fail(e, "ot_neumann_solve");
  if (flag) return fail(OT_ETIMEOUT, "ot_neumann_solve: a bounded device wait expired in a tensor-core GEMM");
  return OT_OK;
}

// The same solve repeated n_rep times on one plan, bracketed by CUDA events
// on the caller's stream after one untimed solve: the device time of one
// solve (the operand split and the four GEMMs for split BF16), without the
// plan's set-up.
extern "C" int ot_neumann_solve_timed(const float* X, float* Y, int32_t B, int32_t H, int32_t W, double c,
                                      int32_t precision, int32_t n_rep, double* ms_per_solve, void* cuda_stream) {
  if (!X || !Y || !ms_per_solve) return fail(OT_EINVAL, "ot_neumann_solve_timed: NULL argument");
  if (B < 1 || H < 1 || W < 1) return fail(OT_EINVAL, "ot_neumann_solve_timed: B, H, W must be >= 1");
  if (!(c >= 0) || !isfinite(c)) return fail(OT_EINVAL, "ot_neumann_solve_timed: c must be >= 0");
  if (precision != OT_PREC_FP32 && precision != OT_PREC_SPLIT_BF16 && precision != OT_PREC_SPLIT_BF16_3)
    return fail(OT_EINVAL, "ot_neumann_solve_timed: unknown precision %d", precision);
  if (n_rep < 1) return fail(OT_EINVAL, "ot_neumann_solve_timed: n_rep must be >= 1");
  if ((double)B * H * W > 2.0e9) return fail(OT_EINVAL, "ot_neumann_solve_timed: problem too large");
  DctPlan* p = nullptr;
  int rc = dct_plan_create(B, H, W, c, precision, &p);
  if (rc != OT_OK) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = dct_plan_solve(p, X, W, Y, W, st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int k = 0; k < n_rep && e == cudaSuccess; ++k) e = dct_plan_solve(p, X, W, Y, W, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  int flag = 0;
  if (e == cudaSuccess && p->err) e = cudaMemcpy(&flag, p->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dct_plan_destroy(p);
  if (e != cudaSuccess) return cuda_fail(e, "ot_neumann_solve_timed");
  if (flag) return fail(OT_ETIMEOUT, "ot_neumann_solve_timed: a bounded device wait expired in a tensor-core GEMM");
  *ms_per_solve = ms / n_rep;
  return OT_OK;
}
