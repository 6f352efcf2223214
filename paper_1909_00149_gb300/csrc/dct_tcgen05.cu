// Tensor-core (tcgen05) GEMMs for the DCT-II Neumann solve, split-BF16.
//
// Each of the four transforms of dct_solve.cu is D = A B^T with A = [rows][K]
// (the batch folded into the rows) and B = [N][K] a DCT matrix, both K-major.
// FP32-level accuracy from BF16 tensor cores by a 2-piece split of every
// operand, x = x_hi + x_lo (x_hi = bf16(x), x_lo = bf16(x - x_hi)), and three
// products per K step accumulated in FP32 in tensor memory:
//   D += A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T     (the A_lo B_lo term ~2^-18 is dropped)
// Per CTA: a 128 x NT tile of D (NT <= 256), K in 64-element chunks staged by
// TMA with 128-byte swizzle into two shared-memory stages.  One thread issues
// the TMA copies and the tcgen05.mma instructions; completion is signalled by
// tcgen05.commit to mbarriers.  All four warps then read the accumulator with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows) and run the
// epilogue: optional spectral scaling, optional per-problem transpose, output
// either as the next GEMM's BF16 hi/lo operand or as FP32.
// Every mbarrier wait is bounded; on expiry the CTA records an error, waits
// (bounded) for its copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/otprox.h"
#include "dct_plan.cuh"
#include "otprox_internal.cuh"
#include "tc_util.cuh"

namespace otp {
namespace {
using namespace tc;

constexpr int kTM = 128;                 // tile rows (TMEM lanes)
constexpr int kKC = 64;                  // K chunk: 64 bf16 = 128 bytes (one swizzle row)
constexpr int kStages = 2;
constexpr int kABytes = kTM * kKC * 2;   // one A operand tile (hi or lo): 16 KB

struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

struct TcEpi {
  int M, N, K;                // GEMM extents
  int rows_per_prob;          // rows of one problem (for the transpose / scaling)
  const float* inv_lam;       // scaling table [row-in-problem][n] (SCALE)
  int lam_ld;
  __nv_bfloat16* out_hi;      // OUT_BF16
  __nv_bfloat16* out_lo;
  float* out_f;               // FP32 output
  long long out_ld;           // row pitch of the output (elements)
};

template <int NT>
constexpr uint32_t stage_bytes() {
  return 2u * kABytes + 2u * NT * kKC * 2;
}

template <int NT>
constexpr int tmem_cols() {
  return NT <= 32 ? 32 : NT <= 64 ? 64 : NT <= 128 ? 128 : 256;
}

template <int NT>
constexpr size_t tc_smem() {
  return 1024 + (size_t)kStages * stage_bytes<NT>();
}

template <int NT, bool TRANS, bool SCALE, bool OUT_BF16>
__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, const TcEpi ep, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (s_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * NT;
  constexpr uint32_t SB = stage_bytes<NT>();
  constexpr uint32_t IDESC = bf16_idesc(kTM, NT);
  const int nchunks = (ep.K + kKC - 1) / kKC;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(s_u32(&bar_full[s]), 1);
      bar_init(s_u32(&bar_empty[s]), 1);
    }
    bar_init(s_u32(&bar_done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(s_u32(&s_tmem), tmem_cols<NT>());
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;

  auto stage_ptr = [&](int s) { return smem + (size_t)s * SB; };
  auto issue = [&](int s, int c) {
    unsigned char* st = stage_ptr(s);
    const uint32_t b = s_u32(&bar_full[s]);
    bar_expect(b, SB);
    tma2d(s_u32(st), &maps.a_hi, c * kKC, m0, b);
    tma2d(s_u32(st + kABytes), &maps.a_lo, c * kKC, m0, b);
    tma2d(s_u32(st + 2 * kABytes), &maps.b_hi, c * kKC, n0, b);
    tma2d(s_u32(st + 2 * kABytes + NT * kKC * 2), &maps.b_lo, c * kKC, n0, b);
  };

  if (tid == 0) {
    bool ok = true;
    for (int c = 0; c < nchunks && c < kStages; ++c) issue(c, c);
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % kStages;
      const uint32_t ph = (uint32_t)((c / kStages) & 1);
      if (!bar_wait(s_u32(&bar_full[s]), ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = s_u32(stage_ptr(s)), a_lo = a_hi + kABytes;
      const uint32_t b_hi = a_hi + 2 * kABytes, b_lo = b_hi + NT * kKC * 2;
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {      // K = 16 per instruction: 32 bytes along the row
        const uint32_t off = kk * 32;
        const uint64_t dah = sw128_desc(a_hi + off), dal = sw128_desc(a_lo + off);
        const uint64_t dbh = sw128_desc(b_hi + off), dbl = sw128_desc(b_lo + off);
        mma_bf16(tmem, dah, dbh, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, IDESC, 1u);
        mma_bf16(tmem, dal, dbh, IDESC, 1u);
      }
      mma_commit(s_u32(&bar_empty[s]));
      if (c + kStages < nchunks) {
        if (!bar_wait(s_u32(&bar_empty[s]), ph)) { ok = false; break; }
        issue(s, c + kStages);
      }
    }
    // bar_done tracks every MMA issued so far (tcgen05.commit covers all prior ones)
    mma_commit(s_u32(&bar_done));
    if (!ok) {
      s_fail = 1;
      atomicExch(err, 1);
      // bounded waits for the MMAs and the copies still in flight before the
      // tensor and shared memory are released
      (void)bar_wait(s_u32(&bar_done), 0);
      for (int s = 0; s < kStages; ++s) (void)bar_wait(s_u32(&bar_full[s]), 0);
    }
  }
  __syncthreads();
  bool done = !s_fail && bar_wait(s_u32(&bar_done), 0);
  done = __syncthreads_and(done) != 0;
  if (done) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + warp * 32 + lane;            // this thread's tile row
    const bool row_ok = m < ep.M;
    const int b = row_ok ? m / ep.rows_per_prob : 0, i = row_ok ? m % ep.rows_per_prob : 0;
#pragma unroll 1
    for (int cc = 0; cc < NT / 32; ++cc) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
      if (!row_ok) continue;
      const int nb = n0 + cc * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = nb + j;
        if (n >= ep.N) break;
        float x = v[j];
        if (SCALE) x *= __ldg(ep.inv_lam + (long long)i * ep.lam_ld + n);
        const long long o = TRANS ? ((long long)b * ep.N + n) * ep.out_ld + i : (long long)m * ep.out_ld + n;
        if (OUT_BF16) {
          const __nv_bfloat16 hi = __float2bfloat16_rn(x);
          ep.out_hi[o] = hi;
          ep.out_lo[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
        } else {
          ep.out_f[o] = x;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, tmem_cols<NT>());
  }
}

// X (FP32, rows of pitch x_ld) -> BF16 hi/lo rows of pitch ld (K = cols).
__global__ void split_bf16_kernel(const float* __restrict__ X, long long x_ld, int rows, int cols,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long long ld) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    const float x = X[r * x_ld + c];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[r * ld + c] = h;
    lo[r * ld + c] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// ------------------------------------------------------------------ host side
// 2-D BF16 map over [rows][K] with row pitch ld elements (extent K, rows);
// box = 64 x box_rows with 128-byte swizzle.
int encode_bf16_map(CUtensorMap* m, const void* base, long long K, long long rows, long long ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tc::encode_fn();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }
int ntile_for(int N) {
  const int n = N > 256 ? 256 : round_up(N, 16);
  return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256;
}

uint16_t f2bf_bits(float x) {   // round to nearest even
  uint32_t u;
  memcpy(&u, &x, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
float bf_bits2f(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

struct TcPlan {
  int KpH, KpW;
  // B operands (hi, lo): CW [W][KpW], CH [H][KpH], CHt [H][KpH], CWt [W][KpW]
  uint16_t* mats;
  __nv_bfloat16 *cw_hi, *cw_lo, *ch_hi, *ch_lo, *cht_hi, *cht_lo, *cwt_hi, *cwt_lo;
  // work operands (hi, lo): bufA [B*H][KpW], bufB1 / bufB2 [B*W][KpH]
  __nv_bfloat16* work;
  __nv_bfloat16 *a_hi, *a_lo, *b1_hi, *b1_lo, *b2_hi, *b2_lo;
  TcMaps g1, g2, g3, g4;
  int* err;
};

template <int NT, bool TRANS, bool SCALE, bool OUT_BF16>
cudaError_t launch_tc(const TcMaps& maps, const TcEpi& ep, int* err, cudaStream_t st) {
  static unsigned long long attr_set = 0;
  if (needs_setup(attr_set)) {
    const cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<NT, TRANS, SCALE, OUT_BF16>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<NT>());
    if (e != cudaSuccess) return e;
    mark_setup(attr_set);
  }
  const dim3 grid((ep.M + kTM - 1) / kTM, (ep.N + NT - 1) / NT);
  tc_gemm_kernel<NT, TRANS, SCALE, OUT_BF16><<<grid, 128, tc_smem<NT>(), st>>>(maps, ep, err);
  return cudaGetLastError();
}

template <bool TRANS, bool SCALE, bool OUT_BF16>
cudaError_t launch_tc_n(int NT, const TcMaps& maps, const TcEpi& ep, int* err, cudaStream_t st) {
  switch (NT) {
    case 32: return launch_tc<32, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    case 64: return launch_tc<64, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    case 128: return launch_tc<128, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    default: return launch_tc<256, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
  }
}

}  // namespace

int dct_tc_create(DctPlan* p) {
  TcPlan* t = (TcPlan*)calloc(1, sizeof(TcPlan));
  if (!t) return fail(OT_ENOMEM, "dct tc plan: host allocation");
  p->tc = t;
  const int B = p->B, H = p->H, W = p->W;
  t->KpH = round_up(H, 64);
  t->KpW = round_up(W, 64);
  const size_t nW = (size_t)W * t->KpW, nH = (size_t)H * t->KpH;
  // host: BF16 hi/lo of C_W, C_H, C_H^T, C_W^T with padded pitch
  std::vector<uint16_t> host(4 * (nW + nH), 0);
  const std::vector<double> CH = dct_matrix(H), CW = dct_matrix(W);
  auto put = [&](size_t base_hi, size_t base_lo, const std::vector<double>& C, int n, int ld, bool tr) {
    for (int r = 0; r < n; ++r)
      for (int k = 0; k < n; ++k) {
        const double v = tr ? C[(size_t)k * n + r] : C[(size_t)r * n + k];
        const uint16_t hb = f2bf_bits((float)v);
        host[base_hi + (size_t)r * ld + k] = hb;
        host[base_lo + (size_t)r * ld + k] = f2bf_bits((float)(v - (double)bf_bits2f(hb)));
      }
  };
  const size_t o_cw = 0, o_ch = 2 * nW, o_cht = 2 * nW + 2 * nH, o_cwt = 2 * nW + 4 * nH;
  put(o_cw, o_cw + nW, CW, W, t->KpW, false);
  put(o_ch, o_ch + nH, CH, H, t->KpH, false);
  put(o_cht, o_cht + nH, CH, H, t->KpH, true);
  put(o_cwt, o_cwt + nW, CW, W, t->KpW, true);
  cudaError_t e = cudaMalloc(&t->mats, host.size() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(t->mats, host.data(), host.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "dct tc plan: matrices");
  __nv_bfloat16* m = reinterpret_cast<__nv_bfloat16*>(t->mats);
  t->cw_hi = m + o_cw;
  t->cw_lo = m + o_cw + nW;
  t->ch_hi = m + o_ch;
  t->ch_lo = m + o_ch + nH;
  t->cht_hi = m + o_cht;
  t->cht_lo = m + o_cht + nH;
  t->cwt_hi = m + o_cwt;
  t->cwt_lo = m + o_cwt + nW;
  const size_t nA = (size_t)B * H * t->KpW, nB = (size_t)B * W * t->KpH;
  e = cudaMalloc(&t->work, (2 * nA + 4 * nB) * sizeof(__nv_bfloat16) + 256);
  if (e == cudaSuccess) e = cudaMemset(t->work, 0, (2 * nA + 4 * nB) * sizeof(__nv_bfloat16) + 256);
  if (e != cudaSuccess) return cuda_fail(e, "dct tc plan: work buffers");
  t->a_hi = t->work;
  t->a_lo = t->a_hi + nA;
  t->b1_hi = t->a_lo + nA;
  t->b1_lo = t->b1_hi + nB;
  t->b2_hi = t->b1_lo + nB;
  t->b2_lo = t->b2_hi + nB;
  t->err = reinterpret_cast<int*>(t->b2_lo + nB);
  if (!p->err) p->err = t->err;
  // G1: A = X split [B*H][KpW] (K = W), B = C_W [W][KpW] (N = W)
  // G2: A = U^T [B*W][KpH] (K = H), B = C_H [H][KpH] (N = H)
  // G3: A = V' [B*W][KpH] (K = H), B = C_H^T [H][KpH] (N = H)
  // G4: A = P^T [B*H][KpW] (K = W), B = C_W^T [W][KpW] (N = W)
  const int ntW = ntile_for(W), ntH = ntile_for(H);
  int rc = 0;
  rc |= encode_bf16_map(&t->g1.a_hi, t->a_hi, W, (long long)B * H, t->KpW, kTM);
  rc |= encode_bf16_map(&t->g1.a_lo, t->a_lo, W, (long long)B * H, t->KpW, kTM);
  rc |= encode_bf16_map(&t->g1.b_hi, t->cw_hi, W, W, t->KpW, ntW);
  rc |= encode_bf16_map(&t->g1.b_lo, t->cw_lo, W, W, t->KpW, ntW);
  rc |= encode_bf16_map(&t->g2.a_hi, t->b1_hi, H, (long long)B * W, t->KpH, kTM);
  rc |= encode_bf16_map(&t->g2.a_lo, t->b1_lo, H, (long long)B * W, t->KpH, kTM);
  rc |= encode_bf16_map(&t->g2.b_hi, t->ch_hi, H, H, t->KpH, ntH);
  rc |= encode_bf16_map(&t->g2.b_lo, t->ch_lo, H, H, t->KpH, ntH);
  rc |= encode_bf16_map(&t->g3.a_hi, t->b2_hi, H, (long long)B * W, t->KpH, kTM);
  rc |= encode_bf16_map(&t->g3.a_lo, t->b2_lo, H, (long long)B * W, t->KpH, kTM);
  rc |= encode_bf16_map(&t->g3.b_hi, t->cht_hi, H, H, t->KpH, ntH);
  rc |= encode_bf16_map(&t->g3.b_lo, t->cht_lo, H, H, t->KpH, ntH);
  rc |= encode_bf16_map(&t->g4.a_hi, t->a_hi, W, (long long)B * H, t->KpW, kTM);
  rc |= encode_bf16_map(&t->g4.a_lo, t->a_lo, W, (long long)B * H, t->KpW, kTM);
  rc |= encode_bf16_map(&t->g4.b_hi, t->cwt_hi, W, W, t->KpW, ntW);
  rc |= encode_bf16_map(&t->g4.b_lo, t->cwt_lo, W, W, t->KpW, ntW);
  if (rc != 0) return fail(OT_ECUDA, "dct tc plan: cuTensorMapEncodeTiled failed (%d)", rc);
  return OT_OK;
}

void dct_tc_destroy(DctPlan* p) {
  TcPlan* t = (TcPlan*)p->tc;
  if (!t) return;
  cudaFree(t->mats);
  cudaFree(t->work);
  free(t);
  p->tc = nullptr;
}

cudaError_t dct_tc_solve(DctPlan* p, const float* X, long long x_ld, float* Y, long long y_ld, cudaStream_t st) {
  TcPlan* t = (TcPlan*)p->tc;
  int* err = p->err;
  const int B = p->B, H = p->H, W = p->W;
  const int ntW = ntile_for(W), ntH = ntile_for(H);
  split_bf16_kernel<<<152 * 8, 256, 0, st>>>(X, x_ld, B * H, W, t->a_hi, t->a_lo, t->KpW);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcEpi ep;
  memset(&ep, 0, sizeof ep);
  // G1: U^T = (X C_W^T)^T -> b1 [B*W][KpH]
  ep.M = B * H; ep.N = W; ep.K = W; ep.rows_per_prob = H;
  ep.out_hi = t->b1_hi; ep.out_lo = t->b1_lo; ep.out_ld = t->KpH;
  e = launch_tc_n<true, false, true>(ntW, t->g1, ep, err, st);
  if (e != cudaSuccess) return e;
  // G2: Xhat^T / lam -> b2 [B*W][KpH]
  ep.M = B * W; ep.N = H; ep.K = H; ep.rows_per_prob = W; ep.inv_lam = p->inv_lam; ep.lam_ld = H;
  ep.out_hi = t->b2_hi; ep.out_lo = t->b2_lo; ep.out_ld = t->KpH;
  e = launch_tc_n<false, true, true>(ntH, t->g2, ep, err, st);
  if (e != cudaSuccess) return e;
  // G3: P = Xhat'^T C_H, stored transposed -> a [B*H][KpW]
  ep.M = B * W; ep.N = H; ep.K = H; ep.rows_per_prob = W; ep.inv_lam = nullptr;
  ep.out_hi = t->a_hi; ep.out_lo = t->a_lo; ep.out_ld = t->KpW;
  e = launch_tc_n<true, false, true>(ntH, t->g3, ep, err, st);
  if (e != cudaSuccess) return e;
  // G4: Y = P^T C_W (FP32)
  ep.M = B * H; ep.N = W; ep.K = W; ep.rows_per_prob = H;
  ep.out_hi = ep.out_lo = nullptr; ep.out_f = Y; ep.out_ld = y_ld;
  return launch_tc_n<false, false, false>(ntW, t->g4, ep, err, st);
}

}  // namespace otp
