// Tensor-core (tcgen05) GEMMs for the DCT-II Neumann solve, split-BF16.
//
// Each of the four transforms of dct_solve.cu is D = A B^T with A = [rows][K]
// (the batch folded into the rows) and B = [N][K] a DCT matrix, both K-major.
// Near-FP32 accuracy from BF16 tensor cores by splitting every operand into
// NP BF16 pieces and accumulating their leading products in FP32 in tensor
// memory, the leading product hh in one accumulator and the corrections
// (2^-8 of it and below) in a second, so that adding a correction into a
// value dominated by hh does not cost its low bits at every K step (with one
// accumulator the 3-piece split lost about 2^-23 of the total per addition,
// 2.8e-5 relative at K = 1024); the two are added once in the epilogue:
//   NP = 2: x = x_h + x_l (x_h = bf16(x), x_l = bf16(x - x_h)); three products
//           per K step, D += A_h B_h^T + A_h B_l^T + A_l B_h^T (A_l B_l, about
//           2^-18 of the result, dropped): about 2^-17 relative per product;
//   NP = 3: x = x_h + x_m + x_l exactly for every FP32 x (8 + 8 + 8
//           significant bits); the six products of weight >= 2^-16, hh, hm,
//           mh, mm, hl, lh (ml, lm, ll, below 2^-24, dropped): the error of
//           FP32 arithmetic.
// Per CTA: a 128 x NT tile of D (NT <= 256 for NP = 2, <= 128 for NP = 3, so
// that two stages fit in shared memory), K in 64-element chunks staged by
// TMA with 128-byte swizzle into two shared-memory stages.  One thread issues
// the TMA copies and the tcgen05.mma instructions; completion is signalled by
// tcgen05.commit to mbarriers.  All four warps then read the accumulator with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows) and run the
// epilogue: optional spectral scaling, optional per-problem transpose, output
// either as the next GEMM's NP BF16 pieces or as FP32.
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

constexpr int kMaxPieces = 3;

struct TcMaps {
  CUtensorMap a[kMaxPieces], b[kMaxPieces];   // piece 0 = hi, then (mid,) lo
};

struct TcEpi {
  int M, N, K;                // GEMM extents
  int rows_per_prob;          // rows of one problem (for the transpose / scaling)
  const float* inv_lam;       // scaling table [row-in-problem][n] (SCALE)
  int lam_ld;
  __nv_bfloat16* out[kMaxPieces];   // OUT_BF16: the pieces of the next GEMM's operand
  float* out_f;               // FP32 output
  long long out_ld;           // row pitch of the output (elements)
};

template <int NT, int NP>
constexpr uint32_t stage_bytes() {
  return (uint32_t)NP * kABytes + (uint32_t)NP * NT * kKC * 2;
}

// Two FP32 accumulators of NT columns each: the leading product (hh) in the
// first, the correction products in the second, added in the epilogue.
template <int NT>
constexpr int tmem_cols() {
  return NT <= 16 ? 32 : NT <= 32 ? 64 : NT <= 64 ? 128 : NT <= 128 ? 256 : 512;
}

template <int NT, int NP>
constexpr size_t tc_smem() {
  return 1024 + (size_t)kStages * stage_bytes<NT, NP>();
}

// The NP pieces of x, highest first (NP = 3: exact; NP = 2: x_l rounded).
template <int NP>
__device__ __forceinline__ void split_pieces(float x, __nv_bfloat16 (&p)[kMaxPieces]) {
  p[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p[0]);
  p[1] = __float2bfloat16_rn(r1);
  if (NP == 3) p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
}

template <int NT, int NP, bool TRANS, bool SCALE, bool OUT_BF16>
__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ TcMaps maps, const TcEpi ep, int* __restrict__ err) {
  static_assert(NP == 2 || NP == 3, "two or three pieces");
  static_assert(tc_smem<NT, NP>() <= 227 * 1024, "two stages must fit in shared memory");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (s_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * NT;
  constexpr uint32_t SB = stage_bytes<NT, NP>();
  constexpr uint32_t kBBytes = NT * kKC * 2;   // one B operand tile
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
#pragma unroll
    for (int q = 0; q < NP; ++q) tma2d(s_u32(st + q * kABytes), &maps.a[q], c * kKC, m0, b);
#pragma unroll
    for (int q = 0; q < NP; ++q) tma2d(s_u32(st + NP * kABytes + q * kBBytes), &maps.b[q], c * kKC, n0, b);
  };

  if (tid == 0) {
    bool ok = true;
    for (int c = 0; c < nchunks && c < kStages; ++c) issue(c, c);
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % kStages;
      const uint32_t ph = (uint32_t)((c / kStages) & 1);
      if (!bar_wait(s_u32(&bar_full[s]), ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = s_u32(stage_ptr(s)), b0 = a0 + NP * kABytes;
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {      // K = 16 per instruction: 32 bytes along the row
        const uint32_t off = kk * 32;
        const uint64_t dah = sw128_desc(a0 + off), dal = sw128_desc(a0 + kABytes + off);
        const uint64_t dbh = sw128_desc(b0 + off), dbl = sw128_desc(b0 + kBBytes + off);
        const uint32_t first = (c > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, dah, dbh, IDESC, first);                 // hh into the first accumulator
        mma_bf16(tmem + NT, dah, dbl, IDESC, first);            // corrections into the second
        mma_bf16(tmem + NT, dal, dbh, IDESC, 1u);
        if (NP == 3) {   // pieces: 0 = h, 1 = m, 2 = l; add mm, hl, lh
          const uint64_t dam = dal, dbm = dbl;
          const uint64_t da3 = sw128_desc(a0 + 2 * kABytes + off), db3 = sw128_desc(b0 + 2 * kBBytes + off);
          mma_bf16(tmem + NT, dam, dbm, IDESC, 1u);
          mma_bf16(tmem + NT, dah, db3, IDESC, 1u);
          mma_bf16(tmem + NT, da3, dbh, IDESC, 1u);
        }
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
    // untransposed output: the warp's 32 x 32 block goes through shared
    // memory (the stage buffers are idle once the accumulator is complete),
    // so that a lane holds a column and each store covers a row segment
    float* tw = reinterpret_cast<float*>(smem) + warp * 32 * 33;
#pragma unroll 1
    for (int cc = 0; cc < NT / 32; ++cc) {
      float v[32], w[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(NT + cc * 32), w);
      const int nb = n0 + cc * 32;
      if (TRANS) {
        if (!row_ok) continue;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = nb + j;
          if (n >= ep.N) break;
          float x = v[j] + w[j];
          if (SCALE) x *= __ldg(ep.inv_lam + (long long)i * ep.lam_ld + n);
          const long long o = ((long long)b * ep.N + n) * ep.out_ld + i;
          if (OUT_BF16) {
            __nv_bfloat16 pc[kMaxPieces];
            split_pieces<NP>(x, pc);
#pragma unroll
            for (int q = 0; q < NP; ++q) ep.out[q][o] = pc[q];
          } else {
            ep.out_f[o] = x;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) tw[lane * 33 + j] = v[j] + w[j];
        __syncwarp();
        const int n = nb + lane;
        for (int r = 0; r < 32; ++r) {
          const int mr = m0 + warp * 32 + r;
          if (mr >= ep.M) break;
          if (n < ep.N) {
            float x = tw[r * 33 + lane];
            if (SCALE) x *= __ldg(ep.inv_lam + (long long)(mr % ep.rows_per_prob) * ep.lam_ld + n);
            const long long o = (long long)mr * ep.out_ld + n;
            if (OUT_BF16) {
              __nv_bfloat16 pc[kMaxPieces];
              split_pieces<NP>(x, pc);
#pragma unroll
              for (int q = 0; q < NP; ++q) ep.out[q][o] = pc[q];
            } else {
              ep.out_f[o] = x;
            }
          }
        }
        __syncwarp();
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

// X (FP32, rows of pitch x_ld) -> NP BF16 piece rows of pitch ld (K = cols).
template <int NP>
__global__ void split_bf16_kernel(const float* __restrict__ X, long long x_ld, int rows, int cols,
                                  __nv_bfloat16* __restrict__ p0, __nv_bfloat16* __restrict__ p1,
                                  __nv_bfloat16* __restrict__ p2, long long ld) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    __nv_bfloat16 pc[kMaxPieces];
    split_pieces<NP>(X[r * x_ld + c], pc);
    p0[r * ld + c] = pc[0];
    p1[r * ld + c] = pc[1];
    if (NP == 3) p2[r * ld + c] = pc[2];
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
int ntile_for(int N, int np) {
  const int cap = np == 3 ? 128 : 256;
  const int n = N > cap ? cap : round_up(N, 16);
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
  int np;                     // pieces per operand (2 or 3)
  int KpH, KpW;
  // B operands, np pieces each: CW [W][KpW], CH [H][KpH], CHt [H][KpH], CWt [W][KpW]
  uint16_t* mats;
  __nv_bfloat16 *cw[kMaxPieces], *ch[kMaxPieces], *cht[kMaxPieces], *cwt[kMaxPieces];
  // work operands, np pieces each: bufA [B*H][KpW], bufB1 / bufB2 [B*W][KpH]
  __nv_bfloat16* work;
  __nv_bfloat16 *a[kMaxPieces], *b1[kMaxPieces], *b2[kMaxPieces];
  TcMaps g1, g2, g3, g4;
  int* err;
};

template <int NT, int NP, bool TRANS, bool SCALE, bool OUT_BF16>
cudaError_t launch_tc(const TcMaps& maps, const TcEpi& ep, int* err, cudaStream_t st) {
  static unsigned long long attr_set = 0;
  if (needs_setup(attr_set)) {
    const cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<NT, NP, TRANS, SCALE, OUT_BF16>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<NT, NP>());
    if (e != cudaSuccess) return e;
    mark_setup(attr_set);
  }
  const dim3 grid((ep.M + kTM - 1) / kTM, (ep.N + NT - 1) / NT);
  tc_gemm_kernel<NT, NP, TRANS, SCALE, OUT_BF16><<<grid, 128, tc_smem<NT, NP>(), st>>>(maps, ep, err);
  return cudaGetLastError();
}

template <bool TRANS, bool SCALE, bool OUT_BF16>
cudaError_t launch_tc_n(int NT, int np, const TcMaps& maps, const TcEpi& ep, int* err, cudaStream_t st) {
  if (np == 3) {
    switch (NT) {
      case 32: return launch_tc<32, 3, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
      case 64: return launch_tc<64, 3, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
      default: return launch_tc<128, 3, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    }
  }
  switch (NT) {
    case 32: return launch_tc<32, 2, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    case 64: return launch_tc<64, 2, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    case 128: return launch_tc<128, 2, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
    default: return launch_tc<256, 2, TRANS, SCALE, OUT_BF16>(maps, ep, err, st);
  }
}

}  // namespace

int dct_tc_create(DctPlan* p) {
  TcPlan* t = (TcPlan*)calloc(1, sizeof(TcPlan));
  if (!t) return fail(OT_ENOMEM, "dct tc plan: host allocation");
  p->tc = t;
  const int B = p->B, H = p->H, W = p->W;
  const int np = p->precision == OT_PREC_SPLIT_BF16_3 ? 3 : 2;
  t->np = np;
  t->KpH = round_up(H, 64);
  t->KpW = round_up(W, 64);
  const size_t nW = (size_t)W * t->KpW, nH = (size_t)H * t->KpH;
  // host: the np BF16 pieces of C_W, C_H, C_H^T, C_W^T with padded pitch
  // (piece q of a matrix at base + q * n)
  std::vector<uint16_t> host((size_t)np * 2 * (nW + nH), 0);
  const std::vector<double> CH = dct_matrix(H), CW = dct_matrix(W);
  auto put = [&](size_t base, size_t n_el, const std::vector<double>& C, int n, int ld, bool tr) {
    for (int r = 0; r < n; ++r)
      for (int k = 0; k < n; ++k) {
        double v = tr ? C[(size_t)k * n + r] : C[(size_t)r * n + k];
        for (int q = 0; q < np; ++q) {   // each piece takes the bf16 rounding of what is left
          const uint16_t b = f2bf_bits((float)v);
          host[base + q * n_el + (size_t)r * ld + k] = b;
          v -= (double)bf_bits2f(b);
        }
      }
  };
  const size_t o_cw = 0, o_ch = np * nW, o_cht = np * (nW + nH), o_cwt = np * (nW + 2 * nH);
  put(o_cw, nW, CW, W, t->KpW, false);
  put(o_ch, nH, CH, H, t->KpH, false);
  put(o_cht, nH, CH, H, t->KpH, true);
  put(o_cwt, nW, CW, W, t->KpW, true);
  cudaError_t e = cudaMalloc(&t->mats, host.size() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(t->mats, host.data(), host.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "dct tc plan: matrices");
  __nv_bfloat16* m = reinterpret_cast<__nv_bfloat16*>(t->mats);
  for (int q = 0; q < np; ++q) {
    t->cw[q] = m + o_cw + q * nW;
    t->ch[q] = m + o_ch + q * nH;
    t->cht[q] = m + o_cht + q * nH;
    t->cwt[q] = m + o_cwt + q * nW;
  }
  const size_t nA = (size_t)B * H * t->KpW, nB = (size_t)B * W * t->KpH;
  const size_t nwork = (size_t)np * (nA + 2 * nB);
  e = cudaMalloc(&t->work, nwork * sizeof(__nv_bfloat16) + 256);
  if (e == cudaSuccess) e = cudaMemset(t->work, 0, nwork * sizeof(__nv_bfloat16) + 256);
  if (e != cudaSuccess) return cuda_fail(e, "dct tc plan: work buffers");
  __nv_bfloat16* w = t->work;
  for (int q = 0; q < np; ++q) t->a[q] = w + q * nA;
  w += np * nA;
  for (int q = 0; q < np; ++q) t->b1[q] = w + q * nB;
  w += np * nB;
  for (int q = 0; q < np; ++q) t->b2[q] = w + q * nB;
  w += np * nB;
  t->err = reinterpret_cast<int*>(w);
  if (!p->err) p->err = t->err;
  // G1: A = X split [B*H][KpW] (K = W), B = C_W [W][KpW] (N = W)
  // G2: A = U^T [B*W][KpH] (K = H), B = C_H [H][KpH] (N = H)
  // G3: A = V' [B*W][KpH] (K = H), B = C_H^T [H][KpH] (N = H)
  // G4: A = P^T [B*H][KpW] (K = W), B = C_W^T [W][KpW] (N = W)
  const int ntW = ntile_for(W, np), ntH = ntile_for(H, np);
  int rc = 0;
  for (int q = 0; q < np; ++q) {
    rc |= encode_bf16_map(&t->g1.a[q], t->a[q], W, (long long)B * H, t->KpW, kTM);
    rc |= encode_bf16_map(&t->g1.b[q], t->cw[q], W, W, t->KpW, ntW);
    rc |= encode_bf16_map(&t->g2.a[q], t->b1[q], H, (long long)B * W, t->KpH, kTM);
    rc |= encode_bf16_map(&t->g2.b[q], t->ch[q], H, H, t->KpH, ntH);
    rc |= encode_bf16_map(&t->g3.a[q], t->b2[q], H, (long long)B * W, t->KpH, kTM);
    rc |= encode_bf16_map(&t->g3.b[q], t->cht[q], H, H, t->KpH, ntH);
    rc |= encode_bf16_map(&t->g4.a[q], t->a[q], W, (long long)B * H, t->KpW, kTM);
    rc |= encode_bf16_map(&t->g4.b[q], t->cwt[q], W, W, t->KpW, ntW);
  }
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
  const int B = p->B, H = p->H, W = p->W, np = t->np;
  const int ntW = ntile_for(W, np), ntH = ntile_for(H, np);
  if (np == 3)
    split_bf16_kernel<3><<<152 * 8, 256, 0, st>>>(X, x_ld, B * H, W, t->a[0], t->a[1], t->a[2], t->KpW);
  else
    split_bf16_kernel<2><<<152 * 8, 256, 0, st>>>(X, x_ld, B * H, W, t->a[0], t->a[1], nullptr, t->KpW);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TcEpi ep;
  memset(&ep, 0, sizeof ep);
  auto outs = [&](__nv_bfloat16* const* dst) {
    for (int q = 0; q < kMaxPieces; ++q) ep.out[q] = q < np ? dst[q] : nullptr;
  };
  // G1: U^T = (X C_W^T)^T -> b1 [B*W][KpH]
  ep.M = B * H; ep.N = W; ep.K = W; ep.rows_per_prob = H;
  outs(t->b1); ep.out_ld = t->KpH;
  e = launch_tc_n<true, false, true>(ntW, np, t->g1, ep, err, st);
  if (e != cudaSuccess) return e;
  // G2: Xhat^T / lam -> b2 [B*W][KpH]
  ep.M = B * W; ep.N = H; ep.K = H; ep.rows_per_prob = W; ep.inv_lam = p->inv_lam; ep.lam_ld = H;
  outs(t->b2); ep.out_ld = t->KpH;
  e = launch_tc_n<false, true, true>(ntH, np, t->g2, ep, err, st);
  if (e != cudaSuccess) return e;
  // G3: P = Xhat'^T C_H, stored transposed -> a [B*H][KpW]
  ep.M = B * W; ep.N = H; ep.K = H; ep.rows_per_prob = W; ep.inv_lam = nullptr;
  outs(t->a); ep.out_ld = t->KpW;
  e = launch_tc_n<true, false, true>(ntH, np, t->g3, ep, err, st);
  if (e != cudaSuccess) return e;
  // G4: Y = P^T C_W (FP32)
  ep.M = B * H; ep.N = W; ep.K = W; ep.rows_per_prob = H;
  for (int q = 0; q < kMaxPieces; ++q) ep.out[q] = nullptr;
  ep.out_f = Y; ep.out_ld = y_ld;
  return launch_tc_n<false, false, false>(ntW, np, t->g4, ep, err, st);
}

}  // namespace otp
