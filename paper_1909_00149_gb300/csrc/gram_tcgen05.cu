// Gram matrix G = X^T X of the SVT (Algorithm 3 line 10, Sec. IV-B.1) on the
// tcgen05 tensor cores.
//
// X is N x T with the T columns stored as rows of N floats (row t at X + t ld),
// so G[t][s] = sum_n X[t][n] X[s][n] is a product of two K-major operands
// (K = pixels).  FP32 accuracy from BF16 tensor cores by an exact 3-piece
// split x = h + m + l (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)) and
// the six products whose size is above 2^-26 |x|^2:
//   G += H H^T + H M^T + M H^T + M M^T + H L^T + L H^T.
// The pixel range is split over the CTAs (one per SM); each CTA streams its
// range in chunks of 64 pixels:
//   warp 0 (one lane): TMA loads of the FP32 chunk [TP rows][64] into a ring
//                      of stages,
//   warps 2-5:         split each chunk into the three BF16 pieces, written
//                      K-major with the 128-byte swizzle the MMA expects,
//   warp 1 (one lane): issues the MMAs into one FP32 accumulator in tensor
//                      memory (128 lanes x TP columns),
// and warps 2-5 finally read the accumulator (tcgen05.ld) and store the
// CTA's partial Gram in FP64; a second kernel sums the partials in a fixed
// order.  Every mbarrier wait is bounded; on expiry the CTA sets the error
// flag, waits (bounded) for its copies and MMAs, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "otprox_internal.cuh"
#include "tc_util.cuh"

namespace otp {
namespace {
using namespace tc;

constexpr int kGK = 64;                  // pixels per chunk: 64 bf16 = one 128-byte swizzled row
constexpr int kGThreads = 192;
constexpr int kPieceBytes = 128 * 128;   // one BF16 piece, 128 rows (TMEM lanes) x 128 bytes
constexpr int kSetBytes = 3 * kPieceBytes;

template <int TP>
constexpr int gram_stages() { return TP == 128 ? 3 : 4; }
template <int TP>
constexpr uint32_t gram_stage_bytes() { return (uint32_t)TP * kGK * 4; }
template <int TP>
constexpr size_t gram_tc_smem() { return 1024 + 2 * (size_t)kSetBytes + (size_t)gram_stages<TP>() * gram_stage_bytes<TP>(); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int TP>
__global__ void __launch_bounds__(kGThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap xmap, int T, int nchunks, double* __restrict__ partials,
               int* __restrict__ err) {
  constexpr int NS = gram_stages<TP>();
  constexpr uint32_t SB = gram_stage_bytes<TP>();
  constexpr uint32_t IDESC = bf16_idesc(128, TP);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (s_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sets = smem;                                   // 2 x [H | M | L] BF16 pieces
  unsigned char* stages = smem + 2 * kSetBytes;                 // NS x FP32 [TP][64]
  __shared__ __align__(8) uint64_t full[NS], freef[NS], conv[2], freeb[2], done;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = (int)((long long)blockIdx.x * nchunks / gridDim.x);
  const int c1 = (int)((long long)(blockIdx.x + 1) * nchunks / gridDim.x);
  const int nc = c1 - c0;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      bar_init(s_u32(&full[s]), 1);
      bar_init(s_u32(&freef[s]), 4);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(s_u32(&conv[b]), 4);
      bar_init(s_u32(&freeb[b]), 1);
    }
    bar_init(s_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(s_u32(&s_tmem), TP);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {   // producer
      int issued = 0;
      for (int c = 0; c < nc; ++c) {
        const int s = c % NS;
        if (c >= NS && !bar_wait(s_u32(&freef[s]), (uint32_t)((c / NS - 1) & 1))) { ok = false; break; }
        bar_expect(s_u32(&full[s]), SB);
        tma2d(s_u32(stages + (size_t)s * SB), &xmap, (c0 + c) * kGK, 0, s_u32(&full[s]));
        issued = c + 1;
      }
      // copies still in flight must land before the CTA's shared memory goes away
      for (int c = issued - NS < 0 ? 0 : issued - NS; c < issued; ++c)
        (void)bar_wait(s_u32(&full[c % NS]), (uint32_t)((c / NS) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      for (int c = 0; c < nc; ++c) {
        const int b = c & 1;
        if (!bar_wait(s_u32(&conv[b]), (uint32_t)((c >> 1) & 1))) { ok = false; break; }
        fence_after_sync();
        const uint32_t h = s_u32(sets + (size_t)b * kSetBytes), m = h + kPieceBytes, l = m + kPieceBytes;
#pragma unroll
        for (int kk = 0; kk < kGK / 16; ++kk) {   // K = 16 per instruction: 32 bytes along the row
          const uint32_t o = kk * 32;
          const uint64_t dh = sw128_desc(h + o), dm = sw128_desc(m + o), dl = sw128_desc(l + o);
          mma_bf16(tmem, dh, dh, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
          mma_bf16(tmem, dh, dm, IDESC, 1u);
          mma_bf16(tmem, dm, dh, IDESC, 1u);
          mma_bf16(tmem, dm, dm, IDESC, 1u);
          mma_bf16(tmem, dh, dl, IDESC, 1u);
          mma_bf16(tmem, dl, dh, IDESC, 1u);
        }
        mma_commit(s_u32(&freeb[b]));
      }
      mma_commit(s_u32(&done));   // tracks every MMA issued above
      if (!ok) (void)bar_wait(s_u32(&done), 0);
    }
  } else {
    // splitters: 128 threads, a task is one row and one 8-pixel group of the chunk
    const int q0 = tid - 64;
    for (int c = 0; c < nc && ok; ++c) {
      const int s = c % NS, b = c & 1;
      if (!bar_wait(s_u32(&full[s]), (uint32_t)((c / NS) & 1))) { ok = false; break; }
      if (c >= 2 && !bar_wait(s_u32(&freeb[b]), (uint32_t)(((c >> 1) - 1) & 1))) { ok = false; break; }
      const float* src = reinterpret_cast<const float*>(stages + (size_t)s * SB);
      unsigned char* dst = sets + (size_t)b * kSetBytes;
#pragma unroll
      for (int i = 0; i < TP * 8 / 128; ++i) {
        const int q = q0 + 128 * i;
        const int row = q >> 3, g = q & 7;
        const float4 u0 = *reinterpret_cast<const float4*>(src + row * kGK + g * 8);
        const float4 u1 = *reinterpret_cast<const float4*>(src + row * kGK + g * 8 + 4);
        const float x[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        float h[8], m[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          h[j] = __bfloat162float(__float2bfloat16_rn(x[j]));
          const float r1 = x[j] - h[j];
          m[j] = __bfloat162float(__float2bfloat16_rn(r1));
          l[j] = r1 - m[j];
        }
        const uint32_t off = (uint32_t)row * 128 + (uint32_t)((g ^ (row & 7)) << 4);
        *reinterpret_cast<uint4*>(dst + off) =
            make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
        *reinterpret_cast<uint4*>(dst + kPieceBytes + off) =
            make_uint4(pack_bf16(m[0], m[1]), pack_bf16(m[2], m[3]), pack_bf16(m[4], m[5]), pack_bf16(m[6], m[7]));
        *reinterpret_cast<uint4*>(dst + 2 * kPieceBytes + off) =
            make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) {
        bar_arrive(s_u32(&conv[b]));
        bar_arrive(s_u32(&freef[s]));
      }
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ... (tile rows t)
    const bool fin = ok && bar_wait(s_u32(&done), 0);
    const int quad = warp & 3;
    if (fin && 32 * quad < TP) {
      fence_after_sync();
      const int t = 32 * quad + lane;
      double* out = partials + (size_t)blockIdx.x * TP * TP + (size_t)t * TP;
#pragma unroll 1
      for (int cc = 0; cc < TP / 32; ++cc) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int sidx = 32 * cc + j;
          out[sidx] = (t < T && sidx < T) ? (double)v[j] : 0.0;
        }
      }
    }
    if (!fin) ok = false;
  }
  if (!ok) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, TP);
  }
}

template <int TP>
cudaError_t launch_gram_tc(const CUtensorMap& m, int T, int nchunks, int grid, double* partials, int* err,
                           cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(gram_tc_kernel<TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem<TP>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  gram_tc_kernel<TP><<<grid, kGThreads, gram_tc_smem<TP>(), st>>>(m, T, nchunks, partials, err);
  return cudaGetLastError();
}

}  // namespace

int svt_gram_tc_blocks(long long N) {
  const long long nch = (N + kGK - 1) / kGK;
  return (int)(nch < 152 ? nch : 152);
}

// Partial Grams (FP64, [grid][TP][TP]) of the N x T matrix X (row t at X + t ld)
// on the tensor cores; TP = 32, 64 or 128 (T > 16).  ld * 4 must be a
// multiple of 16 bytes and X 16-byte aligned (the TMA rules).
cudaError_t svt_launch_gram_tc(const float* X, long long ld, long long N, int T, double* partials, int* err,
                               cudaStream_t st) {
  const int TP = svt_padded_T(T);
  if (TP < 32 || (ld * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  // one cached map: the RPCA solver calls this every iteration on the same buffer
  static thread_local struct { const float* X; long long ld, N; int T; CUtensorMap m; bool valid; } cache = {};
  if (!cache.valid || cache.X != X || cache.ld != ld || cache.N != N || cache.T != T) {
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)T};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kGK, (cuuint32_t)TP};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(&cache.m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      cache.valid = false;
      return cudaErrorInvalidValue;
    }
    cache.X = X;
    cache.ld = ld;
    cache.N = N;
    cache.T = T;
    cache.valid = true;
  }
  const int nchunks = (int)((N + kGK - 1) / kGK);
  const int grid = svt_gram_tc_blocks(N);
  switch (TP) {
    case 32: return launch_gram_tc<32>(cache.m, T, nchunks, grid, partials, err, st);
    case 64: return launch_gram_tc<64>(cache.m, T, nchunks, grid, partials, err, st);
    default: return launch_gram_tc<128>(cache.m, T, nchunks, grid, partials, err, st);
  }
}

}  // namespace otp
