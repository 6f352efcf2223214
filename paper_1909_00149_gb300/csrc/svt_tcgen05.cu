// The two dense contractions of the SVT (Algorithm 3 line 10, Sec. IV-B.1)
// on the tcgen05 tensor cores: the Gram matrix G = X^T X and the apply
// Y = X Wm (gram_tc_kernel, apply_tc_kernel below).
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
//   warps 2-9:         split each chunk into the three BF16 pieces, written
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
constexpr int kSplitWarps = 8;           // splitter warps (two per SM sub-partition, to hide latency)
constexpr int kGThreads = 64 + 32 * kSplitWarps;
constexpr int kPieceBytes = 128 * 128;   // one BF16 piece, 128 rows (TMEM lanes) x 128 bytes
constexpr int kSetBytes = 3 * kPieceBytes;

template <int TP>
constexpr int gram_stages() { return TP == 128 ? 3 : 4; }
template <int TP>
constexpr uint32_t gram_stage_bytes() { return (uint32_t)TP * kGK * 4; }
template <int TP>
constexpr size_t gram_tc_smem() { return 1024 + 2 * (size_t)kSetBytes + (size_t)gram_stages<TP>() * gram_stage_bytes<TP>(); }


// Exact 3-piece BF16 split of 8 values, two at a time (cvt.rn.bf16x2.f32):
// x = h + m + l with h = bf16(x), m = bf16(x - h), l = bf16(x - h - m).
__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<const uint32_t*>(&v); }
__device__ __forceinline__ void split8(const float (&x)[8], uint4& H, uint4& M, uint4& L) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 v = make_float2(x[2 * p], x[2 * p + 1]);
    const __nv_bfloat162 hb = __float22bfloat162_rn(v);
    const float2 hf = __bfloat1622float2(hb);
    const float2 r = make_float2(v.x - hf.x, v.y - hf.y);
    const __nv_bfloat162 mb = __float22bfloat162_rn(r);
    const float2 mf = __bfloat1622float2(mb);
    const __nv_bfloat162 lb = __float22bfloat162_rn(make_float2(r.x - mf.x, r.y - mf.y));
    h[p] = bf2_bits(hb);
    m[p] = bf2_bits(mb);
    l[p] = bf2_bits(lb);
  }
  H = make_uint4(h[0], h[1], h[2], h[3]);
  M = make_uint4(m[0], m[1], m[2], m[3]);
  L = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void bulk_store(void* gdst, uint32_t ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

template <int TP>
__global__ void __launch_bounds__(kGThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap xmap, int T, int nchunks, float* __restrict__ partials,
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
      bar_init(s_u32(&freef[s]), kSplitWarps);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(s_u32(&conv[b]), kSplitWarps);
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
    // splitters: a task is one row and one 8-pixel group of the chunk
    const int q0 = tid - 64;
    for (int c = 0; c < nc && ok; ++c) {
      const int s = c % NS, b = c & 1;
      if (!bar_wait(s_u32(&full[s]), (uint32_t)((c / NS) & 1))) { ok = false; break; }
      if (c >= 2 && !bar_wait(s_u32(&freeb[b]), (uint32_t)(((c >> 1) - 1) & 1))) { ok = false; break; }
      const float* src = reinterpret_cast<const float*>(stages + (size_t)s * SB);
      unsigned char* dst = sets + (size_t)b * kSetBytes;
#pragma unroll
      for (int i = 0; i < TP * 8 / (32 * kSplitWarps); ++i) {
        const int q = q0 + 32 * kSplitWarps * i;
        const int row = q >> 3, g = q & 7;
        const float4 u0 = *reinterpret_cast<const float4*>(src + row * kGK + g * 8);
        const float4 u1 = *reinterpret_cast<const float4*>(src + row * kGK + g * 8 + 4);
        const float x[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        uint4 H, M, L;
        split8(x, H, M, L);
        const uint32_t off = (uint32_t)row * 128 + (uint32_t)((g ^ (row & 7)) << 4);
        *reinterpret_cast<uint4*>(dst + off) = H;
        *reinterpret_cast<uint4*>(dst + kPieceBytes + off) = M;
        *reinterpret_cast<uint4*>(dst + 2 * kPieceBytes + off) = L;
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) {
        bar_arrive(s_u32(&conv[b]));
        bar_arrive(s_u32(&freef[s]));
      }
    }
    // epilogue (warps 2-5): warp w reads TMEM lanes 32 (w % 4) ... (rows t).
    // The partial is symmetric, so thread t writes its row as column t of a
    // shared-memory tile (conflict-free), and one bulk copy stores the tile.
    const bool fin = ok && bar_wait(s_u32(&done), 0);
    const int quad = warp & 3;
    float* tile = reinterpret_cast<float*>(stages);            // the FP32 ring is idle now
    if (warp < 6) {
      if (fin && 32 * quad < TP) {
        fence_after_sync();
        const int t = 32 * quad + lane;
#pragma unroll 1
        for (int cc = 0; cc < TP / 32; ++cc) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(32 * cc), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int sidx = 32 * cc + j;
            tile[sidx * TP + t] = (t < T && sidx < T) ? v[j] : 0.f;
          }
        }
      }
      fence_async_shared();
      asm volatile("bar.sync 1, 128;" ::: "memory");          // warps 2-5 only
      if (fin && tid == 64) bulk_store(partials + (size_t)blockIdx.x * TP * TP, s_u32(tile), TP * TP * 4);
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
cudaError_t launch_gram_tc(const CUtensorMap& m, int T, int nchunks, int grid, float* partials, int* err,
                           cudaStream_t st) {
  static unsigned long long attr = 0;
  if (needs_setup(attr)) {
    const cudaError_t e =
        cudaFuncSetAttribute(gram_tc_kernel<TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem<TP>());
    if (e != cudaSuccess) return e;
    mark_setup(attr);
  }
  gram_tc_kernel<TP><<<grid, kGThreads, gram_tc_smem<TP>(), st>>>(m, T, nchunks, partials, err);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ apply
// Y = X Wm: Y[t][n] = sum_s Wm[t][s] X[s][n] (Wm = V diag(f) V^T is
// symmetric), i.e. D = A B^T with A = Wm (M = frames t, padded to 128 rows;
// K = frames s, padded to 64) and B[n][s] = X[s][n] (N = a tile of 128
// pixels).  B is K-major only after a transpose, which the splitter warps do
// while they cut each FP32 tile into its three BF16 pieces; Wm is split once
// per CTA.  The six products of the Gram give FP32 accuracy.  Per CTA, over
// its pixel tiles (persistent):
//   warp 0 (one lane): TMA loads of X tiles [TP frames][128 pixels],
//   warps 2-9:         transpose + split into the BF16 pieces of B,
//   warp 1 (one lane): 24 MMAs per tile into one of two TMEM accumulators
//                      (128 lanes x 128 columns each),
//   warps 10-13:       read the accumulator; each warp holding rows t < TP
//                      writes 32 x 32 blocks into a 128-byte-swizzled,
//                      double-buffered staging box that one lane stores
//                      with a TMA tile store (rows t >= T and pixels >= N
//                      fall outside the map and are not written).
constexpr int kAN = 128;                     // pixels per tile (MMA N)
constexpr int kAEpi = 2 + kSplitWarps;        // first epilogue warp
constexpr int kAThreads = 32 * (kAEpi + 4);
constexpr int kAStages = 2;
constexpr int kABPiece = kAN * 128;          // one BF16 piece of B: 128 pixel rows x 64 frames
constexpr int kABSet = 3 * kABPiece;
constexpr int kAAPiece = 128 * 128;          // one BF16 piece of A: 128 rows x 64 frames
template <int TP>
constexpr uint32_t apply_stage_bytes() { return (uint32_t)TP * kAN * 4; }
constexpr int kAStgBytes = 32 * 32 * 4;       // one staging box: 32 rows x 32 pixels, FP32
template <int TP>
constexpr size_t apply_tc_smem() {
  return 1024 + 3 * (size_t)kAAPiece + 2 * (size_t)kABSet + (size_t)kAStages * apply_stage_bytes<TP>() +
         (size_t)(TP / 32) * 2 * kAStgBytes;
}


template <int TP>
__global__ void __launch_bounds__(kAThreads, 1)
apply_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
                const float* __restrict__ Wm, int T, long long N, int ntiles, int* __restrict__ err) {
  constexpr uint32_t SB = apply_stage_bytes<TP>();
  constexpr uint32_t IDESC = bf16_idesc(128, kAN);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (s_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* apieces = smem;                              // [H | M | L] of Wm
  unsigned char* bsets = smem + 3 * kAAPiece;                 // 2 x [H | M | L] of X^T
  unsigned char* stages = bsets + 2 * kABSet;                 // kAStages x FP32 [TP][128]
  unsigned char* stg = stages + (size_t)kAStages * SB;        // [TP / 32][2] staging boxes
  __shared__ __align__(8) uint64_t full[kAStages], freef[kAStages], conv[2], freeb[2], tfull[2], tfree[2], aready,
      drain;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < kAStages; ++s) {
      bar_init(s_u32(&full[s]), 1);
      bar_init(s_u32(&freef[s]), kSplitWarps);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(s_u32(&conv[b]), kSplitWarps);
      bar_init(s_u32(&freeb[b]), 1);
      bar_init(s_u32(&tfull[b]), 1);
      bar_init(s_u32(&tfree[b]), 4);
    }
    bar_init(s_u32(&aready), kSplitWarps);
    bar_init(s_u32(&drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero every BF16 piece once: rows t >= T of A and frames s >= TP stay zero
  for (int i = tid; i < (3 * kAAPiece + 2 * kABSet) / 16; i += kAThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_async_shared();
  if (warp == 0) tmem_alloc(s_u32(&s_tmem), 2 * kAN);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = s_tmem;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {   // producer
      int issued = 0;
      for (int i = 0; i < nmine; ++i) {
        const int s = i % kAStages;
        if (i >= kAStages && !bar_wait(s_u32(&freef[s]), (uint32_t)((i / kAStages - 1) & 1))) { ok = false; break; }
        bar_expect(s_u32(&full[s]), SB);
        tma2d(s_u32(stages + (size_t)s * SB), &xmap, ((int)blockIdx.x + i * (int)gridDim.x) * kAN, 0,
              s_u32(&full[s]));
        issued = i + 1;
      }
      for (int i = issued - kAStages < 0 ? 0 : issued - kAStages; i < issued; ++i)
        (void)bar_wait(s_u32(&full[i % kAStages]), (uint32_t)((i / kAStages) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      if (!bar_wait(s_u32(&aready), 0)) ok = false;
      for (int i = 0; i < nmine && ok; ++i) {
        const int b = i & 1;
        if (!bar_wait(s_u32(&conv[b]), (uint32_t)((i >> 1) & 1))) { ok = false; break; }
        if (i >= 2 && !bar_wait(s_u32(&tfree[b]), (uint32_t)(((i >> 1) - 1) & 1))) { ok = false; break; }
        fence_after_sync();
        const uint32_t ah = s_u32(apieces), am = ah + kAAPiece, al = am + kAAPiece;
        const uint32_t bh = s_u32(bsets + (size_t)b * kABSet), bm = bh + kABPiece, bl = bm + kABPiece;
        const uint32_t acc = tmem + (uint32_t)(b * kAN);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t o = kk * 32;
          const uint64_t dah = sw128_desc(ah + o), dam = sw128_desc(am + o), dal = sw128_desc(al + o);
          const uint64_t dbh = sw128_desc(bh + o), dbm = sw128_desc(bm + o), dbl = sw128_desc(bl + o);
          mma_bf16(acc, dah, dbh, IDESC, kk > 0 ? 1u : 0u);
          mma_bf16(acc, dah, dbm, IDESC, 1u);
          mma_bf16(acc, dam, dbh, IDESC, 1u);
          mma_bf16(acc, dam, dbm, IDESC, 1u);
          mma_bf16(acc, dah, dbl, IDESC, 1u);
          mma_bf16(acc, dal, dbh, IDESC, 1u);
        }
        mma_commit(s_u32(&freeb[b]));
        mma_commit(s_u32(&tfull[b]));
      }
      if (!ok) {   // let every issued MMA finish before the memory is released
        mma_commit(s_u32(&drain));
        (void)bar_wait(s_u32(&drain), 0);
      }
    }
  } else if (warp < kAEpi) {
    // splitters: thread q owns pixel row q % 128 of B and half of its frame groups
    const int q = tid - 64;
    const int px = q & (kAN - 1), half = q >> 7;
    // A = Wm (symmetric), once: rows t < TP, frames s < TP, groups of 8 frames
    for (int task = q; task < TP * (TP / 8); task += 32 * kSplitWarps) {
      const int row = task / (TP / 8), g = task % (TP / 8);
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = __ldg(Wm + (size_t)row * TP + g * 8 + j);
      uint4 H, M, L;
      split8(x, H, M, L);
      const uint32_t off = (uint32_t)row * 128 + (uint32_t)((g ^ (row & 7)) << 4);
      *reinterpret_cast<uint4*>(apieces + off) = H;
      *reinterpret_cast<uint4*>(apieces + kAAPiece + off) = M;
      *reinterpret_cast<uint4*>(apieces + 2 * kAAPiece + off) = L;
    }
    fence_async_shared();
    __syncwarp();
    if (lane == 0) bar_arrive(s_u32(&aready));
    for (int i = 0; i < nmine && ok; ++i) {
      const int s = i % kAStages, b = i & 1;
      if (!bar_wait(s_u32(&full[s]), (uint32_t)((i / kAStages) & 1))) { ok = false; break; }
      if (i >= 2 && !bar_wait(s_u32(&freeb[b]), (uint32_t)(((i >> 1) - 1) & 1))) { ok = false; break; }
      const float* src = reinterpret_cast<const float*>(stages + (size_t)s * SB);
      unsigned char* dst = bsets + (size_t)b * kABSet;
#pragma unroll
      for (int gg = 0; gg < TP / 16; ++gg) {
        const int g = 2 * gg + half;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = src[(g * 8 + j) * kAN + px];
        uint4 H, M, L;
        split8(x, H, M, L);
        const uint32_t off = (uint32_t)px * 128 + (uint32_t)((g ^ (px & 7)) << 4);
        *reinterpret_cast<uint4*>(dst + off) = H;
        *reinterpret_cast<uint4*>(dst + kABPiece + off) = M;
        *reinterpret_cast<uint4*>(dst + 2 * kABPiece + off) = L;
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) {
        bar_arrive(s_u32(&conv[b]));
        bar_arrive(s_u32(&freef[s]));
      }
    }
  } else {
    // epilogue (warps 10-13): warp w reads TMEM lanes 32 (w % 4) ... = rows t
    const int quad = warp & 3;
    const bool live = 32 * quad < TP;         // warp-uniform
    unsigned char* my = stg + (size_t)(live ? quad : 0) * 2 * kAStgBytes;
    int buf = 0;
    for (int i = 0; i < nmine && ok; ++i) {
      const int b = i & 1;
      if (!bar_wait(s_u32(&tfull[b]), (uint32_t)((i >> 1) & 1))) { ok = false; break; }
      fence_after_sync();
      if (live) {
        const int n0 = ((int)blockIdx.x + i * (int)gridDim.x) * kAN;
#pragma unroll 1
        for (int cc = 0; cc < kAN / 32; ++cc) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * kAN + 32 * cc), v);
          unsigned char* box = my + buf * kAStgBytes;
          if (lane == 0) bulk_wait_read<1>();   // the store that last used this box has read it
          __syncwarp();
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4)        // row lane, 16-byte chunk c4, 128-byte swizzle
            *reinterpret_cast<float4*>(box + lane * 128 + ((c4 ^ (lane & 7)) << 4)) =
                make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
          fence_async_shared();
          __syncwarp();
          // a box entirely beyond the last pixel is not stored (stores start in range)
          if (lane == 0 && n0 + 32 * cc < N && 32 * quad < T) {
            tma_store2d(&ymap, s_u32(box), n0 + 32 * cc, 32 * quad);
            bulk_commit();
          }
          buf ^= 1;
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) bar_arrive(s_u32(&tfree[b]));
    }
    if (live && lane == 0) bulk_wait_all();   // the stores complete before the CTA exits
  }
  if (!ok) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, 2 * kAN);
  }
}

template <int TP>
cudaError_t launch_apply_tc(const CUtensorMap& xm, const CUtensorMap& ym, const float* Wm, int T, long long N,
                            int ntiles, int grid, int* err, cudaStream_t st) {
  static unsigned long long attr = 0;
  if (needs_setup(attr)) {
    const cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel<TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)apply_tc_smem<TP>());
    if (e != cudaSuccess) return e;
    mark_setup(attr);
  }
  apply_tc_kernel<TP><<<grid, kAThreads, apply_tc_smem<TP>(), st>>>(xm, ym, Wm, T, N, ntiles, err);
  return cudaGetLastError();
}

// FP32 map over X [T rows][N] (row pitch ld floats), box [box_rows][box_inner];
// 128-byte swizzle when the box rows are exactly 128 bytes (box_inner = 32).
int x_map(CUtensorMap* m, const float* X, long long ld, long long N, int T, int box_inner, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)T};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_inner == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

struct MapCache {
  const float* X;
  long long ld, N;
  int T, bi, br;
  CUtensorMap m;
  bool valid;
};

// One cached map per use: the RPCA solver calls these every iteration on the same buffers.
const CUtensorMap* cached_map(MapCache& c, const float* X, long long ld, long long N, int T, int bi, int br) {
  if (!c.valid || c.X != X || c.ld != ld || c.N != N || c.T != T || c.bi != bi || c.br != br) {
    c.valid = false;
    if (x_map(&c.m, X, ld, N, T, bi, br) != 0) return nullptr;
    c.X = X;
    c.ld = ld;
    c.N = N;
    c.T = T;
    c.bi = bi;
    c.br = br;
    c.valid = true;
  }
  return &c.m;
}
}  // namespace

int svt_gram_tc_blocks(long long N) {
  const long long nch = (N + kGK - 1) / kGK;
  return (int)(nch < 152 ? nch : 152);
}

// Partial Grams (FP32, [grid][TP][TP]) of the N x T matrix X (row t at X + t ld)
// on the tensor cores; TP = 32, 64 or 128 (T > 16).  ld * 4 must be a
// multiple of 16 bytes and X 16-byte aligned (the TMA rules).
cudaError_t svt_launch_gram_tc(const float* X, long long ld, long long N, int T, float* partials, int* err,
                               cudaStream_t st) {
  const int TP = svt_padded_T(T);
  if (TP < 32 || (ld * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
  static thread_local MapCache cache = {};
  const CUtensorMap* m = cached_map(cache, X, ld, N, T, kGK, TP);
  if (!m) return cudaErrorInvalidValue;
  const int nchunks = (int)((N + kGK - 1) / kGK);
  const int grid = svt_gram_tc_blocks(N);
  switch (TP) {
    case 32: return launch_gram_tc<32>(*m, T, nchunks, grid, partials, err, st);
    case 64: return launch_gram_tc<64>(*m, T, nchunks, grid, partials, err, st);
    default: return launch_gram_tc<128>(*m, T, nchunks, grid, partials, err, st);
  }
}

}  // namespace otp

namespace otp {

int svt_apply_tc_blocks(long long N) {
  const long long nt = (N + kAN - 1) / kAN;
  return (int)(nt < 152 ? nt : 152);
}

// Y = X Wm on the tensor cores for T_pad = 32 or 64 (see apply_tc_kernel).
// X, Y: [T][N] with row pitch ld / ldy floats; ld, ldy multiples of 4 and X,
// Y 16-byte aligned (the TMA rules).
cudaError_t svt_launch_apply_tc(const float* X, long long ld, long long N, int T, const float* Wm, float* Y,
                                long long ldy, int* err, cudaStream_t st) {
  const int TP = svt_padded_T(T);
  if ((TP != 32 && TP != 64) || ld % 4 != 0 || ldy % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(Y) & 15) != 0)
    return cudaErrorInvalidValue;
  static thread_local MapCache xcache = {};
  static thread_local MapCache ycache[2] = {};   // the RPCA solver alternates two output planes
  static thread_local int ynext = 0;
  const CUtensorMap* xm = cached_map(xcache, X, ld, N, T, kAN, TP);
  const CUtensorMap* ym = nullptr;
  for (int k = 0; k < 2 && !ym; ++k)
    if (ycache[k].valid && ycache[k].X == Y && ycache[k].ld == ldy && ycache[k].N == N && ycache[k].T == T)
      ym = &ycache[k].m;
  if (!ym) {
    ym = cached_map(ycache[ynext], Y, ldy, N, T, 32, 32);
    ynext ^= 1;
  }
  if (!xm || !ym) return cudaErrorInvalidValue;
  const int ntiles = (int)((N + kAN - 1) / kAN);
  const int grid = svt_apply_tc_blocks(N);
  return TP == 32 ? launch_apply_tc<32>(*xm, *ym, Wm, T, N, ntiles, grid, err, st)
                  : launch_apply_tc<64>(*xm, *ym, Wm, T, N, ntiles, grid, err, st);
}

}  // namespace otp
