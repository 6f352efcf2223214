// Many Algorithm 1 problems of uneven size in one launch per iteration.
//
// A batch holds n_seq sequences; sequence i is B_i independent frame pairs of
// H_i x W_i (the T_i - 1 pairs of a T_i-frame video, Alg. 3 line 11 / the
// prox of eq. Prox_UOT for each pair).  All sequences' planes live in one
// slab, plane-major: for each of the 11 state planes the sequences follow
// one another, so sequence i's plane is base + off_i.  Each sequence keeps
// its own geometry and its own step sizes (Theorem 1 with its own
// lambda_max).
//
// One iteration is one persistent launch over a work list of tiles: the
// active sequences' tiles are numbered consecutively (prefix sums), and each
// CTA walks the list with a grid stride, mapping a tile number to (sequence,
// tile) by binary search over the prefix sums in shared memory, then runs
// the same tile body as the one-problem tiled kernel (prox_tile.cuh), so
// every pixel's arithmetic, and hence every iterate, equals the one-problem
// result bit for bit.  Check iterations write one partial-sum row per tile
// at the sequence's tile offset; a segmented fixed-order FP64 reduction then
// gives every sequence its own residuals, and sequences that met the
// tolerance leave the work list.  A check interval (an even number of
// iterations, so that all active sequences share the ping-pong parity) is
// captured once as a CUDA graph; the work list is data, so the graph stays
// valid as sequences finish.  Two iteration kernels walk the list: this
// file's tiled kernel (tile height 8 or 16 rows, 1-4 CTAs per SM) and the
// TMA pipeline of prox_tma.cu (one CTA per SM, per-sequence tensor maps);
// ot_prox_batch_autotune times every candidate on the loaded problems and
// keeps the fastest.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"
#include "prox_tile.cuh"

using namespace otp;

namespace {

using SeqDesc = BatchSeq;
constexpr int kMaxSeq = kBatchMaxSeq;

template <int MODE, bool BAL, bool RED, int TH>
__global__ void __launch_bounds__(kTiledThreads, 2)
prox_batch_kernel(const SeqDesc* __restrict__ seqs, const int* __restrict__ act, int parity, const BatchPlanes P,
                  double* __restrict__ partials) {
  // act[0] = n_act; act[1 .. n_act]: active sequence ids; act[1 + n_act + k]:
  // tile prefix of the first k active sequences (k = 0..n_act).  The work
  // list is data, so a captured graph stays valid when sequences finish.
  __shared__ int s_seq[kMaxSeq];
  __shared__ int s_pre[kMaxSeq + 1];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int n_act = act[0];
  for (int k = tid; k < n_act; k += kTiledThreads) s_seq[k] = act[1 + k];
  for (int k = tid; k <= n_act; k += kTiledThreads) s_pre[k] = act[1 + n_act + k];
  __syncthreads();
  const int total = s_pre[n_act];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = n_act - 1;                      // largest k with s_pre[k] <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    const SeqDesc& d = seqs[s_seq[lo]];
    const int t = w - s_pre[lo];
    StatePtrs S;
    // selects, not P.Mx[parity]: a runtime index into a kernel parameter would go through local memory
    S.Mx_in = (parity ? P.Mx[1] : P.Mx[0]) + d.off;
    S.My_in = (parity ? P.My[1] : P.My[0]) + d.off;
    S.a_in = (parity ? P.a[1] : P.a[0]) + d.off;
    S.Mx_out = (parity ? P.Mx[0] : P.Mx[1]) + d.off;
    S.My_out = (parity ? P.My[0] : P.My[1]) + d.off;
    S.a_out = (parity ? P.a[0] : P.a[1]) + d.off;
    S.x0 = P.x0 + d.off;
    S.x1 = P.x1 + d.off;
    S.r = P.r + d.off;
    S.p0 = P.p0 + d.off;
    S.p1 = P.p1 + d.off;
    tile::prox_tile<MODE, BAL, RED, TH>(d.G, d.C, S, t, RED ? partials + (size_t)(d.tile0 + t) * kNumSums : nullptr);
    __syncthreads();   // the tile body's shared arrays are reused by the next tile
  }
}

// Per active sequence k (one CTA each): FP64 sum of its tiles' partial rows
// in a fixed order (lanes stride over tiles, then the 32 lanes of each of 8
// warps, then the warps in order).  out[seq][kNumSums].
__global__ void __launch_bounds__(256)
segment_sums_kernel(const SeqDesc* __restrict__ seqs, const int* __restrict__ act, const double* __restrict__ partials,
                    double* __restrict__ out) {
  __shared__ double red[8][kNumSums];
  if ((int)blockIdx.x >= act[0]) return;   // one CTA per sequence; the active ones come first
  const int seq = act[1 + blockIdx.x];
  const SeqDesc d = seqs[seq];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double v[kNumSums];
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) v[k] = 0.0;
  for (int t = tid; t < d.ntiles; t += 256) {
    const double* row = partials + (size_t)(d.tile0 + t) * kNumSums;
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) v[k] += row[k];
  }
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (tid < kNumSums) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][tid];
    out[(size_t)seq * kNumSums + tid] = t;
  }
}

typedef void (*BatchKernel)(const SeqDesc*, const int*, int, const BatchPlanes, double*);

template <int MODE, bool BAL, bool RED>
BatchKernel pick_th(int th) {
  return th == 8 ? prox_batch_kernel<MODE, BAL, RED, 8> : prox_batch_kernel<MODE, BAL, RED, 16>;
}

BatchKernel pick_kernel(int mode, bool bal, bool red, int th) {
#define OTP_PICK(M, BL)                                                              \
  if (mode == M && bal == BL) return red ? pick_th<M, BL, true>(th) : pick_th<M, BL, false>(th);
  OTP_PICK(0, false)
  OTP_PICK(0, true)
  OTP_PICK(1, false)
  OTP_PICK(1, true)
  OTP_PICK(2, false)
  OTP_PICK(2, true)
#undef OTP_PICK
  return nullptr;
}

}  // namespace

#define OT_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

struct ot_prox_batch {
  ot_prox_params prm;                 // the shared parameters (B, H, W unused)
  cudaStream_t stream;
  int n_seq;
  std::vector<SeqDesc> host;          // per-sequence descriptors (host copy)
  std::vector<int> iters;             // iterations run by each sequence in the current solve
  std::vector<char> active;
  SeqDesc* dseqs;
  int* dact;                          // n_act, [n_act] ids, then [n_act + 1] prefix
  float* slab;
  BatchPlanes P;
  size_t plane_elems;                 // all sequences, one plane
  double* partials;                   // [max tiles][kNumSums]
  double* dsums;                      // [n_seq][kNumSums]
  double* hsums;                      // pinned mirror
  int* hact;                          // pinned work list
  int n_act, act_tiles;
  int parity;
  int kernel, tile_rows, ctas_per_sm, n_sm;   // kernel: OT_KERNEL_TILED or OT_KERNEL_TMA
  int* derr;                          // TMA pipeline: bounded-wait error flag
  int* herr;
  int max_tiles;
  cudaGraphExec_t graph;              // one check interval
  int graph_n, graph_par;
};

namespace {

int tiles_of(const Geometry& G, int th) {
  return G.B * ((G.Wp + kTW - 1) / kTW) * ((G.H + th - 1) / th);
}

// Tile counts and offsets for the current tile height; descriptors to the device.
int set_tiles(ot_prox_batch* h) {
  int t0 = 0;
  const int th = h->kernel == OT_KERNEL_TMA ? kTH : h->tile_rows;
  for (auto& d : h->host) {
    d.G.tiles_x = (d.G.Wp + kTW - 1) / kTW;
    d.G.tiles_y = (d.G.H + th - 1) / th;
    d.ntiles = d.G.B * d.G.tiles_x * d.G.tiles_y;
    d.tile0 = t0;
    t0 += d.ntiles;
  }
  OT_CUDA(cudaMemcpyAsync(h->dseqs, h->host.data(), h->host.size() * sizeof(SeqDesc), cudaMemcpyHostToDevice,
                          h->stream),
          "batch: descriptors");
  return OT_OK;
}

// The work list of the active sequences (ids, then tile prefix sums).  The
// pinned host copy is rewritten, so earlier copies from it must have landed.
int upload_work(ot_prox_batch* h) {
  OT_CUDA(cudaStreamSynchronize(h->stream), "batch: work list sync");
  int n = 0;
  for (int i = 0; i < h->n_seq; ++i)
    if (h->active[i]) h->hact[1 + n++] = i;
  int pre = 0;
  for (int k = 0; k < n; ++k) {
    h->hact[1 + n + k] = pre;
    pre += h->host[h->hact[1 + k]].ntiles;
  }
  h->hact[1 + 2 * n] = pre;
  h->hact[0] = n;
  h->n_act = n;
  h->act_tiles = pre;
  OT_CUDA(cudaMemcpyAsync(h->dact, h->hact, (2 * (size_t)n + 2) * sizeof(int), cudaMemcpyHostToDevice, h->stream),
          "batch: work list");
  return OT_OK;
}

int grid_of(const ot_prox_batch* h) {
  const int g = h->n_sm * h->ctas_per_sm;
  return h->act_tiles < g ? (h->act_tiles > 0 ? h->act_tiles : 1) : g;
}

cudaError_t launch_iter(ot_prox_batch* h, bool red) {
  cudaError_t e;
  if (h->kernel == OT_KERNEL_TMA) {
    const int grid = h->act_tiles < h->n_sm ? (h->act_tiles > 0 ? h->act_tiles : 1) : h->n_sm;
    e = launch_prox_tma_batch(h->prm.mode, h->prm.balanced != 0, red, h->dseqs, h->dact, h->parity, h->P,
                              h->partials, h->derr, grid, h->stream);
  } else {
    BatchKernel k = pick_kernel(h->prm.mode, h->prm.balanced != 0, red, h->tile_rows);
    const dim3 block(kTX, kTY);
    k<<<grid_of(h), block, 0, h->stream>>>(h->dseqs, h->dact, h->parity, h->P, h->partials);
    e = cudaGetLastError();
  }
  h->parity ^= 1;
  return e;
}

// n iterations of every active sequence; the last one reduces, and the
// per-sequence sums are copied to the pinned host mirror.
int enqueue_interval(ot_prox_batch* h, int n, bool sums) {
  for (int k = 0; k < n; ++k) OT_CUDA(launch_iter(h, sums && k == n - 1), "batch: iteration");
  if (sums) {
    segment_sums_kernel<<<h->n_seq, 256, 0, h->stream>>>(h->dseqs, h->dact, h->partials, h->dsums);
    OT_CUDA(cudaGetLastError(), "batch: segment sums");
    OT_CUDA(cudaMemcpyAsync(h->hsums, h->dsums, (size_t)h->n_seq * kNumSums * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream),
            "batch: sums copy");
    OT_CUDA(cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "batch: error flag");
  }
  return OT_OK;
}

void destroy_graph(ot_prox_batch* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_n = 0;
}

// One check interval; replayed from a graph when the stream allows capture.
int run_interval(ot_prox_batch* h, int n) {
  if (!h->prm.use_graph || h->stream == nullptr || (n & 1)) return enqueue_interval(h, n, true);
  if (!h->graph || h->graph_n != n || h->graph_par != h->parity) {
    destroy_graph(h);
    const int par = h->parity;
    h->graph_par = par;
    cudaGraph_t g = nullptr;
    OT_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "batch: capture");
    const int rc = enqueue_interval(h, n, true);
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    h->parity = par;
    if (rc != OT_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "batch: capture end");
    const cudaError_t e3 = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return cuda_fail(e3, "batch: graph instantiate");
    h->graph_n = n;
  }
  OT_CUDA(cudaGraphLaunch(h->graph, h->stream), "batch: graph launch");
  h->parity ^= (n & 1);
  return OT_OK;
}

bool seq_sums_bad(const double* s) {
  if (s[7] > 0) return true;
  for (int k = 0; k < 7; ++k)
    if (!isfinite(s[k])) return true;
  return false;
}

}  // namespace

extern "C" {

int ot_prox_batch_destroy(ot_prox_batch_t h) {
  if (!h) return OT_OK;
  destroy_graph(h);
  cudaFree(h->slab);
  cudaFree(h->dseqs);
  cudaFree(h->dact);
  cudaFree(h->partials);
  cudaFree(h->derr);
  if (h->herr) cudaFreeHost(h->herr);
  if (h->hsums) cudaFreeHost(h->hsums);
  if (h->hact) cudaFreeHost(h->hact);
  delete h;
  return OT_OK;
}

int ot_prox_batch_create(int32_t n_seq, const int32_t* B, const int32_t* H, const int32_t* W,
                         const ot_prox_params* common, void* cuda_stream, ot_prox_batch_t* out) {
  if (!out || !B || !H || !W || !common) return fail(OT_EINVAL, "ot_prox_batch_create: NULL argument");
  *out = nullptr;
  if (n_seq < 1 || n_seq > kMaxSeq) return fail(OT_EINVAL, "ot_prox_batch_create: n_seq must be in [1, %d]", kMaxSeq);
  const ot_prox_params p = *common;
  if (p.mode < 0 || p.mode > 2) return fail(OT_EINVAL, "ot_prox_batch_create: unknown mode %d", p.mode);
  if (p.norm != OT_NORM_ISO && p.norm != OT_NORM_ANISO) return fail(OT_EINVAL, "ot_prox_batch_create: unknown norm");
  if (p.p_exp != 1 && p.p_exp != 2) return fail(OT_EINVAL, "ot_prox_batch_create: p_exp must be 1 or 2");
  if (!(p.mu > 0) || !(p.rho > 0) || !isfinite(p.mu) || !isfinite(p.rho))
    return fail(OT_EINVAL, "ot_prox_batch_create: mu and rho must be > 0");
  if (p.tau1 > 0 || p.tau2 > 0)
    return fail(OT_EINVAL, "ot_prox_batch_create: steps are per sequence (Theorem 1); leave tau1, tau2 at 0");
  if (p.check_every < 2 || (p.check_every & 1))
    return fail(OT_EINVAL, "ot_prox_batch_create: check_every must be even and >= 2");
  if (!(p.tol >= 0) || p.max_iter < 0) return fail(OT_EINVAL, "ot_prox_batch_create: tol >= 0, max_iter >= 0");
  ot_prox_batch* h = new ot_prox_batch();
  h->prm = p;
  h->stream = (cudaStream_t)cuda_stream;
  h->n_seq = n_seq;
  h->kernel = OT_KERNEL_TMA;
  h->tile_rows = 16;
  h->ctas_per_sm = 2;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    h->n_sm = 152;
  const int n_id = ot_n_identity_blocks(p.mode, p.balanced);
  size_t off = 0;
  int max_tiles8 = 0;
  for (int i = 0; i < n_seq; ++i) {
    if (B[i] < 1 || H[i] < 1 || W[i] < 1) {
      ot_prox_batch_destroy(h);
      return fail(OT_EINVAL, "ot_prox_batch_create: sequence %d: B, H, W must be >= 1", i);
    }
    SeqDesc d;
    memset(&d, 0, sizeof d);
    d.G.B = B[i];
    d.G.H = H[i];
    d.G.W = W[i];
    d.G.Wp = (W[i] + 3) / 4 * 4;
    d.G.plane = (long long)d.G.H * d.G.Wp;
    const double L = ot_lambda_max(H[i], W[i]) + n_id;
    if (!(L > 0)) {
      ot_prox_batch_destroy(h);
      return fail(OT_EINVAL, "ot_prox_batch_create: sequence %d has no free variables", i);
    }
    const double t = 0.99 / sqrt(L);
    d.C.tau1 = (float)t;
    d.C.tau2 = (float)t;
    d.C.cp = (float)(t / (p.rho + t));
    d.C.cx = (float)(p.rho / (p.rho + t));
    d.C.ca = (float)(p.rho * t / (p.rho + t));
    d.C.mu_tau1 = (float)(p.mu * t);
    d.C.r2 = (float)(1.0 / (1.0 + 2.0 * p.mu * t));
    d.C.iso = p.norm == OT_NORM_ISO;
    d.C.pexp = p.p_exp;
    d.off = (long long)off;
    off += (size_t)d.G.B * d.G.plane;
    max_tiles8 += tiles_of(d.G, 8);
    h->host.push_back(d);
  }
  h->plane_elems = off;
  h->max_tiles = max_tiles8;            // the smallest tile height has the most tiles
  h->iters.assign(n_seq, 0);
  h->active.assign(n_seq, 1);
  if ((double)off * 11 * 4 > 2.6e11) {
    ot_prox_batch_destroy(h);
    return fail(OT_ENOMEM, "ot_prox_batch_create: state would exceed device memory");
  }
  cudaError_t e = cudaMalloc(&h->slab, off * 11 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->dseqs, (size_t)n_seq * sizeof(SeqDesc));
  if (e == cudaSuccess) e = cudaMalloc(&h->dact, (2 * (size_t)n_seq + 2) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, ((size_t)h->max_tiles + (size_t)n_seq) * kNumSums * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hsums, (size_t)n_seq * kNumSums * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hact, (2 * (size_t)n_seq + 2) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h->herr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = prepare_prox_tma_batch(p.mode, p.balanced != 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->slab, 0, off * 11 * sizeof(float), h->stream);
  if (e != cudaSuccess) {
    ot_prox_batch_destroy(h);
    return cuda_fail(e, "ot_prox_batch_create: allocation");
  }
  h->dsums = h->partials + (size_t)h->max_tiles * kNumSums;
  float* q = h->slab;
  h->P.Mx[0] = q; q += off;
  h->P.Mx[1] = q; q += off;
  h->P.My[0] = q; q += off;
  h->P.My[1] = q; q += off;
  h->P.a[0] = q; q += off;
  h->P.a[1] = q; q += off;
  h->P.x0 = q; q += off;
  h->P.x1 = q; q += off;
  h->P.r = q; q += off;
  h->P.p0 = q; q += off;
  h->P.p1 = q;
  if (h->herr) *h->herr = 0;
  // per-sequence tensor maps of the TMA pipeline, for both parities of M, a
  int rc = OT_OK;
  for (int i = 0; i < n_seq && rc == OT_OK; ++i) {
    SeqDesc& d = h->host[i];
    int bw, bh, r2 = 0;
    for (int par = 0; par < 2; ++par) {
      TmaMaps& m = d.maps[par];
      tma_box(0, &bw, &bh);
      r2 |= encode_plane_map(&m.a, h->P.a[par] + d.off, d.G, bw, bh);
      tma_box(1, &bw, &bh);
      r2 |= encode_plane_map(&m.Mx, h->P.Mx[par] + d.off, d.G, bw, bh);
      r2 |= encode_plane_map(&m.My, h->P.My[par] + d.off, d.G, bw, bh);
      tma_box(2, &bw, &bh);
      r2 |= encode_plane_map(&m.x0, h->P.x0 + d.off, d.G, bw, bh);
      r2 |= encode_plane_map(&m.x1, h->P.x1 + d.off, d.G, bw, bh);
      r2 |= encode_plane_map(&m.r, h->P.r + d.off, d.G, bw, bh);
      r2 |= encode_plane_map(&m.p0, h->P.p0 + d.off, d.G, bw, bh);
      r2 |= encode_plane_map(&m.p1, h->P.p1 + d.off, d.G, bw, bh);
    }
    if (r2 != 0) h->kernel = OT_KERNEL_TILED;   // no TMA maps: the tiled kernel only
  }
  rc = set_tiles(h);
  if (rc == OT_OK) rc = upload_work(h);
  if (rc == OT_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "ot_prox_batch_create: sync");
  }
  if (rc != OT_OK) {
    ot_prox_batch_destroy(h);
    return rc;
  }
  *out = h;
  return OT_OK;
}

int ot_prox_batch_set_input(ot_prox_batch_t h, int32_t seq, const float* p0, const float* p1) {
  if (!h || !p0 || !p1) return fail(OT_EINVAL, "ot_prox_batch_set_input: NULL argument");
  if (seq < 0 || seq >= h->n_seq) return fail(OT_EINVAL, "ot_prox_batch_set_input: no sequence %d", seq);
  const SeqDesc& d = h->host[seq];
  const size_t wb = (size_t)d.G.W * sizeof(float), pitch = (size_t)d.G.Wp * sizeof(float);
  const size_t rows = (size_t)d.G.B * d.G.H;
  OT_CUDA(cudaMemcpy2DAsync(h->P.p0 + d.off, pitch, p0, wb, wb, rows, cudaMemcpyDefault, h->stream), "batch: p0");
  OT_CUDA(cudaMemcpy2DAsync(h->P.p1 + d.off, pitch, p1, wb, wb, rows, cudaMemcpyDefault, h->stream), "batch: p1");
  return OT_OK;
}

int ot_prox_batch_reset(ot_prox_batch_t h) {
  if (!h) return fail(OT_EINVAL, "ot_prox_batch_reset: NULL handle");
  OT_CUDA(cudaMemsetAsync(h->slab, 0, h->plane_elems * 9 * sizeof(float), h->stream), "ot_prox_batch_reset");
  h->parity = 0;
  for (int i = 0; i < h->n_seq; ++i) {
    h->active[i] = 1;
    h->iters[i] = 0;
  }
  return upload_work(h);
}

int ot_prox_batch_step(ot_prox_batch_t h, int32_t n_iter) {
  if (!h) return fail(OT_EINVAL, "ot_prox_batch_step: NULL handle");
  if (n_iter < 0) return fail(OT_EINVAL, "ot_prox_batch_step: n_iter must be >= 0");
  if (h->n_act == 0) return OT_OK;
  for (int k = 0; k < n_iter; ++k) OT_CUDA(launch_iter(h, false), "ot_prox_batch_step");
  for (int i = 0; i < h->n_seq; ++i)
    if (h->active[i]) h->iters[i] += n_iter;
  return OT_OK;
}

int ot_prox_batch_solve(ot_prox_batch_t h, ot_prox_batch_result* res, int32_t* launches) {
  if (!h || !res) return fail(OT_EINVAL, "ot_prox_batch_solve: NULL argument");
  for (int i = 0; i < h->n_seq; ++i) {
    res[i].iters = h->iters[i];
    res[i].status = OT_ENOTCONV;
    res[i].res_pri = res[i].res_fp = INFINITY;
  }
  int n_launch = 0, done_iters = 0;
  const int ce = h->prm.check_every;
  while (h->n_act > 0 && done_iters < h->prm.max_iter) {
    int rc = run_interval(h, ce);
    if (rc != OT_OK) return rc;
    n_launch += ce + 1;
    done_iters += ce;
    OT_CUDA(cudaStreamSynchronize(h->stream), "ot_prox_batch_solve: sync");
    if (*h->herr) return fail(OT_ETIMEOUT, "ot_prox_batch_solve: a bounded device wait expired in the TMA pipeline");
    bool changed = false;
    for (int i = 0; i < h->n_seq; ++i) {
      if (!h->active[i]) continue;
      h->iters[i] += ce;
      const double* s = h->hsums + (size_t)i * kNumSums;
      res[i].iters = h->iters[i];
      res[i].res_pri = sqrt(s[0]) / fmax(sqrt(s[6]), 1e-30);
      res[i].res_fp = sqrt(s[1]) / fmax(sqrt(s[2]), 1e-30);
      if (seq_sums_bad(s)) {
        res[i].status = OT_ENONFINITE;
        h->active[i] = 0;
        changed = true;
      } else if (fmax(res[i].res_pri, res[i].res_fp) <= h->prm.tol) {
        res[i].status = OT_OK;
        h->active[i] = 0;
        changed = true;
      }
    }
    if (changed) {
      rc = upload_work(h);
      if (rc != OT_OK) return rc;
    }
  }
  if (launches) *launches = n_launch;
  // the next call starts a fresh solve from the current iterates of every sequence
  for (int i = 0; i < h->n_seq; ++i) h->active[i] = 1;
  int rc = upload_work(h);
  if (rc != OT_OK) return rc;
  for (int i = 0; i < h->n_seq; ++i)
    if (res[i].status == OT_ENONFINITE) return fail(OT_ENONFINITE, "ot_prox_batch_solve: sequence %d is not finite", i);
  for (int i = 0; i < h->n_seq; ++i)
    if (res[i].status != OT_OK) return fail(OT_ENOTCONV, "ot_prox_batch_solve: max_iter reached before every sequence met tol");
  return OT_OK;
}

int ot_prox_batch_get_state(ot_prox_batch_t h, int32_t seq, float* Mx, float* My, float* x0, float* x1, float* r,
                            float* a) {
  if (!h) return fail(OT_EINVAL, "ot_prox_batch_get_state: NULL handle");
  if (seq < 0 || seq >= h->n_seq) return fail(OT_EINVAL, "ot_prox_batch_get_state: no sequence %d", seq);
  const SeqDesc& d = h->host[seq];
  const size_t wb = (size_t)d.G.W * sizeof(float), pitch = (size_t)d.G.Wp * sizeof(float);
  const size_t rows = (size_t)d.G.B * d.G.H;
  const float* src[6] = {h->P.Mx[h->parity] + d.off, h->P.My[h->parity] + d.off,
                         (h->prm.mode == OT_MODE_PROX ? h->P.x0 : h->P.p0) + d.off,
                         (h->prm.mode != OT_MODE_EVAL ? h->P.x1 : h->P.p1) + d.off, h->P.r + d.off,
                         h->P.a[h->parity] + d.off};
  float* dst[6] = {Mx, My, x0, x1, r, a};
  for (int k = 0; k < 6; ++k)
    if (dst[k])
      OT_CUDA(cudaMemcpy2DAsync(dst[k], wb, src[k], pitch, wb, rows, cudaMemcpyDefault, h->stream),
              "ot_prox_batch_get_state");
  OT_CUDA(cudaStreamSynchronize(h->stream), "ot_prox_batch_get_state: sync");
  return OT_OK;
}

int ot_prox_batch_set_config(ot_prox_batch_t h, int32_t kernel, int32_t tile_rows, int32_t ctas_per_sm) {
  if (!h) return fail(OT_EINVAL, "ot_prox_batch_set_config: NULL handle");
  if (kernel != OT_KERNEL_TILED && kernel != OT_KERNEL_TMA)
    return fail(OT_EINVAL, "ot_prox_batch_set_config: kernel must be OT_KERNEL_TILED or OT_KERNEL_TMA");
  if (tile_rows != 8 && tile_rows != 16) return fail(OT_EINVAL, "ot_prox_batch_set_config: tile_rows must be 8 or 16");
  if (ctas_per_sm < 1 || ctas_per_sm > 8) return fail(OT_EINVAL, "ot_prox_batch_set_config: ctas_per_sm in [1, 8]");
  h->kernel = kernel;
  h->tile_rows = tile_rows;
  h->ctas_per_sm = ctas_per_sm;
  destroy_graph(h);
  int rc = set_tiles(h);
  if (rc == OT_OK) rc = upload_work(h);
  return rc;
}

// Time every (tile height, CTAs per SM) candidate on the loaded problems
// (plain iterations, CUDA events, after one warm-up launch) and keep the
// fastest.  The iterates advance by the timed iterations; call
// ot_prox_batch_reset afterwards for a cold start.
int ot_prox_batch_autotune(ot_prox_batch_t h, int32_t* kernel, int32_t* tile_rows, int32_t* ctas_per_sm,
                           float* best_ms) {
  if (!h) return fail(OT_EINVAL, "ot_prox_batch_autotune: NULL handle");
  // candidates: the TMA pipeline (one CTA per SM), then the tiled kernel
  // with 8 or 16 rows per tile and 1, 2 or 4 CTAs per SM
  struct Cand { int kernel, th, cp; };
  std::vector<Cand> cands;
  if (h->kernel == OT_KERNEL_TMA) cands.push_back({OT_KERNEL_TMA, 16, 1});
  for (int th : {8, 16})
    for (int cp : {1, 2, 4}) cands.push_back({OT_KERNEL_TILED, th, cp});
  float best = INFINITY;
  Cand bc = cands[0];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OT_CUDA(cudaEventCreate(&e0), "autotune: event");
  OT_CUDA(cudaEventCreate(&e1), "autotune: event");
  int rc = OT_OK;
  for (size_t c = 0; c < cands.size() && rc == OT_OK; ++c) {
    {
      rc = ot_prox_batch_set_config(h, cands[c].kernel, cands[c].th, cands[c].cp);
      if (rc != OT_OK) break;
      cudaError_t e = launch_iter(h, false);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = launch_iter(h, false);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = cuda_fail(e, "ot_prox_batch_autotune");
      else if (ms < best) {
        best = ms;
        bc = cands[c];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != OT_OK) return rc;
  rc = ot_prox_batch_set_config(h, bc.kernel, bc.th, bc.cp);
  if (kernel) *kernel = bc.kernel;
  if (tile_rows) *tile_rows = bc.th;
  if (ctas_per_sm) *ctas_per_sm = bc.cp;
  if (best_ms) *best_ms = best / 4.f;
  return rc;
}

}  // extern "C"
