// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/otprox.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace otp {

// One-time setup per device (a kernel's attributes belong to the context of
// the device it runs on): needs_setup is true until mark_setup has recorded
// the current device in `done` (devices 0-63; others always set up).
inline bool needs_setup(unsigned long long done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  return !(done & (1ull << dev));
}
inline void mark_setup(unsigned long long& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) done |= 1ull << dev;
}

// ----------------------------------------------------------------- tiling
// Tiled Algorithm 1 iteration: a CTA owns kTH rows x kTW columns of one
// problem; 32 x 8 threads, each thread a float4 column group on kRPT rows.
constexpr int kTW = 128;
constexpr int kTH = 16;
constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kRPT = kTH / kTY;
constexpr int kTiledThreads = kTX * kTY;
// Resident kernel: one CTA iterates a whole problem in shared memory.
constexpr int kResidentThreads = 512;
constexpr size_t kResidentSmemCap = 200 * 1024;
// Reduction quantities of a stopping check (FP64 sums):
//  0 ||K(z')||^2      1 ||(z',a') - (z,a)||^2   2 ||(z',a')||^2
//  3 ||M'||_{2,1}     4 sum |r'| (or r'^2)      5 sum_free (x' - p)^2
//  6 ||p0||^2 + ||p1||^2                        7 non-finite count
constexpr int kNumSums = 8;

struct Geometry {
  int B, H, W, Wp;         // Wp: row pitch in floats, multiple of 4
  long long plane;         // H * Wp
  int tiles_x, tiles_y;
};

struct IterCoeffs {
  float tau1, tau2;
  float cp, cx, ca;        // x-step: x' = max(cp p + cx x -/+ ca a, 0)
  float mu_tau1;           // r-step threshold (p = 1)
  float r2;                // r-step scale 1 / (1 + 2 mu tau1) (p = 2)
  int iso;                 // 1: ||.||_{2,1}; 0: anisotropic l1
  int pexp;                // 1 or 2
};

// One iteration's buffers.  M and a are ping-ponged (their neighbours are
// read); x and r are updated in place (only their own pixel is read).
struct StatePtrs {
  const float* Mx_in;
  const float* My_in;
  const float* a_in;
  float* Mx_out;
  float* My_out;
  float* a_out;
  float* x0;
  float* x1;
  float* r;
  const float* p0;
  const float* p1;
};

// Temporally blocked Algorithm 1 (prox_temporal.cu): a CTA of 512 threads
// stages a 136 x 45 tile (34 float4 groups; 128 own columns with 4 halo
// columns each side, own rows with a halo of 2 or 4 rows above and below) and
// runs up to 4 iterations on it.  Every plane is ping-ponged.
constexpr int kTbGroups = 34;
constexpr int kTbThreadRows = 15;
constexpr int kTbRowsPerThread = 3;
constexpr int kTbExtRows = kTbThreadRows * kTbRowsPerThread;
constexpr int kTbThreads = 512;
struct TbPtrs {
  const float *Mx_in, *My_in, *a_in, *x0_in, *x1_in, *r_in;
  float *Mx_out, *My_out, *a_out, *x0_out, *x1_out, *r_out;
  const float *p0, *p1;
};

// TMA descriptors of the planes one iteration reads (ping-pong resolved).
struct TmaMaps {
  CUtensorMap a, Mx, My, x0, x1, r, p0, p1;
};

// Batched Algorithm 1 (prox_batch.cu, prox_tma.cu): the sequences' planes
// share one slab per state plane (sequence i at base + off); each sequence
// has its own geometry, step sizes and, for the TMA pipeline, tensor maps
// per ping-pong parity of M, a (in device memory, 64-byte aligned).
struct BatchPlanes {
  float *Mx[2], *My[2], *a[2];
  float *x0, *x1, *r, *p0, *p1;
};
struct BatchSeq {
  TmaMaps maps[2];
  Geometry G;
  IterCoeffs C;
  long long off;      // element offset of the sequence in every plane
  int tile0;          // first tile of the sequence in the partial-sum rows
  int ntiles;         // tiles of one iteration at the current tile height
};
constexpr int kBatchMaxSeq = 256;   // sequences per batch (work list in shared memory)
cudaError_t prepare_prox_tma_batch(int mode, bool balanced);
cudaError_t launch_prox_tma_batch(int mode, bool balanced, bool reduce, const BatchSeq* seqs, const int* act,
                                  int parity, const BatchPlanes& P, double* partials, int* err, int grid,
                                  cudaStream_t st);

struct CertCoeffs {
  double mu, rho;
  int iso, pexp, mode, balanced;
};

// ----------------------------------------------------------------- launchers
int tiled_num_ctas(const Geometry& g);
cudaError_t launch_prox_tiled(int mode, bool balanced, bool reduce, const Geometry& g,
                              const IterCoeffs& c, const StatePtrs& s, double* partials,
                              cudaStream_t st);

// Temporal blocking: `depth` iterations per pass (2..4) selects the halo
// (2 rows for depth 2, 4 otherwise); a launch runs n_sub <= halo iterations.
int temporal_halo(int depth);
int temporal_tile_rows(int depth);
int temporal_num_ctas(const Geometry& g, int depth);
// Raise the kernels' dynamic shared-memory limits (once, outside any capture).
cudaError_t prepare_prox_temporal(int mode, bool balanced, int depth);
cudaError_t launch_prox_temporal(int mode, bool balanced, bool reduce, int depth, int n_sub, const Geometry& g,
                                 const IterCoeffs& c, const TbPtrs& s, double* partials, cudaStream_t st);

size_t resident_smem_bytes(const Geometry& g, int mode, bool balanced);
bool resident_fits(const Geometry& g, int mode, bool balanced);
// Raise the kernel's dynamic shared-memory limit (once, outside any capture).
cudaError_t prepare_prox_resident(int mode, bool balanced, const Geometry& g);
// n_iter iterations in place on (Mx, My, a, x0, x1, r); the last one writes
// per-problem partial sums to partials[B][kNumSums] when reduce_last.
cudaError_t launch_prox_resident(int mode, bool balanced, const Geometry& g, const IterCoeffs& c,
                                 float* Mx, float* My, float* a, float* x0, float* x1, float* r,
                                 const float* p0, const float* p1, int n_iter, bool reduce_last,
                                 double* partials, cudaStream_t st);

// Persistent TMA-fed iteration (prox_tma.cu): one CTA per SM (grid =
// min(tiles, SMs)); partials[grid][kNumSums] when reduce; *err set to 1 if a
// bounded mbarrier wait expired.
cudaError_t prepare_prox_tma(int mode, bool balanced);
cudaError_t launch_prox_tma(int mode, bool balanced, bool reduce, const TmaMaps& maps, const Geometry& g,
                            const IterCoeffs& c, const StatePtrs& s, double* partials, int* err, int grid,
                            cudaStream_t st);
// Encode a TMA descriptor for a [B][H][Wp] plane with a box_w x box_h box;
// 0 on success.  tma_box(0|1|2) gives the box of a / M / pointwise planes.
int encode_plane_map(CUtensorMap* map, const float* base, const Geometry& g, int box_w, int box_h);
int tma_box(int which, int* w, int* h);

// Solver planes from a predicted state pred [B][4][H][W] (Mx, My, r, a);
// r, x0, x1 may be null (not a variable); gate > 0 keeps the prediction only
// near mass (warm_start.cu).
cudaError_t launch_warm_start(const float* pred, const Geometry& G, float* Mx, float* My, float* r, float* a,
                              float* x0, float* x1, const float* p0, const float* p1, float rho, float gate,
                              cudaStream_t st);

// Sum partials[n][kNumSums] in a fixed order into out[kNumSums].
cudaError_t launch_finalize_sums(const double* partials, int n, double* out, cudaStream_t st);

// Evaluation of a state without iterating: the check sums of the state
// itself (quantities 0, 2..7; 1 is 0) into partials, plus the certificate:
// cert_partials[n][4] = {max ||D*a||, dual objective, primal-feasible
// objective, unused} finalised into cert_out[4].
int cert_num_blocks(const Geometry& g);
cudaError_t launch_evaluate(const Geometry& g, const CertCoeffs& cc, const float* Mx,
                            const float* My, const float* a, const float* x0, const float* x1,
                            const float* r, const float* p0, const float* p1, double* partials,
                            double* sums_out, double* cert_partials, double* cert_out,
                            cudaStream_t st);

// ----------------------------------------------------------------- projection form
struct AdmmCoeffs {
  float beta, inv_beta;      // ADMM penalty and 1/beta (flux threshold)
  float rb, inv_1rb;         // rho * beta and 1 / (1 + rho * beta) (x-step)
  float mu_over_beta;        // r threshold (p = 1)
  float r2;                  // 1 / (1 + 2 mu / beta)  (p = 2)
  int iso, pexp, free0, free1, balanced;
};
// z, w, u: 5 planes each (Mx, My, x0, x1, r; frozen x and balanced r unused)
struct AdmmPlanes {
  float* z[5];
  float* w[5];
  float* u[5];
  float* k;      // K(z + u) - k0
  float* y;      // (K K^T)^{-1} k
  float* a;      // beta y
  const float* p0;
  const float* p1;
};
int admm_num_blocks(const Geometry& g);
cudaError_t admm_launch_z(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce, double* partials,
                          cudaStream_t st);
cudaError_t admm_launch_rhs(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce,
                            double* partials, cudaStream_t st);
cudaError_t admm_launch_w(const Geometry& g, const AdmmCoeffs& c, const AdmmPlanes& P, bool reduce, double* partials,
                          cudaStream_t st);

// DCT-II Neumann solve (dct_solve.cu)
struct DctPlan;
int dct_plan_create(int B, int H, int W, double c, int precision, DctPlan** out);
void dct_plan_destroy(DctPlan* p);
cudaError_t dct_plan_solve(DctPlan* p, const float* X, long long x_ld, float* Y, long long y_ld, cudaStream_t st);
// Route the tensor-core kernels' timeout flag to the owner's device flag.
void dct_plan_set_error_flag(DctPlan* p, int* derr);

// ----------------------------------------------------------------- RPCA
struct RpcaGeom {
  int T, H, W, Wp;
  long long plane;         // H * Wp
};
struct RpcaCoeffs {
  float lam, rho;
};
// Frame planes [T][H][Wp] (X, L, A, Tm, D, Y, S, LD) and pair planes
// [T-1][H][Wp] (z = prox x0, w = prox x1, Bz, Cw, p0, p1, zprev, wprev).
struct RpcaPlanes {
  float *X, *L, *A, *Tm, *D, *Y, *S, *LD;
  float* Tn;                // the SVT output of this outer iteration (Tm holds the previous one)
  float *z, *w, *Bz, *Cw, *p0, *p1, *zprev, *wprev;
  // signed-foreground variant only: S+ and S- frame planes (S = S+ - S-);
  // every pair plane then holds both signs, S- at sgn_off floats after S+
  float *Sp, *Sm;
  long long sgn_off;
};
int rpca_num_blocks(const RpcaGeom& g);
cudaError_t rpca_launch_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                            cudaStream_t st);
cudaError_t rpca_launch_post(const RpcaGeom& g, const RpcaPlanes& P, double* partials, cudaStream_t st);
// post of outer iteration k and pre of k + 1 in one pass (slot 0 sums only)
cudaError_t rpca_launch_post_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                                 cudaStream_t st);
// for T padded to TP in {16, 32, 64}: the same pass preceded by the SVT
// apply of iteration k (T^k = LD^k Wm, Wm TP x TP row-major, computed per
// chunk in shared memory; P.Tn written only when store_tn) and followed by
// iteration k + 1's Gram matrix: FP32 partials gpart[rpca_gram_parts(g)][TP][TP],
// reduced in the same cooperative launch into G (TP x TP doubles); bar: two
// zero-initialised unsigned ints owned by the caller (its grid barrier);
// err is set if the barrier wait expires; writes nrows slot-0 rows of partials
int rpca_gram_parts(const RpcaGeom& g);
cudaError_t rpca_launch_apply_post_pre_gram(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, int TP,
                                            const float* Wm, int store_tn, double* partials, int nrows, float* gpart,
                                            double* G, unsigned* bar, int* err, cudaStream_t st);
// the fused pass's grid barrier alone on `ctas` cooperative CTAs, its count
// preset (diagnostic: ot_debug_grid_barrier)
cudaError_t grid_barrier_probe(int ctas, unsigned preset, int* err, unsigned* generation);
cudaError_t rpca_launch_sumsq(const RpcaGeom& g, const float* Y, double* partials, cudaStream_t st);
// signed-foreground variant (rpca_pn_kernels.cu): lines 4-9 and 12-15 for S+
// and S-, residual sums in the same slots as rpca_launch_pre / _post
cudaError_t rpca_launch_pn_pre(const RpcaGeom& g, const RpcaCoeffs& c, const RpcaPlanes& P, double* partials,
                               cudaStream_t st);
cudaError_t rpca_launch_pn_post(const RpcaGeom& g, const RpcaPlanes& P, double* partials, cudaStream_t st);

// ----------------------------------------------------------------- SVT
int svt_padded_T(int T);                       // 16, 32, 64 or 128
float svt_tolerance(int T);                    // Jacobi stopping tolerance
int svt_gram_blocks(long long N);
int svt_apply_blocks(long long N, int T, int* gy);
cudaError_t svt_prepare();
cudaError_t svt_launch_gram(const float* X, long long ld, long long N, int T, double* partials, double* G, int* err,
                            cudaStream_t st);
// tensor-core partial Grams (gram_tcgen05.cu); T > 16
int svt_gram_tc_blocks(long long N);
cudaError_t svt_launch_gram_tc(const float* X, long long ld, long long N, int T, float* partials, int* err,
                               cudaStream_t st);
cudaError_t svt_launch_eig(const double* G, int T, int warm, float theta, int max_sweeps, float tol, float* V_io,
                           float* Wm, float* sig, int* sweeps, cudaStream_t st);
cudaError_t svt_launch_apply(const float* X, long long ld, long long N, int T, const float* Wm, float* Y,
                             long long ldy, bool reduce, double* partials, int* err, cudaStream_t st);
// tensor-core apply (svt_tcgen05.cu); T_pad = 32 or 64
int svt_apply_tc_blocks(long long N);
cudaError_t svt_launch_apply_tc(const float* X, long long ld, long long N, int T, const float* Wm, float* Y,
                                long long ldy, int* err, cudaStream_t st);

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace otp
