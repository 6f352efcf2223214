// Warm start of Algorithm 1 from a predicted state (Sec. III-B warm-starts
// the iterates from a cache; here the cache is a network's prediction).
//
// pred is [B][4][H][W] (channels Mx, My, r, a, the layout the warm-start
// network writes).  Mx, My, r and a go to the solver's current planes, with
// the flux zeroed on the slots that have no edge (Mx on the last row, My on
// the last column).  A free x is set from the x-step's fixed point, which is
// the optimality condition of the (1/2 rho) ||x - p||^2 term given a:
// x0 = max(p0 + rho a, 0), x1 = max(p1 - rho a, 0).
//
// Gate: with gate > 0 the prediction is taken only at pixels where p0 + p1
// exceeds gate somewhere in the 5 x 5 neighbourhood; elsewhere the frames
// hold (almost) no mass, the converged state is (almost) zero, and the
// state is written as for a zero prediction (M = r = a = 0, x = p).
#include <cuda_runtime.h>

#include "otprox_internal.cuh"

namespace otp {
namespace {

constexpr int kGateR = 2;   // gate neighbourhood radius

__global__ void warm_start_kernel(const float* __restrict__ pred, Geometry G, float* __restrict__ Mx,
                                  float* __restrict__ My, float* __restrict__ r, float* __restrict__ a,
                                  float* __restrict__ x0, float* __restrict__ x1, const float* __restrict__ p0,
                                  const float* __restrict__ p1, float rho, float gate) {
  const long long hw = (long long)G.H * G.W;
  const long long total = (long long)G.B * hw;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / hw;
    const int i = (int)((idx / G.W) % G.H), j = (int)(idx % G.W);
    const float* src = pred + b * 4 * hw + (long long)i * G.W + j;
    const long long o = b * G.plane + (long long)i * G.Wp + j;
    bool use = true;
    if (gate > 0.f) {
      float m = 0.f;
      for (int di = -kGateR; di <= kGateR; ++di)
        for (int dj = -kGateR; dj <= kGateR; ++dj) {
          const int ii = i + di, jj = j + dj;
          if (ii >= 0 && ii < G.H && jj >= 0 && jj < G.W) {
            const long long q = b * G.plane + (long long)ii * G.Wp + jj;
            m = fmaxf(m, p0[q] + p1[q]);
          }
        }
      use = m > gate;
    }
    const float av = use ? src[3 * hw] : 0.f;
    Mx[o] = (i == G.H - 1 || !use) ? 0.f : src[0];
    My[o] = (j == G.W - 1 || !use) ? 0.f : src[hw];
    if (r) r[o] = use ? src[2 * hw] : 0.f;
    a[o] = av;
    if (x0) x0[o] = fmaxf(fmaf(rho, av, p0[o]), 0.f);
    if (x1) x1[o] = fmaxf(fmaf(-rho, av, p1[o]), 0.f);
  }
}

}  // namespace

cudaError_t launch_warm_start(const float* pred, const Geometry& G, float* Mx, float* My, float* r, float* a,
                              float* x0, float* x1, const float* p0, const float* p1, float rho, float gate,
                              cudaStream_t st) {
  const long long total = (long long)G.B * G.H * G.W;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  warm_start_kernel<<<(int)blocks, 256, 0, st>>>(pred, G, Mx, My, r, a, x0, x1, p0, p1, rho, gate);
  return cudaGetLastError();
}

}  // namespace otp
