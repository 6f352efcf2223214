// The Algorithm 1 solver handle (opaque in the C ABI), shared by the
// translation units that drive it: otprox_api.cu and the RPCA runtime.
#pragma once

#include <cuda_runtime.h>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"

struct ot_prox {
  using Geometry = otp::Geometry;
  using IterCoeffs = otp::IterCoeffs;
  using TmaMaps = otp::TmaMaps;
  ot_prox_params prm;
  cudaStream_t stream;
  Geometry G;
  IterCoeffs C;
  size_t plane_elems;        // B * H * Wp
  float* slab;
  float* Mx[2];
  float* My[2];
  float* a[2];
  float* x0;
  float* x1;
  float* r;
  float* p0;
  float* p1;
  int cur;                   // ping-pong index of the current M, a
  bool resident;
  bool tma;
  int tma_grid;              // persistent CTAs (one per SM, at most one per tile)
  TmaMaps maps[2];           // by ping-pong parity of the input M, a
  int* derr;                 // device error flag (bounded waits)
  int* herr;                 // pinned host mirror
  double* partials;          // [max(n_ctas, n_cert)][kNumSums]
  double* cert_partials;     // [n_cert][4]
  double* dsums;             // device: [kNumSums] sums + [4] certificate
  double* hsums;             // pinned host mirror
  cudaGraphExec_t graph[2];  // one check interval, by starting parity
  int graph_n;
  // projection form (algorithm OT_ALG_PROJECTION)
  bool admm;
  float* admm_slab;          // z[5], w[5], u[5], k, y
  otp::AdmmPlanes AP;
  otp::AdmmCoeffs AC;
  otp::DctPlan* dct;
  int n_id;                  // identity blocks of K: the Laplacian shift c
  // temporal blocking (OT_KERNEL_TEMPORAL): x0, x1, r are ping-ponged with
  // M and a; x0 / x1 / r above point at the copies of parity cur
  bool tb;
  int tb_depth;
  float* x0s[2];
  float* x1s[2];
  float* rs[2];
};

// Cap the persistent TMA kernel's grid at (SMs - k) CTAs (otprox_api.cu).
void prox_reserve_sms(ot_prox* h, int k);
