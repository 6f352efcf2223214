// Plan of the DCT-II Neumann solve, shared by the FP32 path (dct_solve.cu)
// and the tensor-core path (dct_tcgen05.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace otp {

struct DctPlan {
  int B, H, W;
  double c;
  int precision;
  // FP32 transform matrices (row-major n x n): C and C^T for each axis
  float *CH, *CHt, *CW, *CWt;
  float* inv_lam;     // [W][H]: 1 / (lam_W[l] + lam_H[k] + c), 0 for a zero mode
  float* work;        // [B][max(H,W)]^2 scratch
  void* tc;           // tensor-core plan (split BF16), or null
  int* err;           // device flag set by a tensor-core kernel whose bounded wait expired
};

// Orthonormal DCT-II matrix C[k][m] = s_k cos(pi (m + 1/2) k / n) and the
// path-Laplacian eigenvalues 4 sin^2(pi k / 2n), in double.
std::vector<double> dct_matrix(int n);
std::vector<double> path_laplacian_eigs(int n);

int dct_tc_create(DctPlan* p);
void dct_tc_destroy(DctPlan* p);
cudaError_t dct_tc_solve(DctPlan* p, const float* X, long long x_ld, float* Y, long long y_ld, cudaStream_t st);

}  // namespace otp
