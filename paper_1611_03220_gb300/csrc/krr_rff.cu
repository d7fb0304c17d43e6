// Random Fourier features, Section 2.2 of the paper:
//   Z[i, j] = sqrt(2/s) cos(x_i . w_j + b_j)
// with w_j ~ N(0, sigma^-2 I) and b_j ~ U[0, 2 pi) supplied by the caller
// (the feature step of Algorithm 1).  The sqrt(2/s) scale makes E[Z Z^T] = K; the
// printed s^-1/2 omits the factor 2 of E[cos(a + b) cos(c + b)].
//
// One FP32 register-tiled GEMM X W (128 x 128 tile per CTA, 8 x 8 per
// thread, 8-deep coordinate chunks through shared memory) with the cos
// epilogue fused, so the n x s pre-activation never reaches HBM.
#include "krr_internal.cuh"

namespace krr {
namespace {

constexpr int BM = 128, BN = 128, DC = 8;

__global__ void __launch_bounds__(256)
rff_kernel(const float* __restrict__ X, int n, int d, int ldx, const float* __restrict__ W,
           const float* __restrict__ b, int s, float scale, float* __restrict__ Z, int ldz) {
  __shared__ float As[DC][BM + 4];
  __shared__ float Bs[DC][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  for (int c0 = 0; c0 < d; c0 += DC) {
    __syncthreads();
    for (int e = tid; e < BM * DC; e += 256) {
      int rr = e / DC, t = e % DC;
      int i = i0 + rr, dd = c0 + t;
      As[t][rr] = (i < n && dd < d) ? X[(size_t)i * ldx + dd] : 0.f;
    }
    for (int e = tid; e < BN * DC; e += 256) {
      int t = e / BN, cc = e % BN;
      int j = j0 + cc, dd = c0 + t;
      Bs[t][cc] = (j < s && dd < d) ? W[(size_t)dd * s + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < DC; ++t) {
      float a[8], bb[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = As[t][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 8; ++c) bb[c] = Bs[t][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], bb[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int j = j0 + tx + 16 * c;
    if (j >= s) continue;
    float bj = b[j];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      int i = i0 + ty + 16 * r;
      if (i < n) Z[(size_t)i * ldz + j] = scale * cosf(acc[r][c] + bj);
    }
  }
}

}  // namespace

void launch_rff(cudaStream_t st, const float* X, int n, int d, int ldx, const float* W,
                const float* b, int s, float* Z, int ldz) {
  dim3 grid((n + BM - 1) / BM, (s + BN - 1) / BN);
  float scale = (float)sqrt(2.0 / (double)s);
  rff_kernel<<<grid, 256, 0, st>>>(X, n, d, ldx, W, b, s, scale, Z, ldz);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
