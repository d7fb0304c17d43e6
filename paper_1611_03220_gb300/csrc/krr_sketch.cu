// TensorSketch features of the polynomial kernel (Section 2.2; the kernel of
// the experiments in Section 6 is k(x, z) = (gamma x^T z + c)^q).
//
// With x~ = [sqrt(gamma) x, sqrt(c)] (the last coordinate only when c > 0),
// the degree-q TensorSketch is
//   phi(x)[H] = sum over (i_1 .. i_q) with (h_1(i_1) + ... + h_q(i_q)) mod s = H
//               of g_1(i_1) ... g_q(i_q) x~_{i_1} ... x~_{i_q},
// i.e. the circular convolution of the q CountSketches CS_t(x~)[h_t(i)] +=
// g_t(i) x~_i.  E phi(x)^T phi(z) = (x~^T z~)^q = (gamma x^T z + c)^q.
//
// One warp per point, with its s-long accumulators in shared memory:
//   * q >= 2: the d~^2 terms of the first two factors are scattered with
//     shared-memory atomics (the convolution of two sparse vectors);
//   * every further factor convolves the dense s-vector with the d~ nonzeros
//     of its CountSketch, one nonzero at a time, lanes over the s positions
//     (distinct targets per nonzero, so no atomics);
// then the row is written out coalesced.  All arithmetic is FP32.
#include <algorithm>
#include <cmath>

#include "krr_internal.cuh"

namespace krr {
namespace {

__device__ __forceinline__ float xt_coord(const float* __restrict__ x, int d, int t, float sg,
                                          float sc) {
  return t < d ? sg * x[t] : sc;
}

__global__ void tensorsketch_kernel(const float* __restrict__ X, int n, int d, int ldx,
                                    const int* __restrict__ hash, const signed char* __restrict__ sign,
                                    int q, int dd, int s, float sg, float sc,
                                    float* __restrict__ Z, int ldz) {
  extern __shared__ float sbuf[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* A = sbuf + (size_t)warp * 2 * s;
  float* B = A + s;
  for (int i = blockIdx.x * warps + warp; i < n; i += gridDim.x * warps) {
    const float* x = X + (size_t)i * ldx;
    for (int j = lane; j < s; j += 32) A[j] = 0.f;
    __syncwarp();
    if (q == 1) {
      for (int t = lane; t < dd; t += 32)
        atomicAdd(&A[hash[t]], (float)sign[t] * xt_coord(x, d, t, sg, sc));
    } else {
      const int pairs = dd * dd;
      for (int e = lane; e < pairs; e += 32) {
        const int t1 = e % dd, t2 = e / dd;   // the first factor's index runs fastest
        int H = hash[t1] + hash[dd + t2];
        if (H >= s) H -= s;
        const float v = (float)(sign[t1] * sign[dd + t2]) * xt_coord(x, d, t1, sg, sc) *
                        xt_coord(x, d, t2, sg, sc);
        atomicAdd(&A[H], v);
      }
    }
    __syncwarp();
    for (int f = 2; f < q; ++f) {
      for (int j = lane; j < s; j += 32) B[j] = 0.f;
      __syncwarp();
      for (int t = 0; t < dd; ++t) {
        const float v = (float)sign[f * dd + t] * xt_coord(x, d, t, sg, sc);
        const int sh = hash[f * dd + t];
        if (v != 0.f) {
          for (int j = lane; j < s; j += 32) {
            int H = j + sh;
            if (H >= s) H -= s;
            B[H] = fmaf(v, A[j], B[H]);
          }
        }
        __syncwarp();
      }
      float* tmp = A;
      A = B;
      B = tmp;
    }
    float* z = Z + (size_t)i * ldz;
    for (int j = lane; j < s; j += 32) z[j] = A[j];
    __syncwarp();
  }
}

// Subsampled randomized Hadamard transform of each row (Section 4):
// z2 = s2^-1/2 P H D z1, one CTA per row.  The row, multiplied by the random
// signs and zero-padded to m (a power of two), is transformed in shared memory
// by the in-place butterflies of H_m's recursive definition (log2 m passes of
// (a + b, a - b) on pairs h apart), then the sampled entries are written.
__global__ void srht_kernel(const float* __restrict__ Z1, int n, int s1, int ldz1,
                            const signed char* __restrict__ signs, int m,
                            const int* __restrict__ rows, int s2, float scale,
                            float* __restrict__ Z2, int ldz2) {
  extern __shared__ float buf[];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const float* z = Z1 + (size_t)i * ldz1;
    for (int j = threadIdx.x; j < m; j += blockDim.x)
      buf[j] = j < s1 ? (float)signs[j] * z[j] : 0.f;
    __syncthreads();
    for (int hh = 1; hh < m; hh <<= 1) {
      for (int p = threadIdx.x; p < (m >> 1); p += blockDim.x) {
        const int j = (p / hh) * 2 * hh + (p % hh);
        const float a = buf[j], b = buf[j + hh];
        buf[j] = a + b;
        buf[j + hh] = a - b;
      }
      __syncthreads();
    }
    float* out = Z2 + (size_t)i * ldz2;
    for (int k = threadIdx.x; k < s2; k += blockDim.x) out[k] = scale * buf[rows[k]];
    __syncthreads();
  }
}

}  // namespace

void launch_tensorsketch(cudaStream_t st, const float* X, int n, int d, int ldx, const int* hash,
                         const signed char* sign, int q, int s, double gamma, double c, float* Z,
                         int ldz) {
  const int dd = d + (c > 0.0 ? 1 : 0);
  const size_t per_warp = (size_t)2 * s * sizeof(float);
  const size_t budget = 200 * 1024;
  if (per_warp > budget) throw Error{KRR_EUNSUPPORTED, "tensorsketch: s too large (s <= 25600)"};
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, budget / per_warp));
  const size_t smem = per_warp * warps;
  static size_t attr = 0;
  if (attr < smem) {
    KRR_CUDA(cudaFuncSetAttribute(tensorsketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = smem;
  }
  const int blocks = std::min((n + warps - 1) / warps, 8 * sm_count());
  tensorsketch_kernel<<<blocks, 32 * warps, smem, st>>>(
      X, n, d, ldx, hash, sign, q, dd, s, (float)std::sqrt(gamma), (float)std::sqrt(c), Z, ldz);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr

namespace krr {

void launch_srht(cudaStream_t st, const float* Z1, int n, int s1, int ldz1,
                 const signed char* signs, int m, const int* rows, int s2, float* Z2, int ldz2) {
  const size_t smem = (size_t)m * sizeof(float);
  if (smem > 200 * 1024) throw Error{KRR_EUNSUPPORTED, "srht: m too large (m <= 32768)"};
  static size_t attr = 0;
  if (attr < smem) {
    KRR_CUDA(cudaFuncSetAttribute(srht_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = smem;
  }
  const int blocks = std::min(n, 8 * sm_count());
  srht_kernel<<<blocks, 512, smem, st>>>(Z1, n, s1, ldz1, signs, m, rows, s2,
                                         (float)(1.0 / std::sqrt((double)s2)), Z2, ldz2);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
