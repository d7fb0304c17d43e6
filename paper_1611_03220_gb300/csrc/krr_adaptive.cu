// Adaptive sketch size (Section 5, Theorem 4).  Starting from a small s, the
// random-feature matrix Z (n x s) is tested against Theorem 4's first
// condition,
//   ||(I - P) K (I - P)||_2 <= 0.1 lambda,
// P the orthogonal projection on the eigenvectors of Z Z^T whose eigenvalues
// exceed 0.05 lambda, by power iteration; s doubles until the test passes.
//
// P from the s x s Gram matrix G = Z^T Z (same eigenvalues as Z Z^T, with
// eigenvectors v_k <-> u_k = Z v_k / sqrt(t_k)):
//   P = Z Q Z^T,   Q = G^-1 Pi,   Pi the spectral projection of G on t > tau.
// Pi = (I + sign(B)) / 2 with B = (G - tau I)(G + tau I)^-1 = I - 2 tau (G + tau I)^-1,
// whose eigenvalues (t - tau)/(t + tau) lie in (-1, 1) and keep the sign of
// t - tau on the scale of tau rather than of ||G||; sign(B) by the
// Newton-Schulz iteration X <- X (3 I - X^2) / 2 (FP64 s x s products).
// G^-1 on Pi's range is (G + delta I)^-1 with delta = 1e-3 tau (a relative
// change below 1e-3 of P's eigenvalues there).  The inverses come from the
// FP64 Cholesky factorisation and triangular inverse of the preconditioner
// set-up.
#include <algorithm>
#include <cmath>
#include <vector>

#include "krr_internal.cuh"

namespace krr {
namespace {

// out = a A + b I (s x s); A may alias out.
__global__ void axpi_kernel(const double* A, int s, double a, double b, double* out) {
  const size_t total = (size_t)s * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = a * A[e] + ((e / s) == (e % s) ? b : 0.0);
}

// part[blk, j] = sum over this block's rows of Z[i, j] x[i]  (Z n x s FP32)
__global__ void zt_x_kernel(const float* __restrict__ Z, int n, int s, const double* __restrict__ x,
                            int rows_per_block, double* __restrict__ part) {
  const int r0 = blockIdx.x * rows_per_block, r1 = min(n, r0 + rows_per_block);
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    double acc = 0.0;
    for (int i = r0; i < r1; ++i) acc = fma((double)Z[(size_t)i * s + j], x[i], acc);
    part[(size_t)blockIdx.x * s + j] = acc;
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int nb, int s,
                                 double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)b * s + j];
    out[j] = acc;
  }
}

// y = Q u (s x s FP64 times s)
__global__ void gemv_d_kernel(const double* __restrict__ Q, int s, const double* __restrict__ u,
                              double* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= s) return;
  double acc = 0.0;
  for (int j = lane; j < s; j += 32) acc = fma(Q[(size_t)warp * s + j], u[j], acc);
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) y[warp] = acc;
}

// out = x - Z v  (Z n x s FP32, v s FP64)
__global__ void x_minus_zv_kernel(const float* __restrict__ Z, int n, int s,
                                  const double* __restrict__ v, const double* __restrict__ x,
                                  double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double acc = 0.0;
  for (int j = lane; j < s; j += 32) acc = fma((double)Z[(size_t)warp * s + j], v[j], acc);
  for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) out[warp] = x[warp] - acc;
}

__global__ void scale_kernel(double* x, int n, double a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] *= a;
}

void gemm_d(cudaStream_t st, const double* A, const double* B, double* C, int s, int ta, int tb,
            double alpha, double beta) {
  launch_gemm_d(st, s, s, s, alpha, A, s, ta, B, s, tb, beta, C, s);
}

void axpi(cudaStream_t st, const double* A, int s, double a, double b, double* out) {
  axpi_kernel<<<std::min(8 * sm_count(), (int)(((size_t)s * s + 255) / 256)), 256, 0, st>>>(
      A, s, a, b, out);
  KRR_CHECK_LAUNCH();
}

}  // namespace

size_t adaptive_work_elems(int n, int s) {
  const int nb = std::max(1, std::min(8 * sm_count(), (n + 63) / 64));
  return (size_t)5 * s * s + (size_t)nb * s + 2 * (size_t)s + tri_inverse_scratch_elems(s);
}

void adaptive_projector(cudaStream_t st, const double* G, int s, double tau, int ns_iters,
                        double* work, int* info_dev, int* info_host) {
  const size_t ss = (size_t)s * s;
  double* A = work;
  double* B = A + ss;
  double* C = B + ss;
  double* D = C + ss;
  double* Q = D + ss;
  double* tri = work + 5 * ss;   // scratch of the triangular inverse
  auto chol_inv = [&](double shift) {
    // C = (G + shift I)^-1 = L^-T L^-1
    axpi(st, G, s, 1.0, shift, A);
    launch_cholesky(st, A, s, info_dev);
    KRR_CUDA(cudaMemcpyAsync(info_host, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaStreamSynchronize(st));
    if (*info_host != 0)
      throw Error{KRR_ECHOL, "adaptive sketch: G + shift I is not positive definite"};
    KRR_CUDA(cudaMemsetAsync(B, 0, ss * sizeof(double), st));
    launch_tri_inverse(st, A, s, B, tri);
    gemm_d(st, B, B, C, s, 1, 0, 1.0, 0.0);
  };
  // B0 = I - 2 tau (G + tau I)^-1, then its sign by Newton-Schulz
  chol_inv(tau);
  axpi(st, C, s, -2.0 * tau, 1.0, A);
  for (int it = 0; it < ns_iters; ++it) {
    gemm_d(st, A, A, B, s, 0, 0, 1.0, 0.0);
    KRR_CUDA(cudaMemcpyAsync(C, A, ss * sizeof(double), cudaMemcpyDeviceToDevice, st));
    gemm_d(st, A, B, C, s, 0, 0, -0.5, 1.5);
    std::swap(A, C);
  }
  // D = Pi = (I + sign) / 2; Q = (G + delta I)^-1 Pi
  axpi(st, A, s, 0.5, 0.5, D);
  // chol_inv writes A, B, C: A no longer holds the sign once D is formed
  A = work;
  B = A + ss;
  C = B + ss;
  chol_inv(1e-3 * tau);
  gemm_d(st, C, D, Q, s, 0, 0, 1.0, 0.0);
}

const double* adaptive_q(const double* work, int s) { return work + 4 * (size_t)s * s; }

void apply_i_minus_p(cudaStream_t st, const float* Z, int n, int s, const double* work,
                     const double* x, double* out) {
  const size_t ss = (size_t)s * s;
  const double* Q = work + 4 * ss;
  double* part = const_cast<double*>(work) + 5 * ss + tri_inverse_scratch_elems(s);
  const int nb = std::max(1, std::min(8 * sm_count(), (n + 63) / 64));
  double* u = part + (size_t)nb * s;
  double* v = u + s;
  const int rpb = (n + nb - 1) / nb;
  zt_x_kernel<<<nb, 256, 0, st>>>(Z, n, s, x, rpb, part);
  KRR_CHECK_LAUNCH();
  sum_parts_kernel<<<std::max(1, (s + 255) / 256), 256, 0, st>>>(part, nb, s, u);
  KRR_CHECK_LAUNCH();
  gemv_d_kernel<<<(s * 32 + 255) / 256, 256, 0, st>>>(Q, s, u, v);
  KRR_CHECK_LAUNCH();
  x_minus_zv_kernel<<<(n * 32 + 255) / 256, 256, 0, st>>>(Z, n, s, v, x, out);
  KRR_CHECK_LAUNCH();
}

void launch_scale_d(cudaStream_t st, double* x, int n, double a) {
  scale_kernel<<<std::min(8 * sm_count(), (n + 255) / 256), 256, 0, st>>>(x, n, a);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
