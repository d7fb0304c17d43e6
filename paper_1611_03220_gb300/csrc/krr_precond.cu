// Random-feature preconditioner M = Z Z^T + lambda_p I (Section 3.1,
// Algorithm 1):
//   G = Z^T Z + lambda_p I_s              gram_kernel / gram_finalize_kernel
//   L L^T = G (lower, FP64)               potrf / trsm / syrk kernels
//   L^-1 (for the ZL apply form)          diag_inv / offdiag_inv kernels
//   U = L^-1 Z^T (paper's apply form)     form_u_kernel
//   M^-1 r = (r - Z L^-T L^-1 Z^T r) / lambda_p   or  (r - U^T U r) / lambda_p
// The paper forms U so that the apply is GEMM-only; here both forms exist.
// The triangular solves of the ZL form use the explicit inverse L^-1 computed
// once at set-up, so each per-iteration solve is a pair of triangular
// matrix-vector products spread over all SMs instead of a serial
// substitution.
//
// Precision: Z is stored FP32 or BF16.  With BF16 storage the Gram matrix is
// formed from the rounded values (their pairwise products are exact in FP32),
// so the factors describe exactly the operator that is applied, and
// M stays symmetric positive definite by construction.  All s x s work is
// FP64; every n-long reduction accumulates in FP64.
#include "krr_internal.cuh"

namespace krr {
namespace {

constexpr int NB = 64;   // block size of every s x s kernel

// One stored feature: FP32 (0), BF16 (1) or an 8-bit fixed-point q / 128 (2).
template <int BF16>
__device__ __forceinline__ float zload(const void* Zs, size_t idx) {
  if (BF16 == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Zs)[idx]);
  if (BF16 == 2) return (float)reinterpret_cast<const signed char*>(Zs)[idx] * 0.0078125f;
  return reinterpret_cast<const float*>(Zs)[idx];
}

__global__ void copy_z_kernel(const float* __restrict__ Z, int n, int s, int ldz, void* Zs,
                              int bf16) {
  const size_t total = (size_t)n * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t i = e / s, j = e % s;
    float v = Z[i * ldz + j];
    if (bf16)
      reinterpret_cast<__nv_bfloat16*>(Zs)[e] = __float2bfloat16_rn(v);
    else
      reinterpret_cast<float*>(Zs)[e] = v;
  }
}

// ----------------------------------------------------------------- Gram --
// One CTA per (lower tile pair, row chunk).  With BF16 storage each 16-row
// slab is summed in FP32 (exact products, short sums) and then added to
// FP64 accumulators; with FP32 storage products and sums are FP64.
constexpr int GR = 16;

__device__ __forceinline__ void tile_pair(int p, int& I, int& J) {
  int i = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

template <int BF16>
__global__ void __launch_bounds__(256)
gram_kernel(const void* __restrict__ Zs, int n, int s, double* __restrict__ part,
            int rows_per_chunk) {
  __shared__ float As[GR][NB + 4];
  __shared__ float Bs[GR][NB + 4];
  int I, J;
  tile_pair(blockIdx.x, I, J);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(n, r0 + rows_per_chunk);
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int base = r0; base < r1; base += GR) {
    __syncthreads();
    for (int e = tid; e < GR * NB; e += 256) {
      int t = e / NB, col = e % NB;
      int row = base + t;
      int ca = I * NB + col, cb = J * NB + col;
      As[t][col] = (row < r1 && ca < s) ? zload<BF16>(Zs, (size_t)row * s + ca) : 0.f;
      Bs[t][col] = (row < r1 && cb < s) ? zload<BF16>(Zs, (size_t)row * s + cb) : 0.f;
    }
    __syncthreads();
    if (BF16) {
      float a32[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) a32[r][c] = 0.f;
#pragma unroll
      for (int t = 0; t < GR; ++t)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            a32[r][c] = fmaf(As[t][ty + 16 * r], Bs[t][tx + 16 * c], a32[r][c]);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += (double)a32[r][c];
    } else {
#pragma unroll
      for (int t = 0; t < GR; ++t)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            acc[r][c] = fma((double)As[t][ty + 16 * r], (double)Bs[t][tx + 16 * c], acc[r][c]);
    }
  }
  double* out = part + (size_t)blockIdx.y * s * s;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int row = I * NB + ty + 16 * r;
    if (row >= s) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int col = J * NB + tx + 16 * c;
      if (col < s) out[(size_t)row * s + col] = acc[r][c];
    }
  }
}

__global__ void gram_finalize_kernel(const double* __restrict__ part, int nchunk, int s,
                                     double lam_p, double* __restrict__ G) {
  const size_t total = (size_t)s * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / s), j = (int)(e % s);
    if (i < j) continue;
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += part[(size_t)c * total + e];
    if (i == j) v += lam_p;
    G[(size_t)i * s + j] = v;
    G[(size_t)j * s + i] = v;
  }
}

// ------------------------------------------------------------- Cholesky --
// Right-looking blocked LL^T with 64-wide panels.  info != 0 stops every
// later kernel; it holds 1 + the first column whose pivot was not > 0.

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int s, int kb, int* info) {
  if (*info) return;
  __shared__ double a[NB][NB + 1];
  __shared__ int fail;
  const int o = kb * NB, nb = min(NB, s - o), tid = threadIdx.x;
  if (tid == 0) fail = 0;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    a[i][j] = (j <= i) ? A[(size_t)(o + i) * s + o + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double v = a[j][j];
      if (!(v > 0.0)) {
        fail = 1;
        *info = o + j + 1;
      } else {
        a[j][j] = sqrt(v);
      }
    }
    __syncthreads();
    if (fail) return;
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) a[i][j] /= a[j][j];
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int ii = j + 1 + e / m, ll = j + 1 + e % m;
      if (ll <= ii) a[ii][ll] -= a[ii][j] * a[ll][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    A[(size_t)(o + i) * s + o + j] = (j <= i) ? a[i][j] : 0.0;
  }
}

// Panel below the diagonal block: B := B L_kk^-T, one thread per row.
__global__ void __launch_bounds__(NB) trsm_panel_kernel(double* A, int s, int kb, const int* info) {
  if (*info) return;
  __shared__ double L[NB][NB + 1];
  __shared__ double B[NB][NB + 1];
  const int o = kb * NB, nb = min(NB, s - o);
  const int r0 = o + nb + blockIdx.x * NB, nr = min(NB, s - r0);
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += NB) {
    int i = e / nb, j = e % nb;
    L[i][j] = A[(size_t)(o + i) * s + o + j];
  }
  for (int e = tid; e < nr * nb; e += NB) {
    int i = e / nb, j = e % nb;
    B[i][j] = A[(size_t)(r0 + i) * s + o + j];
  }
  __syncthreads();
  if (tid < nr) {
    for (int j = 0; j < nb; ++j) {
      double v = B[tid][j];
      for (int m = 0; m < j; ++m) v -= B[tid][m] * L[j][m];
      B[tid][j] = v / L[j][j];
    }
  }
  __syncthreads();
  for (int e = tid; e < nr * nb; e += NB) {
    int i = e / nb, j = e % nb;
    A[(size_t)(r0 + i) * s + o + j] = B[i][j];
  }
}

// Trailing update A[I, J] -= P_I P_J^T for lower tile pairs past panel kb.
__global__ void __launch_bounds__(256) syrk_update_kernel(double* A, int s, int kb, const int* info) {
  if (*info) return;
  __shared__ double Pa[16][NB + 1];
  __shared__ double Pb[16][NB + 1];
  int Ip, Jp;
  tile_pair(blockIdx.x, Ip, Jp);
  const int I = kb + 1 + Ip, J = kb + 1 + Jp;
  const int o = kb * NB, nb = min(NB, s - o);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int m0 = 0; m0 < nb; m0 += 16) {
    __syncthreads();
    for (int e = tid; e < 16 * NB; e += 256) {
      int row = e / 16, t = e % 16;
      int ra = I * NB + row, rb = J * NB + row, m = m0 + t;
      Pa[t][row] = (ra < s && m < nb) ? A[(size_t)ra * s + o + m] : 0.0;
      Pb[t][row] = (rb < s && m < nb) ? A[(size_t)rb * s + o + m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          acc[r][c] = fma(Pa[t][ty + 16 * r], Pb[t][tx + 16 * c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int row = I * NB + ty + 16 * r;
    if (row >= s) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int col = J * NB + tx + 16 * c;
      if (col < s && col <= row) A[(size_t)row * s + col] -= acc[r][c];
    }
  }
}

__global__ void zero_upper_kernel(double* A, int s) {
  const size_t total = (size_t)s * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / s), j = (int)(e % s);
    if (j > i) A[e] = 0.0;
  }
}

// -------------------------------------------------------- FP64 products --
// C = alpha op(A) op(B) + beta C with op(A) m x k, op(B) k x n, row-major
// with leading dimensions; op(X) = X^T when tX.  64 x 64 output tiles of
// 16 x 16 threads, 4 x 4 results each, K in slabs of 16 through shared
// memory.  C must not alias A or B.
constexpr int GT = 64;
constexpr int GKS = 16;

__global__ void __launch_bounds__(256)
gemm_f64_kernel(int m, int n, int k, double alpha, const double* __restrict__ A, int lda, int ta,
                const double* __restrict__ B, int ldb, int tb, double beta,
                double* __restrict__ C, int ldc) {
  __shared__ double As[GKS][GT + 1];
  __shared__ double Bs[GKS][GT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int k0 = 0; k0 < k; k0 += GKS) {
    for (int e = threadIdx.x; e < GKS * GT; e += 256) {
      const int t = ta ? e / GT : e % GKS, r = ta ? e % GT : e / GKS;
      const int i = i0 + r, kk = k0 + t;
      As[t][r] = (i < m && kk < k) ? (ta ? A[(size_t)kk * lda + i] : A[(size_t)i * lda + kk]) : 0.0;
    }
    for (int e = threadIdx.x; e < GKS * GT; e += 256) {
      const int t = tb ? e % GKS : e / GT, c = tb ? e / GKS : e % GT;
      const int j = j0 + c, kk = k0 + t;
      Bs[t][c] = (j < n && kk < k) ? (tb ? B[(size_t)j * ldb + kk] : B[(size_t)kk * ldb + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < GKS; ++t)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(As[t][ty + 16 * r], Bs[t][tx + 16 * c], acc[r][c]);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= n) continue;
      double* cp = C + (size_t)i * ldc + j;
      *cp = alpha * acc[r][c] + (beta != 0.0 ? beta * *cp : 0.0);
    }
  }
}

// ------------------------------------------------------ triangular inverse --
// Diagonal blocks: D_kk = L_kk^-1 by forward substitution, one column per
// thread.
__global__ void __launch_bounds__(NB) diag_inv_kernel(const double* L, int s, double* Linv) {
  __shared__ double a[NB][NB + 1];
  __shared__ double x[NB][NB + 1];
  const int o = blockIdx.x * NB, nb = min(NB, s - o), t = threadIdx.x;
  for (int e = t; e < nb * nb; e += NB) {
    int i = e / nb, j = e % nb;
    a[i][j] = L[(size_t)(o + i) * s + o + j];
  }
  __syncthreads();
  if (t < nb) {
    for (int i = 0; i < nb; ++i) {
      if (i < t) {
        x[i][t] = 0.0;
        continue;
      }
      double v = (i == t) ? 1.0 : 0.0;
      for (int m = t; m < i; ++m) v -= a[i][m] * x[m][t];
      x[i][t] = v / a[i][i];
    }
  }
  __syncthreads();
  for (int e = t; e < nb * nb; e += NB) {
    int i = e / nb, j = e % nb;
    Linv[(size_t)(o + i) * s + o + j] = x[i][j];
  }
}


__global__ void transpose_d_kernel(const double* __restrict__ A, int s, double* __restrict__ B) {
  __shared__ double t[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int i = by + r, j = bx + threadIdx.x;
    t[r][threadIdx.x] = (i < s && j < s) ? A[(size_t)i * s + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int i = bx + r, j = by + threadIdx.x;
    if (i < s && j < s) B[(size_t)i * s + j] = t[threadIdx.x][r];
  }
}

// ------------------------------------------------------------ U = L^-1 Z^T --
template <int BF16>
__global__ void __launch_bounds__(256)
form_u_kernel(const double* __restrict__ Linv, const void* __restrict__ Zs, int n, int s,
              float* __restrict__ U) {
  __shared__ double Pa[16][NB + 1];
  __shared__ double Pb[16][NB + 1];
  const int a0 = blockIdx.y * NB, i0 = blockIdx.x * NB;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int bmax = min(s, a0 + NB);
  for (int b0 = 0; b0 < bmax; b0 += 16) {
    __syncthreads();
    for (int e = tid; e < 16 * NB; e += 256) {
      int row = e / 16, t = e % 16;
      int a = a0 + row, b = b0 + t;
      Pa[t][row] = (a < s && b < s) ? Linv[(size_t)a * s + b] : 0.0;
      int i = i0 + row;
      Pb[t][row] = (i < n && b < s) ? (double)zload<BF16>(Zs, (size_t)i * s + b) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          acc[r][c] = fma(Pa[t][ty + 16 * r], Pb[t][tx + 16 * c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int a = a0 + ty + 16 * r;
    if (a >= s) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = i0 + tx + 16 * c;
      if (i < n) U[(size_t)a * n + i] = (float)acc[r][c];
    }
  }
}

}  // namespace

int gram_chunks(int n, int s) {
  int T = (s + NB - 1) / NB;
  int pairs = T * (T + 1) / 2;
  int nch = (2 * sm_count() + pairs - 1) / pairs;
  int maxch = (n + 255) / 256;
  if (nch > maxch) nch = maxch;
  // keep the partial buffer under 512 MiB
  size_t per = (size_t)s * s * sizeof(double);
  while (nch > 1 && per * nch > (size_t(512) << 20)) --nch;
  return nch < 1 ? 1 : nch;
}

void launch_copy_z(cudaStream_t st, const float* Z, int n, int s, int ldz, void* Zs, int bf16) {
  int nb = 8 * sm_count();
  copy_z_kernel<<<nb, 256, 0, st>>>(Z, n, s, ldz, Zs, bf16);
  KRR_CHECK_LAUNCH();
}

void launch_gram(cudaStream_t st, const void* Zs, int bf16, int n, int s, double lam_p,
                 double* G, double* part, int nchunk) {
  int T = (s + NB - 1) / NB;
  int pairs = T * (T + 1) / 2;
  int rpc = (n + nchunk - 1) / nchunk;
  rpc = (rpc + GR - 1) / GR * GR;
  dim3 grid(pairs, nchunk);
  if (bf16)
    gram_kernel<1><<<grid, 256, 0, st>>>(Zs, n, s, part, rpc);
  else
    gram_kernel<0><<<grid, 256, 0, st>>>(Zs, n, s, part, rpc);
  KRR_CHECK_LAUNCH();
  gram_finalize_kernel<<<8 * sm_count(), 256, 0, st>>>(part, nchunk, s, lam_p, G);
  KRR_CHECK_LAUNCH();
}

void launch_cholesky(cudaStream_t st, double* A, int s, int* info) {
  const int T = (s + NB - 1) / NB;
  KRR_CUDA(cudaMemsetAsync(info, 0, sizeof(int), st));
  for (int kb = 0; kb < T; ++kb) {
    potrf_diag_kernel<<<1, 256, 0, st>>>(A, s, kb, info);
    KRR_CHECK_LAUNCH();
    if (kb + 1 < T) {
      int rows = s - (kb + 1) * NB;
      trsm_panel_kernel<<<(rows + NB - 1) / NB, NB, 0, st>>>(A, s, kb, info);
      KRR_CHECK_LAUNCH();
      int Tt = T - kb - 1;
      syrk_update_kernel<<<Tt * (Tt + 1) / 2, 256, 0, st>>>(A, s, kb, info);
      KRR_CHECK_LAUNCH();
    }
  }
  zero_upper_kernel<<<8 * sm_count(), 256, 0, st>>>(A, s);
  KRR_CHECK_LAUNCH();
}

namespace {
// Recursive blocked inverse of the lower triangle L[o:o+m, o:o+m] (m a
// multiple of NB or the tail of the matrix): with L = [L11 0; L21 L22],
// L^-1 = [X11 0; X21 X22], X21 = -X22 L21 X11.  The diagonal NB-blocks are
// already inverted; each level adds two FP64 products, so the work is in a
// few large GEMMs rather than a serial sweep of block rows.  T: scratch of
// at least (m/2) x (m/2) doubles (ld s).
void tri_inverse_rec(cudaStream_t st, const double* L, int s, double* Linv, int o, int m,
                     double* T) {
  if (m <= NB) return;
  const int nb = (m + NB - 1) / NB;
  const int h = (nb / 2) * NB;          // split at a block boundary
  const int m2 = m - h;
  tri_inverse_rec(st, L, s, Linv, o, h, T);
  tri_inverse_rec(st, L, s, Linv, o + h, m2, T);
  // T = L21 X11 (m2 x h), then X21 = -X22 T (m2 x h)
  dim3 g1((h + GT - 1) / GT, (m2 + GT - 1) / GT);
  gemm_f64_kernel<<<g1, 256, 0, st>>>(m2, h, h, 1.0, L + (size_t)(o + h) * s + o, s, 0,
                                      Linv + (size_t)o * s + o, s, 0, 0.0, T, s);
  KRR_CHECK_LAUNCH();
  gemm_f64_kernel<<<g1, 256, 0, st>>>(m2, h, m2, -1.0, Linv + (size_t)(o + h) * s + o + h, s, 0,
                                      T, s, 0, 0.0, Linv + (size_t)(o + h) * s + o, s);
  KRR_CHECK_LAUNCH();
}
}  // namespace

size_t tri_inverse_scratch_elems(int s) { return ((size_t)s / 2 + NB) * (size_t)s; }

void launch_tri_inverse(cudaStream_t st, const double* L, int s, double* Linv, double* scratch) {
  const int T = (s + NB - 1) / NB;
  KRR_CUDA(cudaMemsetAsync(Linv, 0, (size_t)s * s * sizeof(double), st));
  diag_inv_kernel<<<T, NB, 0, st>>>(L, s, Linv);
  KRR_CHECK_LAUNCH();
  if (T > 1) tri_inverse_rec(st, L, s, Linv, 0, s, scratch);
}

void launch_gemm_d(cudaStream_t st, int m, int n, int k, double alpha, const double* A, int lda,
                   int ta, const double* B, int ldb, int tb, double beta, double* C, int ldc) {
  dim3 g((n + GT - 1) / GT, (m + GT - 1) / GT);
  gemm_f64_kernel<<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
  KRR_CHECK_LAUNCH();
}

void launch_transpose_d(cudaStream_t st, const double* A, int s, double* B) {
  dim3 grid((s + 31) / 32, (s + 31) / 32), block(32, 8);
  transpose_d_kernel<<<grid, block, 0, st>>>(A, s, B);
  KRR_CHECK_LAUNCH();
}

void launch_form_u(cudaStream_t st, const double* Linv, const void* Zs, int bf16, int n, int s,
                   float* U) {
  dim3 grid((n + NB - 1) / NB, (s + NB - 1) / NB);
  if (bf16 == 2)
    form_u_kernel<2><<<grid, 256, 0, st>>>(Linv, Zs, n, s, U);
  else if (bf16)
    form_u_kernel<1><<<grid, 256, 0, st>>>(Linv, Zs, n, s, U);
  else
    form_u_kernel<0><<<grid, 256, 0, st>>>(Linv, Zs, n, s, U);
  KRR_CHECK_LAUNCH();
}


}  // namespace krr
