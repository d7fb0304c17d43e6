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

template <int BF16>
__device__ __forceinline__ float zload(const void* Zs, size_t idx) {
  if (BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Zs)[idx]);
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

// Off-diagonal block (I, J), J < I:
//   Linv[I, J] = -D_II * sum_{q = J*NB}^{I*NB-1} L[I, q] Linv[q, J].
// Launched once per block row I (blocks J = 0..I-1 in parallel) because
// block row I reads every earlier block row.
__global__ void __launch_bounds__(256)
offdiag_inv_kernel(const double* L, int s, int I, double* Linv) {
  extern __shared__ double sm[];
  double* Sacc = sm;                    // NB x (NB+1): the sum
  double* Dt = sm + NB * (NB + 1);      // NB x (NB+1): D_II
  __shared__ double Pa[16][NB + 1];
  __shared__ double Pb[16][NB + 1];
  const int J = blockIdx.x;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int oI = I * NB, nI = min(NB, s - oI);
  const int oJ = J * NB;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int q0 = oJ; q0 < oI; q0 += 16) {
    __syncthreads();
    for (int e = tid; e < 16 * NB; e += 256) {
      int row = e / 16, t = e % 16;
      int q = q0 + t;
      Pa[t][row] = (row < nI && q < oI) ? L[(size_t)(oI + row) * s + q] : 0.0;
    }
    for (int e = tid; e < 16 * NB; e += 256) {
      int t = e / NB, col = e % NB;
      int q = q0 + t;
      Pb[t][col] = (q < oI) ? Linv[(size_t)q * s + oJ + col] : 0.0;
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
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) Sacc[(ty + 16 * r) * (NB + 1) + tx + 16 * c] = acc[r][c];
  for (int e = tid; e < NB * NB; e += 256) {
    int i = e / NB, j = e % NB;
    Dt[i * (NB + 1) + j] = (i < nI && j < nI) ? Linv[(size_t)(oI + i) * s + oI + j] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < nI * NB; e += 256) {
    int i = e / NB, j = e % NB;
    double v = 0.0;
    for (int m = 0; m <= i; ++m) v = fma(Dt[i * (NB + 1) + m], Sacc[m * (NB + 1) + j], v);
    Linv[(size_t)(oI + i) * s + oJ + j] = -v;
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

void launch_tri_inverse(cudaStream_t st, const double* L, int s, double* Linv) {
  const int T = (s + NB - 1) / NB;
  KRR_CUDA(cudaMemsetAsync(Linv, 0, (size_t)s * s * sizeof(double), st));
  diag_inv_kernel<<<T, NB, 0, st>>>(L, s, Linv);
  KRR_CHECK_LAUNCH();
  const size_t smem = 2 * NB * (NB + 1) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    KRR_CUDA(cudaFuncSetAttribute(offdiag_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr_set = true;
  }
  for (int I = 1; I < T; ++I) {
    offdiag_inv_kernel<<<I, 256, smem, st>>>(L, s, I, Linv);
    KRR_CHECK_LAUNCH();
  }
}

void launch_transpose_d(cudaStream_t st, const double* A, int s, double* B) {
  dim3 grid((s + 31) / 32, (s + 31) / 32), block(32, 8);
  transpose_d_kernel<<<grid, block, 0, st>>>(A, s, B);
  KRR_CHECK_LAUNCH();
}

void launch_form_u(cudaStream_t st, const double* Linv, const void* Zs, int bf16, int n, int s,
                   float* U) {
  dim3 grid((n + NB - 1) / NB, (s + NB - 1) / NB);
  if (bf16)
    form_u_kernel<1><<<grid, 256, 0, st>>>(Linv, Zs, n, s, U);
  else
    form_u_kernel<0><<<grid, 256, 0, st>>>(Linv, Zs, n, s, U);
  KRR_CHECK_LAUNCH();
}


}  // namespace krr
