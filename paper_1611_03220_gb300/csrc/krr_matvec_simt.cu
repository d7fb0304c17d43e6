// SIMT kernel-matrix products Q = K(Xr, Xc) V + shift V.
//
// The Gaussian kernel of the paper's experiments (Section 5),
// k(x, z) = exp(-||x - z||^2 / (2 sigma^2)), is evaluated on the fly and
// never stored; Section 3.1 names this product the dominant per-iteration
// cost.  Two SIMT variants live here:
//   * FP64: squared distances summed from coordinate differences in FP64
//     (the definition, no cancellation), FP64 exp and accumulation.  It is
//     the parity path and the FP64 solver's product.
//   * FP32: the plain single-precision comparator.  Distances by the
//     expansion ||x||^2 + ||z||^2 - 2 x.z with a register-tiled FFMA
//     micro-kernel, expf, FP32 accumulation within a tile.
// Both split the column range over grid.y and reduce the per-split partial
// sums in a second, deterministic pass.
#include "krr_internal.cuh"

namespace krr {

namespace {

constexpr int M64_ROWS = 128;   // rows per CTA, one per thread
constexpr int M64_TJ = 32;      // columns per shared tile
constexpr int M64_DC = 16;      // coordinates per chunk

int choose_split(int row_blocks, int col_tiles) {
  int target = 4 * sm_count();
  int ns = (target + row_blocks - 1) / row_blocks;
  if (ns < 1) ns = 1;
  if (ns > col_tiles) ns = col_tiles;
  return ns;
}

// DS = 1 evaluates the derivative dK/dlog(sigma) = D o K instead of K, with
// D_ij = ||x_i - x_j||^2 / sigma^2 = -2 g ||x_i - x_j||^2 (g = -1 / (2 sigma^2)).
// DS = 2 evaluates the polynomial kernel (g x_i.x_j + pc)^pq of Section 6
// (g = gamma), the dot product accumulated in FP64.
template <int DS>
__global__ void __launch_bounds__(M64_ROWS)
mv_fp64_kernel(const float* __restrict__ Xr, int nr, int ldxr,
               const float* __restrict__ Xc, int nc, int ldxc, int d, double g,
               const double* __restrict__ V, int k, int ldv,
               double* __restrict__ part, int tiles_per_split, double pc = 0.0, int pq = 1) {
  __shared__ float xs[M64_TJ][M64_DC + 1];
  __shared__ double vs[M64_TJ][KRR_MAX_RHS];
  const int tid = threadIdx.x;
  const int i = blockIdx.x * M64_ROWS + tid;
  const bool row_ok = i < nr;
  double q[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) q[c] = 0.0;

  const int ntiles = (nc + M64_TJ - 1) / M64_TJ;
  const int t0 = blockIdx.y * tiles_per_split;
  const int t1 = min(ntiles, t0 + tiles_per_split);
  for (int tile = t0; tile < t1; ++tile) {
    const int j0 = tile * M64_TJ;
    double acc[M64_TJ];
#pragma unroll
    for (int jj = 0; jj < M64_TJ; ++jj) acc[jj] = 0.0;
    for (int c0 = 0; c0 < d; c0 += M64_DC) {
      __syncthreads();
      for (int e = tid; e < M64_TJ * M64_DC; e += M64_ROWS) {
        int jj = e / M64_DC, t = e % M64_DC;
        int j = j0 + jj, dd = c0 + t;
        xs[jj][t] = (j < nc && dd < d) ? Xc[(size_t)j * ldxc + dd] : 0.0f;
      }
      __syncthreads();
      float xi[M64_DC];
#pragma unroll
      for (int t = 0; t < M64_DC; ++t)
        xi[t] = (row_ok && c0 + t < d) ? Xr[(size_t)i * ldxr + c0 + t] : 0.0f;
#pragma unroll
      for (int jj = 0; jj < M64_TJ; ++jj) {
        double a = acc[jj];
#pragma unroll
        for (int t = 0; t < M64_DC; ++t) {
          if (DS == 2) {
            a = fma((double)xi[t], (double)xs[jj][t], a);
          } else {
            double df = (double)xi[t] - (double)xs[jj][t];
            a = fma(df, df, a);
          }
        }
        acc[jj] = a;
      }
    }
    __syncthreads();
    for (int e = tid; e < M64_TJ * k; e += M64_ROWS) {
      int jj = e / k, c = e % k;
      int j = j0 + jj;
      vs[jj][c] = (j < nc) ? V[(size_t)j * ldv + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < M64_TJ; ++jj) {
      double kv;
      if (DS == 2) {
        const double base = fma(g, acc[jj], pc);
        kv = base;
        for (int e = 1; e < pq; ++e) kv *= base;
      } else {
        kv = exp(g * acc[jj]);
        if (DS) kv *= -2.0 * g * acc[jj];
      }
#pragma unroll
      for (int c = 0; c < KRR_MAX_RHS; ++c)
        if (c < k) q[c] = fma(kv, vs[jj][c], q[c]);
    }
  }
  if (row_ok) {
    double* out = part + ((size_t)blockIdx.y * nr + i) * k;
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) out[c] = q[c];
  }
}

template <typename T, typename P>
__global__ void reduce_split_kernel(const P* __restrict__ part, int nsplit, int nr, int k,
                                    const T* __restrict__ V, int ldv, double shift,
                                    T* __restrict__ Q, int ldq) {
  const size_t total = (size_t)nr * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e % k);
    double s = 0.0;
    for (int y = 0; y < nsplit; ++y) s += (double)part[(size_t)y * total + e];
    if (shift != 0.0) s += shift * (double)V[(size_t)i * ldv + c];
    Q[(size_t)i * ldq + c] = (T)s;
  }
}

// ------------------------------------------------------------------ FP32 --
constexpr int M32_BM = 128, M32_BN = 128, M32_DC = 8;

__global__ void rownorm_f32_kernel(const float* __restrict__ X, int n, int ld, int d,
                                   float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int t = 0; t < d; ++t) {
    float v = X[(size_t)i * ld + t];
    s = fmaf(v, v, s);
  }
  out[i] = s;
}

__global__ void __launch_bounds__(256)
mv_fp32_kernel(const float* __restrict__ Xr, int nr, int ldxr,
               const float* __restrict__ Xc, int nc, int ldxc, int d, float g,
               const float* __restrict__ nrm_r, const float* __restrict__ nrm_c,
               int same, const float* __restrict__ V, int k, int ldv,
               float* __restrict__ part, int tiles_per_split) {
  __shared__ float As[M32_DC][M32_BM + 4];
  __shared__ float Bs[M32_DC][M32_BN + 4];
  __shared__ float vs[M32_BN][KRR_MAX_RHS + 1];
  __shared__ float racc[M32_BM][KRR_MAX_RHS + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * M32_BM;
  for (int e = tid; e < M32_BM * (KRR_MAX_RHS + 1); e += 256) (&racc[0][0])[e] = 0.f;
  float ni[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int i = i0 + ty + 16 * r;
    ni[r] = i < nr ? nrm_r[i] : 0.f;
  }
  const int ntiles = (nc + M32_BN - 1) / M32_BN;
  const int tt0 = blockIdx.y * tiles_per_split;
  const int tt1 = min(ntiles, tt0 + tiles_per_split);
  for (int tile = tt0; tile < tt1; ++tile) {
    const int j0 = tile * M32_BN;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    for (int c0 = 0; c0 < d; c0 += M32_DC) {
      __syncthreads();
      for (int e = tid; e < M32_BM * M32_DC; e += 256) {
        int rr = e / M32_DC, t = e % M32_DC;
        int i = i0 + rr, j = j0 + rr, dd = c0 + t;
        As[t][rr] = (i < nr && dd < d) ? Xr[(size_t)i * ldxr + dd] : 0.f;
        Bs[t][rr] = (j < nc && dd < d) ? Xc[(size_t)j * ldxc + dd] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < M32_DC; ++t) {
        float a[8], b[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r] = As[t][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 8; ++c) b[c] = Bs[t][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
      }
    }
    __syncthreads();
    for (int e = tid; e < M32_BN * k; e += 256) {
      int jj = e / k, c = e % k;
      int j = j0 + jj;
      vs[jj][c] = j < nc ? V[(size_t)j * ldv + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      int j = j0 + tx + 16 * c;
      float nj = j < nc ? nrm_c[j] : 0.f;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        int i = i0 + ty + 16 * r;
        float dist = fmaxf(ni[r] + nj - 2.f * acc[r][c], 0.f);
        float kv = expf(g * dist);
        if (same && i == j) kv = 1.f;
        acc[r][c] = kv;
      }
    }
    for (int cc = 0; cc < k; ++cc) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float p = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) p = fmaf(acc[r][c], vs[tx + 16 * c][cc], p);
        p += __shfl_xor_sync(0xffffffffu, p, 8);
        p += __shfl_xor_sync(0xffffffffu, p, 4);
        p += __shfl_xor_sync(0xffffffffu, p, 2);
        p += __shfl_xor_sync(0xffffffffu, p, 1);
        if (tx == 0) racc[ty + 16 * r][cc] += p;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < M32_BM * k; e += 256) {
    int rr = e / k, c = e % k;
    int i = i0 + rr;
    if (i < nr) part[((size_t)blockIdx.y * nr + i) * k + c] = racc[rr][c];
  }
}

}  // namespace

size_t mv_fp64_part_elems(int nr, int nc, int k) {
  int rb = (nr + M64_ROWS - 1) / M64_ROWS;
  int ct = (nc + M64_TJ - 1) / M64_TJ;
  return (size_t)choose_split(rb, ct) * nr * k;
}

void launch_mv_fp64(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                    int nc, int ldxc, int d, double sigma, double shift, const double* V,
                    int k, int ldv, double* Q, int ldq, double* part, int dsigma) {
  int rb = (nr + M64_ROWS - 1) / M64_ROWS;
  int ct = (nc + M64_TJ - 1) / M64_TJ;
  int ns = choose_split(rb, ct);
  int tps = (ct + ns - 1) / ns;
  ns = (ct + tps - 1) / tps;
  double g = -1.0 / (2.0 * sigma * sigma);
  if (dsigma)
    mv_fp64_kernel<1><<<dim3(rb, ns), M64_ROWS, 0, st>>>(Xr, nr, ldxr, Xc, nc, ldxc, d, g, V, k,
                                                          ldv, part, tps);
  else
    mv_fp64_kernel<0><<<dim3(rb, ns), M64_ROWS, 0, st>>>(Xr, nr, ldxr, Xc, nc, ldxc, d, g, V, k,
                                                          ldv, part, tps);
  KRR_CHECK_LAUNCH();
  int nb = (int)std::min<size_t>(((size_t)nr * k + 255) / 256, (size_t)8 * sm_count());
  reduce_split_kernel<double, double><<<nb, 256, 0, st>>>(part, ns, nr, k, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

// Q = P(Xr, Xc) V + shift V for the polynomial kernel (gamma x.z + c)^q in FP64.
void launch_mv_fp64_poly(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                         int nc, int ldxc, int d, double gamma, double c, int q, double shift,
                         const double* V, int k, int ldv, double* Q, int ldq, double* part) {
  int rb = (nr + M64_ROWS - 1) / M64_ROWS;
  int ct = (nc + M64_TJ - 1) / M64_TJ;
  int ns = choose_split(rb, ct);
  int tps = (ct + ns - 1) / ns;
  ns = (ct + tps - 1) / tps;
  mv_fp64_kernel<2><<<dim3(rb, ns), M64_ROWS, 0, st>>>(Xr, nr, ldxr, Xc, nc, ldxc, d, gamma, V,
                                                        k, ldv, part, tps, c, q);
  KRR_CHECK_LAUNCH();
  int nb = (int)std::min<size_t>(((size_t)nr * k + 255) / 256, (size_t)8 * sm_count());
  reduce_split_kernel<double, double><<<nb, 256, 0, st>>>(part, ns, nr, k, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

// Same product with the split count limited so the partial sums fit in a
// caller-provided scratch of `cap` doubles (nr * k <= cap is required).
void launch_mv_fp64_capped(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                           int nc, int ldxc, int d, double sigma, double shift, const double* V,
                           int k, int ldv, double* Q, int ldq, double* part, size_t cap) {
  int rb = (nr + M64_ROWS - 1) / M64_ROWS;
  int ct = (nc + M64_TJ - 1) / M64_TJ;
  int ns = choose_split(rb, ct);
  const size_t per = (size_t)nr * k;
  if (per == 0 || per > cap) throw Error{KRR_EINVAL, "product too large for the scratch"};
  if ((size_t)ns * per > cap) ns = (int)(cap / per);
  int tps = (ct + ns - 1) / ns;
  ns = (ct + tps - 1) / tps;
  double g = -1.0 / (2.0 * sigma * sigma);
  mv_fp64_kernel<0><<<dim3(rb, ns), M64_ROWS, 0, st>>>(Xr, nr, ldxr, Xc, nc, ldxc, d, g, V, k,
                                                        ldv, part, tps);
  KRR_CHECK_LAUNCH();
  int nb = (int)std::min<size_t>(((size_t)nr * k + 255) / 256, (size_t)8 * sm_count());
  reduce_split_kernel<double, double><<<nb, 256, 0, st>>>(part, ns, nr, k, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

size_t mv_fp32_part_elems(int nr, int nc, int k) {
  int rb = (nr + M32_BM - 1) / M32_BM;
  int ct = (nc + M32_BN - 1) / M32_BN;
  return (size_t)choose_split(rb, ct) * nr * k;
}

void launch_mv_fp32(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                    int nc, int ldxc, int d, double sigma, double shift, const float* V,
                    int k, int ldv, float* Q, int ldq, float* nrm_r, float* nrm_c,
                    float* part) {
  const bool same = (Xr == Xc) && (nr == nc) && (ldxr == ldxc);
  rownorm_f32_kernel<<<(nr + 255) / 256, 256, 0, st>>>(Xr, nr, ldxr, d, nrm_r);
  KRR_CHECK_LAUNCH();
  if (!same) {
    rownorm_f32_kernel<<<(nc + 255) / 256, 256, 0, st>>>(Xc, nc, ldxc, d, nrm_c);
    KRR_CHECK_LAUNCH();
  }
  int rb = (nr + M32_BM - 1) / M32_BM;
  int ct = (nc + M32_BN - 1) / M32_BN;
  int ns = choose_split(rb, ct);
  int tps = (ct + ns - 1) / ns;
  ns = (ct + tps - 1) / tps;
  float g = (float)(-1.0 / (2.0 * sigma * sigma));
  mv_fp32_kernel<<<dim3(rb, ns), 256, 0, st>>>(Xr, nr, ldxr, Xc, nc, ldxc, d, g, nrm_r,
                                                same ? nrm_r : nrm_c, same ? 1 : 0, V, k, ldv,
                                                part, tps);
  KRR_CHECK_LAUNCH();
  int nb = (int)std::min<size_t>(((size_t)nr * k + 255) / 256, (size_t)8 * sm_count());
  reduce_split_kernel<float, float><<<nb, 256, 0, st>>>(part, ns, nr, k, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
