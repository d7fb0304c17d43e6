// Conjugate-gradient vector kernels (the PCG step of Algorithm 1: PCG on
// (K + lambda I) c = y with the random-feature preconditioner).
//
// Each column of the n x k block iterates independently (Section 5 asks the
// stopping test to hold for every right-hand side): per column the scalars
// alpha = r.z / p.q and beta = r'.z' / r.z, the recursive ||r||^2 and the
// active flag live in a CgScalars block in device memory, so the loop never
// reads anything back to the host.  Every reduction is a grid-wide column
// sum: warp shuffles, one partial per CTA, and the last CTA to finish
// (atomic counter) adds the partials in CTA order, which keeps the result
// deterministic, and then updates the scalars.
#include <algorithm>

#include "krr_cgstep.cuh"

namespace krr {
namespace {

constexpr int CT = 256;           // threads per CTA
constexpr int NW = CT / 32;

constexpr int C_INIT = CGC_INIT, C_RZ = CGC_RZ, C_ALPHA = CGC_ALPHA, C_XR = CGC_XR,
              C_NORM = CGC_NORM;

int cg_blocks(int n) {
  int b = (n + CT - 1) / CT;
  int cap = 2 * sm_count();
  return b < 1 ? 1 : (b > cap ? cap : b);
}

__device__ __forceinline__ bool grid_colsum(double (&v)[KRR_MAX_RHS], int k, double* part,
                                            unsigned int* counter, double (&tot)[KRR_MAX_RHS]) {
  return grid_colsum_nt<CT>(v, k, part, counter, blockIdx.x, gridDim.x, tot);
}

__device__ __forceinline__ bool bad(double x) { return cg_bad(x); }

template <typename T>
__global__ void __launch_bounds__(CT)
cg_init_kernel(CgScalars* sc, const double* __restrict__ Y, int ldy, const T* __restrict__ R,
               int n, int k, double tol, int max_iter, double* part, double* hist,
               int hist_cap) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        double y = Y[(size_t)i * ldy + c];
        v[c] = fma(y, y, v[c]);
      }
  }
  if (!grid_colsum(v, k, part, &sc->counter[C_INIT], tot)) return;
  // second pass for ||r0||^2 runs in cg_rz_first; here rr = ||y||^2 as a start
  sc->k = k;
  sc->iter = 0;
  sc->max_iter = max_iter;
  sc->flags = 0;
  sc->hist = hist;
  sc->hist_cap = hist ? hist_cap : 0;
  int any = 0;
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    if (c < k) {
      sc->yy[c] = tot[c];
      sc->tol2[c] = tol * tol * tot[c];
      sc->rr[c] = tot[c];
      sc->active[c] = tot[c] > 0.0 ? 1 : 0;
      any |= sc->active[c];
      if (bad(tot[c])) sc->flags |= FLAG_NAN;
    } else {
      sc->yy[c] = 0.0;
      sc->tol2[c] = 0.0;
      sc->rr[c] = 0.0;
      sc->active[c] = 0;
    }
    sc->iters[c] = 0;
    sc->rz_keep[c] = sc->rz[c];
    sc->alpha[c] = sc->beta[c] = sc->rz[c] = sc->pq[c] = 0.0;
  }
  sc->run = (any && max_iter > 0 && !(sc->flags & FLAG_NAN)) ? 1 : 0;
}

// rz = r.z, rr = r.r and p = z for the first iteration.
template <typename T>
__global__ void __launch_bounds__(CT)
cg_rz_first_kernel(CgScalars* sc, const T* __restrict__ R, const T* __restrict__ Z,
                   T* __restrict__ P, int n, int k, double* part) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
  double w[KRR_MAX_RHS], tot2[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = w[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        size_t e = (size_t)i * k + c;
        double r = (double)R[e], z = (double)Z[e];
        v[c] = fma(r, z, v[c]);
        w[c] = fma(r, r, w[c]);
        P[e] = Z[e];
      }
  }
  // two column sums packed into one: first k entries r.z, next k entries r.r
  double vv[KRR_MAX_RHS];
  const int k2 = 2 * k <= KRR_MAX_RHS ? 2 * k : 0;
  if (k2) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c) vv[c] = c < k ? v[c] : (c < k2 ? w[c - k] : 0.0);
    if (!grid_colsum(vv, k2, part, &sc->counter[C_RZ], tot)) return;
    for (int c = 0; c < k; ++c) tot2[c] = tot[k + c];
  } else {
    // k > KRR_MAX_RHS / 2: use r.z only; rr keeps its ||y||^2 start value
    if (!grid_colsum(v, k, part, &sc->counter[C_RZ], tot)) return;
    for (int c = 0; c < k; ++c) tot2[c] = sc->rr[c];
  }
  for (int c = 0; c < k; ++c) {
    sc->rz[c] = tot[c];
    sc->rr[c] = tot2[c];
    if (bad(tot[c])) sc->flags |= FLAG_NAN;
    if (sc->active[c]) {
      if (tot2[c] <= sc->tol2[c]) {
        sc->active[c] = 0;  // x0 already meets the tolerance
      } else if (!(tot[c] > 0.0)) {
        sc->flags |= FLAG_BREAKDOWN;
        sc->active[c] = 0;
      }
    }
  }
}

// Restart with the previous direction kept: sums r.z, r.r and r.P (P in the
// previous units), then per column the coefficients of p = a_z z + a_p P,
// stored in alpha (a_z) and beta (a_p) until the first iteration overwrites
// them.  With P' = s P and beta = r.z / (s^2 rz_keep):
//   p = z + beta (P' - (r.P' / r.z) z),  so  r.p = r.z  exactly.
template <typename T>
__global__ void __launch_bounds__(CT)
cg_restart_kernel(CgScalars* sc, const T* __restrict__ R, const T* __restrict__ Z,
                  const T* __restrict__ P, int n, int k, ColScale s, double* part) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
    for (int c = 0; c < k; ++c) {
      const size_t e = (size_t)i * k + c;
      const double r = (double)R[e];
      v[c] = fma(r, (double)Z[e], v[c]);
      v[k + c] = fma(r, r, v[k + c]);
      v[2 * k + c] = fma(r, (double)P[e], v[2 * k + c]);
    }
  }
  if (!grid_colsum(v, 3 * k, part, &sc->counter[C_RZ], tot)) return;
  for (int c = 0; c < k; ++c) {
    const double rz = tot[c], rr = tot[k + c], rp = s.v[c] * tot[2 * k + c];
    const double rzk = s.v[c] * s.v[c] * sc->rz_keep[c];
    sc->rz[c] = rz;
    sc->rr[c] = rr;
    double az = 1.0, ap = 0.0;
    if (bad(rz) || bad(rr)) sc->flags |= FLAG_NAN;
    if (sc->active[c]) {
      if (rr <= sc->tol2[c]) {
        sc->active[c] = 0;
      } else if (!(rz > 0.0)) {
        sc->flags |= FLAG_BREAKDOWN;
        sc->active[c] = 0;
      } else if (rzk > 0.0 && !bad(rzk) && !bad(rp)) {
        const double beta = rz / rzk;
        az = 1.0 - beta * rp / rz;
        ap = beta * s.v[c];
      }
    }
    sc->alpha[c] = az;
    sc->beta[c] = ap;
  }
}

template <typename T>
__global__ void __launch_bounds__(CT)
cg_restart_p_kernel(const CgScalars* sc, T* __restrict__ P, const T* __restrict__ Z, int n,
                    int k) {
  double az[KRR_MAX_RHS], ap[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    az[c] = c < k ? sc->alpha[c] : 0.0;
    ap[c] = c < k ? sc->beta[c] : 0.0;
  }
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        const size_t e = (size_t)i * k + c;
        P[e] = (T)(az[c] * (double)Z[e] + ap[c] * (double)P[e]);
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(CT)
cg_alpha_kernel(CgScalars* sc, const T* __restrict__ P, const T* __restrict__ Q, int n, int k,
                double* part) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        size_t e = (size_t)i * k + c;
        v[c] = fma((double)P[e], (double)Q[e], v[c]);
      }
  }
  if (!grid_colsum(v, k, part, &sc->counter[C_ALPHA], tot)) return;
  cg_alpha_finish(sc, tot, k);
}

template <typename T>
__global__ void __launch_bounds__(CT)
cg_update_xr_kernel(CgScalars* sc, T* __restrict__ X, T* __restrict__ R, const T* __restrict__ P,
                    const T* __restrict__ Q, int n, int k, double* part) {
  double a[KRR_MAX_RHS], v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    a[c] = c < k ? sc->alpha[c] : 0.0;
    v[c] = 0.0;
  }
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        size_t e = (size_t)i * k + c;
        double r = (double)R[e];
        if (a[c] != 0.0) {
          X[e] = (T)((double)X[e] + a[c] * (double)P[e]);
          r = r - a[c] * (double)Q[e];
          R[e] = (T)r;
          r = (double)R[e];
        }
        v[c] = fma(r, r, v[c]);
      }
  }
  if (!grid_colsum(v, k, part, &sc->counter[C_XR], tot)) return;
  cg_xr_finish(sc, tot, k);
}

template <typename T>
__global__ void __launch_bounds__(CT)
cg_rz_kernel(CgScalars* sc, const T* __restrict__ R, const T* __restrict__ Z, int n, int k,
             double* part) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        size_t e = (size_t)i * k + c;
        v[c] = fma((double)R[e], (double)Z[e], v[c]);
      }
  }
  if (!grid_colsum(v, k, part, &sc->counter[C_RZ], tot)) return;
  cg_rz_finish(sc, tot, k);
}

template <typename T>
__global__ void __launch_bounds__(CT)
cg_update_p_kernel(const CgScalars* sc, T* __restrict__ P, const T* __restrict__ Z, int n, int k) {
  double b[KRR_MAX_RHS];
  int act[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    b[c] = c < k ? sc->beta[c] : 0.0;
    act[c] = c < k ? sc->active[c] : 0;
  }
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k && act[c]) {
        size_t e = (size_t)i * k + c;
        P[e] = (T)((double)Z[e] + b[c] * (double)P[e]);
      }
  }
}

// The tensor-core product's chunk sums finished and p.q reduced in the same
// pass: q_i = ra_i sum_ch part[ch, i] + shift p_i (FP64 sum over the chunks,
// rounded to T), then alpha = r.z / p.q as in cg_alpha_kernel.
template <typename T>
__global__ void __launch_bounds__(CT)
cg_reduce_alpha_kernel(CgScalars* sc, const float* __restrict__ part, int nchunk, int n_rpad,
                       int kv, const float* __restrict__ ra, double shift,
                       const T* __restrict__ P, T* __restrict__ Q, int n, int k, double* cpart) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
    const double rai = (double)ra[i];
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        double s = 0.0;
        for (int ch = 0; ch < nchunk; ++ch) s += (double)part[((size_t)ch * n_rpad + i) * kv + c];
        s *= rai;
        const size_t e = (size_t)i * k + c;
        const double p = (double)P[e];
        if (shift != 0.0) s += shift * p;
        const T q = (T)s;
        Q[e] = q;
        v[c] = fma(p, (double)q, v[c]);
      }
  }
  if (!grid_colsum(v, k, cpart, &sc->counter[C_ALPHA], tot)) return;
  cg_alpha_finish(sc, tot, k);
}

// p = z + beta p for the active columns (update != 0), then the product's
// weights w[j, c] = ra_j p[j, c] over the padded n_pad x kv block (zero for
// rows >= n and columns >= k), as the product's own weight kernel forms them.
template <typename T>
__global__ void __launch_bounds__(CT)
cg_update_pw_kernel(const CgScalars* sc, T* __restrict__ P, const T* __restrict__ Z, int n, int k,
                    int update, const float* __restrict__ ra, int n_pad, int kv,
                    float* __restrict__ w) {
  double b[KRR_MAX_RHS];
  int act[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    b[c] = c < k ? sc->beta[c] : 0.0;
    act[c] = (update && c < k) ? sc->active[c] : 0;
  }
  for (int i = blockIdx.x * CT + threadIdx.x; i < n_pad; i += gridDim.x * CT) {
    const float rai = i < n ? ra[i] : 0.f;
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c) {
      if (c >= kv) break;
      float wv = 0.f;
      if (i < n && c < k) {
        const size_t e = (size_t)i * k + c;
        T p = P[e];
        if (act[c]) {
          p = (T)((double)Z[e] + b[c] * (double)p);
          P[e] = p;
        }
        wv = rai * (float)p;
      }
      w[(size_t)i * kv + c] = wv;
    }
  }
}

__global__ void cg_tail_kernel(CgScalars* sc, cudaGraphConditionalHandle cond) {
  cg_tail_finish(sc, cond);
}

__global__ void batch_gate_kernel(CgScalars* const* scs, const unsigned long long* conds,
                                  int nsolve) {
  for (int i = threadIdx.x; i < nsolve; i += blockDim.x)
    cudaGraphSetConditional((cudaGraphConditionalHandle)conds[i], scs[i]->run ? 1u : 0u);
}

__global__ void batch_tail_kernel(CgScalars* const* scs, int nsolve,
                                  cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int i = 0; i < nsolve; ++i) any |= scs[i]->run;
  cudaGraphSetConditional(cond, any ? 1u : 0u);
}

// ------------------------------------------------------------ elementwise --
template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ a, int n, int k, int lda, B* __restrict__ b,
                               int ldb, ColScale sc) {
  const size_t total = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / k), c = (int)(e % k);
    b[(size_t)i * ldb + c] = (B)((double)a[(size_t)i * lda + c] * sc.v[c]);
  }
}

template <typename D>
__global__ void axpy_d_kernel(const D* __restrict__ dl, int n, int k, int ldd, double* __restrict__ c,
                              int ldc, ColScale sc) {
  const size_t total = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / k), q = (int)(e % k);
    c[(size_t)i * ldc + q] += sc.v[q] * (double)dl[(size_t)i * ldd + q];
  }
}

__global__ void sub_d_kernel(const double* __restrict__ y, int ldy, const double* __restrict__ a,
                             int lda, int n, int k, double* __restrict__ r, int ldr) {
  const size_t total = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e / k), c = (int)(e % k);
    r[(size_t)i * ldr + c] = y[(size_t)i * ldy + c] - a[(size_t)i * lda + c];
  }
}

template <typename T>
__global__ void __launch_bounds__(CT)
colnorm2_kernel(const T* __restrict__ a, int n, int k, int lda, double* out, double* part,
                unsigned int* counter) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) {
        double x = (double)a[(size_t)i * lda + c];
        v[c] = fma(x, x, v[c]);
      }
  }
  if (!grid_colsum(v, k, part, counter, tot)) return;
  for (int c = 0; c < k; ++c) out[c] = tot[c];
}

// out[0] = sum_{i,c} a[i, c] b[i, c], one grid-wide FP64 sum.
__global__ void __launch_bounds__(CT)
dot_d_kernel(const double* __restrict__ a, int lda, const double* __restrict__ b, int ldb, int n,
             int k, double* out, double* part, unsigned int* counter) {
  double v[KRR_MAX_RHS], tot[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) v[c] = 0.0;
  for (int i = blockIdx.x * CT + threadIdx.x; i < n; i += gridDim.x * CT) {
    double s = 0.0;
    for (int c = 0; c < k; ++c) s = fma(a[(size_t)i * lda + c], b[(size_t)i * ldb + c], s);
    v[0] += s;
  }
  if (!grid_colsum(v, 1, part, counter, tot)) return;
  out[0] = tot[0];
}

// Column mean in two deterministic passes: per-slab column sums, then the
// slabs added in order.
constexpr int MEAN_ROWS = 128;

__global__ void colsum_slab_kernel(const float* __restrict__ X, int n, int ld, int d,
                                   double* __restrict__ part) {
  const int r0 = blockIdx.x * MEAN_ROWS, r1 = min(n, r0 + MEAN_ROWS);
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    double s = 0.0;
    for (int i = r0; i < r1; ++i) s += (double)X[(size_t)i * ld + t];
    part[(size_t)blockIdx.x * d + t] = s;
  }
}

__global__ void colmean_finish_kernel(const double* __restrict__ part, int nslab, int n, int d,
                                      double* __restrict__ mu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d) return;
  double s = 0.0;
  for (int b = 0; b < nslab; ++b) s += part[(size_t)b * d + t];
  mu[t] = s / (double)n;
}

int ew_blocks(size_t total) {
  size_t b = (total + 255) / 256;
  size_t cap = (size_t)8 * sm_count();
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

size_t cg_part_elems(int n, int k) {
  (void)k;
  // also the partials of the fused reductions, whose kernels run up to two
  // CTAs per SM whatever n is
  return (size_t)std::max(cg_blocks(n), 2 * sm_count()) * KRR_MAX_RHS;
}

template <typename T>
void launch_cg_init(cudaStream_t st, CgScalars* sc, const double* Y, int ldy, const T* R, int n,
                    int k, double tol, int max_iter, double* part, double* hist, int hist_cap) {
  (void)R;
  cg_init_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, Y, ldy, R, n, k, tol, max_iter, part, hist,
                                                 hist_cap);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_rz_first(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, T* P, int n,
                        int k, double* part) {
  cg_rz_first_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, R, Z, P, n, k, part);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_restart(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, T* P, int n,
                       int k, const ColScale& s, double* part) {
  if (3 * k > KRR_MAX_RHS)
    throw Error{KRR_EINVAL, "cg_restart: needs 3 k <= KRR_MAX_RHS"};
  cg_restart_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, R, Z, P, n, k, s, part);
  KRR_CHECK_LAUNCH();
  cg_restart_p_kernel<T><<<ew_blocks((size_t)n), CT, 0, st>>>(sc, P, Z, n, k);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_alpha(cudaStream_t st, CgScalars* sc, const T* P, const T* Q, int n, int k,
                     double* part) {
  cg_alpha_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, P, Q, n, k, part);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_update_xr(cudaStream_t st, CgScalars* sc, T* X, T* R, const T* P, const T* Q,
                         int n, int k, double* part) {
  cg_update_xr_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, X, R, P, Q, n, k, part);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_rz(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, int n, int k,
                  double* part) {
  cg_rz_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, R, Z, n, k, part);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_update_p(cudaStream_t st, CgScalars* sc, T* P, const T* Z, int n, int k) {
  cg_update_p_kernel<T><<<ew_blocks((size_t)n), CT, 0, st>>>(sc, P, Z, n, k);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_reduce_alpha(cudaStream_t st, CgScalars* sc, const float* part, int nchunk,
                            int n_rpad, int kv, const float* ra, double shift, const T* P, T* Q,
                            int n, int k, double* cpart) {
  cg_reduce_alpha_kernel<T><<<cg_blocks(n), CT, 0, st>>>(sc, part, nchunk, n_rpad, kv, ra, shift,
                                                        P, Q, n, k, cpart);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_cg_update_pw(cudaStream_t st, CgScalars* sc, T* P, const T* Z, int n, int k,
                         int update, const float* ra, int n_pad, int kv, float* w) {
  cg_update_pw_kernel<T><<<ew_blocks((size_t)n_pad), CT, 0, st>>>(sc, P, Z, n, k, update, ra,
                                                                  n_pad, kv, w);
  KRR_CHECK_LAUNCH();
}

template void launch_cg_reduce_alpha<float>(cudaStream_t, CgScalars*, const float*, int, int,
                                            int, const float*, double, const float*, float*,
                                            int, int, double*);
template void launch_cg_update_pw<float>(cudaStream_t, CgScalars*, float*, const float*, int,
                                         int, int, const float*, int, int, float*);

void launch_cg_tail(cudaStream_t st, CgScalars* sc, unsigned long long cond) {
  cg_tail_kernel<<<1, 1, 0, st>>>(sc, (cudaGraphConditionalHandle)cond);
  KRR_CHECK_LAUNCH();
}

void launch_batch_gate(cudaStream_t st, CgScalars* const* scs, const unsigned long long* conds,
                       int nsolve) {
  batch_gate_kernel<<<1, 128, 0, st>>>(scs, conds, nsolve);
  KRR_CHECK_LAUNCH();
}

void launch_batch_tail(cudaStream_t st, CgScalars* const* scs, int nsolve,
                       unsigned long long cond) {
  batch_tail_kernel<<<1, 1, 0, st>>>(scs, nsolve, (cudaGraphConditionalHandle)cond);
  KRR_CHECK_LAUNCH();
}

void launch_dot_d(cudaStream_t st, const double* a, int lda, const double* b, int ldb, int n,
                  int k, double* out, double* part, unsigned int* counter) {
  dot_d_kernel<<<cg_blocks(n), CT, 0, st>>>(a, lda, b, ldb, n, k, out, part, counter);
  KRR_CHECK_LAUNCH();
}

void launch_colmean(cudaStream_t st, const float* X, int n, int ld, int d, double* mu,
                    double* slab) {
  const int nslab = (n + MEAN_ROWS - 1) / MEAN_ROWS;
  colsum_slab_kernel<<<nslab, 128, 0, st>>>(X, n, ld, d, slab);
  KRR_CHECK_LAUNCH();
  colmean_finish_kernel<<<(d + 127) / 128, 128, 0, st>>>(slab, nslab, n, d, mu);
  KRR_CHECK_LAUNCH();
}

template <typename A, typename B>
void launch_convert(cudaStream_t st, const A* a, int n, int k, int lda, B* b, int ldb,
                    const ColScale& scale) {
  convert_kernel<A, B><<<ew_blocks((size_t)n * k), 256, 0, st>>>(a, n, k, lda, b, ldb, scale);
  KRR_CHECK_LAUNCH();
}

template <typename D>
void launch_axpy_d(cudaStream_t st, const D* dl, int n, int k, int ldd, double* c, int ldc,
                   const ColScale& scale) {
  axpy_d_kernel<D><<<ew_blocks((size_t)n * k), 256, 0, st>>>(dl, n, k, ldd, c, ldc, scale);
  KRR_CHECK_LAUNCH();
}

void launch_sub_d(cudaStream_t st, const double* y, int ldy, const double* a, int lda, int n,
                  int k, double* r, int ldr) {
  sub_d_kernel<<<ew_blocks((size_t)n * k), 256, 0, st>>>(y, ldy, a, lda, n, k, r, ldr);
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_colnorm2(cudaStream_t st, const T* a, int n, int k, int lda, double* out,
                     double* part, unsigned int* counter) {
  colnorm2_kernel<T><<<cg_blocks(n), CT, 0, st>>>(a, n, k, lda, out, part, counter);
  KRR_CHECK_LAUNCH();
}

#define KRR_CG_INST(T)                                                                        \
  template void launch_cg_init<T>(cudaStream_t, CgScalars*, const double*, int, const T*, int, \
                                  int, double, int, double*, double*, int);                   \
  template void launch_cg_rz_first<T>(cudaStream_t, CgScalars*, const T*, const T*, T*, int,  \
                                      int, double*);                                          \
  template void launch_cg_restart<T>(cudaStream_t, CgScalars*, const T*, const T*, T*, int,   \
                                     int, const ColScale&, double*);                          \
  template void launch_cg_alpha<T>(cudaStream_t, CgScalars*, const T*, const T*, int, int,     \
                                   double*);                                                  \
  template void launch_cg_update_xr<T>(cudaStream_t, CgScalars*, T*, T*, const T*, const T*,   \
                                       int, int, double*);                                    \
  template void launch_cg_rz<T>(cudaStream_t, CgScalars*, const T*, const T*, int, int,        \
                                double*);                                                     \
  template void launch_cg_update_p<T>(cudaStream_t, CgScalars*, T*, const T*, int, int);       \
  template void launch_colnorm2<T>(cudaStream_t, const T*, int, int, int, double*, double*,    \
                                   unsigned int*);                                            \
  template void launch_axpy_d<T>(cudaStream_t, const T*, int, int, int, double*, int,          \
                                 const ColScale&);
KRR_CG_INST(float)
KRR_CG_INST(double)
template void launch_convert<double, float>(cudaStream_t, const double*, int, int, int, float*,
                                            int, const ColScale&);
template void launch_convert<float, double>(cudaStream_t, const float*, int, int, int, double*,
                                            int, const ColScale&);
template void launch_convert<double, double>(cudaStream_t, const double*, int, int, int,
                                             double*, int, const ColScale&);

}  // namespace krr
