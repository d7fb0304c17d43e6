// Device-side pieces of one PCG iteration (Algorithm 1) shared by the CG
// vector kernels and the kernels that fuse a CG step into their own pass
// (the chunk sums of the product, the two streamed GEMVs of the apply).
//
// grid_colsum_nt: a deterministic grid-wide column sum.  Each CTA reduces its
// per-thread values (warp shuffles, then a fixed order over warps), writes one
// partial per column, and the last CTA to arrive (atomic counter) adds the
// partials in CTA order with a fixed tree.  The "*_finish" functions are the
// scalar updates the last CTA's thread 0 then makes.
#pragma once

#include "krr_internal.cuh"

namespace krr {

// Sums v[c] (c < k) over `ncta` participating CTAs, this one being `cta`.
// True in thread 0 of the last CTA, with tot[c] the totals.  Every thread of a
// participating CTA must call it; part holds ncta x KRR_MAX_RHS doubles.
template <int NT>
__device__ bool grid_colsum_nt(double (&v)[KRR_MAX_RHS], int k, double* part,
                               unsigned int* counter, int cta, int ncta,
                               double (&tot)[KRR_MAX_RHS]) {
  constexpr int NW = NT / 32;
  __shared__ double red[NW][KRR_MAX_RHS];
  __shared__ int last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    if (c >= k) break;
    double x = v[c];
    for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][c] = x;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int q = 0; q < NW; ++q) s += red[q][threadIdx.x];
    part[cta * KRR_MAX_RHS + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)ncta - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double loc[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) loc[c] = 0.0;
  for (int b = threadIdx.x; b < ncta; b += NT) {
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) loc[c] += __ldcg(&part[b * KRR_MAX_RHS + c]);
  }
  __syncthreads();  // red is reused
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    if (c >= k) break;
    double x = loc[c];
    for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][c] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  for (int c = 0; c < k; ++c) {
    double t = 0.0;
    for (int q = 0; q < NW; ++q) t += red[q][c];
    tot[c] = t;
  }
  *counter = 0u;
  return true;
}

__device__ __forceinline__ bool cg_bad(double x) { return isnan(x) || isinf(x); }

// alpha = r.z / p.q per active column (tot = p.q).
__device__ inline void cg_alpha_finish(CgScalars* sc, const double (&tot)[KRR_MAX_RHS], int k) {
  for (int c = 0; c < k; ++c) {
    sc->pq[c] = tot[c];
    double a = 0.0;
    if (sc->active[c]) {
      if (cg_bad(tot[c])) {
        sc->flags |= FLAG_NAN;
      } else if (!(tot[c] > 0.0)) {
        sc->flags |= FLAG_BREAKDOWN;
      } else {
        a = sc->rz[c] / tot[c];
      }
    }
    sc->alpha[c] = a;
    if (sc->iter < sc->hist_cap) sc->hist[((size_t)sc->iter * 2) * KRR_MAX_RHS + c] = a;
  }
}

// ||r||^2 after the x, r update (tot = r.r); a column whose residual meets
// its tolerance stops.
__device__ inline void cg_xr_finish(CgScalars* sc, const double (&tot)[KRR_MAX_RHS], int k) {
  for (int c = 0; c < k; ++c) {
    sc->rr[c] = tot[c];
    if (cg_bad(tot[c])) sc->flags |= FLAG_NAN;
    if (sc->active[c]) {
      sc->iters[c] += 1;
      if (tot[c] <= sc->tol2[c]) sc->active[c] = 0;
    }
  }
}

// beta = r'.z' / r.z per active column (tot = r'.z').
__device__ inline void cg_rz_finish(CgScalars* sc, const double (&tot)[KRR_MAX_RHS], int k) {
  for (int c = 0; c < k; ++c) {
    double b = 0.0;
    if (sc->active[c]) {
      if (cg_bad(tot[c])) {
        sc->flags |= FLAG_NAN;
      } else if (!(tot[c] > 0.0)) {
        sc->flags |= FLAG_BREAKDOWN;
      } else {
        b = tot[c] / sc->rz[c];
      }
      sc->rz[c] = tot[c];
    }
    sc->beta[c] = b;
    if (sc->iter < sc->hist_cap) sc->hist[((size_t)sc->iter * 2 + 1) * KRR_MAX_RHS + c] = b;
  }
}

// iter += 1 and the continue decision; sets the graph's WHILE condition when
// `cond` is nonzero.
__device__ inline void cg_tail_finish(CgScalars* sc, cudaGraphConditionalHandle cond) {
  int any = 0;
  for (int c = 0; c < sc->k; ++c) any |= sc->active[c];
  sc->iter += 1;
  bool stop = !any || (sc->flags & (FLAG_BREAKDOWN | FLAG_NAN));
  if (!stop && sc->iter >= sc->max_iter) {
    sc->flags |= FLAG_CAP;
    stop = true;
  }
  sc->run = stop ? 0 : 1;
  if (cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// Counter slots of CgScalars::counter used by the reductions.
enum CgCounter : int { CGC_INIT = 0, CGC_RZ = 1, CGC_ALPHA = 2, CGC_XR = 3, CGC_NORM = 4 };

}  // namespace krr
