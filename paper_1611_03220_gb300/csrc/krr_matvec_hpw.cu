// High-precision kernel-matrix products for any dimension, on the FP32 pipes:
//   DS = 0:  Q = K(Xr, Xc) V + shift V
//   DS = 1:  Q = (D o K)(Xr, Xc) V,  D_ij = ||xr_i - xc_j||^2 / sigma^2
// with V and Q in FP64 and each K_ij to about 1e-13 relative (the Gaussian
// kernel of Section 5; the product is the per-iteration cost named in
// Section 3.1).  It serves the refinement residual when d > 64 (the tensor-
// core digit product needs d <= 64), products with distinct row and column
// sets (prediction) and the derivative products of the hyper-parameter
// gradient.
//
// Squared distances come from the norm expansion of the FP32 inputs in
// float-float arithmetic: each product a b is split exactly into fl(a b) and
// fma(a, b, -fl(a b)) and summed with two-sum, ||x||^2 is accumulated in FP64
// and split into two floats, and d2 = n_i + n_j - 2 x_i.x_j keeps about
// 2^-48 (n_i + n_j) absolute error.  exp2 (krr_ff.cuh) and the contraction
// with V (split into two floats) are float-float.
//
// Tiling: a CTA owns 64 rows and a chunk of 64-column tiles.  Its 256
// threads compute 4 x 4 pairs each from 16-coordinate slabs in shared
// memory; each finished 64 x 64 kernel block passes through shared memory to
// the row-sum stage, where threads own (row, right-hand side) pairs.  Partial
// sums per chunk are written in FP64 and added in chunk order by a second
// kernel.
#include <cmath>

#include "krr_ff.cuh"
#include "krr_internal.cuh"

namespace krr {
namespace {

using ff::exp2_ff;
using ff::NTAB;
using ff::two_sum;

constexpr int TM = 64;        // rows per CTA
constexpr int TN = 64;        // columns per tile
constexpr int TK = 16;        // coordinates per slab
constexpr int HT = 256;       // threads
constexpr int SP = TM + 4;    // padded slab row
constexpr int KP = TN + 1;    // padded kernel-block row

struct HpwParams {
  const float* Xr;
  const float* Xc;
  int nr, nc, ldxr, ldxc, d, k, ldv;
  const double* V;
  const float* nrm_r;  // nr x 2: ||xr_i||^2 as (hi, lo)
  const float* nrm_c;  // nc x 2
  double* part;        // nchunk x nr x k
  int cpc;             // column tiles per chunk
  float ch, cl;        // log2(e) / (2 sigma^2) as a float pair
  float sh, sl;        // 1 / sigma^2 as a float pair (DS = 1)
  float tab[2 * NTAB];
};

// (ph, pl) ~= (ah + al) (bh + bl)
__device__ __forceinline__ void mul_ff(float ah, float al, float bh, float bl, float& ph,
                                       float& pl) {
  ph = ah * bh;
  pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
}

template <int DS, int KV>
__global__ void __launch_bounds__(HT)
hpw_kernel(const __grid_constant__ HpwParams p) {
  extern __shared__ __align__(16) float hsm[];
  float* As = hsm;                         // TK x SP
  float* Bs = As + TK * SP;                // TK x SP
  float* Kh = Bs + TK * SP;                // TM x KP
  float* Kl = Kh + TM * KP;                // TM x KP
  float* Vh = Kl + TM * KP;                // TN x KV
  float* Vl = Vh + TN * KV;                // TN x KV
  float* nrr = Vl + TN * KV;               // TM x 2
  float* nrc = nrr + 2 * TM;               // TN x 2
  float* tab = nrc + 2 * TN;               // 2 NTAB

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * TM;
  const int ct0 = blockIdx.y * p.cpc;
  const int nct = (p.nc + TN - 1) / TN;
  const int ct1 = min(nct, ct0 + p.cpc);
  for (int e = tid; e < 2 * NTAB; e += HT) tab[e] = p.tab[e];
  for (int e = tid; e < 2 * TM; e += HT) {
    const int i = r0 + (e >> 1);
    nrr[e] = i < p.nr ? p.nrm_r[2 * i + (e & 1)] : 0.f;
  }
  // row-sum stage: NP (row, rhs) pairs per thread, JS threads per pair
  constexpr int NPAIR = TM * KV;
  constexpr int JS = NPAIR >= HT ? 1 : HT / NPAIR;
  constexpr int NP = NPAIR >= HT ? NPAIR / HT : 1;
  constexpr int JW = TN / JS;
  float qh[NP], ql[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) qh[q] = ql[q] = 0.f;

  for (int ct = ct0; ct < ct1; ++ct) {
    const int c0 = ct * TN;
    __syncthreads();  // the previous tile's row-sum stage is done with Kh, Vh
    for (int e = tid; e < TN * KV; e += HT) {
      const int j = e / KV, c = e % KV;
      const double v = (c0 + j < p.nc && c < p.k) ? p.V[(size_t)(c0 + j) * p.ldv + c] : 0.0;
      const float vh = (float)v;
      Vh[e] = vh;
      Vl[e] = (float)(v - (double)vh);
    }
    for (int e = tid; e < 2 * TN; e += HT) {
      const int j = c0 + (e >> 1);
      nrc[e] = j < p.nc ? p.nrm_c[2 * j + (e & 1)] : 0.f;
    }
    // ---------------------------------------------- x_i . x_j, float-float
    float dh[4][4], dl[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) dh[a][b] = dl[a][b] = 0.f;
    for (int t0 = 0; t0 < p.d; t0 += TK) {
      __syncthreads();
      for (int e = tid; e < TK * TM; e += HT) {
        const int row = e / TK, t = e % TK;
        const int i = r0 + row, j = c0 + row, tt = t0 + t;
        As[t * SP + row] = (i < p.nr && tt < p.d) ? p.Xr[(size_t)i * p.ldxr + tt] : 0.f;
        Bs[t * SP + row] = (j < p.nc && tt < p.d) ? p.Xc[(size_t)j * p.ldxc + tt] : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int t = 0; t < TK; ++t) {
        float av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[t * SP + ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[t * SP + tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float pr = av[a] * bv[b];
            const float pe = fmaf(av[a], bv[b], -pr);
            float s, e;
            two_sum(dh[a][b], pr, s, e);
            dh[a][b] = s;
            dl[a][b] += e + pe;
          }
      }
    }
    // ----------------------------------------- kernel entries, float-float
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int il = ty + 16 * a;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int jl = tx + 16 * b;
        // d2 = n_i + n_j - 2 x_i.x_j
        float s, e, s2, e2;
        two_sum(nrr[2 * il], nrc[2 * jl], s, e);
        two_sum(s, -2.f * dh[a][b], s2, e2);
        const float lo = e + e2 + nrr[2 * il + 1] + nrc[2 * jl + 1] - 2.f * dl[a][b];
        float d2h = s2 + lo;
        float d2l = lo - (d2h - s2);
        if (d2h <= 0.f) {
          d2h = 0.f;
          d2l = 0.f;
        }
        float xh, xl;
        mul_ff(d2h, d2l, p.ch, p.cl, xh, xl);
        float kh, kl;
        exp2_ff(-xh, -xl, tab, kh, kl);
        if (DS) {
          float gh, gl;
          mul_ff(d2h, d2l, p.sh, p.sl, gh, gl);
          float th, tl;
          mul_ff(kh, kl, gh, gl, th, tl);
          kh = th;
          kl = tl;
        }
        Kh[il * KP + jl] = kh;
        Kl[il * KP + jl] = kl;
      }
    }
    __syncthreads();
    // ----------------------------------------------- row sums K V, per pair
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int pair = (tid / JS) + q * (HT / JS);
      const int row = pair % TM, c = pair / TM;
      const int j0 = (tid % JS) * JW;
#pragma unroll 4
      for (int jj = 0; jj < JW; ++jj) {
        const int j = j0 + jj;
        float ph, pl;
        mul_ff(Kh[row * KP + j], Kl[row * KP + j], Vh[j * KV + c], Vl[j * KV + c], ph, pl);
        float s, e;
        two_sum(qh[q], ph, s, e);
        qh[q] = s;
        ql[q] += e + pl;
      }
    }
  }
  // combine the JS column parts of each pair (float-float), write FP64 partials
#pragma unroll
  for (int q = 0; q < NP; ++q) {
#pragma unroll
    for (int off = 1; off < JS; off <<= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, qh[q], off);
      const float ol = __shfl_xor_sync(0xffffffffu, ql[q], off);
      float s, e;
      two_sum(qh[q], oh, s, e);
      qh[q] = s;
      ql[q] += e + ol;
    }
    const int pair = (tid / JS) + q * (HT / JS);
    const int row = pair % TM, c = pair / TM;
    const int i = r0 + row;
    if (tid % JS == 0 && i < p.nr && c < p.k)
      p.part[((size_t)blockIdx.y * p.nr + i) * p.k + c] = (double)qh[q] + (double)ql[q];
  }
}

// nrm[i] = ||x_i||^2 in FP64, stored as two floats; one warp per row.
__global__ void hpw_norms_kernel(const float* __restrict__ X, int n, int ld, int d,
                                 float* __restrict__ nrm) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double s = 0.0;
  for (int t = lane; t < d; t += 32) {
    const double v = (double)X[(size_t)warp * ld + t];
    s = fma(v, v, s);
  }
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const float h = (float)s;
    nrm[2 * warp] = h;
    nrm[2 * warp + 1] = (float)(s - (double)h);
  }
}

// Q[i, c] = sum_ch part[ch, i, c] (in order) + shift V[i, c]
__global__ void hpw_reduce_kernel(const double* __restrict__ part, int nchunk, int nr, int k,
                                  const double* __restrict__ V, int ldv, double shift,
                                  double* __restrict__ Q, int ldq) {
  const size_t total = (size_t)nr * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e % k);
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[((size_t)ch * nr + i) * k + c];
    if (shift != 0.0) s += shift * V[(size_t)i * ldv + c];
    Q[(size_t)i * ldq + c] = s;
  }
}

int kv_of(int k) {
  if (k <= 1) return 1;
  if (k <= 2) return 2;
  if (k <= 4) return 4;
  if (k <= 8) return 8;
  return 16;
}

size_t smem_of(int kv) {
  return sizeof(float) *
         (2 * TK * SP + 2 * TM * KP + 2 * TN * kv + 2 * TM + 2 * TN + 2 * NTAB);
}

// Column chunks: enough CTAs for about four per SM.
int chunks_of(int nr, int nc) {
  const int rt = (nr + TM - 1) / TM, nct = (nc + TN - 1) / TN;
  int nch = (4 * sm_count() + rt - 1) / rt;
  if (nch > nct) nch = nct;
  if (nch < 1) nch = 1;
  return nch;
}

template <int DS, int KV>
void launch(cudaStream_t st, const HpwParams& p, dim3 grid) {
  const size_t sm = smem_of(KV);
  static bool attr = false;
  if (!attr) {
    KRR_CUDA(cudaFuncSetAttribute(hpw_kernel<DS, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    attr = true;
  }
  hpw_kernel<DS, KV><<<grid, HT, sm, st>>>(p);
  KRR_CHECK_LAUNCH();
}

template <int DS>
void dispatch_kv(int kv, cudaStream_t st, const HpwParams& p, dim3 grid) {
  switch (kv) {
    case 1: launch<DS, 1>(st, p, grid); break;
    case 2: launch<DS, 2>(st, p, grid); break;
    case 4: launch<DS, 4>(st, p, grid); break;
    case 8: launch<DS, 8>(st, p, grid); break;
    default: launch<DS, 16>(st, p, grid); break;
  }
}

}  // namespace

size_t mv_hpw_part_elems(int nr, int nc, int k) {
  return (size_t)chunks_of(nr, nc) * nr * k;
}

void launch_mv_hpw(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc, int nc,
                   int ldxc, int d, double sigma, double shift, const double* V, int k, int ldv,
                   double* Q, int ldq, double* part, float* nrm_r, float* nrm_c, int dsigma) {
  hpw_norms_kernel<<<(nr * 32 + 255) / 256, 256, 0, st>>>(Xr, nr, ldxr, d, nrm_r);
  KRR_CHECK_LAUNCH();
  const bool same = (Xr == Xc && nr == nc && ldxr == ldxc);
  if (!same) {
    hpw_norms_kernel<<<(nc * 32 + 255) / 256, 256, 0, st>>>(Xc, nc, ldxc, d, nrm_c);
    KRR_CHECK_LAUNCH();
  }
  HpwParams p;
  p.Xr = Xr;
  p.Xc = Xc;
  p.nr = nr;
  p.nc = nc;
  p.ldxr = ldxr;
  p.ldxc = ldxc;
  p.d = d;
  p.k = k;
  p.ldv = ldv;
  p.V = V;
  p.nrm_r = nrm_r;
  p.nrm_c = same ? nrm_r : nrm_c;
  const int nch = chunks_of(nr, nc);
  const int nct = (nc + TN - 1) / TN;
  p.cpc = (nct + nch - 1) / nch;
  p.part = part;
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);
  p.ch = (float)c;
  p.cl = (float)(c - (double)p.ch);
  const double is2 = 1.0 / (sigma * sigma);
  p.sh = (float)is2;
  p.sl = (float)(is2 - (double)p.sh);
  for (int j = 0; j < NTAB; ++j) {
    const double v = std::exp2((double)j / NTAB);
    const float hi = (float)v;
    p.tab[2 * j] = hi;
    p.tab[2 * j + 1] = (float)(v - (double)hi);
  }
  const int nch_used = (nct + p.cpc - 1) / p.cpc;
  const dim3 grid((nr + TM - 1) / TM, nch_used);
  const int kv = kv_of(k);
  if (dsigma)
    dispatch_kv<1>(kv, st, p, grid);
  else
    dispatch_kv<0>(kv, st, p, grid);
  const size_t total = (size_t)nr * k;
  hpw_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      part, nch_used, nr, k, V, ldv, dsigma ? 0.0 : shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
