// High-precision kernel-matrix product on the BF16 tensor cores, for the
// residual of the iterative refinement:
//   Q = K(X, X) V + shift V,   K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)),
// with V and Q in FP64 and K_ij accurate to about 1e-13 relative (the paper's
// Gaussian kernel, Section 5; the product is the per-iteration cost named in
// Section 3.1).  GB300's FP64 pipe runs at about 1/64 of FP32, so the FP64
// arithmetic is replaced by exact integer products on the tensor cores and
// float-float arithmetic on the FP32 pipes.
//
// 1. Fixed-point slices.  With u_i = sqrt(log2 e)/sigma (x_i - mu) (FP64) and
//    E_i the exponent of max_t |u_it|, every coordinate is cut into five
//    signed base-512 digits relative to 2^E_i:
//      u_it ~= 2^(E_i - 8) (q0 + q1 2^-9 + q2 2^-18 + q3 2^-27 + q4 2^-36),
//    |q| <= 256, each digit exact in BF16 (every integer in [-256, 256] is).
//    The kernel computes the kernel of these truncated points (error below
//    2^(E_i - 45) per coordinate).
// 2. Dot products from exact integer sums.  For a pair of row/column tiles
//    the tensor core accumulates, per level m = a + b, the sums
//    L_m = sum_{a+b=m} sum_t q_ia q_jb in FP32 in TMEM.  For m <= 3 every
//    term and partial sum is an integer of magnitude at most
//    (m + 1) 64 2^16 <= 2^24 (d <= 64), so L_0..L_3 are exact.  Level 4
//    shares the level-3 accumulator: its five pair products are summed
//    first, and the first level-3 product scales that input by 2^-9 (the
//    MMA's input-D scale), leaving L_3 + 2^-9 L_4 with a rounding error of
//    2^-24 of a term already weighted 2^-27.  15 slice-pair GEMMs per tile.
// 3. Float-float epilogue.  u_i.u_j = 2^(E_i+E_j-16) sum_m 2^-9m L_m, then
//    arg = u_i.u_j - n_i/2 - n_j/2 (n_i = ||u_i||^2 split into two floats),
//    2^arg by a table-driven reduction (256-entry table of 2^(j/256), after
//    P. T. P. Tang's table method, 1989) and a degree-4 Taylor polynomial on
//    |r ln 2| <= ln 2 / 512, and the row sums K_ij v_j accumulated as
//    float-float pairs.  Each K_ij carries about 1e-13 relative error.
//
// Pipeline (one persistent CTA per SM, 320 threads): warp 0 loads by TMA the
// row tile's five slices once per work item and streams the column tiles'
// slices through a ring of stages; warp 1 issues the MMAs into one of two
// TMEM buffers (4 accumulators x 64 columns each, 512 columns in all); warps
// 2-9 run the epilogue.  Every mbarrier wait is bounded.
#include <cuda.h>

#include <cmath>
#include <cstring>

#include "krr_ff.cuh"
#include "krr_internal.cuh"
#include "krr_tc.cuh"
#include "krr_tc_ptx.cuh"

namespace krr {

namespace {

using namespace ptx;
using ff::exp2_ff;
using ff::NTAB;
using ff::two_sum;

constexpr int BM = 128;
constexpr int BN = 64;
constexpr int KP = 64;                 // padded coordinates (d <= 64)
constexpr int NSL = 5;                 // slices
constexpr int NLEV = 4;                // accumulators: L0, L1, L2, L3 + 2^-9 L4
constexpr int NUM_EPI = 8;
constexpr int THREADS = 32 * (2 + NUM_EPI);
constexpr int TMEM_COLS = 512;         // 2 buffers x 4 levels x 64 columns
constexpr int A_SLICE = BM * KP * 2;   // 16 KiB
constexpr int B_SLICE = BN * KP * 2;   // 8 KiB
constexpr int A_BYTES = NSL * A_SLICE;
constexpr int B_BYTES = NSL * B_SLICE;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

struct HpParams {
  int n_rt, n_ct, nchunk, cpc, n_pad;
  const float* rowd;    // n_pad x 4: (a_hi, a_lo, 2^(E-8), 0), a = -||u~||^2 / 2
  const float* cold;    // n_pad x CW: (b_hi, b_lo, 2^(E-8), 0, vh[KV], vl[KV])
  float* part;          // nchunk x n_pad x 2KV float-float partial row sums
  int* err;
  float tab[2 * NTAB];  // 2^(j/256) as (hi, lo) pairs
};

// Column-tile stages: three, or two when the column records are long.
template <int KV>
constexpr int ns_of() {
  return KV >= 16 ? 2 : 3;
}


template <int KV, int CW>
__global__ void __launch_bounds__(THREADS, 1)
hp_matvec_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 HpParams p) {
  constexpr int NS = ns_of<KV>();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                   // A_BYTES
  uint8_t* sB = sA + A_BYTES;                           // NS x B_BYTES
  float* cbuf = (float*)(sB + NS * B_BYTES);            // 2 x BN x CW
  float* comb = cbuf + 2 * BN * CW;                     // BM x 2KV
  float* tab = comb + BM * 2 * KV;                      // 2 NTAB
  uint64_t* bars = (uint64_t*)(tab + 2 * NTAB);
  uint64_t* full = bars;
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* cfull = tempty + 2;
  uint64_t* cempty = cfull + 2;
  uint64_t* afull = cempty + 2;
  uint64_t* aempty = afull + 1;
  uint64_t* drain = aempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.n_rt * p.nchunk;

  for (int e = threadIdx.x; e < 2 * NTAB; e += THREADS) tab[e] = p.tab[e];
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), NUM_EPI);
      mbar_init(smem_u32(&cfull[s]), 1);
      mbar_init(smem_u32(&cempty[s]), NUM_EPI);
    }
    mbar_init(smem_u32(afull), 1);
    mbar_init(smem_u32(aempty), 1);
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0, cs = 0, cph = 0, aph = 0, issued = 0;
      bool ok = true, a_pending = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int rt = item / p.nchunk, ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        // row tile slices, resident for the whole item
        if (!(ok = mbar_wait(smem_u32(aempty), aph ^ 1, abort_flag, p.err))) break;
        mbar_expect_tx(smem_u32(afull), A_BYTES);
        for (int a = 0; a < NSL; ++a)
          tma_load_2d(smem_u32(sA + a * A_SLICE), &tmA, 0, a * p.n_pad + rt * BM, smem_u32(afull));
        a_pending = true;
        aph ^= 1;
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&cempty[cs]), cph ^ 1, abort_flag, p.err))) break;
          fence_proxy_async_smem();   // the readers' loads before the refill
          mbar_expect_tx(smem_u32(&cfull[cs]), BN * CW * 4);
          bulk_load(smem_u32(cbuf + cs * BN * CW), p.cold + (size_t)ct * BN * CW, BN * CW * 4,
                    smem_u32(&cfull[cs]));
          cs ^= 1;
          if (cs == 0) cph ^= 1;
          if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
          const uint32_t sb = smem_u32(sB + st * B_BYTES);
          mbar_expect_tx(smem_u32(&full[st]), B_BYTES);
          for (int b = 0; b < NSL; ++b)
            tma_load_2d(sb + b * B_SLICE, &tmB, 0, b * p.n_pad + ct * BN, smem_u32(&full[st]));
          ++issued;
          if (++st == NS) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA can exit
        uint32_t s2 = st, p2 = ph;
        const uint32_t nout = issued < (uint32_t)NS ? issued : (uint32_t)NS;
        for (uint32_t q = 0; q < nout; ++q) {
          if (s2 == 0) {
            s2 = NS - 1;
            p2 ^= 1;
          } else {
            --s2;
          }
          mbar_drain(smem_u32(&full[s2]), p2);
        }
        if (a_pending) mbar_drain(smem_u32(afull), aph ^ 1);
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t st = 0, ph = 0, acc = 0, aph = 0, afp = 0;
      bool ok = true, any = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        if (!(ok = mbar_wait(smem_u32(afull), afp, abort_flag, p.err))) break;
        afp ^= 1;
        fence_after();
        const uint32_t sa = smem_u32(sA);
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
          fence_after();
          const uint32_t sb = smem_u32(sB + st * B_BYTES);
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const uint32_t d = tmem + (acc * NLEV + m) * BN;
#pragma unroll
            for (int a = 0; a <= m; ++a) {
              const int b = m - a;
#pragma unroll
              for (int kk = 0; kk < KP / 16; ++kk) {
                mma_bf16(d, sdesc(sa + a * A_SLICE + kk * 32), sdesc(sb + b * B_SLICE + kk * 32),
                         IDESC, (a > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          {
            // level 4 first, then level 3 on top of 2^-9 times it
            const uint32_t d = tmem + (acc * NLEV + 3) * BN;
#pragma unroll
            for (int a = 0; a <= 4; ++a) {
#pragma unroll
              for (int kk = 0; kk < KP / 16; ++kk) {
                mma_bf16(d, sdesc(sa + a * A_SLICE + kk * 32),
                         sdesc(sb + (4 - a) * B_SLICE + kk * 32), IDESC,
                         (a > 0 || kk > 0) ? 1u : 0u);
              }
            }
#pragma unroll
            for (int a = 0; a <= 3; ++a) {
#pragma unroll
              for (int kk = 0; kk < KP / 16; ++kk) {
                const uint64_t da = sdesc(sa + a * A_SLICE + kk * 32);
                const uint64_t db = sdesc(sb + (3 - a) * B_SLICE + kk * 32);
                if (a == 0 && kk == 0)
                  mma_bf16_scale9(d, da, db, IDESC);
                else
                  mma_bf16(d, da, db, IDESC, 1u);
              }
            }
          }
          any = true;
          mma_commit(smem_u32(&empty[st]));
          mma_commit(smem_u32(&tfull[acc]));
          if (++st == NS) {
            st = 0;
            ph ^= 1;
          }
          acc ^= 1;
          if (acc == 0) aph ^= 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(aempty));  // row tile free once this item's MMAs finish
      }
      if (any) {
        mma_commit(smem_u32(drain));
        mbar_drain(smem_u32(drain), 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int rloc = quad * 32 + lane;
    uint32_t acc = 0, aph = 0, cs = 0, cph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const int rt = item / p.nchunk, ch = item % p.nchunk;
      const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
      const int row = rt * BM + rloc;
      const float4 rd = *reinterpret_cast<const float4*>(p.rowd + (size_t)row * 4);
      const float ah = rd.x, al = rd.y, sci = rd.z;
      float qh[KV], ql[KV];
#pragma unroll
      for (int c = 0; c < KV; ++c) qh[c] = ql[c] = 0.f;
      for (int ct = ct0; ok && ct < ct1; ++ct) {
        if (!(ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        if (!(ok = mbar_wait(smem_u32(&cfull[cs]), cph, abort_flag, p.err))) break;
        fence_after();
        const float* cb = cbuf + cs * BN * CW;
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
          const int col0 = half * 32 + cc * 16;
          uint32_t L[NLEV][16];
          const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + acc * NLEV * BN + col0;
#pragma unroll
          for (int m = 0; m < NLEV; ++m) tmem_ld16_nowait(tbase + m * BN, L[m]);
          tmem_wait_ld(L[0]);
#pragma unroll
          for (int m = 1; m < NLEV; ++m) tmem_keep(L[m]);
          if (cc == 1) {
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float* cj = cb + (col0 + j) * CW;
            const float4 cd = *reinterpret_cast<const float4*>(cj);
            // scaled dot product from the exact level sums
            const float l0 = __uint_as_float(L[0][j]);
            const float t1 = __uint_as_float(L[1][j]) * 0x1p-9f;
            const float t2 = __uint_as_float(L[2][j]) * 0x1p-18f;
            float sh, sl, e2;
            two_sum(l0, t1, sh, sl);
            two_sum(sh, t2, sh, e2);
            sl += e2;
            sl = fmaf(__uint_as_float(L[3][j]), 0x1p-27f, sl);
            const float sc = sci * cd.z;
            const float dh = sh * sc, dl = sl * sc;
            // arg = u_i.u_j - n_i/2 - n_j/2 (log2 of K_ij)
            float t, te, u, ue;
            two_sum(dh, ah, t, te);
            two_sum(t, cd.x, u, ue);
            const float lo = te + ue + dl + al + cd.y;
            float xh = u + lo;
            float xl = lo - (xh - u);
            float kh, kl;
            exp2_ff(xh, xl, tab, kh, kl);
            // q += K_ij v_j in float-float
#pragma unroll
            for (int c = 0; c < KV; ++c) {
              const float vh = cj[4 + c], vl = cj[4 + KV + c];
              const float ph = kh * vh;
              float pl = fmaf(kh, vh, -ph);
              pl = fmaf(kh, vl, pl);
              pl = fmaf(kl, vh, pl);
              float s, e;
              two_sum(qh[c], ph, s, e);
              qh[c] = s;
              ql[c] += e + pl;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&cempty[cs]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
        cs ^= 1;
        if (cs == 0) cph ^= 1;
      }
      // combine the two column halves, write the item's partial row sums
      if (half == 1) {
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          comb[rloc * 2 * KV + c] = qh[c];
          comb[rloc * 2 * KV + KV + c] = ql[c];
        }
      }
      bar_sync<NUM_EPI * 32>();
      if (half == 0 && ok) {
        float* out = p.part + ((size_t)ch * p.n_pad + row) * 2 * KV;
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          float s, e;
          two_sum(qh[c], comb[rloc * 2 * KV + c], s, e);
          out[c] = s;
          out[KV + c] = ql[c] + comb[rloc * 2 * KV + KV + c] + e;
        }
      }
      if (bar_or<NUM_EPI * 32>(!ok || *abort_flag)) break;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------ helpers ----
// Per row: u = scale (x - mu) in FP64, E = exponent of max |u|, five base-512
// digits per coordinate (exact in BF16), a = -||u~||^2 / 2 as two floats.
__global__ void hp_prep_kernel(const float* __restrict__ X, int n, int ld, int d,
                               const double* __restrict__ mu, double scale, int n_pad,
                               __nv_bfloat16* __restrict__ slices, float* __restrict__ rowd) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_pad) return;
  const int i = warp;
  double u[2] = {0.0, 0.0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    if (i < n && t < d) u[h] = scale * ((double)X[(size_t)i * ld + t] - mu[t]);
  }
  double m = fmax(fabs(u[0]), fabs(u[1]));
  for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  int E = 0;
  if (m > 0.0) frexp(m, &E);  // m = f 2^E, f in [0.5, 1): |u| / 2^E < 1
  double nrm = 0.0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    double w = ldexp(u[h], 8 - E);  // |w| < 256
    double q[NSL];
#pragma unroll
    for (int a = 0; a < NSL; ++a) {
      q[a] = rint(w);                // |q| <= 256
      w = (w - q[a]) * 512.0;        // |w| <= 256
    }
    const double ut =
        ldexp(q[0] + q[1] * 0x1p-9 + q[2] * 0x1p-18 + q[3] * 0x1p-27 + q[4] * 0x1p-36, E - 8);
    nrm += ut * ut;
#pragma unroll
    for (int a = 0; a < NSL; ++a)
      slices[((size_t)a * n_pad + i) * KP + t] = __float2bfloat16_rn((float)q[a]);
  }
  for (int off = 16; off; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0) {
    const double a = -0.5 * nrm;
    const float ah = (float)a;
    const float al = (float)(a - (double)ah);
    float4 r;
    r.x = ah;
    r.y = al;
    r.z = (float)ldexp(1.0, E - 8);
    r.w = 0.f;
    *reinterpret_cast<float4*>(rowd + (size_t)i * 4) = r;
  }
}

// Column data for one product: (b_hi, b_lo, 2^(E-8), 0, vh[KV], vl[KV]).
__global__ void hp_cold_kernel(const float* __restrict__ rowd, const double* __restrict__ V,
                               int n, int k, int ldv, int n_pad, int kv, int cw,
                               float* __restrict__ cold) {
  const size_t total = (size_t)n_pad * cw;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / cw), f = (int)(e % cw);
    float v;
    if (f < 4) {
      v = (f < 3) ? rowd[(size_t)j * 4 + f] : 0.f;
    } else if (f >= 4 + 2 * kv) {
      v = 0.f;  // record padding to a multiple of four floats
    } else {
      const int c = (f - 4) % kv, lo = (f - 4) / kv;
      const double x = (j < n && c < k) ? V[(size_t)j * ldv + c] : 0.0;
      const float xh = (float)x;
      v = lo ? (float)(x - (double)xh) : xh;
    }
    cold[e] = v;
  }
}

// Q[i, c] = sum_ch (hi + lo) in FP64 + shift V[i, c]
__global__ void hp_reduce_kernel(const float* __restrict__ part, int nchunk, int n_pad, int kv,
                                 int n, int k, const double* __restrict__ V, int ldv, double shift,
                                 double* __restrict__ Q, int ldq) {
  const size_t total = (size_t)n * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e % k);
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) {
      const float* pr = part + ((size_t)ch * n_pad + i) * 2 * kv;
      s += (double)pr[c] + (double)pr[kv + c];
    }
    if (shift != 0.0) s += shift * V[(size_t)i * ldv + c];
    Q[(size_t)i * ldq + c] = s;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    KRR_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000,
                                              cudaEnableDefault, &r));
    if (r != cudaDriverEntryPointSuccess || !q)
      throw Error{KRR_ECUDA, "cuTensorMapEncodeTiled entry point not found"};
    fn = (EncodeTiledFn)q;
  }
  return fn;
}

void make_map(CUtensorMap* m, const void* base, int rows, int box_rows) {
  cuuint64_t gdim[2] = {(cuuint64_t)KP, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)KP * 2};
  cuuint32_t box[2] = {(cuuint32_t)KP, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                           gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error{KRR_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
}

void ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{KRR_ENOMEM, std::string("high-precision product workspace: ") +
                                cudaGetErrorString(e)};
  }
  b.bytes = bytes;
}

int kv_bucket(int k) {
  if (k <= 1) return 1;
  if (k <= 2) return 2;
  if (k <= 4) return 4;
  if (k <= 8) return 8;
  return 16;
}

// Column record length in floats: 4 + 2 KV rounded up to a multiple of 4 so
// every record starts 16-byte aligned.
__host__ __device__ constexpr int cw_for(int kv) { return (4 + 2 * kv + 3) / 4 * 4; }

template <int KV>
constexpr int cw_of() {
  return cw_for(KV);
}

template <int KV>
size_t smem_bytes() {
  return 1024 + (size_t)A_BYTES + (size_t)ns_of<KV>() * B_BYTES +
         (size_t)2 * BN * cw_of<KV>() * 4 + (size_t)BM * 2 * KV * 4 + 2 * NTAB * 4 + 256;
}

template <int KV>
void launch(cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b, const HpParams& p,
            int grid) {
  static bool attr = false;
  const size_t sm = smem_bytes<KV>();
  if (!attr) {
    KRR_CUDA(cudaFuncSetAttribute(hp_matvec_kernel<KV, cw_of<KV>()>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  hp_matvec_kernel<KV, cw_of<KV>()><<<grid, THREADS, sm, st>>>(a, b, p);
  KRR_CHECK_LAUNCH();
}

int choose_nchunk(int n_rt, int n_ct, int grid) {
  int best = 1;
  double best_eff = 0.0;
  for (int nc = 1; nc <= std::min(n_ct, 64); ++nc) {
    const int cpc = (n_ct + nc - 1) / nc;
    const int nce = (n_ct + cpc - 1) / cpc;
    const long items = (long)n_rt * nce;
    const long waves = (items + grid - 1) / grid;
    const double eff = (double)items / (double)(waves * grid);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = nc;
    }
  }
  return best;
}

}  // namespace

bool hp_supported(int d) { return d >= 1 && d <= KP; }

void hp_prepare(HpState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma) {
  if (t.ready && t.src == X && t.n == n && t.ld == ldx && t.d == d && t.sigma == sigma) return;
  if (!hp_supported(d))
    throw Error{KRR_EUNSUPPORTED, "high-precision tensor-core product needs d <= 64"};
  const int n_pad = (n + BM - 1) / BM * BM;
  ensure(t.mu, (size_t)d * sizeof(double));
  ensure(t.slab, (size_t)((n + 127) / 128) * d * sizeof(double));
  launch_colmean(st, X, n, ldx, d, (double*)t.mu.p, (double*)t.slab.p);
  ensure(t.slices, (size_t)NSL * n_pad * KP * 2);
  ensure(t.rowd, (size_t)n_pad * 4 * sizeof(float));
  const double scale = std::sqrt(1.4426950408889634) / sigma;
  hp_prep_kernel<<<(n_pad * 32 + 255) / 256, 256, 0, st>>>(
      X, n, ldx, d, (const double*)t.mu.p, scale, n_pad, (__nv_bfloat16*)t.slices.p,
      (float*)t.rowd.p);
  KRR_CHECK_LAUNCH();
  make_map(&t.map_a, t.slices.p, NSL * n_pad, BM);
  make_map(&t.map_b, t.slices.p, NSL * n_pad, BN);
  t.src = X;
  t.n = n;
  t.ld = ldx;
  t.d = d;
  t.sigma = sigma;
  t.n_pad = n_pad;
  t.ready = true;
}

void hp_reserve(HpState& t, cudaStream_t st, int k) {
  if (!t.ready) throw Error{KRR_EINVAL, "high-precision product used before hp_prepare"};
  const int kv = kv_bucket(k);
  const int n_rt = t.n_pad / BM, n_ct = t.n_pad / BN;
  const int nreq = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + nreq - 1) / nreq;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  ensure(t.cold, (size_t)t.n_pad * cw_for(kv) * sizeof(float));
  ensure(t.part, (size_t)nchunk * t.n_pad * 2 * kv * sizeof(float));
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
}

void hp_matvec(HpState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma,
               double shift, const double* V, int k, int ldv, double* Q, int ldq) {
  hp_prepare(t, st, X, n, ldx, d, sigma);
  hp_reserve(t, st, k);
  const int kv = kv_bucket(k);
  const int cw = cw_for(kv);
  const int n_rt = t.n_pad / BM, n_ct = t.n_pad / BN;
  const int nreq = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + nreq - 1) / nreq;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  hp_cold_kernel<<<std::min(8 * sm_count(), (int)(((size_t)t.n_pad * cw + 255) / 256)), 256, 0,
                   st>>>((const float*)t.rowd.p, V, n, k, ldv, t.n_pad, kv, cw, (float*)t.cold.p);
  KRR_CHECK_LAUNCH();
  HpParams p;
  p.n_rt = n_rt;
  p.n_ct = n_ct;
  p.nchunk = nchunk;
  p.cpc = cpc;
  p.n_pad = t.n_pad;
  p.rowd = (const float*)t.rowd.p;
  p.cold = (const float*)t.cold.p;
  p.part = (float*)t.part.p;
  p.err = (int*)t.err.p;
  for (int j = 0; j < NTAB; ++j) {
    const double v = std::exp2((double)j / NTAB);
    const float hi = (float)v;
    p.tab[2 * j] = hi;
    p.tab[2 * j + 1] = (float)(v - (double)hi);
  }
  const int items = n_rt * nchunk;
  const int grid = std::min(items, sm_count());
  switch (kv) {
    case 1: launch<1>(st, t.map_a, t.map_b, p, grid); break;
    case 2: launch<2>(st, t.map_a, t.map_b, p, grid); break;
    case 4: launch<4>(st, t.map_a, t.map_b, p, grid); break;
    case 8: launch<8>(st, t.map_a, t.map_b, p, grid); break;
    default: launch<16>(st, t.map_a, t.map_b, p, grid); break;
  }
  const size_t total = (size_t)n * k;
  hp_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      (const float*)t.part.p, nchunk, t.n_pad, kv, n, k, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

void hp_clear_error(HpState& t, cudaStream_t st) {
  if (t.err.p) KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
}

int hp_error(HpState& t, cudaStream_t st) {
  if (!t.err.p) return 0;
  int e = 0;
  KRR_CUDA(cudaMemcpyAsync(&e, t.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  return e;
}

void hp_release(HpState& t) {
  DevBuf* bufs[] = {&t.mu, &t.slab, &t.slices, &t.rowd, &t.cold, &t.part, &t.err};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  t = HpState();
}

}  // namespace krr
