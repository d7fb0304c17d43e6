// Tensor-core set-up of the random-feature preconditioner (Section 2.2 and
// the set-up steps of Algorithm 1) for the mixed-precision solves:
//
//   Z = sqrt(2/s) cos(X W + b)     rff_tc_kernel: X W on tcgen05 from split
//                                  BF16 operands (hi.hi + lo.hi + hi.lo, dot
//                                  products to about 2^-16 relative), the
//                                  cosine and a 7-bit fixed-point rounding in
//                                  the epilogue
//   G = Z^T Z + lambda_p I         gram_tc_kernel: exact, on tcgen05
//
// Fixed-point features.  With 2^e the smallest power of two >= max |z_ij|
// (sqrt(2/s) for random Fourier features) every feature is stored as
//   zs_ij = q_ij / 128,   q_ij = clamp(rint(z_ij 2^(7-e)), -127, 127),
// so z_ij ~= 2^e zs_ij (absolute rounding error <= 2^(e-8)).  The
// preconditioner is built from these quantised features: with
// Zt = 2^e Zs,  (Zt Zt^T + lambda_p I)^-1 = (r - Zs G'^-1 Zs^T r) / lambda_p
// where G' = Zs^T Zs + lambda_p 2^-2e I, so the Woodbury apply runs unchanged
// on Zs.  The apply reads the 8-bit q (one byte per feature, half the bytes
// of BF16); the Gram reads Zs^T in BF16 (q / 128 is exact in BF16).
//
// Exact Gram.  Every product zs_i zs_j = q_i q_j 2^-14 is exact in FP32, and
// a sum of 256 of them is an integer multiple of 2^-14 below 2^8, i.e. fewer
// than 2^22 quanta: the FP32 accumulation in TMEM is exact over 256 rows.
// The epilogue turns each 256-row sum into an integer with one FMA (adding
// 1.5 * 2^23 puts the integer in the low mantissa bits) and accumulates it in
// 32-bit integers (at most 131,072 rows per work item: 131072 * 127^2 < 2^31).
// A finalize kernel adds the items' integer partials in 64 bits and scales by
// 2^-14, so G' is exact -- the factors describe exactly the operator applied,
// and it stays symmetric positive definite whatever lambda_p is.
//
// Both kernels: one persistent CTA per SM, warp 0 issues TMA copies into a
// ring of stages, warp 1 owns 256 TMEM columns (two 128 x 128 FP32
// accumulators) and issues tcgen05.mma (M = 128, N = 128, K = 16), warps 2-9
// are the epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31 and one half of
// the 128 columns).  Every mbarrier wait is bounded; on expiry the kernel
// raises *err, drains its copies and MMAs, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "krr_internal.cuh"
#include "krr_tc.cuh"
#include "krr_tc_ptx.cuh"

namespace krr {
namespace {

using namespace ptx;

constexpr int TM = 128;                 // rows of an output tile
constexpr int TN = 128;                 // columns of an output tile
constexpr int TK = 64;                  // K elements per block (128-byte rows)
constexpr int UK = 16;                  // K of one tcgen05.mma (16-bit operands)
constexpr int OP_BYTES = TM * TK * 2;   // one 128 x 64 BF16 block, 16 KiB
constexpr int NEPI = 8;                 // epilogue warps
constexpr int THREADS = 32 * (2 + NEPI);
constexpr int TMEM_COLS = 2 * TN;
constexpr int RFF_NS = 3;               // stages of 4 blocks (X hi, X lo, W hi, W lo)
constexpr int GRAM_NS = 6;              // stages of 2 blocks (rows I, rows J)
constexpr int CHUNK_KB = 4;             // K-blocks per exact FP32 sum (256 rows)
constexpr int MAX_ROWS_PER_ITEM = 131072;

struct RffParams {
  int n, s, n_pad, s_pad, nkb, n_rt, n_ct;
  const float* b;       // s phases
  float zscale;         // sqrt(2/s) (the plain product's scale with MODE 1)
  float qscale;         // 2^(7-e)
  signed char* Z;       // n x s, ld s: the 8-bit q of Zs = q / 128
  __nv_bfloat16* ZT;    // s_pad x n_pad
  float* F;             // MODE 1: F = zscale X W (n x s, ld ldf), FP32
  int ldf;
  int* err;
};

struct GramParams {
  int nblk, npairs, ksplit, kb_per_item, nkb_total, s_pad;
  int* part;            // ksplit x s_pad x s_pad partial integer sums
  int* err;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// A warp-uniform bounded wait (tcgen05.ld is .sync.aligned: every lane of the
// warp must take the same branch).
__device__ __forceinline__ bool warp_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  const bool ok = mbar_wait(a, parity, abort_flag, err);
  return __all_sync(0xffffffffu, ok);
}

// Lower tile pair p -> (I, J), I >= J, row-major over the lower triangle.
__device__ __forceinline__ void lower_pair(int p, int& I, int& J) {
  int i = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  I = i;
  J = p - i * (i + 1) / 2;
}

// Common prologue: barriers, TMEM allocation.  Returns the TMEM base.
template <int NS>
__device__ __forceinline__ uint32_t setup_ctl(uint64_t* full, uint64_t* empty, uint64_t* tfull,
                                              uint64_t* tempty, uint64_t* drain,
                                              uint32_t* tmem_slot, volatile int* abort_flag) {
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), NEPI);
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  return *tmem_slot;
}

// Let the copies of the last (up to NS) issued stages land after an abort.
template <int NS>
__device__ __forceinline__ void drain_ring(uint64_t* full, uint32_t st, uint32_t ph,
                                           uint32_t issued) {
  const uint32_t nout = issued < (uint32_t)NS ? issued : (uint32_t)NS;
  for (uint32_t q = 0; q < nout; ++q) {
    if (st == 0) {
      st = NS - 1;
      ph ^= 1;
    } else {
      --st;
    }
    mbar_drain(smem_u32(&full[st]), ph);
  }
}

// 64 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    tmem_ld16_nowait(taddr + 16 * q, *reinterpret_cast<uint32_t(*)[16]>(&r[16 * q]));
  tmem_wait_ld(*reinterpret_cast<uint32_t(*)[16]>(&r[0]));
#pragma unroll
  for (int q = 1; q < 4; ++q) tmem_keep(*reinterpret_cast<uint32_t(*)[16]>(&r[16 * q]));
}

// ------------------------------------------------------------ features --
// Work item = (128-row tile of X, 128-column tile of W).  K runs over the
// kp / 64 blocks of the d coordinates; per block the MMA warp issues
// hi.hi + lo.hi + hi.lo (12 MMAs).  MODE 0: the fixed-point random Fourier
// features; MODE 1: the plain product F = zscale X W in FP32 (the dense
// Gaussian projection of the multiple-level sketch).
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
rff_tc_kernel(const __grid_constant__ CUtensorMap tmXh, const __grid_constant__ CUtensorMap tmXl,
              const __grid_constant__ CUtensorMap tmWh, const __grid_constant__ CUtensorMap tmWl,
              RffParams p) {
  constexpr int NS = RFF_NS;
  constexpr int STAGE = 4 * OP_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + NS * STAGE);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.n_rt * p.n_ct;
  const uint32_t tmem = setup_ctl<NS>(full, empty, tfull, tempty, drain, tmem_slot, abort_flag);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0, issued = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int rt = item / p.n_ct, ct = item % p.n_ct;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
          const uint32_t sa = smem_u32(smem + st * STAGE);
          const uint32_t fb = smem_u32(&full[st]);
          mbar_expect_tx(fb, STAGE);
          tma_load_2d(sa, &tmXh, kb * TK, rt * TM, fb);
          tma_load_2d(sa + OP_BYTES, &tmXl, kb * TK, rt * TM, fb);
          tma_load_2d(sa + 2 * OP_BYTES, &tmWh, kb * TK, ct * TN, fb);
          tma_load_2d(sa + 3 * OP_BYTES, &tmWl, kb * TK, ct * TN, fb);
          ++issued;
          if (++st == (uint32_t)NS) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) drain_ring<NS>(full, st, ph, issued);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TM, TN);
      uint32_t st = 0, ph = 0, acc = 0, aph = 0;
      bool ok = true, any = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
        fence_after();
        const uint32_t d = tmem + acc * TN;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
          fence_after();
          const uint32_t xh = smem_u32(smem + st * STAGE);
          const uint32_t xl = xh + OP_BYTES, wh = xh + 2 * OP_BYTES, wl = xh + 3 * OP_BYTES;
#pragma unroll
          for (int kk = 0; kk < TK / UK; ++kk) {
            mma_bf16(d, sdesc(xh + kk * UK * 2), sdesc(wh + kk * UK * 2), idesc,
                     (kb > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, sdesc(xl + kk * UK * 2), sdesc(wh + kk * UK * 2), idesc, 1u);
            mma_bf16(d, sdesc(xh + kk * UK * 2), sdesc(wl + kk * UK * 2), idesc, 1u);
          }
          any = true;
          mma_commit(smem_u32(&empty[st]));
          if (++st == (uint32_t)NS) {
            st = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&tfull[acc]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
      }
      if (any) {
        mma_commit(smem_u32(drain));
        mbar_drain(smem_u32(drain), 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3, grp = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    uint32_t acc = 0, aph = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const int rt = item / p.n_ct, ct = item % p.n_ct;
      if (!warp_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err)) break;
      fence_after();
      uint32_t raw[64];
      tmem_ld64(tmem + ((uint32_t)(quad * 32) << 16) + acc * TN + grp * 64, raw);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
      acc ^= 1;
      if (acc == 0) aph ^= 1;
      const int i = rt * TM + row;
      const int j0 = ct * TN + grp * 64;
      const bool row_ok = i < p.n;
      if (MODE == 1) {
        if (row_ok) {
          float* fr = p.F + (size_t)i * p.ldf;
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (j0 + c < p.s) fr[j0 + c] = p.zscale * __uint_as_float(raw[c]);
        }
        continue;
      }
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const int j = j0 + c;
        float zs = 0.f;
        if (row_ok && j < p.s) {
          const float z = p.zscale * cosf(__uint_as_float(raw[c]) + __ldg(&p.b[j]));
          const float q = fminf(fmaxf(rintf(z * p.qscale), -127.f), 127.f);
          zs = q * 0.0078125f;
        }
        raw[c] = __float_as_uint(zs);
      }
      // Z^T: for each column the warp's 32 rows are consecutive (64 bytes)
#pragma unroll
      for (int c = 0; c < 64; ++c)
        p.ZT[(size_t)(j0 + c) * p.n_pad + i] = __float2bfloat16_rn(__uint_as_float(raw[c]));
      if (row_ok) {
        signed char* zr = p.Z + (size_t)i * p.s;
        if ((p.s & 15) == 0 && j0 + 64 <= p.s && ((uintptr_t)p.Z & 15) == 0) {
#pragma unroll
          for (int c = 0; c < 64; c += 16) {
            uint32_t wd[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              uint32_t b = 0;
#pragma unroll
              for (int v = 0; v < 4; ++v)
                b |= ((uint32_t)(uint8_t)(signed char)(int)(__uint_as_float(raw[c + 4 * u + v]) * 128.f))
                     << (8 * v);
              wd[u] = b;
            }
            *reinterpret_cast<uint4*>(zr + j0 + c) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
          }
        } else {
          for (int c = 0; c < 64 && j0 + c < p.s; ++c)
            zr[j0 + c] = (signed char)(int)(__uint_as_float(raw[c]) * 128.f);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- Gram --
// Work item = (lower tile pair I >= J of 128 x 128, K range).  Items are
// ordered K range first, so the CTAs running together read the same rows of
// Z^T from L2.  The item's integer sums go to part[split][I*128 + r][J*128 + c].
__global__ void __launch_bounds__(THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmZ, GramParams p) {
  constexpr int NS = GRAM_NS;
  constexpr int STAGE = 2 * OP_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = (uint64_t*)(smem + NS * STAGE);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.npairs * p.ksplit;
  const uint32_t tmem = setup_ctl<NS>(full, empty, tfull, tempty, drain, tmem_slot, abort_flag);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0, issued = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int sp = item / p.npairs;
        int I, J;
        lower_pair(item % p.npairs, I, J);
        const int kb0 = sp * p.kb_per_item, kb1 = min(p.nkb_total, kb0 + p.kb_per_item);
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
          const uint32_t sa = smem_u32(smem + st * STAGE);
          const uint32_t fb = smem_u32(&full[st]);
          mbar_expect_tx(fb, STAGE);
          tma_load_2d(sa, &tmZ, kb * TK, I * TM, fb);
          tma_load_2d(sa + OP_BYTES, &tmZ, kb * TK, J * TN, fb);
          ++issued;
          if (++st == (uint32_t)NS) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) drain_ring<NS>(full, st, ph, issued);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TM, TN);
      uint32_t st = 0, ph = 0, acc = 0, aph = 0;
      bool ok = true, any = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int sp = item / p.npairs;
        const int kb0 = sp * p.kb_per_item, kb1 = min(p.nkb_total, kb0 + p.kb_per_item);
        for (int c0 = kb0; ok && c0 < kb1; c0 += CHUNK_KB) {
          // one exact 256-row sum per accumulator buffer
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          const uint32_t d = tmem + acc * TN;
          for (int kb = c0; kb < c0 + CHUNK_KB; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
            fence_after();
            const uint32_t a = smem_u32(smem + st * STAGE), b = a + OP_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / UK; ++kk)
              mma_bf16(d, sdesc(a + kk * UK * 2), sdesc(b + kk * UK * 2), idesc,
                       (kb > c0 || kk > 0) ? 1u : 0u);
            any = true;
            mma_commit(smem_u32(&empty[st]));
            if (++st == (uint32_t)NS) {
              st = 0;
              ph ^= 1;
            }
          }
          if (!ok) break;
          mma_commit(smem_u32(&tfull[acc]));
          acc ^= 1;
          if (acc == 0) aph ^= 1;
        }
      }
      if (any) {
        mma_commit(smem_u32(drain));
        mbar_drain(smem_u32(drain), 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3, grp = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    uint32_t acc = 0, aph = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
      const int sp = item / p.npairs;
      int I, J;
      lower_pair(item % p.npairs, I, J);
      const int kb0 = sp * p.kb_per_item, kb1 = min(p.nkb_total, kb0 + p.kb_per_item);
      int isum[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) isum[c] = 0;
      for (int c0 = kb0; c0 < kb1; c0 += CHUNK_KB) {
        if (!(ok = warp_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        fence_after();
        uint32_t raw[64];
        tmem_ld64(tmem + ((uint32_t)(quad * 32) << 16) + acc * TN + grp * 64, raw);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
        // v = m 2^-14 with |m| < 2^22: v 2^14 + 1.5 2^23 holds m in its low
        // mantissa bits exactly
#pragma unroll
        for (int c = 0; c < 64; ++c)
          isum[c] += __float_as_int(fmaf(__uint_as_float(raw[c]), 16384.f, 12582912.f)) -
                     0x4B400000;
      }
      if (!ok) break;
      int* out = p.part + ((size_t)sp * p.s_pad + (size_t)I * TM + row) * p.s_pad + J * TN +
                 grp * 64;
#pragma unroll
      for (int c = 0; c < 64; c += 4)
        *reinterpret_cast<int4*>(out + c) = make_int4(isum[c], isum[c + 1], isum[c + 2], isum[c + 3]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// G[i, j] = G[j, i] = 2^-14 sum_split part[split, i, j] (+ shift on the
// diagonal) for i >= j; integer sums in 64 bits, so the result is exact.
__global__ void gram_tc_finalize_kernel(const int* __restrict__ part, int ksplit, int s,
                                        int s_pad, double shift, double* __restrict__ G) {
  const size_t total = (size_t)s * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / s), j = (int)(e % s);
    if (i < j) continue;
    long long v = 0;
    for (int sp = 0; sp < ksplit; ++sp) v += part[((size_t)sp * s_pad + i) * s_pad + j];
    double g = (double)v * (1.0 / 16384.0);
    if (i == j) g += shift;
    G[(size_t)i * s + j] = g;
    G[(size_t)j * s + i] = g;
  }
}

// hi = bf16(a), lo = bf16(a - hi) of a rows x cols matrix read with element
// (r, c) at A[r * rs + c * cs], written K-major to rows_pad x kp (zero padded).
__global__ void split_rows_kernel(const float* __restrict__ A, int rows, int cols, size_t rs,
                                  size_t cs, int rows_pad, int kp, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  const size_t total = (size_t)rows_pad * kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / kp), c = (int)(e % kp);
    const float a = (r < rows && c < cols) ? A[(size_t)r * rs + (size_t)c * cs] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(a);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(a - __bfloat162float(h));
  }
}

// Largest |Z_ij| as the bit pattern of a non-negative float (atomicMax on int).
__global__ void absmax_kernel(const float* __restrict__ Z, int n, int s, int ldz,
                              int* __restrict__ out) {
  float m = 0.f;
  const size_t total = (size_t)n * s;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(Z[(e / s) * ldz + e % s]));
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_int(m));
}

// Fixed-point features of a caller's Z: q = clamp(rint(z qscale), +-127),
// zs = q / 128 into Zs (n x s) and Zs^T (s_pad x n_pad, zero padded).  The
// scaling by a power of two is exact, so the rounding decision is exactly
// rint(z * qscale) of the FP32 input.
__global__ void quantize_z_kernel(const float* __restrict__ Z, int n, int s, int ldz,
                                  float qscale, int n_pad, int s_pad,
                                  signed char* __restrict__ Zs, __nv_bfloat16* __restrict__ ZT) {
  // 32 x 32 tiles through shared memory so both outputs are written coalesced
  __shared__ float t[32][33];
  const int tiles_j = s_pad / 32;
  const int ntiles = (n_pad / 32) * tiles_j;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (tile / tiles_j) * 32, j0 = (tile % tiles_j) * 32;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int i = i0 + r, j = j0 + threadIdx.x;
      float zs = 0.f;
      if (i < n && j < s) {
        const float q = fminf(fmaxf(rintf(Z[(size_t)i * ldz + j] * qscale), -127.f), 127.f);
        zs = q * 0.0078125f;
        Zs[(size_t)i * s + j] = (signed char)(int)q;
      }
      t[r][threadIdx.x] = zs;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y)
      ZT[(size_t)(j0 + r) * n_pad + i0 + threadIdx.x] = __float2bfloat16_rn(t[threadIdx.x][r]);
  }
}

}  // namespace
}  // namespace krr

namespace krr {

int setup_tc_n_pad(int n) { return (n + 255) / 256 * 256; }
int setup_tc_s_pad(int s) { return (s + TN - 1) / TN * TN; }
int setup_tc_kp(int d) { return (d + TK - 1) / TK * TK; }

int fixed_point_exponent(double maxabs) {
  if (!(maxabs > 0.0) || !std::isfinite(maxabs)) return 0;
  int E = 0;
  const double m = std::frexp(maxabs, &E);   // maxabs = m 2^E, m in [1/2, 1)
  return m == 0.5 ? E - 1 : E;
}

namespace {
int gram_ksplit(int n_pad, int npairs) {
  const int nkb = n_pad / TK;
  const int min_split = (n_pad + MAX_ROWS_PER_ITEM - 1) / MAX_ROWS_PER_ITEM;
  const int want = (4 * sm_count() + npairs - 1) / npairs;
  const int max_split = std::max(1, n_pad / 2048);     // at least 8 exact sums per item
  int ks = std::max(min_split, std::min(want, max_split));
  int kbi = (nkb + ks - 1) / ks;
  kbi = (kbi + CHUNK_KB - 1) / CHUNK_KB * CHUNK_KB;
  return (nkb + kbi - 1) / kbi;
}

template <typename K>
void set_smem(K kern, size_t bytes) {
  KRR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}
}  // namespace

size_t gram_tc_part_elems(int n, int s) {
  const int s_pad = setup_tc_s_pad(s), nblk = s_pad / TN;
  return (size_t)gram_ksplit(setup_tc_n_pad(n), nblk * (nblk + 1) / 2) * s_pad * s_pad;
}

void launch_split_rows(cudaStream_t st, const float* A, int rows, int cols, size_t rs, size_t cs,
                       int rows_pad, int kp, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const size_t total = (size_t)rows_pad * kp;
  const int nb = (int)std::min<size_t>((total + 255) / 256, (size_t)8 * sm_count());
  split_rows_kernel<<<nb, 256, 0, st>>>(A, rows, cols, rs, cs, rows_pad, kp, hi, lo);
  KRR_CHECK_LAUNCH();
}

int launch_rff_tc(cudaStream_t st, const float* X, int n, int d, int ldx, const float* W,
                  const float* b, int s, __nv_bfloat16* Xh, __nv_bfloat16* Xl,
                  __nv_bfloat16* Wh, __nv_bfloat16* Wl, signed char* Z, __nv_bfloat16* ZT,
                  int* err) {
  const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s), kp = setup_tc_kp(d);
  launch_split_rows(st, X, n, d, (size_t)ldx, 1, n_pad, kp, Xh, Xl);
  launch_split_rows(st, W, s, d, 1, (size_t)s, s_pad, kp, Wh, Wl);   // W^T: row j = W[:, j]
  CUtensorMap mxh, mxl, mwh, mwl;
  tc_make_map_bf16(&mxh, Xh, n_pad, kp, TM);
  tc_make_map_bf16(&mxl, Xl, n_pad, kp, TM);
  tc_make_map_bf16(&mwh, Wh, s_pad, kp, TN);
  tc_make_map_bf16(&mwl, Wl, s_pad, kp, TN);
  const float zscale = (float)std::sqrt(2.0 / s);
  const int e = fixed_point_exponent((double)zscale);
  RffParams p{};
  p.n = n;
  p.s = s;
  p.n_pad = n_pad;
  p.s_pad = s_pad;
  p.nkb = kp / TK;
  p.n_rt = n_pad / TM;
  p.n_ct = s_pad / TN;
  p.b = b;
  p.zscale = zscale;
  p.qscale = (float)std::ldexp(1.0, 7 - e);
  p.Z = Z;
  p.ZT = ZT;
  p.err = err;
  const size_t sm = 1024 + (size_t)RFF_NS * 4 * OP_BYTES + 256;
  static size_t attr = 0;
  if (attr < sm) {
    set_smem(rff_tc_kernel<0>, sm);
    attr = sm;
  }
  const int grid = std::min(p.n_rt * p.n_ct, sm_count());
  rff_tc_kernel<0><<<grid, THREADS, sm, st>>>(mxh, mxl, mwh, mwl, p);
  KRR_CHECK_LAUNCH();
  return e;
}

int launch_quantize_z(cudaStream_t st, const float* Z, int n, int s, int ldz, signed char* Zs,
                      __nv_bfloat16* ZT, int* scratch) {
  KRR_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int), st));
  const size_t total = (size_t)n * s;
  const int nb = (int)std::min<size_t>((total + 255) / 256, (size_t)8 * sm_count());
  absmax_kernel<<<nb, 256, 0, st>>>(Z, n, s, ldz, scratch);
  KRR_CHECK_LAUNCH();
  int bits = 0;
  KRR_CUDA(cudaMemcpyAsync(&bits, scratch, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  float mx = 0.f;
  memcpy(&mx, &bits, sizeof(float));
  if (!std::isfinite(mx)) throw Error{KRR_ECHOL, "precond_setup: Z holds a NaN or Inf"};
  if (!(mx > 0.f)) throw Error{KRR_EINVAL, "precond_setup: Z is zero"};
  const int e = fixed_point_exponent((double)mx);
  const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s);
  const int tiles = (n_pad / 32) * (s_pad / 32);
  quantize_z_kernel<<<std::min(tiles, 16 * sm_count()), dim3(32, 8), 0, st>>>(
      Z, n, s, ldz, (float)std::ldexp(1.0, 7 - e), n_pad, s_pad, Zs, ZT);
  KRR_CHECK_LAUNCH();
  return e;
}

void launch_gram_tc(cudaStream_t st, const __nv_bfloat16* ZT, int n, int s, double shift,
                    int* part, double* G, int* err) {
  const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s);
  GramParams p;
  p.nblk = s_pad / TN;
  p.npairs = p.nblk * (p.nblk + 1) / 2;
  p.ksplit = gram_ksplit(n_pad, p.npairs);
  p.nkb_total = n_pad / TK;
  int kbi = (p.nkb_total + p.ksplit - 1) / p.ksplit;
  p.kb_per_item = (kbi + CHUNK_KB - 1) / CHUNK_KB * CHUNK_KB;
  p.s_pad = s_pad;
  p.part = part;
  p.err = err;
  CUtensorMap mz;
  tc_make_map_bf16(&mz, ZT, s_pad, n_pad, TM);
  const size_t sm = 1024 + (size_t)GRAM_NS * 2 * OP_BYTES + 256;
  static size_t attr = 0;
  if (attr < sm) {
    set_smem(gram_tc_kernel, sm);
    attr = sm;
  }
  const int grid = std::min(p.npairs * p.ksplit, sm_count());
  gram_tc_kernel<<<grid, THREADS, sm, st>>>(mz, p);
  KRR_CHECK_LAUNCH();
  const size_t total = (size_t)s * s;
  const int nb = (int)std::min<size_t>((total + 255) / 256, (size_t)8 * sm_count());
  gram_tc_finalize_kernel<<<nb, 256, 0, st>>>(part, p.ksplit, s, s_pad, shift, G);
  KRR_CHECK_LAUNCH();
}

void launch_gemm_tc_f32(cudaStream_t st, const float* A, int n, int K, int lda, const float* B,
                        int s, int ldb, float scale, float* F, int ldf, __nv_bfloat16* Ah,
                        __nv_bfloat16* Al, __nv_bfloat16* Bh, __nv_bfloat16* Bl, int* err) {
  const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s), kp = setup_tc_kp(K);
  launch_split_rows(st, A, n, K, (size_t)lda, 1, n_pad, kp, Ah, Al);
  launch_split_rows(st, B, s, K, (size_t)ldb, 1, s_pad, kp, Bh, Bl);
  CUtensorMap mah, mal, mbh, mbl;
  tc_make_map_bf16(&mah, Ah, n_pad, kp, TM);
  tc_make_map_bf16(&mal, Al, n_pad, kp, TM);
  tc_make_map_bf16(&mbh, Bh, s_pad, kp, TN);
  tc_make_map_bf16(&mbl, Bl, s_pad, kp, TN);
  RffParams p{};
  p.n = n;
  p.s = s;
  p.n_pad = n_pad;
  p.s_pad = s_pad;
  p.nkb = kp / TK;
  p.n_rt = n_pad / TM;
  p.n_ct = s_pad / TN;
  p.zscale = scale;
  p.F = F;
  p.ldf = ldf;
  p.err = err;
  const size_t sm = 1024 + (size_t)RFF_NS * 4 * OP_BYTES + 256;
  static size_t attr = 0;
  if (attr < sm) {
    set_smem(rff_tc_kernel<1>, sm);
    attr = sm;
  }
  const int grid = std::min(p.n_rt * p.n_ct, sm_count());
  rff_tc_kernel<1><<<grid, THREADS, sm, st>>>(mah, mal, mbh, mbl, p);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
