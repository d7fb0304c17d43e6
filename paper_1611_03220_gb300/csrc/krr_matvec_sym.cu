// Symmetric fused kernel-matrix product on the tensor cores (tcgen05), one
// right-hand side, d <= 64:
//
//   q = K v + shift v,   K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)),
//
// the per-iteration product of Algorithm 1 (Section 3.1), with K symmetric:
// every exponential serves two entries.  The arithmetic is that of
// tc_matvec_kernel (Gaussian kernel of the rounded, centred, scaled points,
// K_ij = exp2(xh_i.xh_j) ra_i ra_j); only the tiling differs.
//
// Tiling.  Square 128 x 128 tiles (I, J) of row block I and column block J,
// only for I <= J.  A work item is one column block J and a run of its row
// blocks I0 <= I < I1 (I1 <= J + 1).  For every tile the epilogue forms
// E_ij = exp2(S_ij) once and adds
//   E_ij w_j  to the row sum of i     (K_IJ v_J: the tile's row sums)
//   E_ij w_i  to the column sum of j  (K_JI v_I: the tile's column sums,
//                                       skipped on the diagonal tile I = J)
// with w = ra v.  A thread owns one row of the tile (its TMEM lane) and 64 of
// its columns, so the column sums of one item stay in registers (32 packed
// pairs) while its row blocks stream past; they are reduced across lanes (a
// reduce-scatter of 62 shuffles) and across the four row quadrants once per
// item.  The row sums of a tile are complete after one combine across the
// two column halves (shared memory, one named barrier per row quadrant).
//
// Status: correct (it passes the same parity tests as the full product) but
// slower on this GPU -- at n = 65,536 0.845 ms with 16 epilogue warps and
// 0.868 ms with 8, against 0.676 ms for tc_matvec_kernel -- so it is only a
// candidate of the tile-plan autotuner (modes 2 and 3 select it).  The
// epilogue needs about three issue slots per exponential (row FMA, column FMA,
// MUFU) against two in the full product, and every tile ends in a combine of
// its row sums across the column groups (a named barrier per row quadrant);
// ncu put the 8-warp MUFU at 28 % of its peak with fixed-latency and
// TMEM-load stalls on top.  Packed FP32 FMAs, four TMEM accumulators,
// 16-column TMEM chunks with the next one in flight, split row-sum chains and
// twice the epilogue warps each left the time within 3 %.
//
// Output: rowpart[J][i] = sum over columns of J of E_ij w_j (i in I <= J) and
// colpart[c][j] = the column sums of item c of column block J(j); a second
// kernel adds them in FP64 in a fixed order, applies ra_i and the shift.
//
// Structure (one persistent CTA per SM, items dealt round-robin from a host
// list sorted by size): warp 0 issues TMA loads (the item's column block
// once, into one of two resident buffers; each row block into a ring of NS
// stages), warp 1 issues
// the MMAs (M = N = 128, K = 16, four FP32 accumulators in the 512 TMEM
// columns) and warps 2.. are the epilogue (8 or 16 warps).  Every mbarrier wait is
// bounded; on expiry the kernel raises the error flag, drains its own copies
// and MMAs, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "krr_tc.cuh"
#include "krr_tc_ptx.cuh"

namespace krr {
namespace {

using namespace ptx;

constexpr int T = 128;                 // tile edge (rows = columns)
constexpr int SK = 64;                 // K extent (d <= 64, one K-block)
constexpr int SUK = 16;                // K per MMA instruction
constexpr int TILE_BYTES = T * SK * 2; // one 128 x 64 16-bit block
// Epilogue warps: 4 row quadrants x (SNEPI / 4) column groups of SCOLS
// columns; 8 (64 columns per thread) or 16 (32 columns, twice the warps to
// hide TMEM-load and MUFU latency with half the column accumulators).
template <int SNEPI>
struct SymCfg {
  static constexpr int NG = SNEPI / 4;           // column groups
  static constexpr int SCOLS = T / NG;           // columns per epilogue warp
  static constexpr int STHREADS = 32 * (2 + SNEPI);
};
constexpr int SNS_MAX = 6;
constexpr int NACC = 4;                // 128-column accumulators in TMEM
constexpr uint32_t STMEM_COLS = NACC * T;

struct SymParams {
  int n_items;
  const int4* items;   // (J, I0, I1, chunk) per item
  int n_pad;
  int ns;              // ring stages (<= SNS_MAX)
  uint32_t idesc;
  const float* w;      // n_pad weights ra_j v_j (0 for padding)
  float* rowpart;      // n_t x n_pad
  float* colpart;      // chunks x n_pad
  int* err;
};

__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Wait for the outstanding TMEM loads; the registers are operands so that
// no use of them can be scheduled before the wait.
__device__ __forceinline__ void ld_wait(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ void qbar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The exponentials of one 16-column chunk: row sums against the column
// weights wv (shared memory), column sums against this row's weight w_r
// unless the tile is on the diagonal.  All exponentials first (independent
// MUFU work, in place), then paired FMAs (two independent round-to-nearest
// FP32 FMAs per instruction: the same arithmetic as two fmaf, half the issue
// slots).  rs[m] sums the columns 4i + 2m (x) and 4i + 2m + 1 (y) over i:
// four independent chains, so the row sum is no serial dependency; cs[m]
// holds the column sums of columns 2m and 2m + 1 of the chunk.
template <bool DIAG>
__device__ __forceinline__ void chunk_math(uint32_t (&u)[16], const float* wv, float w_r,
                                          float2 (&rs)[4], float2* cs) {
  const float4* w4 = reinterpret_cast<const float4*>(wv);
#pragma unroll
  for (int j = 0; j < 16; ++j) u[j] = __float_as_uint(ex2a(__uint_as_float(u[j])));
  const float2 wr2 = make_float2(w_r, w_r);
#pragma unroll
  for (int j4 = 0; j4 < 4; ++j4) {
    const float4 w = w4[j4];
    const float2 e01 = make_float2(__uint_as_float(u[4 * j4]), __uint_as_float(u[4 * j4 + 1]));
    const float2 e23 =
        make_float2(__uint_as_float(u[4 * j4 + 2]), __uint_as_float(u[4 * j4 + 3]));
    rs[(2 * j4) & 3] = __ffma2_rn(e01, make_float2(w.x, w.y), rs[(2 * j4) & 3]);
    rs[(2 * j4 + 1) & 3] = __ffma2_rn(e23, make_float2(w.z, w.w), rs[(2 * j4 + 1) & 3]);
    if (!DIAG) {
      cs[2 * j4] = __ffma2_rn(e01, wr2, cs[2 * j4]);
      cs[2 * j4 + 1] = __ffma2_rn(e23, wr2, cs[2 * j4 + 1]);
    }
  }
}

template <int SNEPI>
__global__ void __launch_bounds__(SymCfg<SNEPI>::STHREADS, 1)
tc_sym_kernel(const __grid_constant__ CUtensorMap tmX, SymParams p) {
  constexpr int NG = SymCfg<SNEPI>::NG, SCOLS = SymCfg<SNEPI>::SCOLS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int NS = p.ns;
  uint8_t* bres = smem;                            // [2] resident column blocks (item parity)
  uint8_t* ring = smem + 2 * TILE_BYTES;           // NS row blocks
  float* wcol = (float*)(ring + NS * TILE_BYTES);  // [2][T] column weights per item parity
  float* comb = wcol + 2 * T;                      // [2][NG][T] row-sum combine per tile parity
  float* colc = comb + 2 * NG * T;                 // [4][T] column-sum combine
  uint64_t* bars = (uint64_t*)(colc + 4 * T);
  uint64_t* full = bars;
  uint64_t* empty = full + SNS_MAX;
  uint64_t* tfull = empty + SNS_MAX;
  uint64_t* tempty = tfull + NACC;
  uint64_t* bfull = tempty + NACC;
  uint64_t* bempty = bfull + 2;
  uint64_t* drain = bempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SNS_MAX; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < NACC; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), SNEPI);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&bfull[s]), 1);
      mbar_init(smem_u32(&bempty[s]), 1);
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), STMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0, issued = 0, nb = 0, bis = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < p.n_items; item += gridDim.x, ++nb) {
        const int4 it = p.items[item];
        const uint32_t b = nb & 1, bpar = (nb >> 1) & 1;
        if (!(ok = mbar_wait(smem_u32(&bempty[b]), bpar ^ 1, abort_flag, p.err))) break;
        mbar_expect_tx(smem_u32(&bfull[b]), TILE_BYTES);
        tma_load_2d(smem_u32(bres + b * TILE_BYTES), &tmX, 0, it.x * T, smem_u32(&bfull[b]));
        ++bis;
        for (int I = it.y; ok && I < it.z; ++I) {
          if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
          mbar_expect_tx(smem_u32(&full[st]), TILE_BYTES);
          tma_load_2d(smem_u32(ring + st * TILE_BYTES), &tmX, 0, I * T, smem_u32(&full[st]));
          ++issued;
          if (++st == (uint32_t)NS) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        // let the copies of the last (up to NS) stages and column blocks land
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
        // the last two column-block copies (the latest phase of each buffer)
        for (uint32_t m = bis >= 2 ? bis - 2 : 0; m < bis; ++m)
          mbar_drain(smem_u32(&bfull[m & 1]), (m >> 1) & 1);
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t st = 0, ph = 0, acc = 0, aph = 0, nb = 0;
      bool ok = true, any = false;
      for (int item = blockIdx.x; ok && item < p.n_items; item += gridDim.x, ++nb) {
        const int4 it = p.items[item];
        const uint32_t b = nb & 1, bpar = (nb >> 1) & 1;
        if (!(ok = mbar_wait(smem_u32(&bfull[b]), bpar, abort_flag, p.err))) break;
        fence_after();
        const uint32_t sb = smem_u32(bres + b * TILE_BYTES);
        for (int I = it.y; ok && I < it.z; ++I) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
          fence_after();
          const uint32_t sa = smem_u32(ring + st * TILE_BYTES);
          const uint32_t d = tmem + acc * T;
#pragma unroll
          for (int kk = 0; kk < SK / SUK; ++kk)
            mma_bf16(d, sdesc(sa + kk * SUK * 2), sdesc(sb + kk * SUK * 2), p.idesc,
                     kk > 0 ? 1u : 0u);
          any = true;
          mma_commit(smem_u32(&empty[st]));
          mma_commit(smem_u32(&tfull[acc]));
          if (++st == (uint32_t)NS) {
            st = 0;
            ph ^= 1;
          }
          if (++acc == (uint32_t)NACC) {
            acc = 0;
            aph ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bempty[b]));  // the column block is free once the item's MMAs finish
      }
      // every issued MMA has finished before TMEM is released
      if (any) {
        mma_commit(smem_u32(drain));
        mbar_drain(smem_u32(drain), 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - 2;
    const int q = warp & 3;        // TMEM lane quadrant = row quadrant of the tile
    const int g = e >> 2;          // column group: columns SCOLS g .. SCOLS (g + 1) - 1
    const int r = q * 32 + lane;   // row within the tile
    const int et = e * 32 + lane;  // 0 .. 255
    uint32_t acc = 0, aph = 0, tb = 0, ib = 0;
    bool ok = true;
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + g * SCOLS;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
      const int4 it = p.items[item];
      const int J = it.x;
      if (et < T) wcol[ib * T + et] = p.w[(size_t)J * T + et];
      float2 cacc[SCOLS / 2];
#pragma unroll
      for (int j = 0; j < SCOLS / 2; ++j) cacc[j] = make_float2(0.f, 0.f);
      bar_sync<SNEPI * 32>();
      const float* wc = wcol + ib * T + g * SCOLS;
      float w_next = p.w[(size_t)it.y * T + r];
      // SNEPI = 8: chunk 0 of the item's first tile; afterwards the next
      // 16-column chunk (of this tile or the next) is always in flight while
      // the current chunk's exponentials run.  SNEPI = 16: twice the warps
      // hide the latencies instead, and one chunk is in registers at a time
      // (the register budget of 18 warps is 96 per thread).
      constexpr bool PF = SNEPI == 8;
      uint32_t ua[16], ub[16];
      if (PF) {
        if (ok) ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err);
        if (ok) {
          fence_after();
          tmem_ld16_nowait(tq + acc * T, ua);
          ld_wait(ua);
        }
      }
      for (int I = it.y; I < it.z; ++I) {
      if (!PF) {
        const float w_r = p.w[(size_t)I * T + r];
        float2 rs[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rs[m] = make_float2(0.f, 0.f);
        const bool diag = I == J;
        if (ok) ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err);
        if (ok) {
          fence_after();
#pragma unroll
          for (int kc = 0; kc < SCOLS / 16; ++kc) {
            tmem_ld16_nowait(tq + acc * T + kc * 16, ua);
            ld_wait(ua);
            if (kc + 1 == SCOLS / 16) {
              // the tile's last chunk is in registers: the accumulator is free
              fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
            }
            if (diag)
              chunk_math<true>(ua, wc + kc * 16, w_r, rs, cacc + kc * 8);
            else
              chunk_math<false>(ua, wc + kc * 16, w_r, rs, cacc + kc * 8);
          }
        }
        float* cb = comb + tb * NG * T;
        cb[g * T + r] = ((rs[0].x + rs[0].y) + (rs[1].x + rs[1].y)) +
                        ((rs[2].x + rs[2].y) + (rs[3].x + rs[3].y));
        qbar_sync(2 + q, 32 * NG);
        if (g == 0 && ok) {
          float t = cb[r];
#pragma unroll
          for (int gg = 1; gg < NG; ++gg) t += cb[gg * T + r];
          p.rowpart[(size_t)J * p.n_pad + (size_t)I * T + r] = t;
        }
        tb ^= 1;
        if (++acc == (uint32_t)NACC) {
          acc = 0;
          aph ^= 1;
        }
        continue;
      }
        const float w_r = w_next;
        const bool more = I + 1 < it.z;
        if (more) w_next = p.w[(size_t)(I + 1) * T + r];
        float2 rs[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rs[m] = make_float2(0.f, 0.f);
        const bool diag = I == J;
        if (ok) {
#pragma unroll
          for (int kc = 0; kc < SCOLS / 16; ++kc) {
            uint32_t (&cur)[16] = (kc & 1) ? ub : ua;
            uint32_t (&nxt)[16] = (kc & 1) ? ua : ub;
            bool pre = false;
            if (kc + 1 < SCOLS / 16) {
              tmem_ld16_nowait(tq + acc * T + (kc + 1) * 16, nxt);
              pre = true;
            } else if (more) {
              const uint32_t an = acc + 1 == (uint32_t)NACC ? 0 : acc + 1;
              ok = mbar_wait(smem_u32(&tfull[an]), an ? aph : aph ^ 1, abort_flag, p.err);
              if (ok) {
                fence_after();
                tmem_ld16_nowait(tq + an * T, nxt);
                pre = true;
              }
            }
            if (diag)
              chunk_math<true>(cur, wc + kc * 16, w_r, rs, cacc + kc * 8);
            else
              chunk_math<false>(cur, wc + kc * 16, w_r, rs, cacc + kc * 8);
            if (pre) ld_wait(nxt);
            if (kc + 2 == SCOLS / 16) {
              // the tile's last chunk is in registers: the accumulator is free
              fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
            }
          }
        }
        // row sums of the tile: add the column groups (fixed order); every
        // warp of the quadrant passes this barrier once per tile
        float* cb = comb + tb * NG * T;
        cb[g * T + r] = ((rs[0].x + rs[0].y) + (rs[1].x + rs[1].y)) +
                        ((rs[2].x + rs[2].y) + (rs[3].x + rs[3].y));
        qbar_sync(2 + q, 32 * NG);
        if (g == 0 && ok) {
          float t = cb[r];
#pragma unroll
          for (int gg = 1; gg < NG; ++gg) t += cb[gg * T + r];
          p.rowpart[(size_t)J * p.n_pad + (size_t)I * T + r] = t;
        }
        tb ^= 1;
        if (++acc == (uint32_t)NACC) {
          acc = 0;
          aph ^= 1;
        }
      }
      // column sums: reduce-scatter the SCOLS per-row partials across the
      // warp's lanes (lane l ends with the column pair (l mod SCOLS/2) of its
      // group; with 32 columns lanes l and l + 16 then add theirs), then add
      // the four quadrants
      constexpr int NP = SCOLS / 2;   // column pairs per thread
#pragma unroll
      for (int s = NP / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
          const float2 send = up ? cacc[j] : cacc[j + s];
          const float2 keep = up ? cacc[j + s] : cacc[j];
          cacc[j].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, s);
          cacc[j].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, s);
        }
      }
      if (NP < 32) {
#pragma unroll
        for (int s = NP; s < 32; s <<= 1) {
          cacc[0].x += __shfl_xor_sync(0xffffffffu, cacc[0].x, s);
          cacc[0].y += __shfl_xor_sync(0xffffffffu, cacc[0].y, s);
        }
      }
      if (lane < NP) {
        colc[q * T + g * SCOLS + 2 * lane] = cacc[0].x;
        colc[q * T + g * SCOLS + 2 * lane + 1] = cacc[0].y;
      }
      if (bar_or<SNEPI * 32>(!ok || *abort_flag)) break;
      if (q == 0 && lane < NP) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = g * SCOLS + 2 * lane + h;
          p.colpart[(size_t)it.w * p.n_pad + (size_t)J * T + c] =
              (colc[c] + colc[T + c]) + (colc[2 * T + c] + colc[3 * T + c]);
        }
      }
      ib ^= 1;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, STMEM_COLS);
}

// q_i = ra_i (sum_{J >= I} rowpart[J][i] + sum_{c < nch(I)} colpart[c][i]) + shift v_i,
// FP64 sums in a fixed order.  Block: 32 rows x 8 slices of the J range.
__global__ void __launch_bounds__(256)
sym_reduce_kernel(const float* __restrict__ rowpart, const float* __restrict__ colpart,
                  int n_t, int n_pad, int C, const float* __restrict__ ra, int nr,
                  const float* __restrict__ V, int ldv, double shift, float* __restrict__ Q,
                  int ldq) {
  __shared__ double red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + tx;
  double s = 0.0;
  if (i < n_pad) {
    const int I = i / T;
    for (int J = I + ty; J < n_t; J += 8) s += (double)rowpart[(size_t)J * n_pad + i];
    const int nch = (I + C) / C;   // chunks of column block I: ceil((I + 1) / C)
    for (int c = ty; c < nch; c += 8) s += (double)colpart[(size_t)c * n_pad + i];
  }
  red[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && i < nr) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < 8; ++y) t += red[y][tx];
    Q[(size_t)i * ldq] = (float)((double)ra[i] * t + shift * (double)V[(size_t)i * ldv]);
  }
}

// w[j] = ra_j v_j for j < n, 0 for padding.
__global__ void sym_w_kernel(const float* __restrict__ V, int n, int ldv,
                             const float* __restrict__ ra, int n_pad, float* __restrict__ w) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += gridDim.x * blockDim.x)
    w[j] = j < n ? ra[j] * V[(size_t)j * ldv] : 0.f;
}

size_t sym_smem_bytes(int ns, int nepi) {
  return 1024 + (size_t)(2 + ns) * TILE_BYTES + (size_t)(2 * T + 2 * (nepi / 4) * T + 4 * T) * 4 +
         (size_t)(2 * SNS_MAX + 2 * NACC + 4 + 1) * 8 + 16;
}

template <int SNEPI>
void launch_sym(cudaStream_t st, const CUtensorMap& map, const SymParams& p, int grid) {
  const size_t sm = sym_smem_bytes(p.ns, SNEPI);
  static size_t attr = 0;
  if (attr < sm) {
    KRR_CUDA(cudaFuncSetAttribute(tc_sym_kernel<SNEPI>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = sm;
  }
  tc_sym_kernel<SNEPI><<<grid, SymCfg<SNEPI>::STHREADS, sm, st>>>(map, p);
  KRR_CHECK_LAUNCH();
}

}  // namespace

bool sym_supported(const TcOperand& op, int k, int split) {
  return k == 1 && !split && op.kp == SK && op.n_pad % T == 0;
}

// Item list of the symmetric product: for every column block J its row
// blocks 0..J in runs of at most C, sorted by length (longest first, then
// by J) so that the round-robin deal stays balanced.
void sym_items(int n_t, int C, std::vector<int4>& out) {
  out.clear();
  for (int J = 0; J < n_t; ++J)
    for (int c = 0; c * C <= J; ++c)
      out.push_back(make_int4(J, c * C, std::min(J + 1, (c + 1) * C), c));
  std::stable_sort(out.begin(), out.end(),
                   [](const int4& a, const int4& b) { return (a.z - a.y) > (b.z - b.y); });
}

void sym_reserve(TcState& t, cudaStream_t st, const TcOperand& op, int C) {
  const int n_t = op.n_pad / T;
  const int cmax = (n_t + C - 1) / C;
  tc_ensure(t.w, (size_t)op.n_pad * 4);
  tc_ensure(t.sym_rowpart, (size_t)n_t * op.n_pad * 4);
  tc_ensure(t.sym_colpart, (size_t)cmax * op.n_pad * 4);
  if (t.sym_items_nt != n_t || t.sym_items_c != C) {
    std::vector<int4> items;
    sym_items(n_t, C, items);
    tc_ensure(t.sym_items, items.size() * sizeof(int4));
    KRR_CUDA(cudaMemcpyAsync(t.sym_items.p, items.data(), items.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, st));
    KRR_CUDA(cudaStreamSynchronize(st));  // the host list goes out of scope
    t.sym_items_nt = n_t;
    t.sym_items_c = C;
    t.sym_n_items = (int)items.size();
  }
  if (!t.err.p) {
    tc_ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
}

void sym_matvec(TcState& t, cudaStream_t st, const TcOperand& op, int f16, int C, int ns,
                int nr, const float* V, int ldv, double shift, float* Q, int ldq, int nepi) {
  sym_reserve(t, st, op, C);
  const int n_t = op.n_pad / T;
  sym_w_kernel<<<std::min(4 * sm_count(), (op.n_pad + 255) / 256), 256, 0, st>>>(
      V, op.n, ldv, (const float*)op.ra.p, op.n_pad, (float*)t.w.p);
  KRR_CHECK_LAUNCH();
  SymParams p;
  p.n_items = t.sym_n_items;
  p.items = (const int4*)t.sym_items.p;
  p.n_pad = op.n_pad;
  p.ns = std::max(2, std::min(ns > 0 ? ns : 4, SNS_MAX));
  p.idesc = f16 ? idesc_f16(T, T) : idesc_bf16(T, T);
  p.w = (const float*)t.w.p;
  p.rowpart = (float*)t.sym_rowpart.p;
  p.colpart = (float*)t.sym_colpart.p;
  p.err = (int*)t.err.p;
  const int grid = std::min(p.n_items, sm_count());
  if (nepi == 8)
    launch_sym<8>(st, op.map_a, p, grid);
  else
    launch_sym<16>(st, op.map_a, p, grid);
  sym_reduce_kernel<<<op.n_pad / 32, 256, 0, st>>>(
      (const float*)t.sym_rowpart.p, (const float*)t.sym_colpart.p, n_t, op.n_pad, C,
      (const float*)op.ra.p, nr, V, ldv, shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

}  // namespace krr
