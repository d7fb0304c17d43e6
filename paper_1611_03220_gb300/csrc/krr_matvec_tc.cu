// Fused kernel-matrix product on the 5th-generation tensor cores (tcgen05).
//
//   q_i = sum_j exp(-||x_i - x_j||^2 / (2 sigma^2)) v_j  (+ shift v_i)
//
// the per-iteration cost the paper names dominant (Section 3.1), for the
// Gaussian kernel of its experiments (Section 5); K is never written.
//
// Arithmetic.  With c = log2(e) / (2 sigma^2) and xh_i = bf16(sqrt(2c)(x_i - mu))
// (mu the column mean; the kernel is shift invariant),
//   -c ||x_i - x_j||^2  ~=  xh_i.xh_j - nh_i/2 - nh_j/2,   nh_i = ||xh_i||^2,
// so   K_ij = exp2(xh_i.xh_j) * ra_i * ra_j  with ra_i = exp2(-nh_i / 2).
// The tensor core forms S_ij = xh_i.xh_j (BF16 x BF16 products are exact in
// FP32; FP32 accumulation in TMEM), the epilogue evaluates exp2(S_ij) and
// contracts against w_j = ra_j v_j, and ra_i scales the finished row sum.
// This is the Gaussian kernel of the BF16-rounded points xh: the product
// stays a (symmetric positive semi-definite) kernel matrix, and the rounding
// error is what the outer refinement removes.  exp2(S) must not overflow:
// the host requires max nh <= 120.
//
// exp2 is split between two pipes: most entries use the MUFU ex2, and EMU of
// every 32 use a degree-5 polynomial for 2^f on [-1/2, 1/2] on the FMA pipe
// (coefficients fitted for this file: near-minimax in relative error,
// 7.5e-8 in exact arithmetic) with the integer part added to the exponent.
//
// Structure (one persistent CTA per SM):
//   warp 0     TMA producer: per 128 x 256 tile, K-blocks of 64 BF16 of the
//              row tile (A) and the column tile (B) into a ring of NS stages
//              (128-byte swizzle), plus the tile's w block by bulk copy.
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//              and one thread issues tcgen05.mma (M=128, N=256, K=16).
//   warps 2..  NEPI epilogue warps: warp w reads TMEM lanes 32*(w%4)..+31
//              (its row quadrant) and one of NEPI/4 column groups; each
//              thread keeps CH independent accumulator chains per RHS.
// Work items are (row tile, column chunk) pairs dealt round-robin; each item
// writes one partial row sum per chunk, and a second kernel adds the chunks
// in FP64, applies ra_i and the shift.  This kernel is the solvers' BF16
// product for every k; tc_matvec2_kernel (below) contracts on the tensor
// cores instead, for explicit products only (KRR_BF16P).  Every mbarrier wait is bounded: on
// expiry the kernel raises an error flag, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "krr_exp2.cuh"
#include "krr_tc.cuh"
#include "krr_tc_ptx.cuh"

namespace krr {
namespace {

using namespace ptx;

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr int PAD = BM / gcd_c(BM, BN) * BN;  // rows are padded to a multiple of lcm(BM, BN)
constexpr int BK = 64;
constexpr int UK = 16;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 512;

// Per-RHS-width configuration: epilogue warps, w-ring slots, accumulator
// chains, FMA-pipe exponentials per 32 entries.  Chosen by a sweep at
// n = 65536, d = 64 (tile width 128/192/256, 8/12/16 epilogue warps, 0/2/4
// FMA-pipe exponentials per 32, 2/4/8 chains): the epilogue is issue- and
// latency-bound, so moving exponentials to the FMA pipe costs more issue
// slots than it saves MUFU cycles and EMU stays 0.
template <int KV>
struct Cfg {
  static constexpr int NEPI = KV == 1 ? 16 : 8;
  static constexpr int NW = KV <= 12 ? 4 : 3;
  static constexpr int CH = KV <= 4 ? 2 : 1;
  static constexpr int EMU = 0;
  static constexpr int THREADS = 32 * (2 + NEPI);
  static constexpr int COLS = BN / (NEPI / 4);  // columns per epilogue warp
};
constexpr int NS_MAX = 4;

struct TcParams {
  int n_rt, n_ct, nchunk, cpc, nkb;
  int n_rpad;
  int a_res;        // 1: one K-block, the row tile stays in shared memory per item
  int x3;           // split points xh = hi + lo: S = hi.hi + lo.hi + hi.lo (a_res only)
  int ns;           // stages in the ring (<= NS_MAX)
  uint32_t idesc;   // MMA instruction descriptor (BF16 or FP16 operands)
  const float* w;   // n_ct*BN x KV
  float* part;      // nchunk x n_rpad x KV
  int* err;
  int ds_k = 0;     // derivative mode: w columns c < ds_k take exp2(S) S, the rest exp2(S)
  float pg = 0.f, pc = 0.f;  // polynomial mode: entries (pg S + pc)^pq
  int pq = 1;
};

// EMU of every 32 exponentials run on the FMA pipe (a tuner dimension for
// one right-hand side; Cfg<KV>::EMU otherwise).  DS = 1 is the derivative
// mode of the (D o K) product: the first p.ds_k weight columns are
// contracted with exp2(S) S instead of exp2(S).  DS = 2 is the polynomial
// kernel (pg S + pc)^pq of Section 6 on the FMA pipe instead of exp2(S).
template <int KV, int EMU = Cfg<KV>::EMU, int DS = 0>
__global__ void __launch_bounds__(Cfg<KV>::THREADS, 1)
tc_matvec_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                 TcParams p) {
  constexpr int NEPI = Cfg<KV>::NEPI, NW = Cfg<KV>::NW, CH = Cfg<KV>::CH;
  constexpr int COLS = Cfg<KV>::COLS, NG = NEPI / 4;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int NS = p.ns;
  const int sbytes = p.a_res ? B_BYTES : STAGE_BYTES;   // bytes per stage
  const int abytes = p.a_res ? (p.x3 ? 2 * A_BYTES : A_BYTES) : 0;
  uint8_t* abuf = smem;                                  // row tile (hi, lo) when a_res
  uint8_t* stages = smem + abytes;
  float* wbuf = (float*)(stages + NS * sbytes);          // NW x BN x KV
  float* comb = wbuf + NW * BN * KV;                     // (NG-1) x BM x KV
  uint64_t* bars = (uint64_t*)(comb + (NG - 1) * BM * KV);
  uint64_t* full = bars;
  uint64_t* empty = full + NS_MAX;
  uint64_t* tfull = empty + NS_MAX;
  uint64_t* tempty = tfull + 2;
  uint64_t* wfull = tempty + 2;
  uint64_t* wempty = wfull + NW;
  uint64_t* afull = wempty + NW;
  uint64_t* aempty = afull + 1;
  uint64_t* drain = aempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.n_rt * p.nchunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS_MAX; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), NEPI);
    }
    for (int s = 0; s < NW; ++s) {
      mbar_init(smem_u32(&wfull[s]), 1);
      mbar_init(smem_u32(&wempty[s]), NEPI);
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
      uint32_t st = 0, ph = 0, ws = 0, wph = 0, aph = 0, issued = 0;
      bool ok = true, a_pending = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int rt = item / p.nchunk, ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        if (p.a_res) {
          if (!(ok = mbar_wait(smem_u32(aempty), aph ^ 1, abort_flag, p.err))) break;
          mbar_expect_tx(smem_u32(afull), abytes);
          tma_load_2d(smem_u32(abuf), &tmA, 0, rt * BM, smem_u32(afull));
          if (p.x3) tma_load_2d(smem_u32(abuf + A_BYTES), &tmA2, 0, rt * BM, smem_u32(afull));
          a_pending = true;
          aph ^= 1;
        }
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&wempty[ws]), wph ^ 1, abort_flag, p.err))) break;
          fence_proxy_async_smem();   // the readers' loads before the refill
          mbar_expect_tx(smem_u32(&wfull[ws]), BN * KV * 4);
          bulk_load(smem_u32(wbuf + ws * BN * KV), p.w + (size_t)ct * BN * KV, BN * KV * 4,
                    smem_u32(&wfull[ws]));
          if (++ws == NW) {
            ws = 0;
            wph ^= 1;
          }
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
            const uint32_t sa = smem_u32(stages + st * sbytes);
            if (p.a_res) {
              // x3: stage 0 holds the column tile's hi slice, stage 1 its lo slice
              mbar_expect_tx(smem_u32(&full[st]), B_BYTES);
              tma_load_2d(sa, kb == 1 ? &tmB2 : &tmB, 0, ct * BN, smem_u32(&full[st]));
            } else {
              mbar_expect_tx(smem_u32(&full[st]), STAGE_BYTES);
              tma_load_2d(sa, &tmA, kb * BK, rt * BM, smem_u32(&full[st]));
              tma_load_2d(sa + A_BYTES, &tmB, kb * BK, ct * BN, smem_u32(&full[st]));
            }
            ++issued;
            if (++st == (uint32_t)NS) {
              st = 0;
              ph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // let the copies of the last (up to NS) stages and the row tile land
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
        if (p.a_res) {
          if (!(ok = mbar_wait(smem_u32(afull), afp, abort_flag, p.err))) break;
          afp ^= 1;
          fence_after();
        }
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          const uint32_t d = tmem + acc * BN;
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
            fence_after();
            const uint32_t ss = smem_u32(stages + st * sbytes);
            const uint32_t sa = p.a_res ? smem_u32(abuf) : ss;
            const uint32_t sb = p.a_res ? ss : ss + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk)
              mma_bf16(d, sdesc(sa + kk * UK * 2), sdesc(sb + kk * UK * 2), p.idesc,
                       (kb > 0 || kk > 0) ? 1u : 0u);
            if (p.x3 && kb == 0) {
              // lo rows against the hi columns
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk)
                mma_bf16(d, sdesc(sa + A_BYTES + kk * UK * 2), sdesc(sb + kk * UK * 2), p.idesc,
                         1u);
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
        if (!ok) break;
        if (p.a_res) mma_commit(smem_u32(aempty));  // row tile free once the item's MMAs finish
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
    const int quad = warp & 3;
    const int grp = e >> 2;
    const int row = quad * 32 + lane;
    uint32_t acc = 0, aph = 0, ws = 0, wph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const int rt = item / p.nchunk, ch = item % p.nchunk;
      const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
      float q[CH][KV];
#pragma unroll
      for (int h = 0; h < CH; ++h)
#pragma unroll
        for (int c = 0; c < KV; ++c) q[h][c] = 0.f;
      for (int ct = ct0; ok && ct < ct1; ++ct) {
        if (!(ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        if (!(ok = mbar_wait(smem_u32(&wfull[ws]), wph, abort_flag, p.err))) break;
        fence_after();
        const float* wb = wbuf + ws * BN * KV;
        // The accumulator slice is read in 32-column chunks, the next chunk's
        // TMEM load in flight while the current chunk's exponentials run; the
        // TMEM buffer goes back to the MMA warp as soon as the last chunk has
        // landed in registers.
        constexpr int NCH = COLS / 32;
        constexpr int PER = EMU > 0 ? 32 / EMU : 33;
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + acc * BN + grp * COLS;
        uint32_t raw[2][32];
        tmem_ld16_nowait(tbase, *reinterpret_cast<uint32_t(*)[16]>(&raw[0][0]));
        tmem_ld16_nowait(tbase + 16, *reinterpret_cast<uint32_t(*)[16]>(&raw[0][16]));
        tmem_wait_ld(*reinterpret_cast<uint32_t(*)[16]>(&raw[0][0]));
        tmem_keep(*reinterpret_cast<uint32_t(*)[16]>(&raw[0][16]));
        if (NCH == 1) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
        }
#pragma unroll
        for (int cc = 0; cc < NCH; ++cc) {
          const int cur = cc & 1;
          if (cc + 1 < NCH) {
            tmem_ld16_nowait(tbase + (cc + 1) * 32,
                             *reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][0]));
            tmem_ld16_nowait(tbase + (cc + 1) * 32 + 16,
                             *reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][16]));
          }
          // all exponentials of the chunk first (independent), then the contraction
          float sv[DS == 1 ? 32 : 1];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float s = __uint_as_float(raw[cur][j]);
            if (DS == 1) sv[j] = s;
            if (DS == 2) {
              const float b = fmaf(p.pg, s, p.pc);
              float r = b;
              for (int e = 1; e < p.pq; ++e) r *= b;
              raw[cur][j] = __float_as_uint(r);
            } else {
              raw[cur][j] = __float_as_uint((j % PER == PER - 1) ? ex2_fma(s) : ex2_mufu(s));
            }
          }
          const float4* w4 = reinterpret_cast<const float4*>(wb + (grp * COLS + cc * 32) * KV);
          if (KV == 1 && CH == 2) {
            // even columns into q[0], odd into q[1], as paired FP32 FMAs (two
            // independent round-to-nearest FMAs per instruction)
            float2 qq = make_float2(q[0][0], q[CH - 1][0]);
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
              const float4 wv = w4[j4];
              qq = __ffma2_rn(make_float2(__uint_as_float(raw[cur][4 * j4]),
                                          __uint_as_float(raw[cur][4 * j4 + 1])),
                              make_float2(wv.x, wv.y), qq);
              qq = __ffma2_rn(make_float2(__uint_as_float(raw[cur][4 * j4 + 2]),
                                          __uint_as_float(raw[cur][4 * j4 + 3])),
                              make_float2(wv.z, wv.w), qq);
            }
            q[0][0] = qq.x;
            q[CH - 1][0] = qq.y;
          } else {
#pragma unroll
            for (int j4 = 0; j4 < 32 * KV / 4; ++j4) {
              const float4 wv = w4[j4];
              const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int idx = j4 * 4 + u;  // = j * KV + c
                const int j = idx / KV, c = idx % KV;
                float ev = __uint_as_float(raw[cur][j]);
                if (DS == 1 && c < p.ds_k) ev *= sv[j];
                q[j % CH][c] = fmaf(ev, wq[u], q[j % CH][c]);
              }
            }
          }
          if (cc + 1 < NCH) {
            tmem_wait_ld(*reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][0]));
            tmem_keep(*reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][16]));
            if (cc + 2 == NCH) {
              fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&wempty[ws]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
        if (++ws == NW) {
          ws = 0;
          wph ^= 1;
        }
      }
      float qs[KV];
#pragma unroll
      for (int c = 0; c < KV; ++c) {
        float s = q[0][c];
#pragma unroll
        for (int h = 1; h < CH; ++h) s += q[h][c];
        qs[c] = s;
      }
      // combine the column groups (fixed order) and write the partial row sums
      if (grp > 0) {
#pragma unroll
        for (int c = 0; c < KV; ++c) comb[((grp - 1) * BM + row) * KV + c] = qs[c];
      }
      bar_sync<NEPI * 32>();
      if (grp == 0 && ok) {
        float* out = p.part + ((size_t)ch * p.n_rpad + (size_t)rt * BM + row) * KV;
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          float s = qs[c];
#pragma unroll
          for (int g = 1; g < NG; ++g) s += comb[((g - 1) * BM + row) * KV + c];
          out[c] = s;
        }
      }
      if (bar_or<NEPI * 32>(!ok || *abort_flag)) break;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------ two-GEMM variant --
// For many right-hand sides the per-entry FMAs against w dominate the
// epilogue above.  This variant contracts on the tensor cores instead:
//   S = xh_rows . xh_cols^T   GEMM 1 (M=128, N=128), double-buffered in TMEM
//   P = bf16(exp2(S))          epilogue (MUFU), stored to shared memory in the
//                              128-byte-swizzled K-major operand layout
//   D += P . Vt^T              GEMM 2 (M=128, N=16, K=128), Vt = bf16(ra_j v_jc)
// D (128 x 16 FP32 in TMEM) accumulates over the item's column tiles and the
// epilogue writes it as the item's partial row sums.  P carries one more
// BF16 rounding of each kernel entry and Vt one of each weight (2^-9
// relative each).  Unlike the rounding of the points, which leaves a
// Gaussian kernel of nearby points (positive semi-definite), rounding each
// entry perturbs K by about 2^-9 of its entries with independent signs, a
// matrix whose norm grows like sqrt(n) times the typical entry: when K has
// large entries throughout and lambda is small this makes K + lambda I
// indefinite, so the solvers do not use this variant.
//   warp 0  TMA: row tile (resident when d <= 64), column-tile K-blocks, the
//           tile's Vt block (two 64-column boxes).
//   warp 1  MMA: GEMM 1 of tile t, then GEMM 2 of tile t-1 (P of tile t-1 is
//           being written while GEMM 1 of tile t runs).
//   warps 2-17  epilogue: warp w owns TMEM lanes 32*(w%4)..+31 and one of
//           four 32-column quarters of the tile (half of one K-atom of P).
constexpr int BN2 = 128;
constexpr int N2 = 16;
constexpr int NEPI2 = 16;
constexpr int THREADS2 = 32 * (2 + NEPI2);
constexpr int B2_BYTES = BN2 * BK * 2;             // 16 KiB
constexpr int STAGE2_BYTES = A_BYTES + B2_BYTES;   // 32 KiB
constexpr int P_ATOM = BM * 128;                   // 16 KiB: 128 rows x 64 BF16
constexpr int P_BYTES = 2 * P_ATOM;                // 32 KiB
constexpr int V_ATOM = N2 * 128;                   // 2 KiB: 16 rows x 64 BF16
constexpr int V_BYTES = 2 * V_ATOM;                // 4 KiB
constexpr int NV2 = 4;                             // Vt ring slots
constexpr int TMEM_D2 = 2 * BN2;                   // D at TMEM columns 256..271
constexpr uint32_t IDESC1 = idesc_bf16(BM, BN2);
constexpr uint32_t IDESC2 = idesc_bf16(BM, N2);

struct Tc2Params {
  int n_rt, n_ct, nchunk, cpc, nkb, n_rpad, kv;
  int a_res, ns;
  int x3;       // split points as in tc_matvec_kernel (a_res only)
  float* part;  // nchunk x n_rpad x kv
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z,
                                             uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z),
               "r"(w)
               : "memory");
}

__global__ void __launch_bounds__(THREADS2, 1)
tc_matvec2_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmX2,
                  const __grid_constant__ CUtensorMap tmV, Tc2Params p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int NS = p.ns;
  const int sbytes = p.a_res ? B2_BYTES : STAGE2_BYTES;
  const int abytes = p.a_res ? (p.x3 ? 2 * A_BYTES : A_BYTES) : 0;
  uint8_t* abuf = smem;
  uint8_t* stages = smem + abytes;
  uint8_t* pbuf = stages + NS * sbytes;             // 2 x P_BYTES
  uint8_t* vbuf = pbuf + 2 * P_BYTES;               // NV2 x V_BYTES
  uint64_t* bars = (uint64_t*)(vbuf + NV2 * V_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = full + NS_MAX;
  uint64_t* tfull = empty + NS_MAX;
  uint64_t* tempty = tfull + 2;
  uint64_t* pfull = tempty + 2;
  uint64_t* pempty = pfull + 2;
  uint64_t* vfull = pempty + 2;
  uint64_t* vempty = vfull + NV2;
  uint64_t* afull = vempty + NV2;
  uint64_t* aempty = afull + 1;
  uint64_t* dfull = aempty + 1;
  uint64_t* dempty = dfull + 1;
  uint64_t* drain = dempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.n_rt * p.nchunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS_MAX; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), NEPI2);
      mbar_init(smem_u32(&pfull[s]), NEPI2);
      mbar_init(smem_u32(&pempty[s]), 1);
    }
    for (int s = 0; s < NV2; ++s) {
      mbar_init(smem_u32(&vfull[s]), 1);
      mbar_init(smem_u32(&vempty[s]), 1);
    }
    mbar_init(smem_u32(afull), 1);
    mbar_init(smem_u32(aempty), 1);
    mbar_init(smem_u32(dfull), 1);
    mbar_init(smem_u32(dempty), 4);
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
      uint32_t st = 0, ph = 0, vs = 0, vph = 0, aph = 0, issued = 0, vissued = 0;
      bool ok = true, a_pending = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int rt = item / p.nchunk, ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        if (p.a_res) {
          if (!(ok = mbar_wait(smem_u32(aempty), aph ^ 1, abort_flag, p.err))) break;
          mbar_expect_tx(smem_u32(afull), abytes);
          tma_load_2d(smem_u32(abuf), &tmX, 0, rt * BM, smem_u32(afull));
          if (p.x3) tma_load_2d(smem_u32(abuf + A_BYTES), &tmX2, 0, rt * BM, smem_u32(afull));
          a_pending = true;
          aph ^= 1;
        }
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&vempty[vs]), vph ^ 1, abort_flag, p.err))) break;
          const uint32_t sv = smem_u32(vbuf + vs * V_BYTES);
          mbar_expect_tx(smem_u32(&vfull[vs]), V_BYTES);
          tma_load_2d(sv, &tmV, ct * BN2, 0, smem_u32(&vfull[vs]));
          tma_load_2d(sv + V_ATOM, &tmV, ct * BN2 + 64, 0, smem_u32(&vfull[vs]));
          ++vissued;
          if (++vs == NV2) {
            vs = 0;
            vph ^= 1;
          }
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
            const uint32_t sa = smem_u32(stages + st * sbytes);
            if (p.a_res) {
              mbar_expect_tx(smem_u32(&full[st]), B2_BYTES);
              tma_load_2d(sa, kb == 1 ? &tmX2 : &tmX, 0, ct * BN2, smem_u32(&full[st]));
            } else {
              mbar_expect_tx(smem_u32(&full[st]), STAGE2_BYTES);
              tma_load_2d(sa, &tmX, kb * BK, rt * BM, smem_u32(&full[st]));
              tma_load_2d(sa + A_BYTES, &tmX, kb * BK, ct * BN2, smem_u32(&full[st]));
            }
            ++issued;
            if (++st == (uint32_t)NS) {
              st = 0;
              ph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // let the copies still in flight land before the CTA can exit
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
        uint32_t v2 = vs, q2 = vph;
        const uint32_t vout = vissued < (uint32_t)NV2 ? vissued : (uint32_t)NV2;
        for (uint32_t q = 0; q < vout; ++q) {
          if (v2 == 0) {
            v2 = NV2 - 1;
            q2 ^= 1;
          } else {
            --v2;
          }
          mbar_drain(smem_u32(&vfull[v2]), q2);
        }
        if (a_pending) mbar_drain(smem_u32(afull), aph ^ 1);
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t st = 0, ph = 0, acc = 0, aph = 0, afp = 0, pb = 0, pph = 0, vs = 0, vph = 0;
      uint32_t dph = 0;
      bool ok = true, any = false;
      const uint32_t pbase = smem_u32(pbuf), vbase = smem_u32(vbuf);
      // GEMM 2 of the tile whose P sits in buffer pb and whose Vt sits in slot vs
      auto gemm2 = [&](bool first) -> bool {
        if (first) {
          if (!mbar_wait(smem_u32(dempty), dph ^ 1, abort_flag, p.err)) return false;
          dph ^= 1;
        }
        if (!mbar_wait(smem_u32(&pfull[pb]), pph, abort_flag, p.err)) return false;
        if (!mbar_wait(smem_u32(&vfull[vs]), vph, abort_flag, p.err)) return false;
        fence_after();
        const uint32_t pa = pbase + pb * P_BYTES, va = vbase + vs * V_BYTES;
#pragma unroll
        for (int kk = 0; kk < BN2 / UK; ++kk) {
          const uint32_t g = kk >> 2, o = (kk & 3) * UK * 2;
          mma_bf16(tmem + TMEM_D2, sdesc(pa + g * P_ATOM + o), sdesc(va + g * V_ATOM + o), IDESC2,
                   (!first || kk > 0) ? 1u : 0u);
        }
        any = true;
        mma_commit(smem_u32(&pempty[pb]));
        mma_commit(smem_u32(&vempty[vs]));
        pb ^= 1;
        if (pb == 0) pph ^= 1;
        if (++vs == NV2) {
          vs = 0;
          vph ^= 1;
        }
        return true;
      };
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        if (p.a_res) {
          if (!(ok = mbar_wait(smem_u32(afull), afp, abort_flag, p.err))) break;
          afp ^= 1;
          fence_after();
        }
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          const uint32_t d = tmem + acc * BN2;
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
            fence_after();
            const uint32_t ss = smem_u32(stages + st * sbytes);
            const uint32_t sa = p.a_res ? smem_u32(abuf) : ss;
            const uint32_t sb = p.a_res ? ss : ss + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk)
              mma_bf16(d, sdesc(sa + kk * UK * 2), sdesc(sb + kk * UK * 2), IDESC1,
                       (kb > 0 || kk > 0) ? 1u : 0u);
            if (p.x3 && kb == 0) {
#pragma unroll
              for (int kk = 0; kk < BK / UK; ++kk)
                mma_bf16(d, sdesc(sa + A_BYTES + kk * UK * 2), sdesc(sb + kk * UK * 2), IDESC1,
                         1u);
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
          if (ct > ct0 && !(ok = gemm2(ct - 1 == ct0))) break;
        }
        if (!ok) break;
        if (!(ok = gemm2(ct1 - 1 == ct0))) break;
        mma_commit(smem_u32(dfull));
        if (p.a_res) mma_commit(smem_u32(aempty));
      }
      if (any) {
        mma_commit(smem_u32(drain));
        mbar_drain(smem_u32(drain), 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - 2;
    const int quad = warp & 3;
    const int grp = e >> 2;  // 32-column quarter
    const int row = quad * 32 + lane;
    const uint32_t prow = (uint32_t)(grp >> 1) * P_ATOM + (uint32_t)(row >> 3) * 1024u +
                          (uint32_t)(row & 7) * 128u;
    const uint32_t psw = (uint32_t)(row & 7);
    const uint32_t q0 = (uint32_t)(grp & 1) * 4;
    const uint32_t pbase = smem_u32(pbuf);
    uint32_t acc = 0, aph = 0, pb = 0, pph = 0, dph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const int rt = item / p.nchunk, ch = item % p.nchunk;
      const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
      for (int ct = ct0; ok && ct < ct1; ++ct) {
        if (!(ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        fence_after();
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + acc * BN2 + grp * 32;
        uint32_t raw[32];
        tmem_ld16_nowait(tbase, *reinterpret_cast<uint32_t(*)[16]>(&raw[0]));
        tmem_ld16_nowait(tbase + 16, *reinterpret_cast<uint32_t(*)[16]>(&raw[16]));
        tmem_wait_ld(*reinterpret_cast<uint32_t(*)[16]>(&raw[0]));
        tmem_keep(*reinterpret_cast<uint32_t(*)[16]>(&raw[16]));
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          pk[j] = pack_bf16(ex2_mufu(__uint_as_float(raw[2 * j])),
                            ex2_mufu(__uint_as_float(raw[2 * j + 1])));
        // P buffer pb is free once GEMM 2 of two tiles back has read it
        if (!(ok = mbar_wait(smem_u32(&pempty[pb]), pph ^ 1, abort_flag, p.err))) break;
        const uint32_t pa = pbase + pb * P_BYTES + prow;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          st_shared_v4(pa + (((q0 + u) ^ psw) << 4), pk[4 * u], pk[4 * u + 1], pk[4 * u + 2],
                       pk[4 * u + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&pfull[pb]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
        pb ^= 1;
        if (pb == 0) pph ^= 1;
      }
      if (ok) ok = mbar_wait(smem_u32(dfull), dph, abort_flag, p.err);
      dph ^= 1;
      if (ok && grp == 0) {
        fence_after();
        uint32_t dv[16];
        tmem_ld16_nowait(tmem + ((uint32_t)(quad * 32) << 16) + TMEM_D2, dv);
        tmem_wait_ld(dv);
        float* out = p.part + ((size_t)ch * p.n_rpad + (size_t)rt * BM + row) * p.kv;
#pragma unroll
        for (int c = 0; c < N2; ++c)
          if (c < p.kv) out[c] = __uint_as_float(dv[c]);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(dempty));
      }
      if (bar_or<NEPI2 * 32>(!ok || *abort_flag)) break;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------ helpers ----
// xh = bf16(scale (x - mu)) (fp16 with f16) padded to n_pad x kp,
// nh = ||xh||^2, ra = exp2(-nh/2).  With Xlo the points are split,
// xh = hi + lo with lo = bf16(u - hi), and nh is taken of hi + lo.
__global__ void prep_rows_kernel(const float* __restrict__ X, int n, int ld, int d,
                                 const double* __restrict__ mu, double scale, int n_pad, int kp,
                                 int f16, __nv_bfloat16* __restrict__ Xa,
                                 __nv_bfloat16* __restrict__ Xlo, float* __restrict__ ra,
                                 float* __restrict__ nh_out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_pad) return;
  const int i = warp;
  double nh = 0.0;
  for (int t = lane; t < kp; t += 32) {
    double u = 0.0;
    if (i < n && t < d) u = scale * ((double)X[(size_t)i * ld + t] - mu[t]);
    double bv;
    if (f16) {
      const __half hb = __float2half_rn((float)u);
      reinterpret_cast<__half*>(Xa)[(size_t)i * kp + t] = hb;
      bv = (double)__half2float(hb);
    } else {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)u);
      Xa[(size_t)i * kp + t] = b;
      bv = (double)__bfloat162float(b);
    }
    if (Xlo) {
      const __nv_bfloat16 l = __float2bfloat16_rn((float)(u - bv));
      Xlo[(size_t)i * kp + t] = l;
      bv += (double)__bfloat162float(l);
    }
    nh += bv * bv;
  }
  for (int off = 16; off; off >>= 1) nh += __shfl_xor_sync(0xffffffffu, nh, off);
  if (lane == 0) {
    ra[i] = (i < n) ? (float)exp2(-0.5 * nh) : 0.f;
    nh_out[i] = (float)nh;
  }
}

__global__ void max_kernel(const float* __restrict__ a, int n, float* __restrict__ out) {
  __shared__ float red[32];
  float m = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmaxf(m, a[i]);
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) atomicMax((int*)out, __float_as_int(m));
  }
}

// ra[i] = 1 for i < n, 0 for the padding (the polynomial kernel has no row factor).
__global__ void unit_rows_kernel(float* __restrict__ ra, int n, int n_pad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
    ra[i] = i < n ? 1.f : 0.f;
}

// w[j, c] = ra_j v[j, c] for c < k, 0 for padding (rows >= n or c >= k).
__global__ void make_w_kernel(const float* __restrict__ V, int n, int k, int ldv,
                              const float* __restrict__ ra, int n_pad, int kv,
                              float* __restrict__ w) {
  const size_t total = (size_t)n_pad * kv;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / kv), c = (int)(e % kv);
    w[e] = (j < n && c < k) ? ra[j] * V[(size_t)j * ldv + c] : 0.f;
  }
}

// Vt[c, j] = bf16(ra_j v[j, c]) for c < k, 0 for padding; N2 x n_pad, j fastest.
__global__ void make_vt_kernel(const float* __restrict__ V, int n, int k, int ldv,
                               const float* __restrict__ ra, int n_pad,
                               __nv_bfloat16* __restrict__ vt) {
  const size_t total = (size_t)N2 * n_pad;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n_pad), j = (int)(e % n_pad);
    vt[e] = __float2bfloat16_rn((j < n && c < k) ? ra[j] * V[(size_t)j * ldv + c] : 0.f);
  }
}

// Weights of the derivative mode for RHS columns c0 .. c0 + kb - 1: columns
// [0, kb) and [kb, 2 kb) hold ra_j v_j, [2 kb, 3 kb) hold (nh_j / 2) ra_j v_j.
__global__ void make_w_ds_kernel(const float* __restrict__ V, int n, int kb, int c0, int ldv,
                                 const float* __restrict__ ra, const float* __restrict__ nh,
                                 int n_pad, int kv, float* __restrict__ w) {
  const size_t total = (size_t)n_pad * kv;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / kv), c = (int)(e % kv);
    float v = 0.f;
    if (j < n && c < 3 * kb) {
      const int cc = c % kb;
      v = ra[j] * V[(size_t)j * ldv + c0 + cc];
      if (c >= 2 * kb) v *= 0.5f * nh[j];
    }
    w[e] = v;
  }
}

// (D o K) v = -2 ln 2 ra_i (sum_j E_ij S_ij w_j - (nh_i / 2) sum_j E_ij w_j
//             - sum_j E_ij (nh_j / 2) w_j),  E = exp2(S), log2 K_ij = S_ij - nh_i/2 - nh_j/2
__global__ void ds_reduce_kernel(const float* __restrict__ part, int nchunk, int n_rpad, int kv,
                                 int kb, const float* __restrict__ ra,
                                 const float* __restrict__ nh, int nr, int c0,
                                 float* __restrict__ Q, int ldq) {
  const size_t total = (size_t)nr * kb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kb), c = (int)(e % kb);
    double a = 0.0, b = 0.0, cs = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) {
      const float* pr = part + ((size_t)ch * n_rpad + i) * kv;
      a += (double)pr[c];
      b += (double)pr[kb + c];
      cs += (double)pr[2 * kb + c];
    }
    const double r = -1.3862943611198906 * (double)ra[i] * (a - 0.5 * (double)nh[i] * b - cs);
    Q[(size_t)i * ldq + c0 + c] = (float)r;
  }
}

// Q[i, c] = ra_i * sum_ch part[ch, i, c] + shift * V[i, c]
__global__ void tc_reduce_kernel(const float* __restrict__ part, int nchunk, int n_rpad, int kv,
                                 const float* __restrict__ ra, int nr, int k,
                                 const float* __restrict__ V, int ldv, double shift,
                                 float* __restrict__ Q, int ldq) {
  const size_t total = (size_t)nr * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), c = (int)(e % k);
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += (double)part[((size_t)ch * n_rpad + i) * kv + c];
    s *= (double)ra[i];
    if (shift != 0.0) s += shift * (double)V[(size_t)i * ldv + c];
    Q[(size_t)i * ldq + c] = (float)s;
  }
}

// ------------------------------------------------------------ host side --
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

void make_map(CUtensorMap* m, const void* base, int rows, int kp, int box_rows, bool f16) {
  cuuint64_t gdim[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, const_cast<void*>(base), gdim,
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
    throw Error{KRR_ENOMEM, std::string("tensor-core workspace: ") + cudaGetErrorString(e)};
  }
  b.bytes = bytes;
}

int kv_bucket(int k) {
  if (k <= 1) return 1;
  if (k <= 2) return 2;
  if (k <= 4) return 4;
  if (k <= 8) return 8;
  if (k <= 12) return 12;
  return 16;
}

int choose_nchunk(int n_rt, int n_ct, int grid) {
  int best = 1;
  double best_eff = 0.0;
  for (int nc = 1; nc <= std::min(n_ct, 32); ++nc) {
    int cpc = (n_ct + nc - 1) / nc;
    int nce = (n_ct + cpc - 1) / cpc;
    long items = (long)n_rt * nce;
    long waves = (items + grid - 1) / grid;
    double eff = (double)items / (double)(waves * grid);
    // prefer fewer chunks unless the balance gain is real
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = nc;
    }
  }
  return best;
}

template <int KV>
size_t smem_bytes(int a_res, int ns, int x3) {
  constexpr int NW = Cfg<KV>::NW, NG = Cfg<KV>::NEPI / 4;
  return 1024 +
         (a_res ? (size_t)(x3 ? 2 : 1) * A_BYTES + (size_t)ns * B_BYTES
                : (size_t)ns * STAGE_BYTES) +
         (size_t)NW * BN * KV * 4 + (size_t)(NG - 1) * BM * KV * 4 + 256;
}

template <int KV, int EMU = Cfg<KV>::EMU, int DS = 0>
void launch_kernel(cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b,
                   const CUtensorMap& a2, const CUtensorMap& b2, const TcParams& p, int grid) {
  static size_t attr = 0;
  const size_t sm = smem_bytes<KV>(p.a_res, p.ns, p.x3);
  if (attr < sm) {
    KRR_CUDA(cudaFuncSetAttribute(tc_matvec_kernel<KV, EMU, DS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = sm;
  }
  tc_matvec_kernel<KV, EMU, DS><<<grid, Cfg<KV>::THREADS, sm, st>>>(a, b, a2, b2, p);
  KRR_CHECK_LAUNCH();
}

// The polynomial mode for weight blocks of kv = 1, 4 or 16 columns.
void dispatch_poly(int kv, cudaStream_t st, const TcOperand& op, const TcParams& p, int grid) {
  switch (kv) {
    case 1: launch_kernel<1, 0, 2>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 4: launch_kernel<4, Cfg<4>::EMU, 2>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    default: launch_kernel<16, Cfg<16>::EMU, 2>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
  }
}

// The derivative mode for weight blocks of kv = 4, 8, 12 or 16 columns.
void dispatch_ds(int kv, cudaStream_t st, const TcOperand& op, const TcParams& p, int grid) {
  switch (kv) {
    case 4: launch_kernel<4, Cfg<4>::EMU, 1>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 8: launch_kernel<8, Cfg<8>::EMU, 1>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 12: launch_kernel<12, Cfg<12>::EMU, 1>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    default: launch_kernel<16, Cfg<16>::EMU, 1>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
  }
}

// emu: FMA-pipe exponentials per 32 for one right-hand side (0, 2 or 4).
void dispatch(int kv, cudaStream_t st, const TcOperand& op, const TcParams& p, int grid,
              int emu = 0) {
  switch (kv) {
    case 1:
      if (emu == 4)
        launch_kernel<1, 4>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid);
      else if (emu == 2)
        launch_kernel<1, 2>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid);
      else
        launch_kernel<1, 0>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid);
      break;
    case 2: launch_kernel<2>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 4: launch_kernel<4>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 8: launch_kernel<8>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    case 12: launch_kernel<12>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
    default: launch_kernel<16>(st, op.map_a, op.map_b, op.map_a2, op.map_b2, p, grid); break;
  }
}

size_t smem2_bytes(int a_res, int ns, int x3) {
  return 1024 +
         (a_res ? (size_t)(x3 ? 2 : 1) * A_BYTES + (size_t)ns * B2_BYTES
                : (size_t)ns * STAGE2_BYTES) +
         (size_t)2 * P_BYTES + (size_t)NV2 * V_BYTES + 256;
}

void launch_kernel2(cudaStream_t st, const CUtensorMap& x, const CUtensorMap& x2,
                    const CUtensorMap& v, const Tc2Params& p, int grid) {
  static size_t attr = 0;
  const size_t sm = smem2_bytes(p.a_res, p.ns, p.x3);
  if (attr < sm) {
    KRR_CUDA(cudaFuncSetAttribute(tc_matvec2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    attr = sm;
  }
  tc_matvec2_kernel<<<grid, THREADS2, sm, st>>>(x, x2, v, p);
  KRR_CHECK_LAUNCH();
}

// Vt tensor map: N2 rows of n_pad BF16, boxes of 64 columns x N2 rows.
void make_vt_map(CUtensorMap* m, const void* base, int n_pad) {
  cuuint64_t gdim[2] = {(cuuint64_t)n_pad, (cuuint64_t)N2};
  cuuint64_t gstride[1] = {(cuuint64_t)n_pad * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)N2};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                           gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error{KRR_ECUDA, "cuTensorMapEncodeTiled (Vt) failed: " + std::to_string((int)r)};
}

// Prepare one operand set into `op` (split into hi + lo when `split`, FP16
// points when `f16`).
void prep_operand(TcOperand& op, cudaStream_t st, const float* X, int n, int ld, int d,
                  const double* mu, double scale, bool split, bool f16 = false) {
  const int kp = (d + BK - 1) / BK * BK;
  const int n_pad = (n + PAD - 1) / PAD * PAD;
  ensure(op.Xa, (size_t)n_pad * kp * 2);
  if (split) ensure(op.Xlo, (size_t)n_pad * kp * 2);
  ensure(op.ra, (size_t)n_pad * 4);
  ensure(op.nh, (size_t)n_pad * 4 + 16);
  prep_rows_kernel<<<(n_pad * 32 + 255) / 256, 256, 0, st>>>(
      X, n, ld, d, mu, scale, n_pad, kp, f16 ? 1 : 0, (__nv_bfloat16*)op.Xa.p,
      split ? (__nv_bfloat16*)op.Xlo.p : nullptr, (float*)op.ra.p, (float*)op.nh.p);
  KRR_CHECK_LAUNCH();
  op.split = split;
  op.f16 = f16;
  op.src = X;
  op.n = n;
  op.ld = ld;
  op.d = d;
  op.kp = kp;
  op.n_pad = n_pad;
  make_map(&op.map_a, op.Xa.p, n_pad, kp, BM, f16);
  make_map(&op.map_b, op.Xa.p, n_pad, kp, BN, f16);
  make_map(&op.map_a2, split ? op.Xlo.p : op.Xa.p, n_pad, kp, BM, f16);
  make_map(&op.map_b2, split ? op.Xlo.p : op.Xa.p, n_pad, kp, BN, f16);
}

struct Plan {
  int kv, n_rt, n_ct, cpc, nchunk;
  int ns = 0;   // ring stages (0: the default for the operand)
  int sym = 0;  // 1: the symmetric kernel (tiles I <= J), C row blocks per item
  int C = 16;
  int req = 0;  // the chunk request this plan was made from
  int emu = 0;  // exponentials per 32 on the FMA pipe (one right-hand side)
  int nepi = 16;  // the symmetric kernel's epilogue warps (8 or 16)
};

// The tile plan: column chunks per row tile from the wave-balance rule, or
// `req` chunks when req > 0.
Plan plan_for(const TcOperand& op, int k, int gemm2, int req = 0) {
  Plan pl;
  pl.kv = kv_bucket(k);
  pl.n_rt = op.n_pad / BM;
  pl.n_ct = op.n_pad / (gemm2 ? BN2 : BN);
  if (req <= 0) req = choose_nchunk(pl.n_rt, pl.n_ct, sm_count());
  req = std::max(1, std::min(req, pl.n_ct));
  pl.req = req;
  pl.cpc = (pl.n_ct + req - 1) / req;
  pl.nchunk = (pl.n_ct + pl.cpc - 1) / pl.cpc;
  return pl;
}

size_t smem_for(int kv, int a_res, int ns, int x3) {
  switch (kv) {
    case 1: return smem_bytes<1>(a_res, ns, x3);
    case 2: return smem_bytes<2>(a_res, ns, x3);
    case 4: return smem_bytes<4>(a_res, ns, x3);
    case 8: return smem_bytes<8>(a_res, ns, x3);
    case 12: return smem_bytes<12>(a_res, ns, x3);
    default: return smem_bytes<16>(a_res, ns, x3);
  }
}

// ------------------------------------------------------------ autotuner --
// Per problem shape (row tiles, column tiles, K-blocks, RHS bucket, operand
// format) the tuner times the fused product under each candidate plan --
// column chunks per row tile x ring stages x (one RHS) exponentials per 32
// on the FMA pipe, and (one RHS, d <= 64) the symmetric kernel's item length
// x ring stages -- and keeps the fastest in a process-wide table, so each
// shape is timed once per process.  Plans that would need more than 227 KiB
// of shared memory are skipped.  The chunk count changes the order of the
// FP32 partial sums, so a tuned product can differ from the default one in
// the last bits.
struct TuneKey {
  int n_rt, n_ct, nkb, kv, fmt;
  bool operator<(const TuneKey& o) const {
    return std::tie(n_rt, n_ct, nkb, kv, fmt) < std::tie(o.n_rt, o.n_ct, o.nkb, o.kv, o.fmt);
  }
};
struct Tuned {
  int req, ns, sym, C, emu;
  float ms;
  int nepi;
};
std::mutex g_tune_mu;
std::map<TuneKey, Tuned> g_tuned;
constexpr size_t SMEM_LIMIT = 227 * 1024;

int default_ns(int a_res) { return a_res ? 4 : 3; }

}  // namespace

void tc_ensure(DevBuf& b, size_t bytes) { ensure(b, bytes); }

void tc_make_map_bf16(CUtensorMap* m, const void* base, int rows, int row_elems, int box_rows) {
  make_map(m, base, rows, row_elems, box_rows, false);
}

void tc_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma) {
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);  // log2(e) / (2 sigma^2)
  const double scale = std::sqrt(2.0 * c);
  if (t.ready && t.cols.src == X && t.cols.n == n && t.cols.ld == ldx && t.cols.d == d &&
      t.sigma == sigma && t.rows_same)
    return;
  ensure(t.mu, (size_t)d * sizeof(double));
  ensure(t.w, (size_t)((n + 127) / 128) * d * sizeof(double));  // w doubles as the slab scratch
  launch_colmean(st, X, n, ldx, d, (double*)t.mu.p, (double*)t.w.p);
  prep_operand(t.cols, st, X, n, ldx, d, (const double*)t.mu.p, scale, false);
  ensure(t.scal, 16);
  KRR_CUDA(cudaMemsetAsync(t.scal.p, 0, 16, st));
  max_kernel<<<std::min(8 * sm_count(), (t.cols.n_pad + 255) / 256), 256, 0, st>>>(
      (const float*)t.cols.nh.p, t.cols.n_pad, (float*)t.scal.p);
  KRR_CHECK_LAUNCH();
  float mx = 0.f;
  KRR_CUDA(cudaMemcpyAsync(&mx, t.scal.p, sizeof(float), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  if (!(mx <= 120.f))
    throw Error{KRR_EUNSUPPORTED,
                "tensor-core product: ||x - mean||^2 / (2 sigma^2) too large for the factored exp2 "
                "(max " + std::to_string(mx) + " in log2 units); use FP32 or FP64"};
  t.sigma = sigma;
  t.rows_same = true;
  t.ready = true;
}

void tc_prepare_split(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                      double sigma) {
  tc_prepare(t, st, X, n, ldx, d, sigma);
  if (t.split_ready && t.split.src == X && t.split.n == n && t.split.ld == ldx && t.split.d == d &&
      t.split_sigma == sigma)
    return;
  if (t.cols.kp != BK)
    throw Error{KRR_EUNSUPPORTED, "split BF16 product needs d <= 64"};
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);
  prep_operand(t.split, st, X, n, ldx, d, (const double*)t.mu.p, std::sqrt(2.0 * c), true);
  t.split_sigma = sigma;
  t.split_ready = true;
}

void tc_prepare_f16(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                    double sigma) {
  tc_prepare(t, st, X, n, ldx, d, sigma);
  if (t.half_ready && t.half.src == X && t.half.n == n && t.half.ld == ldx && t.half.d == d &&
      t.half_sigma == sigma)
    return;
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);
  // the BF16 set passed the exp2 range check (nh <= 120, so every component
  // is below 11 in magnitude): FP16 holds these points without overflow
  prep_operand(t.half, st, X, n, ldx, d, (const double*)t.mu.p, std::sqrt(2.0 * c), false, true);
  t.half_sigma = sigma;
  t.half_ready = true;
}

void tc_prepare_rows(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr, int d,
                     double sigma, int fmt) {
  if (!t.ready || t.sigma != sigma || t.cols.d != d)
    throw Error{KRR_EINVAL, "row operand prepared before the column operand"};
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);
  prep_operand(t.rows, st, Xr, nr, ldxr, d, (const double*)t.mu.p, std::sqrt(2.0 * c), fmt == 1,
               fmt == 2);
  // the factored exp2 needs xh_i.xh_j <= 120 as well: sqrt(nh_i nh_j) <= max(nh)
  KRR_CUDA(cudaMemsetAsync(t.scal.p, 0, 16, st));
  max_kernel<<<std::min(8 * sm_count(), (t.rows.n_pad + 255) / 256), 256, 0, st>>>(
      (const float*)t.rows.nh.p, t.rows.n_pad, (float*)t.scal.p);
  KRR_CHECK_LAUNCH();
  float mx = 0.f;
  KRR_CUDA(cudaMemcpyAsync(&mx, t.scal.p, sizeof(float), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  if (!(mx <= 120.f))
    throw Error{KRR_EUNSUPPORTED,
                "tensor-core product: a row point is too far from the training mean for the "
                "factored exp2 (||x - mean||^2 / (2 sigma^2) = " + std::to_string(mx) +
                " in log2 units); use FP32, FP64 or HP"};
}

namespace {

TcOperand& operand_of(TcState& t, int fmt) {
  return fmt == 1 ? t.split : (fmt == 2 ? t.half : t.cols);
}

void run_core(TcState& t, cudaStream_t st, TcOperand& op, const Plan& pl, int split, int f16);

// Enqueue one fused product with plan `pl` (w, kernel, chunk sums).
void run_fused(TcState& t, cudaStream_t st, TcOperand& op, const Plan& pl, int split, int f16,
               int nr, const float* V, int k, int ldv, double shift, float* Q, int ldq) {
  if (pl.sym) {
    sym_matvec(t, st, op, f16, pl.C, pl.ns, nr, V, ldv, shift, Q, ldq, pl.nepi);
    return;
  }
  make_w_kernel<<<std::min(8 * sm_count(), (int)(((size_t)op.n_pad * pl.kv + 255) / 256)), 256,
                  0, st>>>(V, op.n, k, ldv, (const float*)op.ra.p, op.n_pad, pl.kv,
                           (float*)t.w.p);
  KRR_CHECK_LAUNCH();
  run_core(t, st, op, pl, split, f16);
  const size_t total = (size_t)nr * k;
  tc_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      (const float*)t.part.p, pl.nchunk, op.n_pad, pl.kv, (const float*)op.ra.p, nr, k, V, ldv,
      shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

// The product kernel alone of plan `pl`: chunk sums of exp2(S) w into t.part
// from the weights already in t.w.
void run_core(TcState& t, cudaStream_t st, TcOperand& op, const Plan& pl, int split, int f16) {
  const int nkb = split ? 2 : op.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  TcParams p;
  p.n_rt = pl.n_rt;
  p.n_ct = pl.n_ct;
  p.nchunk = pl.nchunk;
  p.cpc = pl.cpc;
  p.nkb = nkb;
  p.a_res = a_res;
  p.ns = pl.ns > 0 ? pl.ns : default_ns(a_res);
  p.x3 = split;
  p.idesc = f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN);
  p.n_rpad = op.n_pad;
  p.w = (const float*)t.w.p;
  p.part = (float*)t.part.p;
  p.err = (int*)t.err.p;
  const int items = pl.n_rt * pl.nchunk;
  const int grid = std::min(items, sm_count());
  dispatch(pl.kv, st, op, p, grid, pl.kv == 1 ? pl.emu : 0);
}

// The fused product for a row set other than the columns (prediction, the
// gradient's cross terms): row tiles from `rop` (prepared with the columns'
// mean and scale, so xh_i.xh_j - nh_i/2 - nh_j/2 is still -c ||x_i - x_j||^2),
// column tiles from `cop`; the kernel is the same.
void run_fused_rows(TcState& t, cudaStream_t st, const TcOperand& rop, const TcOperand& cop,
                    int split, int f16, const float* V, int k, int ldv, double shift, float* Q,
                    int ldq) {
  const int kv = kv_bucket(k);
  const int n_rt = rop.n_pad / BM, n_ct = cop.n_pad / BN;
  const int req = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + req - 1) / req;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  ensure(t.w, (size_t)cop.n_pad * kv * 4);
  ensure(t.part, (size_t)nchunk * rop.n_pad * kv * 4);
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
  const int nkb = split ? 2 : cop.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  make_w_kernel<<<std::min(8 * sm_count(), (int)(((size_t)cop.n_pad * kv + 255) / 256)), 256, 0,
                  st>>>(V, cop.n, k, ldv, (const float*)cop.ra.p, cop.n_pad, kv, (float*)t.w.p);
  KRR_CHECK_LAUNCH();
  TcParams p;
  p.n_rt = n_rt;
  p.n_ct = n_ct;
  p.nchunk = nchunk;
  p.cpc = cpc;
  p.nkb = nkb;
  p.a_res = a_res;
  p.ns = default_ns(a_res);
  p.x3 = split;
  p.idesc = f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN);
  p.n_rpad = rop.n_pad;
  p.w = (const float*)t.w.p;
  p.part = (float*)t.part.p;
  p.err = (int*)t.err.p;
  TcOperand mix;   // row maps of rop, column maps of cop
  mix.map_a = rop.map_a;
  mix.map_a2 = rop.map_a2;
  mix.map_b = cop.map_b;
  mix.map_b2 = cop.map_b2;
  const int grid = std::min(n_rt * nchunk, sm_count());
  dispatch(kv, st, mix, p, grid, 0);
  const size_t total = (size_t)rop.n * k;
  tc_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      (const float*)t.part.p, nchunk, rop.n_pad, kv, (const float*)rop.ra.p, rop.n, k, V, ldv,
      shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

// Q = (D o K(Xr, Xc)) V, D_ij = ||x_i - x_j||^2 / sigma^2 = -2 ln 2 log2 K_ij
// (the derivative of K in log sigma) on the rounded points of format fmt, in
// blocks of up to five right-hand sides (three weight columns each).
void run_dsigma(TcState& t, cudaStream_t st, const TcOperand& rop, const TcOperand& cop,
                int split, int f16, const float* V, int k, int ldv, float* Q, int ldq) {
  const int n_rt = rop.n_pad / BM, n_ct = cop.n_pad / BN;
  const int req = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + req - 1) / req;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  const int nkb = split ? 2 : cop.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  TcOperand mix;
  mix.map_a = rop.map_a;
  mix.map_a2 = rop.map_a2;
  mix.map_b = cop.map_b;
  mix.map_b2 = cop.map_b2;
  for (int c0 = 0; c0 < k; c0 += 5) {
    const int kb = std::min(5, k - c0);
    const int kv = kv_bucket(3 * kb);
    ensure(t.w, (size_t)cop.n_pad * kv * 4);
    ensure(t.part, (size_t)nchunk * rop.n_pad * kv * 4);
    if (!t.err.p) {
      ensure(t.err, 16);
      KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
    }
    make_w_ds_kernel<<<std::min(8 * sm_count(), (int)(((size_t)cop.n_pad * kv + 255) / 256)),
                       256, 0, st>>>(V, cop.n, kb, c0, ldv, (const float*)cop.ra.p,
                                     (const float*)cop.nh.p, cop.n_pad, kv, (float*)t.w.p);
    KRR_CHECK_LAUNCH();
    TcParams p;
    p.n_rt = n_rt;
    p.n_ct = n_ct;
    p.nchunk = nchunk;
    p.cpc = cpc;
    p.nkb = nkb;
    p.a_res = a_res;
    p.ns = default_ns(a_res);
    p.x3 = split;
    p.idesc = f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN);
    p.n_rpad = rop.n_pad;
    p.w = (const float*)t.w.p;
    p.part = (float*)t.part.p;
    p.err = (int*)t.err.p;
    p.ds_k = kb;
    dispatch_ds(kv, st, mix, p, std::min(n_rt * nchunk, sm_count()));
    const size_t total = (size_t)rop.n * kb;
    ds_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
        (const float*)t.part.p, nchunk, rop.n_pad, kv, kb, (const float*)rop.ra.p,
        (const float*)rop.nh.p, rop.n, c0, Q, ldq);
    KRR_CHECK_LAUNCH();
  }
}

// Q = P V + shift V for the polynomial kernel P_ij = (gamma xh_i.xh_j + c)^q
// on the rounded points of `op` (ra = 1): the fused kernel in its polynomial
// mode, the same tiles and pipeline as the Gaussian product.
void run_poly(TcState& t, cudaStream_t st, const TcOperand& op, int split, int f16, double gamma,
              double c, int q, const float* V, int k, int ldv, double shift, float* Q, int ldq) {
  const int kv = k <= 1 ? 1 : (k <= 4 ? 4 : 16);
  const int n_rt = op.n_pad / BM, n_ct = op.n_pad / BN;
  const int req = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + req - 1) / req;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  ensure(t.w, (size_t)op.n_pad * kv * 4);
  ensure(t.part, (size_t)nchunk * op.n_pad * kv * 4);
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
  const int nkb = split ? 2 : op.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  make_w_kernel<<<std::min(8 * sm_count(), (int)(((size_t)op.n_pad * kv + 255) / 256)), 256, 0,
                  st>>>(V, op.n, k, ldv, (const float*)op.ra.p, op.n_pad, kv, (float*)t.w.p);
  KRR_CHECK_LAUNCH();
  TcParams p;
  p.n_rt = n_rt;
  p.n_ct = n_ct;
  p.nchunk = nchunk;
  p.cpc = cpc;
  p.nkb = nkb;
  p.a_res = a_res;
  p.ns = default_ns(a_res);
  p.x3 = split;
  p.idesc = f16 ? idesc_f16(BM, BN) : idesc_bf16(BM, BN);
  p.n_rpad = op.n_pad;
  p.w = (const float*)t.w.p;
  p.part = (float*)t.part.p;
  p.err = (int*)t.err.p;
  p.pg = (float)gamma;
  p.pc = (float)c;
  p.pq = q;
  dispatch_poly(kv, st, op, p, std::min(n_rt * nchunk, sm_count()));
  const size_t total = (size_t)op.n * k;
  tc_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      (const float*)t.part.p, nchunk, op.n_pad, kv, (const float*)op.ra.p, op.n, k, V, ldv,
      shift, Q, ldq);
  KRR_CHECK_LAUNCH();
}

// Time the candidate plans of one shape on the prepared operand (scratch
// right-hand sides) and return the fastest.
Tuned tune_shape(TcState& t, cudaStream_t st, TcOperand& op, int k, int fmt) {
  const int split = fmt == 1, f16 = fmt == 2;
  const int nkb = split ? 2 : op.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  const Plan base = plan_for(op, k, 0);
  ensure(t.tune_v, (size_t)op.n * k * 4);
  ensure(t.tune_q, (size_t)op.n * k * 4);
  KRR_CUDA(cudaMemsetAsync(t.tune_v.p, 0, (size_t)op.n * k * 4, st));
  std::vector<int> reqs;
  const int cand[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  std::vector<int> seen;
  for (int r : cand) {
    const Plan pl = plan_for(op, k, 0, r);
    if (std::find(seen.begin(), seen.end(), pl.nchunk) != seen.end()) continue;
    seen.push_back(pl.nchunk);
    reqs.push_back(r == 0 ? base.nchunk : r);
  }
  std::vector<Plan> plans;
  for (int r : reqs)
    for (int ns = 2; ns <= NS_MAX; ++ns) {
      if (smem_for(base.kv, a_res, ns, split) > SMEM_LIMIT) continue;
      for (int emu : {0, 2, 4}) {
        if (emu && base.kv != 1) continue;
        Plan pl = plan_for(op, k, 0, r);
        pl.ns = ns;
        pl.emu = emu;
        plans.push_back(pl);
      }
    }
  if (sym_supported(op, k, split))
    for (int nepi : {8, 16})
      for (int C : {8, 16, 32, 64})
        for (int ns : {3, 4, 6}) {
          Plan pl = base;
          pl.sym = 1;
          pl.C = C;
          pl.ns = ns;
          pl.nepi = nepi;
          plans.push_back(pl);
        }
  cudaEvent_t e0, e1;
  KRR_CUDA(cudaEventCreate(&e0));
  KRR_CUDA(cudaEventCreate(&e1));
  Tuned best{0, default_ns(a_res), 0, 16, 0, 1e30f, 16};
  try {
    for (const Plan& pl : plans) {
      if (pl.sym)
        sym_reserve(t, st, op, pl.C);
      else
        ensure(t.part, (size_t)pl.nchunk * op.n_pad * pl.kv * 4);
      float ms = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        KRR_CUDA(cudaEventRecord(e0, st));
        run_fused(t, st, op, pl, split, f16, op.n, (const float*)t.tune_v.p, k, k, 0.0,
                  (float*)t.tune_q.p, k);
        KRR_CUDA(cudaEventRecord(e1, st));
        KRR_CUDA(cudaEventSynchronize(e1));
        float m = 0.f;
        KRR_CUDA(cudaEventElapsedTime(&m, e0, e1));
        if (rep > 0) ms = std::min(ms, m);   // the first run is a warm-up
      }
      if (getenv("KRR_TRACE"))
        fprintf(stderr,
                "[krr] autotune n_pad=%d kp=%d k=%d fmt=%d: %s chunks=%d C=%d ns=%d emu=%d "
                "%.4f ms\n",
                op.n_pad, op.kp, k, fmt, pl.sym ? "sym" : "full", pl.nchunk, pl.C, pl.ns, pl.emu,
                ms);
      if (ms < best.ms) best = Tuned{pl.req, pl.ns, pl.sym, pl.C, pl.emu, ms, pl.nepi};
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// The plan of the fused product for this shape: the tuned one when the
// handle autotunes (timing it now unless the stream is being captured), else
// the wave-balance rule.
Plan resolve_plan(TcState& t, cudaStream_t st, TcOperand& op, int k, int gemm2, int fmt) {
  // the symmetric kernel is a tuner candidate only: at n = 65,536 it
  // measures 0.845 ms (16 epilogue warps) against 0.676 ms for this kernel
  Plan pl = plan_for(op, k, gemm2);
  if (!gemm2 && (t.autotune == 2 || t.autotune == 3) && sym_supported(op, k, fmt == 1)) {
    pl.sym = 1;   // asked for explicitly: 16 (mode 2) or 8 (mode 3) epilogue warps
    pl.C = 32;
    pl.ns = 6;
    pl.nepi = t.autotune == 2 ? 16 : 8;
    return pl;
  }
  if (gemm2 || t.autotune != 1) return pl;
  const int nkb = fmt == 1 ? 2 : op.kp / BK;
  const TuneKey key{pl.n_rt, pl.n_ct, nkb, pl.kv, fmt};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      Plan q = plan_for(op, k, 0, it->second.req);
      q.ns = it->second.ns;
      q.sym = it->second.sym;
      q.C = it->second.C;
      q.emu = it->second.emu;
      q.nepi = it->second.nepi;
      return q;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KRR_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return pl;
  const Tuned tu = tune_shape(t, st, op, k, fmt);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = tu;
  }
  Plan q = plan_for(op, k, 0, tu.req);
  q.ns = tu.ns;
  q.sym = tu.sym;
  q.C = tu.C;
  q.emu = tu.emu;
  q.nepi = tu.nepi;
  return q;
}

}  // namespace

void tc_set_autotune(TcState& t, int mode) { t.autotune = mode; }

int tc_tuned_shapes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tuned.size();
}

void tc_reserve(TcState& t, cudaStream_t st, int k, int gemm2, int fmt) {
  if (!t.ready) throw Error{KRR_EINVAL, "tensor-core product used before tc_prepare"};
  TcOperand* op = &operand_of(t, fmt);
  int f = fmt;
  if (op->n_pad == 0) {  // that operand set is not prepared yet: size for the plain one
    op = &t.cols;
    f = 0;
  }
  const Plan pl = resolve_plan(t, st, *op, k, gemm2, f);
  if (pl.sym) sym_reserve(t, st, *op, pl.C);
  ensure(t.w, (size_t)t.cols.n_pad * pl.kv * 4);
  ensure(t.part, (size_t)pl.nchunk * t.cols.n_pad * pl.kv * 4);
  if (gemm2 && t.vt.bytes < (size_t)N2 * t.cols.n_pad * 2) {
    ensure(t.vt, (size_t)N2 * t.cols.n_pad * 2);
    make_vt_map(&t.map_v, t.vt.p, t.cols.n_pad);
  }
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
}

void tc_clear_error(TcState& t, cudaStream_t st) {
  if (t.err.p) KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
}

void tc_matvec(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
               int nc, int ldxc, int d, double sigma, double shift, const float* V, int k,
               int ldv, float* Q, int ldq, int split, int gemm2, int f16) {
  const bool same = (Xr == Xc && nr == nc && ldxr == ldxc);
  if (!same && gemm2)
    throw Error{KRR_EUNSUPPORTED, "two-GEMM product: the training system only (Xr == Xc)"};
  if (f16 && (split || gemm2))
    throw Error{KRR_EUNSUPPORTED, "FP16 points: plain product only (no split, no second GEMM)"};
  if (split)
    tc_prepare_split(t, st, Xc, nc, ldxc, d, sigma);
  else if (f16)
    tc_prepare_f16(t, st, Xc, nc, ldxc, d, sigma);
  else
    tc_prepare(t, st, Xc, nc, ldxc, d, sigma);
  const int fmt = split ? 1 : (f16 ? 2 : 0);
  if (!same) {
    tc_prepare_rows(t, st, Xr, nr, ldxr, d, sigma, fmt);
    run_fused_rows(t, st, t.rows, operand_of(t, fmt), split, f16, V, k, ldv, shift, Q, ldq);
    return;
  }
  tc_reserve(t, st, k, gemm2, fmt);
  TcOperand& op = operand_of(t, fmt);
  const Plan pl = resolve_plan(t, st, op, k, gemm2, fmt);
  // split points: the row tile's hi and lo stay resident, each column tile
  // streams its hi and lo slices as two stages
  const int nkb = split ? 2 : op.kp / BK;
  const int a_res = (split || nkb == 1) ? 1 : 0;
  if (gemm2) {
    make_vt_kernel<<<std::min(8 * sm_count(), (int)(((size_t)N2 * op.n_pad + 255) / 256)), 256,
                     0, st>>>(V, nc, k, ldv, (const float*)op.ra.p, op.n_pad,
                              (__nv_bfloat16*)t.vt.p);
    KRR_CHECK_LAUNCH();
    Tc2Params p2;
    p2.n_rt = pl.n_rt;
    p2.n_ct = pl.n_ct;
    p2.nchunk = pl.nchunk;
    p2.cpc = pl.cpc;
    p2.nkb = nkb;
    p2.n_rpad = op.n_pad;
    p2.kv = pl.kv;
    p2.a_res = a_res;
    p2.ns = a_res ? 4 : 3;
    p2.x3 = split;
    p2.part = (float*)t.part.p;
    p2.err = (int*)t.err.p;
    const int grid2 = std::min(pl.n_rt * pl.nchunk, sm_count());
    launch_kernel2(st, op.map_a, op.map_a2, t.map_v, p2, grid2);
    const size_t total2 = (size_t)nr * k;
    tc_reduce_kernel<<<std::min(8 * sm_count(), (int)((total2 + 255) / 256)), 256, 0, st>>>(
        (const float*)t.part.p, pl.nchunk, op.n_pad, pl.kv, (const float*)op.ra.p, nr, k, V, ldv,
        shift, Q, ldq);
    KRR_CHECK_LAUNCH();
    return;
  }
  run_fused(t, st, op, pl, split, f16, nr, V, k, ldv, shift, Q, ldq);
}

bool tc_loop_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                     double sigma, int k, int split, int f16, TcLoop* out) {
  if (f16 && split) return false;
  if (split)
    tc_prepare_split(t, st, X, n, ldx, d, sigma);
  else if (f16)
    tc_prepare_f16(t, st, X, n, ldx, d, sigma);
  else
    tc_prepare(t, st, X, n, ldx, d, sigma);
  const int fmt = split ? 1 : (f16 ? 2 : 0);
  tc_reserve(t, st, k, 0, fmt);
  TcOperand& op = operand_of(t, fmt);
  const Plan pl = resolve_plan(t, st, op, k, 0, fmt);
  if (pl.sym) return false;
  out->ra = (const float*)op.ra.p;
  out->w = (float*)t.w.p;
  out->part = (const float*)t.part.p;
  out->n_pad = op.n_pad;
  out->kv = pl.kv;
  out->nchunk = pl.nchunk;
  return true;
}

void tc_loop_product(TcState& t, cudaStream_t st, int k, int split, int f16) {
  const int fmt = split ? 1 : (f16 ? 2 : 0);
  TcOperand& op = operand_of(t, fmt);
  const Plan pl = resolve_plan(t, st, op, k, 0, fmt);
  if (pl.sym) throw Error{KRR_EINVAL, "loop product: the plan changed since tc_loop_prepare"};
  run_core(t, st, op, pl, split, f16);
}

void tc_dsigma_matvec(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr,
                      const float* Xc, int nc, int ldxc, int d, double sigma, const float* V,
                      int k, int ldv, float* Q, int ldq, int split, int f16) {
  if (f16 && split) throw Error{KRR_EUNSUPPORTED, "FP16 points: no split form"};
  if (split)
    tc_prepare_split(t, st, Xc, nc, ldxc, d, sigma);
  else if (f16)
    tc_prepare_f16(t, st, Xc, nc, ldxc, d, sigma);
  else
    tc_prepare(t, st, Xc, nc, ldxc, d, sigma);
  const int fmt = split ? 1 : (f16 ? 2 : 0);
  TcOperand& cop = operand_of(t, fmt);
  const bool same = (Xr == Xc && nr == nc && ldxr == ldxc);
  if (!same) tc_prepare_rows(t, st, Xr, nr, ldxr, d, sigma, fmt);
  run_dsigma(t, st, same ? cop : t.rows, cop, split, f16, V, k, ldv, Q, ldq);
}

void tc_poly_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d, int fmt) {
  if (fmt == 1 && d > BK) throw Error{KRR_EUNSUPPORTED, "split BF16 product needs d <= 64"};
  TcOperand& op = t.poly;
  if (t.poly_fmt == fmt && op.src == X && op.n == n && op.ld == ldx && op.d == d) return;
  t.poly_fmt = -1;
  ensure(t.mu0, (size_t)d * sizeof(double));
  KRR_CUDA(cudaMemsetAsync(t.mu0.p, 0, (size_t)d * sizeof(double), st));
  prep_operand(op, st, X, n, ldx, d, (const double*)t.mu0.p, 1.0, fmt == 1, fmt == 2);
  unit_rows_kernel<<<std::min(8 * sm_count(), (op.n_pad + 255) / 256), 256, 0, st>>>(
      (float*)op.ra.p, n, op.n_pad);
  KRR_CHECK_LAUNCH();
  ensure(t.scal, 16);
  KRR_CUDA(cudaMemsetAsync(t.scal.p, 0, 16, st));
  max_kernel<<<std::min(8 * sm_count(), (op.n_pad + 255) / 256), 256, 0, st>>>(
      (const float*)op.nh.p, op.n_pad, (float*)t.scal.p);
  KRR_CHECK_LAUNCH();
  float mx = 0.f;
  KRR_CUDA(cudaMemcpyAsync(&mx, t.scal.p, sizeof(float), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  if (!std::isfinite(mx))
    throw Error{KRR_EUNSUPPORTED,
                "polynomial tensor-core product: a point overflows the 16-bit format; use FP64"};
  t.poly_fmt = fmt;
}

void tc_poly_reserve(TcState& t, cudaStream_t st, int k) {
  if (t.poly_fmt < 0) throw Error{KRR_EINVAL, "polynomial product reserved before its operand"};
  const TcOperand& op = t.poly;
  const int kv = k <= 1 ? 1 : (k <= 4 ? 4 : 16);
  const int n_rt = op.n_pad / BM, n_ct = op.n_pad / BN;
  const int req = choose_nchunk(n_rt, n_ct, sm_count());
  const int cpc = (n_ct + req - 1) / req;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  ensure(t.w, (size_t)op.n_pad * kv * 4);
  ensure(t.part, (size_t)nchunk * op.n_pad * kv * 4);
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
}

void tc_poly_matvec(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                    double gamma, double c, int q, double shift, const float* V, int k, int ldv,
                    float* Q, int ldq, int split, int f16) {
  if (f16 && split) throw Error{KRR_EUNSUPPORTED, "FP16 points: no split form"};
  tc_poly_prepare(t, st, X, n, ldx, d, split ? 1 : (f16 ? 2 : 0));
  run_poly(t, st, t.poly, split, f16, gamma, c, q, V, k, ldv, shift, Q, ldq);
}

int tc_error(TcState& t, cudaStream_t st) {
  if (!t.err.p) return 0;
  int e = 0;
  KRR_CUDA(cudaMemcpyAsync(&e, t.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  return e;
}

void tc_release(TcState& t) {
  DevBuf* bufs[] = {&t.cols.Xa, &t.cols.ra, &t.cols.nh, &t.mu,        &t.scal,
                    &t.w,       &t.part,    &t.err,     &t.vt,        &t.split.Xa,
                    &t.split.Xlo, &t.split.ra, &t.split.nh, &t.half.Xa,   &t.half.ra,
                    &t.half.nh, &t.tune_v,  &t.tune_q,  &t.sym_rowpart, &t.sym_colpart,
                    &t.sym_items, &t.rows.Xa, &t.rows.Xlo, &t.rows.ra, &t.rows.nh,
                    &t.poly.Xa, &t.poly.Xlo, &t.poly.ra, &t.poly.nh, &t.mu0};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  t = TcState();
}

}  // namespace krr
