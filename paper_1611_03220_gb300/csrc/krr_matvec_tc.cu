// Fused kernel-matrix product on the 5th-generation tensor cores (tcgen05).
//
//   q_i = sum_j exp(-||x_i - x_j||^2 / (2 sigma^2)) v_j  (+ shift v_i)
//
// the per-iteration cost the paper names dominant (Section 3.1), for the
// Gaussian kernel of its experiments (Section 5); K is never written.
//
// Arithmetic.  With c = log2(e) / (2 sigma^2) and xh_i = bf16(sqrt(2c)(x_i - mu))
// (mu the column mean of the column set; the kernel is shift invariant),
//   -c ||x_i - x_j||^2  ~=  xh_i.xh_j - nh_i/2 - nh_j/2,   nh_i = ||xh_i||^2,
// so   K_ij = exp2(xh_i.xh_j) * ra_i * ra_j  with ra_i = exp2(-nh_i / 2).
// The tensor core forms S_ij = xh_i.xh_j (BF16 x BF16 products are exact in
// FP32; FP32 accumulation in TMEM), the epilogue evaluates exp2 on the MUFU
// and contracts against w_j = ra_j v_j, and ra_i scales the finished row
// sum.  This is the Gaussian kernel of the BF16-rounded points xh: the
// product stays a (symmetric positive semi-definite) kernel matrix, and the
// rounding error is what the outer refinement removes.  exp2(S) must not
// overflow: the host requires max nh <= 120.
//
// Structure (one persistent CTA per SM, 320 threads):
//   warp 0     TMA producer: per 128 x 256 tile, K-blocks of 64 BF16 of the
//              row tile (A) and the column tile (B) into a ring of NS stages
//              (128-byte swizzle), plus the tile's w block by bulk copy.
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//              and one thread issues tcgen05.mma (M=128, N=256, K=16).
//   warps 2-9  epilogue: tcgen05.ld 32 columns at a time, ex2, FMA with w.
//              Warp w reads TMEM lanes 32*(w%4)..+31 (its row quadrant) and
//              columns 128*((w-2)/4)..+127.
// Work items are (row tile, column chunk) pairs dealt round-robin; each item
// writes one partial row sum per chunk, and a second kernel adds the chunks
// in FP64, applies ra_i and the shift.  Every mbarrier wait is bounded: on
// expiry the kernel raises an error flag, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>

#include <cmath>
#include <cstring>

#include "krr_tc.cuh"

namespace krr {
namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int UK = 16;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_EPI = 8;
constexpr int THREADS = 32 * (2 + NUM_EPI);
constexpr int TMEM_COLS = 512;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

constexpr uint32_t IDESC = (1u << 4)                       // D: FP32
                           | (1u << 7)                     // A: BF16
                           | (1u << 10)                    // B: BF16
                           | ((uint32_t)(BN >> 3) << 17)   // N
                           | ((uint32_t)(BM >> 4) << 24);  // M

struct TcParams {
  int n_rt, n_ct, nchunk, cpc, nkb;
  int n_rpad;
  const float* w;   // n_ct*BN x KV
  float* part;      // nchunk x n_rpad x KV
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false (and the CTA abort flag set) when the limit is hit.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 1023u) == 1023u && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(err, 1);
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"((uint64_t)src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NUM_EPI * 32) : "memory");
}

// Barrier over the epilogue warps that also ORs a predicate across them, so
// every epilogue warp takes the same decision to leave the item loop.
__device__ __forceinline__ int epi_bar_or(int pred) {
  int out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}\n"
      : "=r"(out)
      : "r"(pred), "n"(NUM_EPI * 32)
      : "memory");
  return out;
}

template <int KV, int NS>
__global__ void __launch_bounds__(THREADS, 1)
tc_matvec_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 TcParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = smem;
  float* wbuf = (float*)(smem + NS * STAGE_BYTES);                // 2 x BN x KV
  float* comb = wbuf + 2 * BN * KV;                               // BM x KV
  uint64_t* bars = (uint64_t*)(comb + BM * KV);
  uint64_t* full = bars;
  uint64_t* empty = bars + NS;
  uint64_t* tfull = bars + 2 * NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* wfull = tempty + 2;
  uint64_t* wempty = wfull + 2;
  uint64_t* drain = wempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.n_rt * p.nchunk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), NUM_EPI);
      mbar_init(smem_u32(&wfull[s]), 1);
      mbar_init(smem_u32(&wempty[s]), NUM_EPI);
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t st = 0, ph = 0, ws = 0, wph = 0;
      uint32_t issued = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int rt = item / p.nchunk, ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&wempty[ws]), wph ^ 1, abort_flag, p.err))) break;
          mbar_expect_tx(smem_u32(&wfull[ws]), BN * KV * 4);
          bulk_load(smem_u32(wbuf + ws * BN * KV), p.w + (size_t)ct * BN * KV, BN * KV * 4,
                    smem_u32(&wfull[ws]));
          ws ^= 1;
          if (ws == 0) wph ^= 1;
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
            const uint32_t sa = smem_u32(stages + st * STAGE_BYTES);
            mbar_expect_tx(smem_u32(&full[st]), STAGE_BYTES);
            tma_load_2d(sa, &tmA, kb * BK, rt * BM, smem_u32(&full[st]));
            tma_load_2d(sa + A_BYTES, &tmB, kb * BK, ct * BN, smem_u32(&full[st]));
            ++issued;
            if (++st == NS) {
              st = 0;
              ph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // drain: wait for the copies of the last (up to NS) stages to land
        uint32_t s2 = st, p2 = ph;
        for (uint32_t q = 0; q < (issued < (uint32_t)NS ? issued : (uint32_t)NS); ++q) {
          if (s2 == 0) {
            s2 = NS - 1;
            p2 ^= 1;
          } else {
            --s2;
          }
          for (uint32_t it = 0; it < WAIT_LIMIT && !mbar_try(smem_u32(&full[s2]), p2); ++it) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t st = 0, ph = 0, acc = 0, aph = 0;
      bool ok = true;
      bool any = false;
      for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
        const int ch = item % p.nchunk;
        const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          const uint32_t d = tmem + acc * BN;
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
            fence_after();
            const uint32_t sa = smem_u32(stages + st * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk) {
              mma_bf16(d, sdesc(sa + kk * UK * 2), sdesc(sa + A_BYTES + kk * UK * 2),
                       (kb > 0 || kk > 0) ? 1u : 0u);
            }
            any = true;
            mma_commit(smem_u32(&empty[st]));
            if (++st == NS) {
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
      // make sure every issued MMA has finished before TMEM is released
      if (any) {
        mma_commit(smem_u32(drain));
        for (uint32_t it = 0; it < WAIT_LIMIT && !mbar_try(smem_u32(drain), 0); ++it) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    uint32_t acc = 0, aph = 0, ws = 0, wph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
      const int rt = item / p.nchunk, ch = item % p.nchunk;
      const int ct0 = ch * p.cpc, ct1 = min(p.n_ct, ct0 + p.cpc);
      float q[KV];
#pragma unroll
      for (int c = 0; c < KV; ++c) q[c] = 0.f;
      for (int ct = ct0; ok && ct < ct1; ++ct) {
        if (!(ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        if (!(ok = mbar_wait(smem_u32(&wfull[ws]), wph, abort_flag, p.err))) break;
        fence_after();
        const float* wb = wbuf + ws * BN * KV;
#pragma unroll 1
        for (int cc = 0; cc < 4; ++cc) {
          const int col0 = half * 128 + cc * 32;
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + acc * BN + col0, v);
          if (cc == 3) {
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float e = ex2(v[j]);
            const float* wj = wb + (col0 + j) * KV;
#pragma unroll
            for (int c = 0; c < KV; ++c) q[c] = fmaf(e, wj[c], q[c]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&wempty[ws]));
        acc ^= 1;
        if (acc == 0) aph ^= 1;
        ws ^= 1;
        if (ws == 0) wph ^= 1;
      }
      // combine the two column halves and write this item's partial sums
      if (half == 1) {
#pragma unroll
        for (int c = 0; c < KV; ++c) comb[row * KV + c] = q[c];
      }
      epi_bar();
      if (half == 0 && ok) {
        float* out = p.part + ((size_t)ch * p.n_rpad + (size_t)rt * BM + row) * KV;
#pragma unroll
        for (int c = 0; c < KV; ++c) out[c] = q[c] + comb[row * KV + c];
      }
      if (epi_bar_or(!ok || *abort_flag)) break;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ helpers ----
// xh = bf16(scale (x - mu)) padded to n_pad x kp, nh = ||xh||^2, ra = exp2(-nh/2).
__global__ void prep_rows_kernel(const float* __restrict__ X, int n, int ld, int d,
                                 const double* __restrict__ mu, double scale, int n_pad, int kp,
                                 __nv_bfloat16* __restrict__ Xa, float* __restrict__ ra,
                                 float* __restrict__ nh_out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n_pad) return;
  const int i = warp;
  double nh = 0.0;
  for (int t = lane; t < kp; t += 32) {
    float v = 0.f;
    if (i < n && t < d) v = (float)(scale * ((double)X[(size_t)i * ld + t] - mu[t]));
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    Xa[(size_t)i * kp + t] = b;
    double bv = (double)__bfloat162float(b);
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
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    KRR_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                              cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
      throw Error{KRR_ECUDA, "cuTensorMapEncodeTiled entry point not found"};
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

void make_map(CUtensorMap* m, const void* base, int rows, int kp, int box_rows) {
  cuuint64_t gdim[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                           gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{KRR_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
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

template <int KV, int NS>
size_t smem_bytes() {
  return 1024 + (size_t)NS * STAGE_BYTES + (size_t)2 * BN * KV * 4 + (size_t)BM * KV * 4 + 256;
}

template <int KV, int NS>
void launch_kernel(cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b, const TcParams& p,
                   int grid) {
  static bool attr = false;
  const size_t sm = smem_bytes<KV, NS>();
  if (!attr) {
    KRR_CUDA(cudaFuncSetAttribute(tc_matvec_kernel<KV, NS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  tc_matvec_kernel<KV, NS><<<grid, THREADS, sm, st>>>(a, b, p);
  KRR_CHECK_LAUNCH();
}

void dispatch(int kv, cudaStream_t st, const CUtensorMap& a, const CUtensorMap& b,
              const TcParams& p, int grid) {
  switch (kv) {
    case 1: launch_kernel<1, 4>(st, a, b, p, grid); break;
    case 2: launch_kernel<2, 4>(st, a, b, p, grid); break;
    case 4: launch_kernel<4, 4>(st, a, b, p, grid); break;
    case 8: launch_kernel<8, 3>(st, a, b, p, grid); break;
    case 12: launch_kernel<12, 3>(st, a, b, p, grid); break;
    default: launch_kernel<16, 3>(st, a, b, p, grid); break;
  }
}

// Prepare one operand set (rows or columns) into `op`.
void prep_operand(TcOperand& op, cudaStream_t st, const float* X, int n, int ld, int d,
                  const double* mu, double scale) {
  const int kp = (d + BK - 1) / BK * BK;
  const int n_pad = (n + BN - 1) / BN * BN;
  ensure(op.Xa, (size_t)n_pad * kp * 2);
  ensure(op.ra, (size_t)n_pad * 4);
  ensure(op.nh, (size_t)n_pad * 4 + 16);
  prep_rows_kernel<<<(n_pad * 32 + 255) / 256, 256, 0, st>>>(
      X, n, ld, d, mu, scale, n_pad, kp, (__nv_bfloat16*)op.Xa.p, (float*)op.ra.p,
      (float*)op.nh.p);
  KRR_CHECK_LAUNCH();
  op.src = X;
  op.n = n;
  op.ld = ld;
  op.d = d;
  op.kp = kp;
  op.n_pad = n_pad;
  make_map(&op.map_a, op.Xa.p, n_pad, kp, BM);
  make_map(&op.map_b, op.Xa.p, n_pad, kp, BN);
}

}  // namespace

void tc_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma) {
  const double c = 1.4426950408889634 / (2.0 * sigma * sigma);  // log2(e) / (2 sigma^2)
  const double scale = std::sqrt(2.0 * c);
  if (t.ready && t.cols.src == X && t.cols.n == n && t.cols.ld == ldx && t.cols.d == d &&
      t.sigma == sigma && t.rows_same)
    return;
  ensure(t.mu, (size_t)d * sizeof(double));
  ensure(t.w, (size_t)((n + 127) / 128) * d * sizeof(double));  // w doubles as the slab scratch
  launch_colmean(st, X, n, ldx, d, (double*)t.mu.p, (double*)t.w.p);
  prep_operand(t.cols, st, X, n, ldx, d, (const double*)t.mu.p, scale);
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
                "BF16 product: ||x - mean||^2 / (2 sigma^2) too large for the factored exp2 "
                "(max " + std::to_string(mx) + " in log2 units); use FP32 or FP64"};
  t.sigma = sigma;
  t.rows_same = true;
  t.ready = true;
}

void tc_matvec(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
               int nc, int ldxc, int d, double sigma, double shift, const float* V, int k,
               int ldv, float* Q, int ldq) {
  const bool same = (Xr == Xc && nr == nc && ldxr == ldxc);
  if (!same) throw Error{KRR_EUNSUPPORTED, "BF16 product supports the training system (Xr == Xc)"};
  tc_prepare(t, st, Xc, nc, ldxc, d, sigma);
  TcOperand& op = t.cols;
  const int kv = kv_bucket(k);
  const int grid_max = sm_count();
  const int n_rt = op.n_pad / BM, n_ct = op.n_pad / BN;
  const int nchunk_req = choose_nchunk(n_rt, n_ct, grid_max);
  const int cpc = (n_ct + nchunk_req - 1) / nchunk_req;
  const int nchunk = (n_ct + cpc - 1) / cpc;
  tc_reserve(t, st, k);
  make_w_kernel<<<std::min(8 * sm_count(), (int)(((size_t)op.n_pad * kv + 255) / 256)), 256, 0,
                  st>>>(V, nc, k, ldv, (const float*)op.ra.p, op.n_pad, kv, (float*)t.w.p);
  KRR_CHECK_LAUNCH();
  TcParams p;
  p.n_rt = n_rt;
  p.n_ct = n_ct;
  p.nchunk = nchunk;
  p.cpc = cpc;
  p.nkb = op.kp / BK;
  p.n_rpad = op.n_pad;
  p.w = (const float*)t.w.p;
  p.part = (float*)t.part.p;
  p.err = (int*)t.err.p;
  const int items = n_rt * nchunk;
  const int grid = std::min(items, grid_max);
  dispatch(kv, st, op.map_a, op.map_b, p, grid);
  const size_t total = (size_t)nr * k;
  tc_reduce_kernel<<<std::min(8 * sm_count(), (int)((total + 255) / 256)), 256, 0, st>>>(
      (const float*)t.part.p, nchunk, op.n_pad, kv, (const float*)op.ra.p, nr, k, V, ldv, shift,
      Q, ldq);
  KRR_CHECK_LAUNCH();
}

void tc_reserve(TcState& t, cudaStream_t st, int k) {
  const TcOperand& op = t.cols;
  if (!t.ready) throw Error{KRR_EINVAL, "tensor-core product used before tc_prepare"};
  const int kv = kv_bucket(k);
  const int n_rt = op.n_pad / BM, n_ct = op.n_pad / BN;
  const int cpc = (n_ct + choose_nchunk(n_rt, n_ct, sm_count()) - 1) /
                  choose_nchunk(n_rt, n_ct, sm_count());
  const int nchunk = (n_ct + cpc - 1) / cpc;
  ensure(t.w, (size_t)op.n_pad * kv * 4);
  ensure(t.part, (size_t)nchunk * op.n_pad * kv * 4);
  if (!t.err.p) {
    ensure(t.err, 16);
    KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
  }
}

void tc_clear_error(TcState& t, cudaStream_t st) {
  if (t.err.p) KRR_CUDA(cudaMemsetAsync(t.err.p, 0, 16, st));
}

int tc_error(TcState& t, cudaStream_t st) {
  if (!t.err.p) return 0;
  int e = 0;
  KRR_CUDA(cudaMemcpyAsync(&e, t.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  return e;
}

void tc_release(TcState& t) {
  DevBuf* bufs[] = {&t.cols.Xa, &t.cols.ra, &t.cols.nh, &t.mu, &t.scal, &t.w, &t.part, &t.err};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  t = TcState();
}

}  // namespace krr
