// Woodbury apply of the random-feature preconditioner (Section 3.1,
// Algorithm 1):
//   ZL form:  z = (r - Z L^-T L^-1 Z^T r) / lambda_p
//   U form:   z = (r - U^T U r) / lambda_p,   U = L^-1 Z^T
// The ZL form is four steps, each one pass over its operand:
//   zt_kernel    t = Z^T r      GEMV-T over the n x s matrix Z (split over
//                               row slabs; FP32/FP64 slab sums, FP64 merge)
//   sum_kernel   merge the slab partials in FP64
//   trmv_kernel  u = L^-1 t, w = L^-T u   (FP64, explicit inverse from set-up)
//   zw_kernel    z = (r - Z w) / lambda_p GEMV over Z with w staged in
//                               shared memory
// Both GEMVs stream Z once with 16-byte loads (16 fixed-point bytes, 8 BF16
// or 4 FP32 values), so the apply is bound by HBM: about 2 n s b_Z bytes per
// application.  Z is stored as FP32 (ZF = 0), BF16 (ZF = 1) or, for the
// fixed-point features of the mixed solves, 8-bit integers q with
// Z = q / 128 (ZF = 2, exact: the features are q / 128 by construction).
#include <algorithm>
#include <type_traits>

#include "krr_cgstep.cuh"

namespace krr {
namespace {

constexpr int AT = 256;        // threads per CTA
constexpr int ZT_ROWS = 64;    // R rows staged per slab step

int kv_of(int k) {
  if (k <= 1) return 1;
  if (k <= 2) return 2;
  if (k <= 4) return 4;
  if (k <= 8) return 8;
  if (k <= 12) return 12;
  return 16;
}

// Eight Z values from their storage: FP32, BF16 or 8-bit q / 128.
template <int ZF>
__device__ __forceinline__ float zval(const void* Zs, size_t off) {
  if (ZF == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Zs)[off]);
  if (ZF == 2) return (float)reinterpret_cast<const signed char*>(Zs)[off] * 0.0078125f;
  return reinterpret_cast<const float*>(Zs)[off];
}

// Eight consecutive 8-bit codes (one 8-byte word) as the floats q, without
// integer conversions: with the sign bit flipped a code is u = q + 128, the
// byte permute builds the float 2^23 + u, and one subtraction leaves q exactly.
__device__ __forceinline__ float q8f(uint32_t w, uint32_t i) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u + i)) - 8388736.f;
}
__device__ __forceinline__ void unpack_q8(uint2 v, float (&z)[8]) {
  const uint32_t a = v.x ^ 0x80808080u, b = v.y ^ 0x80808080u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    z[q] = q8f(a, q);
    z[4 + q] = q8f(b, q);
  }
}

// The same eight codes as four pairs (q[2p], q[2p + 1]) with paired FP32 adds:
// half the add instructions, and pairs the paired FMAs take directly.
__device__ __forceinline__ void unpack_q8x2(uint2 v, float2 (&z)[4]) {
  const uint32_t a = v.x ^ 0x80808080u, b = v.y ^ 0x80808080u;
  const float2 off = make_float2(-8388736.f, -8388736.f);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    z[p] = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(a, 0x4B000000u, 0x7540u + 2 * p)),
                                  __uint_as_float(__byte_perm(a, 0x4B000000u, 0x7541u + 2 * p))),
                      off);
    z[2 + p] = __fadd2_rn(
        make_float2(__uint_as_float(__byte_perm(b, 0x4B000000u, 0x7540u + 2 * p)),
                    __uint_as_float(__byte_perm(b, 0x4B000000u, 0x7541u + 2 * p))),
        off);
  }
}

// The scale between stage8's values and Z: 1/128 for the 8-bit codes (the
// streamed kernels apply it once to their sums), 1 otherwise.
template <int ZF>
__device__ __forceinline__ constexpr float zscale() { return ZF == 2 ? 0.0078125f : 1.f; }

// Eight consecutive Z values at byte address p of a stage (ZF storage); the
// 8-bit codes come back as q (multiply by zscale<ZF>() for Z).
template <int ZF>
__device__ __forceinline__ void stage8(const uint8_t* p, float (&z)[8]) {
  if (ZF == 1) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __bfloat1622float2(h2[q]);
      z[2 * q] = f.x;
      z[2 * q + 1] = f.y;
    }
  } else if (ZF == 2) {
    unpack_q8(*reinterpret_cast<const uint2*>(p), z);
  } else {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const float4 a = p4[0], b = p4[1];
    z[0] = a.x; z[1] = a.y; z[2] = a.z; z[3] = a.w;
    z[4] = b.x; z[5] = b.y; z[6] = b.z; z[7] = b.w;
  }
}

// Eight consecutive Z values starting at element `off` (n_ok of them valid).
template <int ZF>
__device__ __forceinline__ void load8(const void* Zs, size_t off, int n_ok, bool vec,
                                      float (&z)[8]) {
  if (vec && n_ok >= 8) {
    constexpr int ES = ZF == 1 ? 2 : (ZF == 2 ? 1 : 4);
    stage8<ZF>(reinterpret_cast<const uint8_t*>(Zs) + off * ES, z);
    if (ZF == 2) {
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] *= zscale<ZF>();
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) z[q] = q < n_ok ? zval<ZF>(Zs, off + q) : 0.f;
}

// part[chunk, col, c] = sum_{i in chunk} Z[i, col] R[i, c]; 8 columns per thread.
template <int ZF, typename T, typename ACC, int KV>
__global__ void __launch_bounds__(AT)
zt_kernel(const void* __restrict__ Zs, int n, int s, const T* __restrict__ R, int ldr, int k,
          ACC* __restrict__ part, int rpc, int vec) {
  __shared__ ACC rs[ZT_ROWS][KV];
  const int col0 = (blockIdx.x * AT + threadIdx.x) * 8;
  const int r0 = blockIdx.y * rpc, r1 = min(n, r0 + rpc);
  ACC acc[8][KV];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int c = 0; c < KV; ++c) acc[q][c] = (ACC)0;
  const int n_ok = s - col0;
  for (int base = r0; base < r1; base += ZT_ROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < ZT_ROWS * KV; e += AT) {
      const int rr = e / KV, c = e % KV, i = base + rr;
      rs[rr][c] = (i < r1 && c < k) ? (ACC)R[(size_t)i * ldr + c] : (ACC)0;
    }
    __syncthreads();
    if (n_ok > 0) {
      const int nrow = min(ZT_ROWS, r1 - base);
#pragma unroll 4
      for (int rr = 0; rr < nrow; ++rr) {
        float z[8];
        load8<ZF>(Zs, (size_t)(base + rr) * s + col0, n_ok, vec != 0, z);
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          const ACC rv = rs[rr][c];
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[q][c] = fma((ACC)z[q], rv, acc[q][c]);
        }
      }
    }
  }
  if (n_ok <= 0) return;
  ACC* out = part + (size_t)blockIdx.y * s * KV;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (q >= n_ok) break;
#pragma unroll
    for (int c = 0; c < KV; ++c) out[(size_t)(col0 + q) * KV + c] = acc[q][c];
  }
}

// t[col, c] = sum over chunks (FP64), for c < k (t has leading dimension k).
// A CTA owns 32 consecutive (col, c) entries of the partial rows; its 8
// warps take the chunks round-robin (coalesced 128-byte reads), and the 8
// per-warp sums are added in a fixed order.
template <typename P>
__global__ void __launch_bounds__(256)
sum_kernel(const P* __restrict__ part, int nchunk, int s, int kv, int k, double* __restrict__ t) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t row_len = (size_t)s * kv;
  const size_t e = (size_t)blockIdx.x * 32 + lane;  // index into a partial row
  double v = 0.0;
  if (e < row_len)
    for (int ch = w; ch < nchunk; ch += 8) v += (double)part[(size_t)ch * row_len + e];
  red[w][lane] = v;
  __syncthreads();
  if (w == 0 && e < row_len) {
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += red[q][lane];
    const size_t col = e / kv, c = e % kv;
    if ((int)c < k) t[col * k + c] = acc;
  }
}

// y[a, c] = sum_b A[a, b] x[b, c], b <= a (lower) or b >= a (upper).  A CTA
// takes two rows; four warps share a row (a quarter of its span each), every
// lane keeps eight loads in flight, and the quarters are added in order.
constexpr int TR_ROWS = 2;
constexpr int TR_SPLIT = (AT / 32) / TR_ROWS;

template <int UPPER, int KV>
__global__ void __launch_bounds__(AT)
trmv_kernel(const double* __restrict__ A, int s, const double* __restrict__ x, int k,
            double* __restrict__ y) {
  __shared__ double red[AT / 32][KV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.x * TR_ROWS + warp / TR_SPLIT;
  const int q = warp % TR_SPLIT;
  double acc[2][KV];
#pragma unroll
  for (int c = 0; c < KV; ++c) acc[0][c] = acc[1][c] = 0.0;
  if (a < s) {
    const int lo = UPPER ? a : 0, hi = UPPER ? s : a + 1;
    const int per = (hi - lo + TR_SPLIT - 1) / TR_SPLIT;
    const int qlo = lo + q * per, qhi = min(hi, qlo + per);
    const double* row = A + (size_t)a * s;
    // eight predicated loads in flight per lane, also on the short rows of
    // the triangle (a one-load-at-a-time tail made them latency-bound)
    for (int b = qlo + lane; b < qhi; b += 8 * 32) {
      double av[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = b + 32 * u < qhi ? __ldg(row + b + 32 * u) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < KV; ++c)
          if (c < k && b + 32 * u < qhi)
            acc[u & 1][c] = fma(av[u], __ldg(x + (size_t)(b + 32 * u) * k + c), acc[u & 1][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < KV; ++c) {
    double v = acc[0][c] + acc[1][c];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < TR_ROWS * KV) {
    const int r = threadIdx.x / KV, c = threadIdx.x % KV;
    const int row = blockIdx.x * TR_ROWS + r;
    if (row < s && c < k) {
      double v = 0.0;
      for (int w = 0; w < TR_SPLIT; ++w) v += red[r * TR_SPLIT + w][c];
      y[(size_t)row * k + c] = v;
    }
  }
}

// Zo[i, c] = (R[i, c] - sum_b Z[i, b] w[b, c]) / lambda_p.  Each warp owns 4
// rows; w is staged in shared memory in column chunks of `sch` (transposed,
// [c][b]), lanes take 8 consecutive columns.
constexpr int ZW_ROWS_PER_WARP = 4;
constexpr int ZW_ROWS = ZW_ROWS_PER_WARP * (AT / 32);

template <int ZF, typename T, typename ACC, int KV>
__global__ void __launch_bounds__(AT)
zw_kernel(const void* __restrict__ Zs, int n, int s, const double* __restrict__ w, int k,
          const T* __restrict__ R, int ldr, double inv_lam, T* __restrict__ Zo, int ldo, int sch,
          int vec) {
  extern __shared__ __align__(16) uint8_t zw_smem[];
  ACC* wsm = reinterpret_cast<ACC*>(zw_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * ZW_ROWS + warp * ZW_ROWS_PER_WARP;
  ACC acc[ZW_ROWS_PER_WARP][KV];
#pragma unroll
  for (int r = 0; r < ZW_ROWS_PER_WARP; ++r)
#pragma unroll
    for (int c = 0; c < KV; ++c) acc[r][c] = (ACC)0;
  for (int b0 = 0; b0 < s; b0 += sch) {
    const int nb = min(sch, s - b0);
    __syncthreads();
    // the whole chunk is written (zeros past nb) so no lane reads stale values
    for (int e = threadIdx.x; e < sch * KV; e += AT) {
      const int b = e / KV, c = e % KV;
      wsm[c * sch + b] = (c < k && b < nb) ? (ACC)w[(size_t)(b0 + b) * k + c] : (ACC)0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ZW_ROWS_PER_WARP; ++r) {
      const int i = row0 + r;
      if (i >= n) break;
      for (int bb = lane * 8; bb < nb; bb += 256) {
        float z[8];
        load8<ZF>(Zs, (size_t)i * s + b0 + bb, min(8, nb - bb), vec != 0, z);
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          const ACC* wc = wsm + c * sch + bb;
          ACC a = acc[r][c];
#pragma unroll
          for (int q = 0; q < 8; ++q) a = fma((ACC)z[q], wc[q], a);
          acc[r][c] = a;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < ZW_ROWS_PER_WARP; ++r) {
    const int i = row0 + r;
    if (i >= n) break;
#pragma unroll
    for (int c = 0; c < KV; ++c) {
      if (c >= k) break;
      ACC v = acc[r][c];
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0)
        Zo[(size_t)i * ldo + c] = (T)(((double)R[(size_t)i * ldr + c] - (double)v) * inv_lam);
    }
  }
}

// --------------------------------------------------- streamed GEMVs -------
// The same two GEMVs with Z streamed through shared memory by bulk copies
// (cp.async.bulk into a ring of 64 KiB stages, completion on mbarriers), so
// the bytes in flight per SM no longer depend on registers or occupancy.
// One persistent CTA per SM walks a contiguous range of rows.  Used when the
// rows' byte offsets are 16-byte aligned.
constexpr int SBYTES = 64 * 1024;   // bytes per stage
constexpr int NSTG = 3;             // stages
constexpr uint32_t APPLY_WAIT = 1u << 24;

__device__ __forceinline__ bool stg_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < APPLY_WAIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t sh_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Rows of stage g of a CTA that owns rows [r0, r1), rps rows a stage: first
// to last, or (rev) last to first.  zt walks its rows forwards and zw
// backwards, so zw starts on the rows that zt read last, which are still in
// L2 (Z is larger than L2, but only a little), and the next zt starts on the
// rows that zw read last.
__device__ __forceinline__ void stage_span(int g, int r0, int r1, int rps, bool rev, int& row0,
                                           int& nrow) {
  if (!rev) {
    row0 = r0 + g * rps;
    nrow = min(rps, r1 - row0);
  } else {
    const int hi = r1 - g * rps;
    row0 = max(r0, hi - rps);
    nrow = hi - row0;
  }
}

// Issue the copies of stage `st` (rows [row0, row0 + nrow), columns
// [c0, c0 + seg)) and return; thread 0 only.
__device__ __forceinline__ void stg_issue(uint8_t* ring, uint64_t* full, int st, const uint8_t* Z,
                                          size_t row_bytes, size_t c0_bytes, uint32_t seg_bytes,
                                          int row0, int nrow) {
  // the CTA's generic reads of the stage (ordered before this thread by the
  // barrier in front of a refill) before the async-proxy writes of the copy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const uint32_t bar = sh_u32(&full[st]);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(seg_bytes * (uint32_t)nrow)
               : "memory");
  if ((size_t)seg_bytes == row_bytes) {
    // whole rows: the stage is one contiguous block of Z, one copy (the
    // per-row copies kept thread 0 issuing 32 instructions per stage while
    // the other warps waited at the stage barrier)
    const uint8_t* src = Z + (size_t)row0 * row_bytes;
    const uint32_t dst = sh_u32(ring + (size_t)st * SBYTES);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"((uint64_t)src), "r"(seg_bytes * (uint32_t)nrow), "r"(bar)
        : "memory");
    return;
  }
  for (int rr = 0; rr < nrow; ++rr) {
    const uint8_t* src = Z + (size_t)(row0 + rr) * row_bytes + c0_bytes;
    const uint32_t dst = sh_u32(ring + (size_t)st * SBYTES + (size_t)rr * seg_bytes);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"((uint64_t)src), "r"(seg_bytes), "r"(bar)
        : "memory");
  }
}

// part[cta, col, c] = sum over the CTA's rows of Z[i, col] R[i, c]; thread t
// owns columns c0 + 8t .. c0 + 8t + 7 of the column block blockIdx.x.
// FUSE: R is the residual before the iteration's update; the kernel stages
// r' = r - alpha q instead (alpha from the CG scalars), and the CTAs of
// column block 0 also write x' = x + alpha p and r' (to f.Rn) and reduce
// ||r'||^2 (the stopping test), exactly as the separate x, r update kernel.
template <int ZF, typename T, typename ACC, int KV, int FUSE = 0>
__global__ void __launch_bounds__(AT, 1)
zt_stream_kernel(const void* __restrict__ Zs, int n, int s, const T* __restrict__ R, int ldr,
                 int k, ACC* __restrict__ part, int* err, CgStepArgs<T> f) {
  extern __shared__ __align__(128) uint8_t ring[];
  __shared__ __align__(8) uint64_t full[NSTG];
  constexpr int ES = ZF == 1 ? 2 : (ZF == 2 ? 1 : 4);
  const int cb = blockIdx.x;
  const int c0 = cb * AT * 8;
  const int seg = min(AT * 8, s - c0);                 // columns in this block (multiple of 8)
  const uint32_t seg_bytes = (uint32_t)seg * ES;
  const int rps = SBYTES / (int)seg_bytes;             // rows per stage
  const int rows_per_cta = (n + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  const int nstage = r0 < r1 ? (r1 - r0 + rps - 1) / rps : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTG; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_u32(&full[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int g = 0; g < NSTG && g < nstage; ++g)
      stg_issue(ring, full, g, (const uint8_t*)Zs, (size_t)s * ES, (size_t)c0 * ES, seg_bytes,
                r0 + g * rps, min(rps, r1 - r0 - g * rps));
  }
  // the CTA's rows of R, staged once (the per-row loads would each expose
  // a memory round trip)
  ACC* rsm = reinterpret_cast<ACC*>(ring + (size_t)NSTG * SBYTES);
  __shared__ double alpha_s[FUSE ? KRR_MAX_RHS : 1];
  double vr[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) vr[c] = 0.0;
  if (FUSE) {
    if (threadIdx.x < KRR_MAX_RHS)
      alpha_s[threadIdx.x] = (int)threadIdx.x < k ? f.sc->alpha[threadIdx.x] : 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < (r1 - r0) * KV; e += AT) {
    const int rr = e / KV, c = e % KV;
    ACC val = (ACC)0;
    if (r0 < r1 && c < k) {
      const size_t ei = (size_t)(r0 + rr) * ldr + c;
      if (FUSE) {
        double r = (double)R[ei];
        const double a = alpha_s[c];
        if (a != 0.0) {
          r = (double)(T)(r - a * (double)f.Q[ei]);
          if (blockIdx.x == 0) f.X[ei] = (T)((double)f.X[ei] + a * (double)f.P[ei]);
        }
        if (blockIdx.x == 0) {
          f.Rn[ei] = (T)r;
#pragma unroll
          for (int cc = 0; cc < KV; ++cc)
            if (cc == c) vr[cc] = fma(r, r, vr[cc]);
        }
        val = (ACC)r;
      } else {
        val = (ACC)R[ei];
      }
    }
    rsm[e] = val;
  }
  __syncthreads();
  if (FUSE && blockIdx.x == 0) {
    double tot[KRR_MAX_RHS];
    if (grid_colsum_nt<AT>(vr, k, f.cpart, &f.sc->counter[CGC_XR], blockIdx.y, gridDim.y, tot))
      cg_xr_finish(f.sc, tot, k);
  }
  const int col = threadIdx.x * 8;  // within the block
  const bool mine = col < seg;
  constexpr bool PACKED = ZF == 2 && std::is_same<ACC, float>::value;
  ACC acc[8][KV];
  float2 acc2[PACKED ? 4 : 1][KV];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int c = 0; c < KV; ++c) acc[q][c] = (ACC)0;
#pragma unroll
  for (int p = 0; p < (PACKED ? 4 : 1); ++p)
#pragma unroll
    for (int c = 0; c < KV; ++c) acc2[p][c] = make_float2(0.f, 0.f);
  bool ok = true;
  int g = 0;
  for (; g < nstage; ++g) {
    const int st = g % NSTG;
    const uint32_t parity = (uint32_t)((g / NSTG) & 1);
    ok = __syncthreads_and(ok && stg_wait(sh_u32(&full[st]), parity));
    if (!ok) break;
    const int row0 = r0 + g * rps, nrow = min(rps, r1 - row0);
    const uint8_t* base = ring + (size_t)st * SBYTES;
    if (mine) {
      if constexpr (PACKED) {
        // 8-bit codes, FP32 sums: paired adds and FMAs (the same operations
        // on the same values, half the instructions)
        for (int rr = 0; rr < nrow; ++rr) {
          float2 z2[4];
          unpack_q8x2(*reinterpret_cast<const uint2*>(base + (size_t)rr * seg_bytes + col), z2);
#pragma unroll
          for (int c = 0; c < KV; ++c) {
            const float rv = (float)rsm[(row0 - r0 + rr) * KV + c];
            const float2 r2 = make_float2(rv, rv);
#pragma unroll
            for (int p = 0; p < 4; ++p) acc2[p][c] = __ffma2_rn(z2[p], r2, acc2[p][c]);
          }
        }
      } else {
        for (int rr = 0; rr < nrow; ++rr) {
          float z[8];
          stage8<ZF>(base + (size_t)rr * seg_bytes + col * ES, z);
#pragma unroll
          for (int c = 0; c < KV; ++c) {
            const ACC rv = rsm[(row0 - r0 + rr) * KV + c];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q][c] = fma((ACC)z[q], rv, acc[q][c]);
          }
        }
      }
    }
    __syncthreads();  // every thread is done with the stage
    if (threadIdx.x == 0 && g + NSTG < nstage)
      stg_issue(ring, full, st, (const uint8_t*)Zs, (size_t)s * ES, (size_t)c0 * ES, seg_bytes,
                r0 + (g + NSTG) * rps, min(rps, r1 - r0 - (g + NSTG) * rps));
  }
  if (!ok) {
    // stages g .. g + NSTG - 1 may still have copies in flight: let them land
    if (threadIdx.x == 0) {
      atomicOr(err, 1);
      for (int gg = g; gg < nstage && gg < g + NSTG; ++gg)
        stg_wait(sh_u32(&full[gg % NSTG]), (uint32_t)((gg / NSTG) & 1));
    }
    return;
  }
  if (!mine) return;
  if constexpr (PACKED) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int c = 0; c < KV; ++c) {
        acc[2 * p][c] = acc2[p][c].x;
        acc[2 * p + 1][c] = acc2[p][c].y;
      }
  }
  ACC* out = part + (size_t)blockIdx.y * s * KV;
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int c = 0; c < KV; ++c)
      out[(size_t)(c0 + col + q) * KV + c] = acc[q][c] * (ACC)zscale<ZF>();
}

// Zo[i, c] = (R[i, c] - sum_b Z[i, b] w[b, c]) / lambda_p with whole rows of Z
// streamed; w (s x KV) in shared memory; each warp takes rows of a stage.
// Sixteen warps (one BF16 row each per 64 KiB stage): with eight, the
// shared-memory latency of each row's dot product set the pace.
constexpr int ZAT = 512;

// FUSE: R is the updated residual r' (f.Rn); the kernel also copies it to
// Rout, reduces r'.z and, in the last CTA, forms beta and the loop's continue
// decision, exactly as the separate r.z and tail kernels.
template <int ZF, typename T, typename ACC, int KV, int FUSE = 0>
__global__ void __launch_bounds__(ZAT, 1)
zw_stream_kernel(const void* __restrict__ Zs, int n, int s, const double* __restrict__ w, int k,
                 const T* __restrict__ R, int ldr, double inv_lam, T* __restrict__ Zo, int ldo,
                 int* err, T* __restrict__ Rout, CgStepArgs<T> f) {
  extern __shared__ __align__(128) uint8_t ring[];
  __shared__ __align__(8) uint64_t full[NSTG];
  constexpr int ES = ZF == 1 ? 2 : (ZF == 2 ? 1 : 4);
  ACC* wsm = reinterpret_cast<ACC*>(ring + (size_t)NSTG * SBYTES);  // [c][b]
  const uint32_t row_bytes = (uint32_t)s * ES;
  const int rps = SBYTES / (int)row_bytes;
  const int rows_per_cta = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  const int nstage = r0 < r1 ? (r1 - r0 + rps - 1) / rps : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTG; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_u32(&full[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int g = 0; g < NSTG && g < nstage; ++g) {
      int a0, na;
      stage_span(g, r0, r1, rps, true, a0, na);
      stg_issue(ring, full, g, (const uint8_t*)Zs, row_bytes, 0, row_bytes, a0, na);
    }
  }
  for (int e = threadIdx.x; e < s * KV; e += ZAT) {
    const int b = e / KV, c = e % KV;
    wsm[c * s + b] = c < k ? (ACC)w[(size_t)b * k + c] : (ACC)0;
  }
  // the CTA's rows of R, staged once (a per-row load after the reduction
  // would expose a memory round trip per row)
  double* rsm = reinterpret_cast<double*>(wsm + (size_t)s * KV);
  for (int e = threadIdx.x; e < (r1 - r0) * KV; e += ZAT) {
    const int rr = e / KV, c = e % KV;
    double r = 0.0;
    if (r0 < r1 && c < k) {
      const size_t ei = (size_t)(r0 + rr) * ldr + c;
      const T rv = R[ei];
      if (FUSE) Rout[ei] = rv;
      r = (double)rv;
    }
    rsm[e] = r;
  }
  double vz[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) vz[c] = 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // One right-hand side in FP32 with s <= 2048: each lane keeps its 8 x 8
  // entries of w (columns 8 lane + 256 it + q) in registers for the whole
  // kernel, so a row costs its own bytes only (reading w from shared memory
  // for every row cost twice the row's bytes).
  constexpr bool REGW = KV == 1 && sizeof(ACC) == 4;
  const int nit = s / 256;
  const bool use_reg = REGW && s % 256 == 0 && nit <= 8;
  float wr[8][8];
#pragma unroll
  for (int it = 0; it < 8; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q)
      wr[it][q] = (REGW && use_reg && it < nit) ? (float)wsm[lane * 8 + 256 * it + q] : 0.f;
  bool ok = true;
  int g = 0;
  for (; g < nstage; ++g) {
    const int st = g % NSTG;
    const uint32_t parity = (uint32_t)((g / NSTG) & 1);
    ok = __syncthreads_and(ok && stg_wait(sh_u32(&full[st]), parity));
    if (!ok) break;
    int row0, nrow;
    stage_span(g, r0, r1, rps, true, row0, nrow);
    const uint8_t* base = ring + (size_t)st * SBYTES;
    if (REGW && use_reg) {
      for (int rr = warp; rr < nrow; rr += ZAT / 32) {
        float v;
        if constexpr (ZF == 2) {
          // paired adds and FMAs on the 8-bit codes (the same sums as below)
          float2 a2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            if (it < nit) {
              float2 z2[4];
              unpack_q8x2(*reinterpret_cast<const uint2*>(base + (size_t)rr * row_bytes +
                                                         lane * 8 + 256 * it),
                          z2);
#pragma unroll
              for (int p = 0; p < 4; ++p)
                a2[p & 1] = __ffma2_rn(z2[p], make_float2(wr[it][2 * p], wr[it][2 * p + 1]),
                                       a2[p & 1]);
            }
          }
          v = (a2[0].x + a2[0].y) + (a2[1].x + a2[1].y);
        } else {
          float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            if (it < nit) {
              float z[8];
              stage8<ZF>(base + (size_t)rr * row_bytes + (lane * 8 + 256 * it) * ES, z);
#pragma unroll
              for (int q = 0; q < 8; ++q) a[q & 3] = fmaf(z[q], wr[it][q], a[q & 3]);
            }
          }
          v = (a[0] + a[1]) + (a[2] + a[3]);
        }
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        v *= zscale<ZF>();
        const int i = row0 + rr;
        if (lane == 0 && k > 0) {
          const T zo = (T)((rsm[i - r0] - (double)v) * inv_lam);
          Zo[(size_t)i * ldo] = zo;
          if (FUSE) vz[0] = fma(rsm[i - r0], (double)zo, vz[0]);
        }
      }
    } else
    // one row per warp and pass (RW = 1): sixteen rows of a BF16 stage in one pass
    for (int rr = warp; rr < nrow; rr += 1 * (ZAT / 32)) {
      constexpr int RW = 1;
      const int rb = rr + ZAT / 32;
      const bool two = RW == 2 && rb < nrow;
      ACC acc[RW][KV];
#pragma unroll
      for (int h = 0; h < RW; ++h)
#pragma unroll
        for (int c = 0; c < KV; ++c) acc[h][c] = (ACC)0;
#pragma unroll 2
      for (int b0 = lane * 8; b0 < s; b0 += 256) {
        float z[RW][8];
#pragma unroll
        for (int h = 0; h < RW; ++h) {
          const int row = h ? (two ? rb : rr) : rr;
          stage8<ZF>(base + (size_t)row * row_bytes + b0 * ES, z[h]);
        }
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          ACC wv[8];
          if (sizeof(ACC) == 4) {
            const float4* w4 = reinterpret_cast<const float4*>(wsm + c * s + b0);
            const float4 x0 = w4[0], x1 = w4[1];
            wv[0] = x0.x; wv[1] = x0.y; wv[2] = x0.z; wv[3] = x0.w;
            wv[4] = x1.x; wv[5] = x1.y; wv[6] = x1.z; wv[7] = x1.w;
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) wv[q] = wsm[c * s + b0 + q];
          }
#pragma unroll
          for (int h = 0; h < RW; ++h) {
            // two chains of four (the loop is latency-bound at eight warps)
            ACC x = acc[h][c], y = (ACC)0;
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
              x = fma((ACC)z[h][q], wv[q], x);
              y = fma((ACC)z[h][q + 1], wv[q + 1], y);
            }
            acc[h][c] = x + y;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < RW; ++h) {
        if (h == 1 && !two) break;
        const int i = row0 + (h ? rb : rr);
#pragma unroll
        for (int c = 0; c < KV; ++c) {
          if (c >= k) break;
          // reduce in the accumulator type (FP64 adds are slow on this GPU)
          ACC v = acc[h][c];
          for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          v *= (ACC)zscale<ZF>();
          if (lane == 0) {
            const double r = rsm[(i - r0) * KV + c];
            const T zo = (T)((r - (double)v) * inv_lam);
            Zo[(size_t)i * ldo + c] = zo;
            if (FUSE) vz[c] = fma(r, (double)zo, vz[c]);
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && g + NSTG < nstage) {
      int a0, na;
      stage_span(g + NSTG, r0, r1, rps, true, a0, na);
      stg_issue(ring, full, st, (const uint8_t*)Zs, row_bytes, 0, row_bytes, a0, na);
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicOr(err, 1);
    for (int gg = g; gg < nstage && gg < g + NSTG; ++gg)
      stg_wait(sh_u32(&full[gg % NSTG]), (uint32_t)((gg / NSTG) & 1));
  }
  if (FUSE) {
    double tot[KRR_MAX_RHS];
    if (grid_colsum_nt<ZAT>(vz, k, f.cpart, &f.sc->counter[CGC_RZ], blockIdx.x, gridDim.x,
                            tot)) {
      cg_rz_finish(f.sc, tot, k);
      // a streamed pass that gave up on a copy left z incomplete: stop the loop
      if (*reinterpret_cast<volatile int*>(err)) f.sc->flags |= FLAG_NAN;
      cg_tail_finish(f.sc, (cudaGraphConditionalHandle)f.cond);
    }
  }
}

// U form: t[a, c] = sum_i U[a, i] R[i, c]; one warp per row of U.
template <typename T>
__global__ void ur_kernel(const float* __restrict__ U, int n, int s, const T* __restrict__ R,
                          int k, int ldr, double* __restrict__ t) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= s) return;
  double acc[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) acc[c] = 0.0;
  for (int i = lane; i < n; i += 32) {
    double u = (double)U[(size_t)warp * n + i];
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) acc[c] = fma(u, (double)R[(size_t)i * ldr + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) {
    if (c >= k) break;
    double v = acc[c];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) t[(size_t)warp * k + c] = v;
  }
}

// U form: Zo[i, c] = (R[i, c] - sum_a U[a, i] t[a, c]) / lambda_p; thread per row i.
template <typename T>
__global__ void utt_kernel(const float* __restrict__ U, int n, int s, const double* __restrict__ t,
                           int k, const T* __restrict__ R, int ldr, double inv_lam,
                           T* __restrict__ Zo, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc[KRR_MAX_RHS];
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c) acc[c] = 0.0;
  for (int a = 0; a < s; ++a) {
    double u = (double)U[(size_t)a * n + i];
#pragma unroll
    for (int c = 0; c < KRR_MAX_RHS; ++c)
      if (c < k) acc[c] = fma(u, __ldg(&t[(size_t)a * k + c]), acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KRR_MAX_RHS; ++c)
    if (c < k) Zo[(size_t)i * ldo + c] = (T)(((double)R[(size_t)i * ldr + c] - acc[c]) * inv_lam);
}

struct ApplyPlan {
  int colblocks, nchunk, rpc, kv, sch;
  size_t zw_smem;
};

template <typename ACC>
ApplyPlan plan(int n, int s, int k) {
  ApplyPlan p;
  p.kv = kv_of(k);
  p.colblocks = (s + AT * 8 - 1) / (AT * 8);
  int nch = (4 * sm_count() + p.colblocks - 1) / p.colblocks;
  const int maxch = (n + ZT_ROWS - 1) / ZT_ROWS;
  if (nch > maxch) nch = maxch;
  if (nch < 1) nch = 1;
  p.rpc = (n + nch - 1) / nch;
  p.rpc = (p.rpc + ZT_ROWS - 1) / ZT_ROWS * ZT_ROWS;
  p.nchunk = (n + p.rpc - 1) / p.rpc;
  // w chunk in shared memory: at most 96 KiB, a multiple of 256 columns
  int sch = (int)((96 * 1024) / (p.kv * sizeof(ACC)));
  sch = sch / 256 * 256;
  if (sch < 256) sch = 256;
  const int s256 = (s + 255) / 256 * 256;
  p.sch = sch < s256 ? sch : s256;
  p.zw_smem = (size_t)p.sch * p.kv * sizeof(ACC);
  return p;
}

// Launch shapes of the streamed GEMVs of one apply and whether they apply.
struct StreamPlan {
  bool zt, zw;            // the streamed Z^T r / Z w kernels serve this apply
  int nchunk;             // row chunks of the streamed Z^T r
  size_t zt_bytes, zw_bytes;
};

template <int ZF, typename ACC, int KV>
StreamPlan stream_plan(const Precond& pc, const ApplyPlan& pl) {
  const int n = pc.n, s = pc.s;
  // whole 16-byte groups per row: 8 BF16 / FP32 values, 16 fixed-point bytes
  const bool vec = s % (ZF == 2 ? 16 : 8) == 0;
  const bool err = pc.err.p != nullptr;
  // streamed GEMVs: rows 16-byte aligned; zw also needs w beside the ring
  const size_t w_bytes = (size_t)s * KV * sizeof(ACC);
  const size_t ring_bytes = (size_t)NSTG * SBYTES;
  StreamPlan sp;
  sp.nchunk = std::min(pl.nchunk, std::max(1, sm_count() / pl.colblocks));
  sp.zt_bytes = ring_bytes + (size_t)((n + sp.nchunk - 1) / sp.nchunk) * KV * sizeof(ACC);
  sp.zw_bytes = ring_bytes + w_bytes +
                (size_t)((n + sm_count() - 1) / sm_count()) * KV * sizeof(double);
  constexpr int ES = ZF == 1 ? 2 : (ZF == 2 ? 1 : 4);
  sp.zt = vec && err && sp.zt_bytes <= (size_t)220 * 1024;
  sp.zw = vec && err && (size_t)s * ES <= (size_t)SBYTES && sp.zw_bytes <= (size_t)220 * 1024;
  return sp;
}

// fuse: run the PCG iteration's vector work in the two streamed passes (both
// must be streamed; R is then the residual before the update, and ldr == ldo == k).
template <int ZF, typename T, typename ACC, int KV>
void apply_zl(cudaStream_t st, const Precond& pc, const ApplyPlan& pl, const T* R, int k, int ldr,
              T* Zo, int ldo, double* t1, double* t2, void* part, bool ginv_only = false,
              const CgStepArgs<T>* fuse = nullptr) {
  const int n = pc.n, s = pc.s;
  const int vec = (s % (ZF == 2 ? 16 : 8) == 0) ? 1 : 0;
  int* err = reinterpret_cast<int*>(pc.err.p);
  const StreamPlan sp = stream_plan<ZF, ACC, KV>(pc, pl);
  if (fuse && !(sp.zt && sp.zw && !ginv_only))
    throw Error{KRR_EINVAL, "fused apply: the streamed kernels do not serve this shape"};
  const CgStepArgs<T> nof{};
  int nchunk = pl.nchunk;
  if (sp.zt) {
    nchunk = sp.nchunk;
    auto kz = fuse ? zt_stream_kernel<ZF, T, ACC, KV, 1> : zt_stream_kernel<ZF, T, ACC, KV, 0>;
    KRR_CUDA(cudaFuncSetAttribute(kz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sp.zt_bytes));
    kz<<<dim3(pl.colblocks, nchunk), AT, sp.zt_bytes, st>>>(
        pc.Z.p, n, s, R, ldr, k, reinterpret_cast<ACC*>(part), err, fuse ? *fuse : nof);
  } else {
    zt_kernel<ZF, T, ACC, KV><<<dim3(pl.colblocks, pl.nchunk), AT, 0, st>>>(
        pc.Z.p, n, s, R, ldr, k, reinterpret_cast<ACC*>(part), pl.rpc, vec);
  }
  KRR_CHECK_LAUNCH();
  const int sb = (int)(((size_t)s * KV + 31) / 32);
  sum_kernel<ACC><<<sb, 256, 0, st>>>(reinterpret_cast<const ACC*>(part), nchunk, s, KV, k, t1);
  KRR_CHECK_LAUNCH();
  const int tb = (s + TR_ROWS - 1) / TR_ROWS;
  trmv_kernel<0, KV><<<tb, AT, 0, st>>>(reinterpret_cast<const double*>(pc.Linv.p), s, t1, k, t2);
  KRR_CHECK_LAUNCH();
  trmv_kernel<1, KV><<<tb, AT, 0, st>>>(reinterpret_cast<const double*>(pc.LinvT.p), s, t2, k, t1);
  KRR_CHECK_LAUNCH();
  if (ginv_only) return;  // t1 = G^-1 Z^T R (the random-features solution)
  if (sp.zw) {
    auto kw = fuse ? zw_stream_kernel<ZF, T, ACC, KV, 1> : zw_stream_kernel<ZF, T, ACC, KV, 0>;
    KRR_CUDA(cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sp.zw_bytes));
    // fused: z from the updated residual, which is copied back to R
    const T* Rin = fuse ? fuse->Rn : R;
    T* Rout = fuse ? const_cast<T*>(R) : nullptr;
    kw<<<sm_count(), ZAT, sp.zw_bytes, st>>>(pc.Z.p, n, s, t1, k, Rin, ldr, 1.0 / pc.lam_p, Zo,
                                             ldo, err, Rout, fuse ? *fuse : nof);
    KRR_CHECK_LAUNCH();
    return;
  }
  auto kern = zw_kernel<ZF, T, ACC, KV>;
  if (pl.zw_smem > 48 * 1024)
    KRR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pl.zw_smem));
  kern<<<(n + ZW_ROWS - 1) / ZW_ROWS, AT, pl.zw_smem, st>>>(pc.Z.p, n, s, t1, k, R, ldr,
                                                            1.0 / pc.lam_p, Zo, ldo, pl.sch, vec);
  KRR_CHECK_LAUNCH();
}

template <typename T, typename ACC, int KV>
void apply_zl_kv(cudaStream_t st, const Precond& pc, const ApplyPlan& pl, const T* R, int k,
                 int ldr, T* Zo, int ldo, double* t1, double* t2, void* part,
                 bool ginv_only = false, const CgStepArgs<T>* fuse = nullptr) {
  if (pc.z_bf16 == 2)
    apply_zl<2, T, ACC, KV>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part, ginv_only, fuse);
  else if (pc.z_bf16)
    apply_zl<1, T, ACC, KV>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part, ginv_only, fuse);
  else
    apply_zl<0, T, ACC, KV>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part, ginv_only, fuse);
}

template <typename ACC, int KV>
bool stream_both(const Precond& pc, const ApplyPlan& pl) {
  StreamPlan sp;
  if (pc.z_bf16 == 2)
    sp = stream_plan<2, ACC, KV>(pc, pl);
  else if (pc.z_bf16)
    sp = stream_plan<1, ACC, KV>(pc, pl);
  else
    sp = stream_plan<0, ACC, KV>(pc, pl);
  return sp.zt && sp.zw;
}

// F[i, c] = sum_b Zf[i, b] w[b, c] (FP64 sums): one warp per row.
template <int KV>
__global__ void __launch_bounds__(AT)
feature_gemv_kernel(const float* __restrict__ Zf, int m, int s, const double* __restrict__ w,
                    int k, double* __restrict__ F, int ldf) {
  const int row = (blockIdx.x * AT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= m) return;
  double acc[KV];
#pragma unroll
  for (int c = 0; c < KV; ++c) acc[c] = 0.0;
  const float* zr = Zf + (size_t)row * s;
  for (int b = lane; b < s; b += 32) {
    const double z = (double)zr[b];
#pragma unroll
    for (int c = 0; c < KV; ++c)
      if (c < k) acc[c] = fma(z, w[(size_t)b * k + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KV; ++c) {
    double v = acc[c];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0 && c < k) F[(size_t)row * ldf + c] = v;
  }
}

}  // namespace

size_t apply_part_elems(int n, int s, int k) {
  // in doubles (large enough for either accumulator type)
  ApplyPlan p = plan<double>(n, s, k);
  return (size_t)p.nchunk * s * p.kv;
}

void launch_ginv_zt(cudaStream_t st, const Precond& pc, const double* R, int k, int ldr,
                    double* t1, double* t2, double* part) {
  if (pc.form != KRR_APPLY_ZL) throw Error{KRR_EINVAL, "G^-1 Z^T r needs the ZL factors"};
  const ApplyPlan pl = plan<double>(pc.n, pc.s, k);
  switch (pl.kv) {
    case 1: apply_zl_kv<double, double, 1>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
    case 2: apply_zl_kv<double, double, 2>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
    case 4: apply_zl_kv<double, double, 4>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
    case 8: apply_zl_kv<double, double, 8>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
    case 12: apply_zl_kv<double, double, 12>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
    default: apply_zl_kv<double, double, 16>(st, pc, pl, R, k, ldr, nullptr, 0, t1, t2, part, true); break;
  }
}

void launch_feature_gemv(cudaStream_t st, const float* Zf, int m, int s, const double* w, int k,
                         double* F, int ldf) {
  const int blocks = (int)(((size_t)m * 32 + AT - 1) / AT);
  switch (kv_of(k)) {
    case 1: feature_gemv_kernel<1><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
    case 2: feature_gemv_kernel<2><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
    case 4: feature_gemv_kernel<4><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
    case 8: feature_gemv_kernel<8><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
    case 12: feature_gemv_kernel<12><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
    default: feature_gemv_kernel<16><<<blocks, AT, 0, st>>>(Zf, m, s, w, k, F, ldf); break;
  }
  KRR_CHECK_LAUNCH();
}

template <typename T>
void launch_apply(cudaStream_t st, const Precond& pc, const T* R, int k, int ldr, T* Zo,
                  int ldo, double* t1, double* t2, double* part) {
  const int n = pc.n, s = pc.s;
  const double inv_lam = 1.0 / pc.lam_p;
  if (pc.form == KRR_APPLY_U) {
    const float* U = reinterpret_cast<const float*>(pc.U.p);
    ur_kernel<T><<<(s + 7) / 8, 256, 0, st>>>(U, n, s, R, k, ldr, t1);
    KRR_CHECK_LAUNCH();
    utt_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(U, n, s, t1, k, R, ldr, inv_lam, Zo, ldo);
    KRR_CHECK_LAUNCH();
    return;
  }
  // FP32 slab sums for single-precision vectors, FP64 for the FP64 solve
  typedef typename std::conditional<std::is_same<T, float>::value, float, double>::type ACC;
  const ApplyPlan pl = plan<ACC>(n, s, k);
  switch (pl.kv) {
    case 1: apply_zl_kv<T, ACC, 1>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
    case 2: apply_zl_kv<T, ACC, 2>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
    case 4: apply_zl_kv<T, ACC, 4>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
    case 8: apply_zl_kv<T, ACC, 8>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
    case 12: apply_zl_kv<T, ACC, 12>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
    default: apply_zl_kv<T, ACC, 16>(st, pc, pl, R, k, ldr, Zo, ldo, t1, t2, part); break;
  }
}

bool apply_cg_supported(const Precond& pc, int n, int k) {
  if (pc.form != KRR_APPLY_ZL || !pc.Z.p || pc.n != n || k < 1 || k > KRR_MAX_RHS) return false;
  const ApplyPlan pl = plan<float>(pc.n, pc.s, k);
  switch (pl.kv) {
    case 1: return stream_both<float, 1>(pc, pl);
    case 2: return stream_both<float, 2>(pc, pl);
    case 4: return stream_both<float, 4>(pc, pl);
    case 8: return stream_both<float, 8>(pc, pl);
    case 12: return stream_both<float, 12>(pc, pl);
    default: return stream_both<float, 16>(pc, pl);
  }
}

template <typename T>
void launch_apply_cg(cudaStream_t st, const Precond& pc, T* R, int k, T* Zo, double* t1,
                     double* t2, double* part, const CgStepArgs<T>& f) {
  static_assert(std::is_same<T, float>::value, "the fused apply serves FP32 vectors");
  if (!apply_cg_supported(pc, pc.n, k))
    throw Error{KRR_EINVAL, "fused apply: not available for this preconditioner shape"};
  const ApplyPlan pl = plan<float>(pc.n, pc.s, k);
  switch (pl.kv) {
    case 1: apply_zl_kv<T, float, 1>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
    case 2: apply_zl_kv<T, float, 2>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
    case 4: apply_zl_kv<T, float, 4>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
    case 8: apply_zl_kv<T, float, 8>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
    case 12: apply_zl_kv<T, float, 12>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
    default: apply_zl_kv<T, float, 16>(st, pc, pl, R, k, k, Zo, k, t1, t2, part, false, &f); break;
  }
}

template void launch_apply_cg<float>(cudaStream_t, const Precond&, float*, int, float*, double*,
                                     double*, double*, const CgStepArgs<float>&);

template void launch_apply<float>(cudaStream_t, const Precond&, const float*, int, int, float*,
                                  int, double*, double*, double*);
template void launch_apply<double>(cudaStream_t, const Precond&, const double*, int, int,
                                   double*, int, double*, double*, double*);

}  // namespace krr
