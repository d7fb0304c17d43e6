// One persistent launch for the kernel products of many independent KRR
// problems (the uneven batch): q_p = K_p v_p + lambda_p v_p for every problem
// p whose PCG loop still runs, one right-hand side each, FP16 points.
//
// The arithmetic per problem is tc_matvec_kernel's (Gaussian kernel of the
// rounded, centred, scaled points, K_ij = exp2(xh_i.xh_j) ra_i ra_j; S on
// tcgen05 with FP32 accumulation in TMEM, exp2 on the MUFU, the contraction
// with w_j = ra_j v_j on the FMA pipe, FP64 sums of the column-chunk
// partials).  Only the work list differs: the items of all problems --
// (problem, 128-row tile, column chunk), largest first -- are dealt to one
// persistent CTA per SM, with each problem's TMA descriptors in the kernel's
// parameter block and each item reading its problem's weights and writing its
// partial row sums.  A problem whose loop has stopped (its `run` flag is 0)
// contributes no work.  Row tiles are streamed with the column tiles (no
// resident row tile), which serves every d up to 128 with one code path.
//
// Structure: warp 0 issues the TMA loads (row tile + column tile per K-block
// into a ring of stages, the tile's weights by bulk copy), warp 1 owns 512
// TMEM columns (two 128 x 256 FP32 accumulators) and issues tcgen05.mma
// (M = 128, N = 256, K = 16), warps 2..17 are the epilogue (warp w reads TMEM
// lanes 32 (w % 4) .. + 31 and one of four 64-column groups).  Every mbarrier
// wait is bounded; on expiry the kernel raises the error flag, drains its own
// copies and MMAs, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "krr_exp2.cuh"
#include "krr_tc.cuh"
#include "krr_tc_ptx.cuh"

namespace krr {
namespace {

using namespace ptx;

constexpr int BM = 128, BN = 256, BK = 64, UK = 16;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE = A_BYTES + B_BYTES;
constexpr int NS = 4;            // ring stages
constexpr int NW = 4;            // weight-ring slots
constexpr int NEPI = 16, NG = NEPI / 4, COLS = BN / NG;
constexpr int THREADS = 32 * (2 + NEPI);
constexpr int TMEM_COLS = 2 * BN;

struct BProb {
  const float* w;      // n_ct * BN weights ra_j v_j (0 for padding)
  float* part;         // nchunk x n_rpad partial row sums
  const int* run;      // the problem's PCG loop flag (0: no work)
  int n_ct, cpc, nkb, n_rpad;
};

struct BParams {
  CUtensorMap ma[BATCH_MAX];   // row tiles (128-row boxes)
  CUtensorMap mb[BATCH_MAX];   // column tiles (256-row boxes)
  BProb prob[BATCH_MAX];
  const int4* items;           // (problem, row tile, chunk, 0)
  int n_items;
  uint32_t idesc;
  int* err;
};

__device__ __forceinline__ bool item_live(const BParams& p, int item, int4& it) {
  it = p.items[item];
  return __ldcg(p.prob[it.x].run) != 0;
}

__global__ void __launch_bounds__(THREADS, 1) tc_batch_kernel(const __grid_constant__ BParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = smem;
  float* wbuf = (float*)(stages + NS * STAGE);        // NW x BN
  float* comb = wbuf + NW * BN;                        // (NG - 1) x BM
  uint64_t* full = (uint64_t*)(comb + (NG - 1) * BM);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* wfull = tempty + 2;
  uint64_t* wempty = wfull + NW;
  uint64_t* drain = wempty + NW;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
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
      uint32_t st = 0, ph = 0, ws = 0, wph = 0, issued = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < p.n_items; item += gridDim.x) {
        int4 it;
        if (!item_live(p, item, it)) continue;
        const BProb& pr = p.prob[it.x];
        const int ct0 = it.z * pr.cpc, ct1 = min(pr.n_ct, ct0 + pr.cpc);
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&wempty[ws]), wph ^ 1, abort_flag, p.err))) break;
          fence_proxy_async_smem();   // the readers' loads before the refill
          mbar_expect_tx(smem_u32(&wfull[ws]), BN * 4);
          bulk_load(smem_u32(wbuf + ws * BN), pr.w + (size_t)ct * BN, BN * 4,
                    smem_u32(&wfull[ws]));
          if (++ws == NW) {
            ws = 0;
            wph ^= 1;
          }
          for (int kb = 0; kb < pr.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&empty[st]), ph ^ 1, abort_flag, p.err))) break;
            const uint32_t sa = smem_u32(stages + st * STAGE);
            mbar_expect_tx(smem_u32(&full[st]), STAGE);
            tma_load_2d(sa, &p.ma[it.x], kb * BK, it.y * BM, smem_u32(&full[st]));
            tma_load_2d(sa + A_BYTES, &p.mb[it.x], kb * BK, ct * BN, smem_u32(&full[st]));
            ++issued;
            if (++st == (uint32_t)NS) {
              st = 0;
              ph ^= 1;
            }
          }
        }
      }
      if (!ok) {
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
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t st = 0, ph = 0, acc = 0, aph = 0;
      bool ok = true, any = false;
      for (int item = blockIdx.x; ok && item < p.n_items; item += gridDim.x) {
        int4 it;
        if (!item_live(p, item, it)) continue;
        const BProb& pr = p.prob[it.x];
        const int ct0 = it.z * pr.cpc, ct1 = min(pr.n_ct, ct0 + pr.cpc);
        for (int ct = ct0; ok && ct < ct1; ++ct) {
          if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1, abort_flag, p.err))) break;
          fence_after();
          const uint32_t d = tmem + acc * BN;
          for (int kb = 0; kb < pr.nkb; ++kb) {
            if (!(ok = mbar_wait(smem_u32(&full[st]), ph, abort_flag, p.err))) break;
            fence_after();
            const uint32_t sa = smem_u32(stages + st * STAGE), sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk)
              mma_bf16(d, sdesc(sa + kk * UK * 2), sdesc(sb + kk * UK * 2), p.idesc,
                       (kb > 0 || kk > 0) ? 1u : 0u);
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
    const int e = warp - 2, quad = warp & 3, grp = e >> 2;
    const int row = quad * 32 + lane;
    uint32_t acc = 0, aph = 0, ws = 0, wph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
      int4 it;
      if (!item_live(p, item, it)) continue;
      const BProb& pr = p.prob[it.x];
      const int ct0 = it.z * pr.cpc, ct1 = min(pr.n_ct, ct0 + pr.cpc);
      float2 qq = make_float2(0.f, 0.f);   // even and odd columns
      for (int ct = ct0; ok && ct < ct1; ++ct) {
        if (!(ok = mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, p.err))) break;
        if (!(ok = mbar_wait(smem_u32(&wfull[ws]), wph, abort_flag, p.err))) break;
        fence_after();
        const float* wb = wbuf + ws * BN + grp * COLS;
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + acc * BN + grp * COLS;
        uint32_t raw[2][32];
        tmem_ld16_nowait(tbase, *reinterpret_cast<uint32_t(*)[16]>(&raw[0][0]));
        tmem_ld16_nowait(tbase + 16, *reinterpret_cast<uint32_t(*)[16]>(&raw[0][16]));
        tmem_wait_ld(*reinterpret_cast<uint32_t(*)[16]>(&raw[0][0]));
        tmem_keep(*reinterpret_cast<uint32_t(*)[16]>(&raw[0][16]));
        constexpr int NCH = COLS / 32;
#pragma unroll
        for (int cc = 0; cc < NCH; ++cc) {
          const int cur = cc & 1;
          if (cc + 1 < NCH) {
            tmem_ld16_nowait(tbase + (cc + 1) * 32,
                             *reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][0]));
            tmem_ld16_nowait(tbase + (cc + 1) * 32 + 16,
                             *reinterpret_cast<uint32_t(*)[16]>(&raw[cur ^ 1][16]));
          }
#pragma unroll
          for (int j = 0; j < 32; ++j)
            raw[cur][j] = __float_as_uint(ex2_mufu(__uint_as_float(raw[cur][j])));
          const float4* w4 = reinterpret_cast<const float4*>(wb + cc * 32);
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
      const float qs = qq.x + qq.y;
      if (grp > 0) comb[(grp - 1) * BM + row] = qs;
      bar_sync<NEPI * 32>();
      if (grp == 0 && ok) {
        float s = qs;
#pragma unroll
        for (int g = 1; g < NG; ++g) s += comb[(g - 1) * BM + row];
        pr.part[(size_t)it.z * pr.n_rpad + (size_t)it.y * BM + row] = s;
      }
      if (bar_or<NEPI * 32>(!ok || *abort_flag)) break;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// Per-problem operands of the weight and chunk-sum kernels.
struct BRed {
  const float* ra;       // n_pad row factors (0 for padding)
  const float* V;
  float* Q;
  float* w;              // n_pad weights
  const float* part;     // nchunk x n_pad
  const int* run;
  double shift;
  int n, n_pad, nchunk;
};

// w_p[j] = ra_j v_j (0 for padding) for every running problem p = blockIdx.y.
__global__ void batch_w_kernel(const BRed* __restrict__ tab) {
  const BRed& t = tab[blockIdx.y];
  if (__ldcg(t.run) == 0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < t.n_pad; j += gridDim.x * blockDim.x)
    t.w[j] = j < t.n ? t.ra[j] * t.V[j] : 0.f;
}

// q_p[i] = ra_i sum_ch part[ch, i] + shift v_i (FP64 sums, fixed order).
__global__ void batch_reduce_kernel(const BRed* __restrict__ tab) {
  const BRed& t = tab[blockIdx.y];
  if (__ldcg(t.run) == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < t.n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int ch = 0; ch < t.nchunk; ++ch) s += (double)t.part[(size_t)ch * t.n_pad + i];
    s *= (double)t.ra[i];
    if (t.shift != 0.0) s += t.shift * (double)t.V[i];
    t.Q[i] = (float)s;
  }
}

size_t batch_smem_bytes() {
  return 1024 + (size_t)NS * STAGE + (size_t)NW * BN * 4 + (size_t)(NG - 1) * BM * 4 + 256;
}

void ensure_dev(DevBuf& b, size_t bytes) { tc_ensure(b, bytes); }

}  // namespace

void tc_batch_reserve(BatchState& bs, cudaStream_t st, const std::vector<BatchProb>& probs) {
  const int np = (int)probs.size();
  if (np < 1 || np > BATCH_MAX) throw Error{KRR_EINVAL, "batched product: 1..64 problems"};
  bs.nprob = np;
  bs.chunks.assign(np, 1);
  // column chunks of at most 8 tiles: enough items to balance 152 SMs across
  // problems of 1,000 to 32,768 points, few enough partial sums
  std::vector<int4> items;
  size_t w_elems = 0, part_elems = 0;
  for (int p = 0; p < np; ++p) {
    const TcOperand& op = *probs[p].op;
    if (op.kp > 2 * BK || !op.f16)
      throw Error{KRR_EUNSUPPORTED, "batched product: FP16 points with d <= 128"};
    const int n_rt = op.n_pad / BM, n_ct = op.n_pad / BN;
    const int cpc = std::min(n_ct, 8);
    const int nch = (n_ct + cpc - 1) / cpc;
    bs.chunks[p] = nch;
    for (int rt = 0; rt < n_rt; ++rt)
      for (int ch = 0; ch < nch; ++ch) items.push_back(make_int4(p, rt, ch, 0));
    w_elems += op.n_pad;
    part_elems += (size_t)nch * op.n_pad;
  }
  // largest items first (column tiles x K-blocks), problems interleaved
  auto cost = [&](const int4& it) {
    const TcOperand& op = *probs[it.x].op;
    const int n_ct = op.n_pad / BN, cpc = std::min(n_ct, 8);
    const int tiles = std::min(n_ct, (it.z + 1) * cpc) - it.z * cpc;
    return tiles * (op.kp / BK);
  };
  std::stable_sort(items.begin(), items.end(),
                   [&](const int4& a, const int4& b) { return cost(a) > cost(b); });
  ensure_dev(bs.items, items.size() * sizeof(int4));
  KRR_CUDA(cudaMemcpyAsync(bs.items.p, items.data(), items.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, st));
  bs.n_items = (int)items.size();
  ensure_dev(bs.w, w_elems * 4);
  ensure_dev(bs.part, part_elems * 4);
  ensure_dev(bs.table, (size_t)BATCH_MAX * sizeof(BRed));
  if (!bs.err.p) ensure_dev(bs.err, 16);
  KRR_CUDA(cudaMemsetAsync(bs.err.p, 0, 16, st));
  // the per-problem table (pointers only change with the problems)
  std::vector<BRed> tab(np);
  size_t wo = 0, po = 0;
  for (int p = 0; p < np; ++p) {
    const TcOperand& op = *probs[p].op;
    tab[p] = BRed{(const float*)op.ra.p, probs[p].V, probs[p].Q, (float*)bs.w.p + wo,
                  (const float*)bs.part.p + po, probs[p].run, probs[p].shift, op.n, op.n_pad,
                  bs.chunks[p]};
    wo += op.n_pad;
    po += (size_t)bs.chunks[p] * op.n_pad;
  }
  KRR_CUDA(cudaMemcpyAsync(bs.table.p, tab.data(), np * sizeof(BRed), cudaMemcpyHostToDevice, st));
  KRR_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
  static size_t attr = 0;
  const size_t sm = batch_smem_bytes();
  if (attr < sm) {
    KRR_CUDA(cudaFuncSetAttribute(tc_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    attr = sm;
  }
}

void tc_batch_matvec(BatchState& bs, cudaStream_t st, const std::vector<BatchProb>& probs) {
  const int np = bs.nprob;
  if ((int)probs.size() != np) throw Error{KRR_EINVAL, "batched product: reserve first"};
  int max_pad = 0;
  for (const BatchProb& b : probs) max_pad = std::max(max_pad, b.op->n_pad);
  const BRed* tab = (const BRed*)bs.table.p;
  dim3 gw(std::max(1, std::min(64, (max_pad + 255) / 256)), np);
  batch_w_kernel<<<gw, 256, 0, st>>>(tab);
  KRR_CHECK_LAUNCH();
  BParams p;
  memset(&p, 0, sizeof(p));
  size_t wo = 0, po = 0;
  for (int q = 0; q < np; ++q) {
    const TcOperand& op = *probs[q].op;
    p.ma[q] = op.map_a;
    p.mb[q] = op.map_b;
    const int n_ct = op.n_pad / BN;
    p.prob[q] = BProb{(const float*)bs.w.p + wo, (float*)bs.part.p + po, probs[q].run, n_ct,
                      std::min(n_ct, 8), op.kp / BK, op.n_pad};
    wo += op.n_pad;
    po += (size_t)bs.chunks[q] * op.n_pad;
  }
  p.items = (const int4*)bs.items.p;
  p.n_items = bs.n_items;
  p.idesc = idesc_f16(BM, BN);
  p.err = (int*)bs.err.p;
  tc_batch_kernel<<<std::min(bs.n_items, sm_count()), THREADS, batch_smem_bytes(), st>>>(p);
  KRR_CHECK_LAUNCH();
  batch_reduce_kernel<<<gw, 256, 0, st>>>(tab);
  KRR_CHECK_LAUNCH();
}

int tc_batch_error(BatchState& bs, cudaStream_t st) {
  if (!bs.err.p) return 0;
  int e = 0;
  KRR_CUDA(cudaMemcpyAsync(&e, bs.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  return e;
}

void tc_batch_release(BatchState& bs) {
  for (DevBuf* b : {&bs.items, &bs.table, &bs.w, &bs.part, &bs.err})
    if (b->p) cudaFree(b->p);
  bs = BatchState();
}

}  // namespace krr
