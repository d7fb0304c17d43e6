// Measurement helpers: the kernel-launch counter and the base-2 exponential
// throughput probes that set the exp-bound roofline of the fused product (one
// base-2 exponential per kernel entry): the MUFU ex2 alone, and the MUFU and
// the FMA-pipe polynomial run side by side in a chosen split.
#include <atomic>

#include "krr_exp2.cuh"
#include "krr_internal.cuh"

namespace krr {

namespace {
std::atomic<long long> g_launches{0};
thread_local int g_capturing = 0;
thread_local long long g_captured = 0;

constexpr int EX2_CHAINS = 8;

__device__ __forceinline__ float ex2n(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}

// Independent chains x <- 2^-x keep every value in [0.5, 1] and the MUFU busy.
__global__ void ex2_bench_kernel(float* out, int iters) {
  float x[EX2_CHAINS];
#pragma unroll
  for (int c = 0; c < EX2_CHAINS; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < EX2_CHAINS; ++c) x[c] = ex2n(x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < EX2_CHAINS; ++c) s += x[c];
  if (s == 12345.f) out[0] = s;  // never true; keeps the chains live
}
// 32 independent chains per thread, x <- 2^-x; the first EMU chains use the
// FMA-pipe polynomial and the rest the MUFU, so both pipes run concurrently
// in the ratio EMU : 32 - EMU.
template <int EMU>
__global__ void ex2_mix_kernel(float* out, int iters) {
  float x[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = c < EMU ? ex2_fma(-x[c]) : ex2_mufu(-x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 32; ++c) s += x[c];
  if (s == 12345.f) out[0] = s;  // never true; keeps the chains live
}

template <int EMU>
float time_mix(cudaStream_t st, float* out, int blocks, int threads, int iters,
               cudaEvent_t a, cudaEvent_t b) {
  ex2_mix_kernel<EMU><<<blocks, threads, 0, st>>>(out, 16);  // warm-up
  KRR_CHECK_LAUNCH();
  KRR_CUDA(cudaEventRecord(a, st));
  ex2_mix_kernel<EMU><<<blocks, threads, 0, st>>>(out, iters);
  KRR_CHECK_LAUNCH();
  KRR_CUDA(cudaEventRecord(b, st));
  KRR_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  KRR_CUDA(cudaEventElapsedTime(&ms, a, b));
  return ms;
}
}  // namespace

void count_launch() {
  if (g_capturing)
    ++g_captured;
  else
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

void capture_begin() {
  g_capturing = 1;
  g_captured = 0;
}

long long capture_end() {
  g_capturing = 0;
  return g_captured;
}

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

double bench_ex2(cudaStream_t st, int iters, double* ms_out) {
  const int blocks = 8 * sm_count(), threads = 256;
  float* out = nullptr;
  KRR_CUDA(cudaMalloc(&out, sizeof(float)));
  cudaEvent_t a, b;
  KRR_CUDA(cudaEventCreate(&a));
  KRR_CUDA(cudaEventCreate(&b));
  ex2_bench_kernel<<<blocks, threads, 0, st>>>(out, 64);  // warm-up
  KRR_CHECK_LAUNCH();
  KRR_CUDA(cudaEventRecord(a, st));
  ex2_bench_kernel<<<blocks, threads, 0, st>>>(out, iters);
  KRR_CHECK_LAUNCH();
  KRR_CUDA(cudaEventRecord(b, st));
  KRR_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  KRR_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (ms_out) *ms_out = ms;
  const double n = (double)blocks * threads * (double)iters * EX2_CHAINS;
  return n / (ms * 1e-3);
}

double bench_ex2_mix(cudaStream_t st, int iters, int fma_per_32, double* ms_out) {
  const int blocks = 4 * sm_count(), threads = 256;
  float* out = nullptr;
  KRR_CUDA(cudaMalloc(&out, sizeof(float)));
  cudaEvent_t a, b;
  KRR_CUDA(cudaEventCreate(&a));
  KRR_CUDA(cudaEventCreate(&b));
  float ms = 0.f;
  switch (fma_per_32) {
    case 0: ms = time_mix<0>(st, out, blocks, threads, iters, a, b); break;
    case 2: ms = time_mix<2>(st, out, blocks, threads, iters, a, b); break;
    case 4: ms = time_mix<4>(st, out, blocks, threads, iters, a, b); break;
    case 6: ms = time_mix<6>(st, out, blocks, threads, iters, a, b); break;
    case 8: ms = time_mix<8>(st, out, blocks, threads, iters, a, b); break;
    case 10: ms = time_mix<10>(st, out, blocks, threads, iters, a, b); break;
    case 12: ms = time_mix<12>(st, out, blocks, threads, iters, a, b); break;
    case 16: ms = time_mix<16>(st, out, blocks, threads, iters, a, b); break;
    default: ms = time_mix<32>(st, out, blocks, threads, iters, a, b); break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (ms_out) *ms_out = ms;
  const double n = (double)blocks * threads * (double)iters * 32;
  return n / (ms * 1e-3);
}

}  // namespace krr

extern "C" long long krr_launch_count(void) { return krr::g_launches.load(); }
