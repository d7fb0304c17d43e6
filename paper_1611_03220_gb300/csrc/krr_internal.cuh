// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "krr.h"

namespace krr {

// ---------------------------------------------------------------- errors --
struct Error {
  krr_status st;
  std::string msg;
};

#define KRR_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      throw ::krr::Error{KRR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// Kernel-launch accounting (krr_launch_count): launches made while a loop
// body is being captured into a graph are counted per captured body and
// multiplied by the iterations the graph executes.
void count_launch();
void capture_begin();
long long capture_end();           // launches seen since capture_begin
void add_launches(long long n);
double bench_ex2(cudaStream_t st, int iters, double* ms_out);
// Exponentials per second with fma_per_32 of every 32 on the FMA pipe.
double bench_ex2_mix(cudaStream_t st, int iters, int fma_per_32, double* ms_out);
#define KRR_CHECK_LAUNCH()            \
  do {                                \
    KRR_CUDA(cudaGetLastError());     \
    ::krr::count_launch();            \
  } while (0)

#define KRR_REQUIRE(cond, msg)                                                  \
  do {                                                                          \
    if (!(cond)) throw ::krr::Error{KRR_EINVAL, std::string(msg)};             \
  } while (0)

// ------------------------------------------------------------- workspace --
// A named, grow-only device buffer owned by the handle.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace krr

struct krr_handle;

namespace krr {

// Device scalar block used by the PCG loop (one per handle).
struct CgScalars {
  double rz[KRR_MAX_RHS];      // r.z of the current iteration
  double rz_keep[KRR_MAX_RHS]; // r.z of the previous solve's last step (kept by cg_init)
  double pq[KRR_MAX_RHS];      // p.q
  double alpha[KRR_MAX_RHS];
  double beta[KRR_MAX_RHS];
  double rr[KRR_MAX_RHS];      // ||r||^2 (recursive)
  double yy[KRR_MAX_RHS];      // ||y||^2 of the system being solved
  double tol2[KRR_MAX_RHS];    // (tol ||y||)^2
  int active[KRR_MAX_RHS];     // 1 while the column iterates
  int iters[KRR_MAX_RHS];
  int iter;                    // loop counter
  int max_iter;
  int flags;                   // bit 0 breakdown, bit 1 NaN, bit 2 iteration cap
  int k;
  int run;                     // 1 while the loop should execute another iteration
  unsigned int counter[8];     // last-block-done counters for reductions
  double* hist;                // alpha, beta of the first hist_cap iterations
  int hist_cap;                //   ([iter][2][KRR_MAX_RHS]; null: not recorded)
};

// Rows of the alpha/beta record kept for the condition estimate.
constexpr int CG_HIST_CAP = 4096;

enum : int { FLAG_BREAKDOWN = 1, FLAG_NAN = 2, FLAG_CAP = 4 };

// Per-handle preconditioner state (the set-up step of Algorithm 1).
struct Precond {
  bool ready = false;
  int n = 0, s = 0, form = KRR_APPLY_ZL, z_bf16 = 0;
  int z_fixed_e = 0;  // fixed-point features: Z ~= 2^e Zs (0 otherwise)
  double lam_p = 0.0;
  DevBuf Z;      // n x s (ld = s): FP32 (z_bf16 0), BF16 (1) or 8-bit q (2, Z = q / 128)
  DevBuf L;      // s x s FP64 lower Cholesky factor of G
  DevBuf Linv;   // s x s FP64 lower inverse of L (ZL form)
  DevBuf LinvT;  // s x s FP64, (L^-1)^T, upper (ZL form)
  DevBuf U;      // s x n FP32, U = L^-1 Z^T (U form)
  DevBuf err;    // device flag: a streamed apply's bounded wait expired
};

// ------------------------------------------------------ kernel launchers --
// All launchers enqueue on `st` and throw krr::Error on launch failure.

int sm_count();

// RFF features (krr_rff.cu)
void launch_rff(cudaStream_t st, const float* X, int n, int d, int ldx, const float* W,
                const float* b, int s, float* Z, int ldz);

// SIMT kernel products (krr_matvec_simt.cu).  part: scratch of
// simt_part_elems(...) elements of the accumulator type.
size_t mv_fp64_part_elems(int nr, int nc, int k);
// dsigma = 1: Q = (D o K) V + shift V with D_ij = ||xr_i - xc_j||^2 / sigma^2
// (the derivative of K with respect to log sigma).
void launch_mv_fp64(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                    int nc, int ldxc, int d, double sigma, double shift, const double* V,
                    int k, int ldv, double* Q, int ldq, double* part, int dsigma = 0);
void launch_mv_fp64_capped(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                           int nc, int ldxc, int d, double sigma, double shift, const double* V,
                           int k, int ldv, double* Q, int ldq, double* part, size_t cap);
// High-precision SIMT product for any d (krr_matvec_hpw.cu): float-float
// norm-expansion distances and exp2; part: mv_hpw_part_elems doubles,
// nrm_r / nrm_c: 2 nr / 2 nc floats.  dsigma = 1 gives (D o K) V (no shift).
size_t mv_hpw_part_elems(int nr, int nc, int k);
void launch_mv_hpw(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc, int nc,
                   int ldxc, int d, double sigma, double shift, const double* V, int k, int ldv,
                   double* Q, int ldq, double* part, float* nrm_r, float* nrm_c, int dsigma);
size_t mv_fp32_part_elems(int nr, int nc, int k);
void launch_mv_fp32(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                    int nc, int ldxc, int d, double sigma, double shift, const float* V,
                    int k, int ldv, float* Q, int ldq, float* nrm_r, float* nrm_c,
                    float* part);

// Tensor-core set-up (krr_setup_tc.cu): fixed-point features zs = q / 128
// (q = clamp(rint(z 2^(7-e)), +-127), z ~= 2^e zs) and their exact Gram.
// Padded sizes: Z^T is setup_tc_s_pad(s) x setup_tc_n_pad(n) BF16; the split
// operands are setup_tc_n_pad(n) (X) or setup_tc_s_pad(s) (W^T) x setup_tc_kp(d).
int setup_tc_n_pad(int n);
int setup_tc_s_pad(int s);
int setup_tc_kp(int d);
int fixed_point_exponent(double maxabs);
size_t gram_tc_part_elems(int n, int s);
// Features of X (n x d, ldx) for W (d x s), b (s): Z as the 8-bit q
// (n x s, Zs = q / 128) and Zs^T (BF16); returns e.
int launch_rff_tc(cudaStream_t st, const float* X, int n, int d, int ldx, const float* W,
                  const float* b, int s, __nv_bfloat16* Xh, __nv_bfloat16* Xl,
                  __nv_bfloat16* Wh, __nv_bfloat16* Wl, signed char* Z, __nv_bfloat16* ZT,
                  int* err);
// Fixed-point copy of a caller's FP32 Z (synchronises once for max |Z|); returns e.
int launch_quantize_z(cudaStream_t st, const float* Z, int n, int s, int ldz, signed char* Zs,
                      __nv_bfloat16* ZT, int* scratch);
// F = scale A B^T (A: n x K, B: s x K, FP32 row-major) on tcgen05 from split
// BF16 operands (about 2^-16 of sum |a||b| per entry); the split buffers are
// setup_tc_n_pad(n) / setup_tc_s_pad(s) x setup_tc_kp(K) BF16 each.
void launch_gemm_tc_f32(cudaStream_t st, const float* A, int n, int K, int lda, const float* B,
                        int s, int ldb, float scale, float* F, int ldf, __nv_bfloat16* Ah,
                        __nv_bfloat16* Al, __nv_bfloat16* Bh, __nv_bfloat16* Bl, int* err);
// z2 = s2^-1/2 P H D z1 per row (SRHT, Section 4; krr_sketch.cu): signs (m),
// rows (s2) on the device, m a power of two >= s1.
void launch_srht(cudaStream_t st, const float* Z1, int n, int s1, int ldz1,
                 const signed char* signs, int m, const int* rows, int s2, float* Z2, int ldz2);
// G = Zs^T Zs + shift I (s x s FP64, exact) from Z^T; part: gram_tc_part_elems ints.
void launch_gram_tc(cudaStream_t st, const __nv_bfloat16* ZT, int n, int s, double shift,
                    int* part, double* G, int* err);

// Polynomial kernel (gamma x.z + c)^q of Section 6: TensorSketch features
// (krr_sketch.cu; hash, sign: q x d~ tables on the device, d~ = d + (c > 0))
// and the FP64 SIMT product (krr_matvec_simt.cu; part: mv_fp64_part_elems).
void launch_tensorsketch(cudaStream_t st, const float* X, int n, int d, int ldx, const int* hash,
                         const signed char* sign, int q, int s, double gamma, double c, float* Z,
                         int ldz);
void launch_mv_fp64_poly(cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
                         int nc, int ldxc, int d, double gamma, double c, int q, double shift,
                         const double* V, int k, int ldv, double* Q, int ldq, double* part);

// Adaptive sketch size (krr_adaptive.cu, Theorem 4).  work: adaptive_work_elems
// doubles.  adaptive_projector leaves Q = G^-1 Pi (Pi: the spectral projection
// of G = Z^T Z on eigenvalues above tau) in the work buffer; apply_i_minus_p
// then gives out = (I - Z Q Z^T) x for FP32 Z (n x s) and FP64 x.
size_t adaptive_work_elems(int n, int s);
void adaptive_projector(cudaStream_t st, const double* G, int s, double tau, int ns_iters,
                        double* work, int* info_dev, int* info_host);
void apply_i_minus_p(cudaStream_t st, const float* Z, int n, int s, const double* work,
                     const double* x, double* out);
void launch_scale_d(cudaStream_t st, double* x, int n, double a);

// Preconditioner (krr_precond.cu)
void launch_copy_z(cudaStream_t st, const float* Z, int n, int s, int ldz, void* Zs, int bf16);
void launch_gram(cudaStream_t st, const void* Zs, int bf16, int n, int s, double lam_p,
                 double* G, double* part, int nchunk);
int gram_chunks(int n, int s);
void launch_cholesky(cudaStream_t st, double* A, int s, int* info);
// Linv = L^-1 (lower, FP64) by recursive blocking; scratch: tri_inverse_scratch_elems(s).
size_t tri_inverse_scratch_elems(int s);
void launch_tri_inverse(cudaStream_t st, const double* L, int s, double* Linv, double* scratch);
// C = alpha op(A) op(B) + beta C, FP64, row-major with leading dimensions.
void launch_gemm_d(cudaStream_t st, int m, int n, int k, double alpha, const double* A, int lda,
                   int ta, const double* B, int ldb, int tb, double beta, double* C, int ldc);
void launch_transpose_d(cudaStream_t st, const double* A, int s, double* B);
void launch_form_u(cudaStream_t st, const double* Linv, const void* Zs, int bf16, int n, int s,
                   float* U);
// z = (r - Z Linv^T Linv Z^T r) / lam_p or (r - U^T U r) / lam_p.
// R, Zo: n x k with leading dimension ldr / ldo, element type T (float or double).
// t1, t2: s*k doubles of scratch; part: apply_part_elems doubles of scratch.
size_t apply_part_elems(int n, int s, int k);
// t1 = G^-1 Z^T R (s x k, ld k) with the ZL factors: the first half of the
// apply, which is the random-features ridge solution when R = Y.
void launch_ginv_zt(cudaStream_t st, const Precond& pc, const double* R, int k, int ldr,
                    double* t1, double* t2, double* part);
// F = Zf w: Zf m x s FP32 (ld s), w s x k double (ld k), F m x k (ldf); FP64 sums.
void launch_feature_gemv(cudaStream_t st, const float* Zf, int m, int s, const double* w, int k,
                         double* F, int ldf);
template <typename T>
void launch_apply(cudaStream_t st, const Precond& pc, const T* R, int k, int ldr, T* Zo,
                  int ldo, double* t1, double* t2, double* part);

// The apply with one PCG iteration's vector work fused into its two streamed
// passes over Z (the fused loop body, vectors n x k with ld = k):
//   Z^T pass: r' = r - alpha q and x' = x + alpha p (alpha from sc), written
//             to Rn and X, ||r'||^2 reduced and the stopping test applied;
//   Z w pass: z = M^-1 r' from Rn, r' copied back to R, r'.z reduced, beta
//             and the loop's continue decision (graph condition `cond`).
template <typename T>
struct CgStepArgs {
  CgScalars* sc = nullptr;
  T* X = nullptr;
  const T* P = nullptr;
  const T* Q = nullptr;
  T* Rn = nullptr;            // n x k scratch: the updated residual between the passes
  double* cpart = nullptr;    // cg_part_elems() doubles (the CG reductions' partials)
  unsigned long long cond = 0;
};
// True when launch_apply_cg can serve k right-hand sides (the streamed ZL
// kernels: rows of Z 16-byte aligned, the staged rows within shared memory).
bool apply_cg_supported(const Precond& pc, int n, int k);
template <typename T>
void launch_apply_cg(cudaStream_t st, const Precond& pc, T* R, int k, T* Zo, double* t1,
                     double* t2, double* part, const CgStepArgs<T>& f);

// CG vector kernels (krr_cg.cu).  `part` is cg_part_elems() doubles.
struct ColScale {
  double v[KRR_MAX_RHS];
};
size_t cg_part_elems(int n, int k);
template <typename T>
void launch_cg_init(cudaStream_t st, CgScalars* sc, const double* Y, int ldy, const T* R, int n,
                    int k, double tol, int max_iter, double* part, double* hist = nullptr,
                    int hist_cap = 0);
template <typename T>
void launch_cg_rz_first(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, T* P, int n,
                        int k, double* part);
// Restart that keeps the previous search direction (a residual replacement):
// with r and z = M^-1 r the replaced residual, P the previous solve's last
// direction and s[c] the factor from the previous solve's units to these,
// p = z + beta (s P - (r.(s P) / r.z) z), beta = r.z / (s^2 r.z_previous).
// Needs 3 k <= KRR_MAX_RHS; columns without a usable previous step get p = z.
template <typename T>
void launch_cg_restart(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, T* P, int n,
                       int k, const ColScale& s, double* part);
template <typename T>
void launch_cg_alpha(cudaStream_t st, CgScalars* sc, const T* P, const T* Q, int n, int k,
                     double* part);
template <typename T>
void launch_cg_update_xr(cudaStream_t st, CgScalars* sc, T* X, T* R, const T* P, const T* Q,
                         int n, int k, double* part);
template <typename T>
void launch_cg_rz(cudaStream_t st, CgScalars* sc, const T* R, const T* Z, int n, int k,
                  double* part);
template <typename T>
void launch_cg_update_p(cudaStream_t st, CgScalars* sc, T* P, const T* Z, int n, int k);
// The fused loop body's CG steps (FP32 vectors, the tensor-core product):
// q from the product's chunk sums (nchunk x n_rpad x kv, row factors ra) with
// p.q and alpha in the same pass; and p = z + beta p (update != 0) with the
// product's weights w = ra p (n_pad x kv) for the next iteration.
template <typename T>
void launch_cg_reduce_alpha(cudaStream_t st, CgScalars* sc, const float* part, int nchunk,
                            int n_rpad, int kv, const float* ra, double shift, const T* P, T* Q,
                            int n, int k, double* cpart);
template <typename T>
void launch_cg_update_pw(cudaStream_t st, CgScalars* sc, T* P, const T* Z, int n, int k,
                         int update, const float* ra, int n_pad, int kv, float* w);
// iter += 1; decides whether the loop continues; sets the graph condition
// when `cond` is nonzero (a cudaGraphConditionalHandle).
void launch_cg_tail(cudaStream_t st, CgScalars* sc, unsigned long long cond);
// Lockstep loops over several independent solves (one CgScalars each):
// gate sets the IF condition `conds[i]` of solve i to scs[i]->run; tail sets
// the WHILE condition `cond` to whether any solve still runs.
void launch_batch_gate(cudaStream_t st, CgScalars* const* scs, const unsigned long long* conds,
                       int nsolve);
void launch_batch_tail(cudaStream_t st, CgScalars* const* scs, int nsolve,
                       unsigned long long cond);

// mu[t] = mean_i X[i, t] in FP64, deterministic (slab scratch: ceil(n/128) x d doubles)
void launch_colmean(cudaStream_t st, const float* X, int n, int ld, int d, double* mu,
                    double* slab);

// Elementwise helpers (row-major n x k blocks)
template <typename A, typename B>
void launch_convert(cudaStream_t st, const A* a, int n, int k, int lda, B* b, int ldb,
                    const ColScale& scale);
// c += scale * d (d float or double, c double)
template <typename D>
void launch_axpy_d(cudaStream_t st, const D* dlt, int n, int k, int ldd, double* c, int ldc,
                   const ColScale& scale);
// r = y - a
void launch_sub_d(cudaStream_t st, const double* y, int ldy, const double* a, int lda, int n,
                  int k, double* r, int ldr);
// out[c] = sum_i a[i, c]^2 (FP64), written to device memory
template <typename T>
void launch_colnorm2(cudaStream_t st, const T* a, int n, int k, int lda, double* out,
                     double* part, unsigned int* counter);
// out[0] = sum_{i, c} a[i, c] b[i, c] (FP64), written to device memory
void launch_dot_d(cudaStream_t st, const double* a, int lda, const double* b, int ldb, int n,
                  int k, double* out, double* part, unsigned int* counter);

}  // namespace krr
