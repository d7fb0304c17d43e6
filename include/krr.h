/*
 * krr.h -- C ABI of the GB300 kernel ridge regression library.
 *
 * The library solves the kernel ridge regression system (K + lambda I) c = y
 * (Eq. (1) of Avron, Clarkson, Woodruff, "Faster Kernel Ridge Regression Using
 * Sketching and Preconditioning") for the Gaussian kernel
 * k(x, z) = exp(-||x - z||^2 / (2 sigma^2)) (Section 5) by preconditioned
 * conjugate gradients with the random-Fourier-feature preconditioner
 * Z Z^T + lambda_p I applied through the Woodbury identity (Algorithm 1,
 * Section 3.1).  K is never stored: every product with it is recomputed.
 *
 * Conventions (every entry point):
 *  - Every function returns a krr_status; KRR_OK is 0.  On any other status
 *    krr_last_error(h) returns a message describing the failure.
 *  - Matrices are row-major with an explicit leading dimension (elements).
 *  - Pointers are plain device pointers unless the function says "host or
 *    device": those accept either and stage host buffers through the
 *    library's workspace.  The caller owns every input and output buffer.
 *  - The handle owns its workspace and the preconditioner factors; it
 *    allocates device memory lazily and frees it in krr_destroy.
 *  - All work is enqueued on the handle's stream.  Entry points that return
 *    device results return without synchronising except where a status
 *    depends on device data (the solves, precond setup), which read a few
 *    bytes back at the end.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef KRR_H_
#define KRR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int krr_status;
enum {
  KRR_OK = 0,
  KRR_EINVAL = 1,       /* bad argument (size, pointer, leading dimension)  */
  KRR_ENOMEM = 2,       /* device allocation failed                         */
  KRR_ECUDA = 3,        /* a CUDA runtime call failed                       */
  KRR_ECHOL = 4,        /* Z^T Z + lambda_p I not positive definite         */
  KRR_ENOTCONV = 5,     /* max_iter reached; outputs hold the last iterate  */
  KRR_EBREAKDOWN = 6,   /* p.q <= 0 or r.z <= 0 (indefinite operator)       */
  KRR_ENAN = 7,         /* NaN or Inf met in the iteration                  */
  KRR_ETIMEOUT = 8,     /* a device loop hit its iteration cap              */
  KRR_EUNSUPPORTED = 9  /* valid request this build does not implement      */
};

/* Arithmetic of a kernel-matrix product (the n^2 part of each iteration). */
typedef enum {
  KRR_FP64 = 0,        /* FP64 SIMT: distances from coordinate differences  */
  KRR_FP32 = 1,        /* FP32 SIMT: the plain single-precision path        */
  KRR_BF16 = 2,        /* tcgen05 BF16 tensor cores, FP32 accumulation      */
  KRR_HP = 3,          /* extended precision for refinement residuals       */
  KRR_MIXED = 4,       /* solver only: FP16/BF16 inner PCG + HP refinement  */
  KRR_BF16X3 = 5,      /* tcgen05 BF16 on split points (hi + lo, d <= 64):  */
                       /* hi.hi + lo.hi + hi.lo, about 2^-16 relative dots  */
  KRR_BF16P = 6,       /* KRR_BF16 with the contraction with V on the tensor */
                       /* cores (exp2 values rounded to BF16, 2^-9 each);    */
                       /* products only: the entrywise rounding can make    */
                       /* K + lambda I indefinite, so solvers never use it   */
  KRR_FP16 = 7         /* KRR_BF16 on FP16-rounded points: same tensor rate, */
                       /* 2^-12 instead of 2^-9 relative point rounding     */
} krr_precision;

/* How the preconditioner is applied (Section 3.1). */
typedef enum {
  KRR_APPLY_ZL = 0,    /* z = (r - Z L^-T L^-1 Z^T r) / lambda_p            */
  KRR_APPLY_U = 1      /* z = (r - U^T U r) / lambda_p, U = L^-1 Z^T        */
} krr_apply_form;

/* How the handle stores the features Z of the preconditioner. */
typedef enum {
  KRR_Z_FP32 = 0,      /* FP32 copy; Gram accumulated in FP64 on the SIMT pipes */
  KRR_Z_BF16 = 1,      /* BF16 copy; Gram of the rounded values, FP64 sums     */
  KRR_Z_FIXED = 2      /* 7-bit fixed point: Z ~= 2^e Zs, Zs = q / 128 with     */
                       /* q = clamp(rint(z 2^(7-e)), -127, 127) and 2^e the    */
                       /* smallest power of two >= max |z|; the Gram of Zs is  */
                       /* formed exactly on the tensor cores (integer sums)    */
} krr_z_format;

#define KRR_MAX_RHS 16

typedef struct {
  double tol;          /* relative residual target tau (default 1e-6)        */
  int max_iter;        /* PCG iteration cap (default 1000, Section 5)        */
  double lambda_p;     /* preconditioner ridge; 0 means lambda (Table 2)     */
  int precond;         /* 1: RFF Woodbury preconditioner, 0: plain CG,       */
                       /* 2: keep the handle's preconditioner from the last  */
                       /* krr_precond_setup (any features: caller's,         */
                       /* multiple-level, adaptive) -- single solves only    */
  int precision;       /* krr_precision; KRR_MIXED adds refinement           */
  int apply_form;      /* krr_apply_form                                     */
  int use_graph;       /* 1: PCG loop as a CUDA-graph while node             */
  double inner_tol;    /* KRR_MIXED: inner PCG relative tolerance (0.03)     */
  int max_outer;       /* KRR_MIXED: refinement step cap                     */
  int z_format;        /* krr_z_format of the preconditioner's features;     */
                       /* -1 auto: KRR_Z_FIXED for KRR_MIXED (features and   */
                       /* Gram on the tensor cores), else KRR_Z_FP32         */
  int warm_start;      /* 1: C holds x0 on entry                             */
  int inner_precision; /* KRR_MIXED: product of the inner PCG, KRR_FP16,     */
                       /* KRR_BF16 or KRR_BF16X3 (split points, d <= 64),    */
                       /* or KRR_HP (FP64 vectors and HP products from the   */
                       /* start: PCG in FP64-grade arithmetic throughout)    */
                       /* (0: the default, KRR_FP16)                         */
  int batch_product;   /* krr_pcg_solve_batched, KRR_MIXED: 1 (default) runs  */
                       /* the FP16-point products of all problems (k = 1,    */
                       /* d <= 128) as one persistent launch per iteration;  */
                       /* 0: each problem launches its own                   */
  int keep_direction;  /* KRR_MIXED: 1 continues the previous inner solve's  */
                       /* search direction after the residual is replaced   */
                       /* (k <= 5); 0 (default) restarts each at p = z      */
  int fuse_step;       /* KRR_MIXED, single solves: 1 (default) runs an FP32  */
                       /* inner PCG iteration as 8 launches, the CG vector   */
                       /* updates fused into the passes that read the same   */
                       /* vectors (the product's chunk sums, the apply's two */
                       /* streamed passes over Z); 0: separate CG kernels    */
                       /* (13 launches). Same arithmetic either way.         */
} krr_opts;

typedef struct {
  int status;                       /* same value the call returned          */
  int k;                            /* number of right-hand sides            */
  int iters[KRR_MAX_RHS];           /* PCG iterations per column (all steps) */
  double rel_res[KRR_MAX_RHS];      /* final relative residual per column,   */
                                    /* computed on device in the solve's     */
                                    /* residual arithmetic                   */
  int outer_steps;                  /* refinement steps (KRR_MIXED)          */
  int matvecs;                      /* kernel-matrix products launched       */
  double ms_setup;                  /* features + Gram + Cholesky + factors  */
  double ms_solve;                  /* PCG (and refinement)                  */
  double ms_total;
  double kappa[KRR_MAX_RHS];        /* Lanczos estimate of cond(M^-1 A) per  */
                                    /* column from the CG coefficients of    */
                                    /* its first 4096 steps (the largest     */
                                    /* over a solve's inner loops; 0: none)  */
  double rel_res_rec[KRR_MAX_RHS];  /* relative residual the last loop's     */
                                    /* recurrence reached (in units of ||y|| */
                                    /* for refined solves)                   */
} krr_report;

typedef struct krr_handle krr_handle;

/* Fill *o with the defaults listed above. */
void krr_default_opts(krr_opts* o);

/* Create a handle bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current device. */
krr_status krr_create(krr_handle** h, void* stream);
krr_status krr_destroy(krr_handle* h);
krr_status krr_set_stream(krr_handle* h, void* stream);
const char* krr_last_error(const krr_handle* h);
const char* krr_status_string(krr_status s);

/*
 * Tile-plan autotuning of the tensor-core product (KRR_BF16, KRR_FP16,
 * KRR_BF16X3; the paper has no counterpart, its kernel products are library
 * calls).  With on = 1 the first product of each shape (row tiles, column
 * tiles, K-blocks, RHS bucket, operand format) on this handle times the
 * candidate plans -- column chunks per row tile x TMA ring stages -- on
 * scratch right-hand sides and keeps the fastest for the rest of the
 * process; the first product of a shape therefore synchronises the stream.
 * Solves time their shapes before they capture a graph.  Off (0) by
 * default: the plan then follows a fixed wave-balance rule, and results do
 * not depend on timing.  on = 2 selects, without timing, the symmetric
 * product where it applies (one right-hand side, d <= 64, BF16 or FP16
 * points): only the tiles on and above the block diagonal, each exponential
 * serving K_ij and K_ji (half the exponentials), with 16 epilogue warps;
 * on = 3 the same with 8 epilogue warps.  Batched solves pass the setting to
 * their problems.  `shapes` (may be NULL) receives the number of shapes
 * tuned so far in this process.  Errors: KRR_EINVAL for a NULL handle or on
 * outside 0..3.
 */
krr_status krr_set_autotune(krr_handle* h, int on, int* shapes);

/*
 * Random Fourier features, Section 2.2:
 *   Z[i, j] = sqrt(2/s) * cos(sum_t X[i, t] W[t, j] + b[j]).
 * X: n x d (ldx), W: d x s (lds = s), b: s, Z: n x s output (ldz), all FP32.
 * W has N(0, sigma^-2) entries and b is U[0, 2 pi) for the Gaussian kernel;
 * they are inputs so that callers can reproduce a draw.
 */
krr_status krr_rff_features(krr_handle* h, const float* X, int n, int d, int ldx,
                            const float* W, const float* b, int s,
                            float* Z, int ldz);

/*
 * The same features on the tensor cores in the fixed-point form of
 * KRR_Z_FIXED (the mixed solves' preconditioner): Zq (n x s, ldz >= s, int8,
 * device memory) holds q = clamp(rint(z 2^(7-e)), -127, 127), so
 * Z ~= 2^(e-7) q, with 2^e the smallest power of two >= sqrt(2/s); e is
 * written to *e_out.  X W runs on split BF16 operands (hi.hi + lo.hi +
 * hi.lo), so the cosine's argument carries about 2^-16 of sum_t |x_t||w_t| of
 * error besides FP32 rounding.  X, W, b in device memory.
 */
krr_status krr_rff_features_fixed(krr_handle* h, const float* X, int n, int d, int ldx,
                                  const float* W, const float* b, int s, signed char* Zq, int ldz,
                                  int* e_out);

/*
 * Kernel-matrix product, the per-iteration cost the paper names dominant
 * (Section 3.1, "multiplying the kernel matrix by a vector"):
 *   Q[i, :] = sum_j k(xr_i, xc_j) V[j, :] + shift * V[i, :]
 * Xr: nr x d (ldxr), Xc: nc x d (ldxc), FP32.  V: nc x k (ldv), Q: nr x k
 * (ldq).  V and Q are double for KRR_FP64 and KRR_HP and float for KRR_FP32,
 * KRR_BF16, KRR_FP16, KRR_BF16X3 and KRR_BF16P.  `shift` (lambda of Eq. (1))
 * needs nr == nc and is added
 * only when it is nonzero; pass Xr == Xc for the training system.  The
 * tensor-core products take any row set (Xr != Xc) except KRR_BF16P.
 * 1 <= k <= KRR_MAX_RHS.
 */
krr_status krr_kernel_matvec(krr_handle* h, const float* Xr, int nr, int ldxr,
                             const float* Xc, int nc, int ldxc, int d,
                             double sigma, double shift,
                             const void* V, int k, int ldv, void* Q, int ldq,
                             int precision);

/*
 * Preconditioner set-up of Algorithm 1 and Section 3.1:
 *   G = Z^T Z + lambda_p I_s (FP64 accumulation), L L^T = G (FP64
 *   Cholesky, lower L), then either U = L^-1 Z^T (KRR_APPLY_U, stored FP32
 *   s x n) or L^-1 kept for triangular solves (KRR_APPLY_ZL).
 * Z: n x s (ldz) FP32; the handle keeps its own copy in `z_format`
 * (krr_z_format; KRR_Z_FIXED stores the 8-bit q, one byte per feature, which
 * halves the apply's bytes against BF16).  With KRR_Z_BF16 or KRR_Z_FIXED, G is formed from the
 * stored (rounded) values, so the factors describe exactly the operator
 * applied, (Zt Zt^T + lambda_p I)^-1 with Zt the stored features; with
 * KRR_Z_FIXED that Gram is exact (integer sums on the tensor cores) and the
 * call synchronises once to find max |Z|.  s <= n.
 * Returns KRR_ECHOL when a pivot of the Cholesky factorisation is <= 0 or Z
 * holds a NaN or Inf, KRR_ETIMEOUT when a tensor-core wait hit its limit.
 */
krr_status krr_precond_setup(krr_handle* h, const float* Z, int n, int s, int ldz,
                             double lambda_p, int apply_form, int z_format);

/*
 * Apply the preconditioner inverse of the last krr_precond_setup
 * (the PCG step of Algorithm 1):  Zout = (Z Z^T + lambda_p I)^-1 R.
 * R, Zout: n x k double (ldr, ldo).  1 <= k <= KRR_MAX_RHS.
 */
krr_status krr_precond_apply(krr_handle* h, const double* R, int k, int ldr,
                             double* Zout, int ldo);

/*
 * Algorithm 1 end to end: RFF features from (W, b), preconditioner set-up,
 * PCG from x0 = 0 (or C when opts->warm_start) on (K + lambda I) C = Y,
 * stopping when ||y - (K + lambda I) c|| <= tol ||y|| for every column
 * (Section 5).  X: n x d (ldx) FP32; W: d x s FP32; b: s FP32;
 * Y, C: n x k double (ldy, ldc).  X, W, b, Y and C may be host or device
 * pointers.  With opts->precision == KRR_MIXED the inner PCG runs the
 * tensor-core product of opts->inner_precision (FP16 points by default, or
 * BF16) and an outer refinement loop recomputes the residual
 * in KRR_HP arithmetic and FP64 vectors; when a correction contracts the
 * residual by less than a half, later inner solves use KRR_BF16X3 (d <= 64)
 * and then KRR_HP products.  `rep` (may be NULL) receives the
 * per-column report.  Returns KRR_ENOTCONV if max_iter is reached (C holds
 * the last iterate), KRR_EBREAKDOWN / KRR_ENAN on breakdown.
 */
krr_status krr_pcg_solve(krr_handle* h, const float* X, int n, int d, int ldx,
                         double sigma, double lambda,
                         const float* W, const float* b, int s,
                         const double* Y, int k, int ldy, double* C, int ldc,
                         const krr_opts* opts, krr_report* rep);

/*
 * One independent problem of a batch: the arguments of krr_pcg_solve for
 * one system (K + lambda I) C = Y (Eq. (1)) with its own RFF draw.  Any
 * pointer may be host or device memory.
 */
typedef struct krr_problem {
  const float* X;   /* n x d (ldx) FP32 */
  int n, d, ldx;
  double sigma, lambda;
  const float* W;   /* d x s FP32 (may be NULL when opts->precond == 0) */
  const float* b;   /* s FP32 */
  int s;
  const double* Y;  /* n x k (ldy) */
  int k, ldy;
  double* C;        /* n x k (ldc), output */
  int ldc;
} krr_problem;

/*
 * Algorithm 1 for `nprob` independent problems of any sizes.  The paper
 * solves one problem at a time; this call runs their PCG loops in lockstep
 * inside one CUDA graph launch per refinement round: each problem's
 * iteration sits under its own conditional node, so a converged problem
 * stops costing launches while the others continue, and the graph runs
 * the problems' kernels concurrently (largest n first).  Set-up (features,
 * factors) runs per problem before the loop.  opts applies to every
 * problem (KRR_FP64, KRR_FP32 or KRR_MIXED; warm_start must be 0).
 * reps (may be NULL) receives nprob reports; their ms_* fields are the
 * batch's times.  Returns KRR_OK when every problem converged, otherwise
 * the status of the first problem (in the caller's order) that did not.
 */
krr_status krr_pcg_solve_batched(krr_handle* h, const krr_problem* probs, int nprob,
                                 const krr_opts* opts, krr_report* reps);

/*
 * Random-features method (Section 2.2: the random Fourier features used as
 * the model instead of as a preconditioner): the ridge regression in feature
 * space
 *   w = (Z^T Z + lambda I_s)^-1 Z^T Y,   Z = sqrt(2/s) cos(X W + b),
 * computed with the preconditioner's set-up (FP32 Z, FP64 Gram and Cholesky
 * of Algorithm 1, with lambda_p = lambda) and the first half of its apply
 * (Z^T Y, then L^-1 and L^-T).  By the push-through identity its predictions
 * at the training points are those of kernel ridge regression with the
 * approximate kernel Z Z^T.  X: n x d (ldx) FP32; W: d x s, b: s FP32;
 * Y: n x k double (ldy); Wf: s x k double (ldw) out; 0 < s <= n.  Host or
 * device pointers.  Replaces the handle's preconditioner factors.  Errors:
 * KRR_EINVAL (sizes, s > n, lambda <= 0), KRR_ECHOL (Gram not positive
 * definite).
 */
krr_status krr_rfm_fit(krr_handle* h, const float* X, int n, int d, int ldx,
                       const float* W, const float* b, int s, double lambda,
                       const double* Y, int k, int ldy, double* Wf, int ldw);

/*
 * The random-features predictor F = phi(Xte) Wf with
 * phi(x) = sqrt(2/s) cos(x W + b): Xte m x d (ldx) FP32, W and b as for
 * krr_rfm_fit, Wf s x k double (ldw), F m x k double (ldf); FP64 sums over
 * the s features.  Host or device pointers.
 */
krr_status krr_rfm_predict(krr_handle* h, const float* Xte, int m, int d, int ldx,
                           const float* W, const float* b, int s, const double* Wf,
                           int k, int ldw, double* F, int ldf);

/*
 * Predictor f(x) = sum_i c_i k(x_i, x) (Section 1) at m held-out points:
 *   F = K(Xte, Xtr) C.  Xtr: n x d (ldxtr), Xte: m x d (ldxte) FP32,
 * C: n x k double (ldc), F: m x k double (ldf); host or device pointers
 * (F is written before the call returns when it is a host pointer).
 * precision: KRR_FP64, KRR_HP, KRR_FP32 (FP32 then widened), or a
 * tensor-core product on rounded points, KRR_FP16, KRR_BF16 or KRR_BF16X3
 * (C rounded to FP32; the held-out points rounded with the training mean and
 * scale; KRR_EUNSUPPORTED when a held-out point lies so far from the training
 * mean that the factored exp2 would overflow).  The rounded-point products
 * carry the point rounding's error (about 2^-12 relative of -log K for FP16,
 * 2^-16 for BF16X3), amplified by sum_j |K_ij||c_j| / |f_i|: use them when c
 * does not cancel heavily.
 */
krr_status krr_predict(krr_handle* h, const float* Xtr, int n, int ldxtr,
                       const float* Xte, int m, int ldxte, int d, double sigma,
                       const double* C, int k, int ldc, double* F, int ldf,
                       int precision);

/* --------------------------------------------- batched products ------- */
/* One problem of krr_kernel_matvec_batched. */
typedef struct {
  const float* X;      /* n x d training points (ldx), device              */
  int n, d, ldx;       /* d <= 128                                          */
  double sigma;        /* Gaussian kernel bandwidth                         */
  double shift;        /* lambda: Q = K V + shift V                          */
  const float* V;      /* n x 1 right-hand side, device                     */
  float* Q;            /* n x 1 product, device                             */
} krr_matvec_problem;

/*
 * The kernel products of up to 64 independent problems (the uneven batch of
 * independent KRR problems) in one persistent tensor-core launch: every
 * problem's (128-row tile, column chunk) items in one work list, largest
 * first, dealt to one CTA per SM.  The arithmetic is KRR_FP16's (the
 * Gaussian kernel of the FP16-rounded, centred, scaled points), one
 * right-hand side per problem.  Besides the kernel, one launch forms every
 * problem's weights and one adds the partial sums.  The paper has no
 * counterpart; krr_pcg_solve_batched uses the same launch for its inner
 * solves (opts->batch_product).
 */
krr_status krr_kernel_matvec_batched(krr_handle* h, const krr_matvec_problem* probs,
                                     int count);

/* ------------------------------------------- polynomial kernel -------- */
/*
 * The paper's second kernel (Section 6): k(x, z) = (gamma x^T z + c)^q,
 * gamma > 0, c >= 0, 1 <= q <= 8, with its TensorSketch feature map
 * (Section 2.2) as the preconditioner's features.
 */

/*
 * TensorSketch features Z = phi(X) (Section 2.2): with x~ = [sqrt(gamma) x,
 * sqrt(c)] (the extra coordinate only when c > 0; d~ = d + 1, else d),
 *   phi(x)[H] = sum of g_1(i_1)..g_q(i_q) x~_{i_1}..x~_{i_q} over the index
 *               tuples with (h_1(i_1) + .. + h_q(i_q)) mod s = H,
 * so E phi(x)^T phi(z) = (gamma x^T z + c)^q.  hash: q x d~ int32 in [0, s),
 * sign: q x d~ int8 in {-1, +1} (row t is the t-th CountSketch; host or
 * device, checked on the host: KRR_EINVAL when out of range).  X: n x d
 * (ldx) FP32 on the device, Z: n x s (ldz >= s) FP32 on the device; FP32
 * arithmetic.  s <= 25,600.
 */
krr_status krr_tensorsketch_features(krr_handle* h, const float* X, int n, int d, int ldx,
                                     const int* hash, const signed char* sign, int q, int s,
                                     double gamma, double c, float* Z, int ldz);

/*
 * Polynomial-kernel product Q = P(Xr, Xc) V + shift V, P_ij = (gamma
 * xr_i.xc_j + c)^q.  precision: KRR_FP64 (FP64 dot products, any row set;
 * V, Q double) or, for the training system (Xr == Xc), the fused tensor-core
 * kernel on rounded points, KRR_FP16, KRR_BF16 or KRR_BF16X3 (x rounded
 * without scaling or centring, the power on the FMA pipe; V, Q float;
 * KRR_EUNSUPPORTED when a point overflows FP16/BF16).  Device pointers.
 */
krr_status krr_kernel_matvec_poly(krr_handle* h, const float* Xr, int nr, int ldxr,
                                  const float* Xc, int nc, int ldxc, int d, double gamma,
                                  double c, int q, double shift, const void* V, int k, int ldv,
                                  void* Q, int ldq, int precision);

/*
 * Algorithm 1 for the polynomial kernel: solve (P + lambda I) C = Y with PCG,
 * preconditioned by (Z Z^T + lambda_p I)^-1 through the Woodbury identity,
 * Z the TensorSketch features of X (hash, sign as for
 * krr_tensorsketch_features; unused when opts->precond = 0).  Arguments,
 * staging and report as for krr_pcg_solve; opts->precision is KRR_FP64 (FP64
 * products) or KRR_MIXED (tensor-core inner solves on rounded points,
 * refinement with FP64 residuals).
 */
krr_status krr_poly_pcg_solve(krr_handle* h, const float* X, int n, int d, int ldx, double gamma,
                              double c, int q, double lambda, const int* hash,
                              const signed char* sign, int s, const double* Y, int k, int ldy,
                              double* C, int ldc, const krr_opts* opts, krr_report* rep);

/* ------------------------------------ multiple-level sketching -------- */
/*
 * Features of Algorithm 2 (Section 4) from first-level features Z1 (n x s1,
 * ldz1; random Fourier or TensorSketch features):
 *   Z2 = Z1 S2^T,  S2 = s2^-1/2 P H D  (a subsampled randomized Walsh-Hadamard
 *                                        transform: D = diag(signs), H = H_m,
 *                                        P keeps rows `rows` of H D),
 *   Z3 = s3^-1/2 Z2 G^T                 (G: s3 x s2 standard normal entries).
 * m: a power of two with s1 <= m <= 32768 (Z1's rows are zero-padded to m);
 * signs: m int8 in {-1, +1}; rows: s2 int32 in [0, m) (host or device,
 * checked on the host); s3 <= s2 <= m.  Z1, G (FP32, row-major) and Z3
 * (n x s3, ldz3, FP32) in device memory.  The transform runs per row in
 * shared memory (log2 m butterfly passes); Z2 G^T on tcgen05 from split BF16
 * operands (about 2^-16 of sum |z2||g| per entry).  Feed Z3 to
 * krr_precond_setup and solve with opts->precond = 2.
 */
krr_status krr_multilevel_features(krr_handle* h, const float* Z1, int n, int s1, int ldz1,
                                   const signed char* signs, int m, const int* rows, int s2,
                                   const float* G, int s3, float* Z3, int ldz3);

/* ------------------------------------------ adaptive sketch size ------ */
/*
 * Preconditioner set-up with the number of random Fourier features chosen
 * adaptively (Section 5, Theorem 4), for the Gaussian kernel: from s = s0,
 * features Z of the first s columns of W (d x s_max, row-major) and b are
 * tested against Theorem 4's first condition
 *     ||(I - P) K (I - P)||_2 <= 0.1 lambda,
 * P the orthogonal projection on the eigenvectors of Z Z^T with eigenvalues
 * above 0.05 lambda, by `power_iters` steps of power iteration from x0 (n
 * doubles); s doubles (capped at s_max) until the test passes.  P comes from
 * the s x s Gram matrix: P = Z G^-1 Pi Z^T with Pi the spectral projection of
 * G on eigenvalues above 0.05 lambda, sign(I - 2 tau (G + tau I)^-1) by
 * `ns_iters` Newton-Schulz steps (FP64; 25 resolves eigenvalues within about
 * 1 % of the threshold).  The second condition's test is left out (the paper
 * omits it).  product_precision: the K products of the power iteration,
 * KRR_FP64, KRR_HP or KRR_FP16.  The handle's preconditioner is then set up
 * from the chosen features with lambda_p (0: lambda), apply_form and
 * z_format (krr_z_format; -1: KRR_Z_FP32); solve with opts->precond = 2.
 * *s_out: the chosen s; estimates (may be NULL, room for log2(s_max/s0) + 2
 * values): the power-iteration estimate at each s tried; *tests_out (may be
 * NULL): how many s were tried.  X, W, b, x0: host or device.
 */
krr_status krr_precond_setup_adaptive(krr_handle* h, const float* X, int n, int d, int ldx,
                                      double sigma, double lambda, const float* W,
                                      const float* b, int s_max, int s0, const double* x0,
                                      int power_iters, int ns_iters, int product_precision,
                                      double lambda_p, int apply_form, int z_format, int* s_out,
                                      double* estimates, int* tests_out);

/* --------------------------------------- hyper-parameter gradient ------ */
/*
 * The paper fixes sigma and lambda and does not differentiate the solution.
 * These two calls add the gradient of a held-out loss with respect to
 * log sigma and log lambda, derived from Eq. (1) and the Gaussian kernel of
 * Section 5 (k(x, z) = exp(-||x - z||^2 / (2 sigma^2))):
 *   A = K + lambda I,  c = A^-1 y,  f = K(Xte, X) c,
 *   dK/dlog(sigma) = D o K,  D_ij = ||x_i - x_j||^2 / sigma^2,
 *   dA/dlog(lambda) = lambda I.
 */

/*
 * Derivative product  Q = (D o K)(Xr, Xc) V  (the lambda I term has no
 * sigma dependence, so there is no shift).  Xr: nr x d (ldxr), Xc: nc x d
 * (ldxc) FP32; V: nc x k (ldv), Q: nr x k (ldq) double; device pointers.
 * precision: KRR_FP64 (distances summed from differences, FP64 exp),
 * KRR_HP (float-float SIMT), or the tensor-core product on rounded points
 * (KRR_FP16, KRR_BF16, KRR_BF16X3): S = xh_i.xh_j on tcgen05 and, with
 * log2 K_ij = S_ij - nh_i/2 - nh_j/2, the epilogue contracts exp2(S) S and
 * exp2(S) so that D o K = -2 ln 2 (log2 K) o K is formed without K (V, Q
 * rounded to FP32 on the way).
 * 1 <= k <= KRR_MAX_RHS.  Returns KRR_EINVAL for bad arguments.
 */
krr_status krr_kernel_dsigma_matvec(krr_handle* h, const float* Xr, int nr, int ldxr,
                                    const float* Xc, int nc, int ldxc, int d,
                                    double sigma, const double* V, int k, int ldv,
                                    double* Q, int ldq, int precision);

/*
 * Backward pass of  F = K(Xte, X) (K + lambda I)^-1 Y  for a scalar loss L
 * whose gradient with respect to F is GF = dL/dF:
 *   gbar = K(X, Xte) GF,  w = A^-1 gbar  (adjoint solve: A is symmetric, so
 *   it is Algorithm 1 again with gbar as right-hand side, run with *opts),
 *   grad[0] = dL/dlog(sigma)  = sum(GF o ((Dte o Kte) C)) - sum(w o ((D o K) C)),
 *   grad[1] = dL/dlog(lambda) = -lambda sum(w o C).
 * X: n x d (ldx), Xte: m x d (ldxte) FP32; W (d x s), b (s): the RFF draw
 * for the adjoint solve's preconditioner (may be NULL when
 * opts->precond == 0); C: n x k (ldc) the forward solution; GF: m x k (ldg).
 * These may be host or device pointers.  grad: host array of 2 doubles.
 * Wadj (may be NULL): receives w, n x k (ldw), host or device.  rep (may be
 * NULL) reports the adjoint solve.  The products and the contractions run
 * in FP64; the adjoint solve in opts->precision.  Returns the adjoint
 * solve's status (grad is written in every case once the arguments pass).
 * opts->warm_start must be 0.
 */
krr_status krr_hypergrad(krr_handle* h, const float* X, int n, int d, int ldx,
                         const float* Xte, int m, int ldxte,
                         double sigma, double lambda,
                         const float* W, const float* b, int s,
                         const double* C, int ldc, const double* GF, int k, int ldg,
                         const krr_opts* opts, double* grad,
                         double* Wadj, int ldw, krr_report* rep);

/*
 * Kernel-matrix product that allocates nothing.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc when
 * they need the product -- code that runs while a stream is captured into
 * a CUDA graph (an allocation there breaks the capture), code inside a
 * framework whose caching allocator already holds the GPU's memory, and
 * loops that must avoid the device synchronisation an allocation may cause.
 *
 * Computes the same FP64 product as krr_kernel_matvec(..., KRR_FP64):
 *   Q[i, :] = sum_j k(xr_i, xc_j) V[j, :] + shift * V[i, :]
 * with the same argument meaning and layout (device pointers), enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream); no handle.
 * Its partial sums live in a fixed device array of 2^20 doubles (8 MiB)
 * that every GPU loading the library keeps until the process exits, so
 * nr * k must be at most 1048576; larger requests return KRR_EINVAL without
 * launching.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array: calls whose kernels may overlap on
 * the GPU (other streams, other threads) race and must be serialised by
 * the caller.  Returns KRR_EINVAL for bad arguments, KRR_ECUDA if the
 * lookup or a launch fails.
 */
krr_status krr_kernel_matvec_fp64_noalloc(const float* Xr, int nr, int ldxr,
                                          const float* Xc, int nc, int ldxc, int d,
                                          double sigma, double shift,
                                          const double* V, int k, int ldv,
                                          double* Q, int ldq, void* stream);

/* ------------------------------------------------------- diagnostics --- */
/* The paper has no counterpart for these; they serve measurement. */

/* Number of this library's kernels launched by the calling process so far,
 * kernels inside the PCG graph counted once per executed iteration. */
long long krr_launch_count(void);

/*
 * Throughput of the MUFU base-2 exponential on the handle's device: runs a
 * kernel of independent ex2.approx chains for `iters` steps per thread on
 * every SM and writes results per second to *ex2_per_s and the kernel time
 * to *ms.  Used to state the exp-bound roofline of the fused product.
 */
krr_status krr_bench_ex2(krr_handle* h, int iters, double* ex2_per_s, double* ms);

/*
 * Combined throughput of the two base-2 exponentials the fused products use:
 * every thread runs 32 independent chains for `iters` steps, `fma_per_32` of
 * them through the FMA-pipe polynomial and the rest through the MUFU
 * ex2.approx, so both pipes work at once.  fma_per_32 is one of 0, 2, 4, 6,
 * 8, 10, 12, 16, 32 (else KRR_EINVAL).  Writes exponentials per second to
 * *exp2_per_s and the kernel time to *ms (may be NULL).  The best rate over
 * the splits is the exp-bound roofline of the fused product.
 */
krr_status krr_bench_ex2_mix(krr_handle* h, int iters, int fma_per_32, double* exp2_per_s,
                             double* ms);

#ifdef __cplusplus
}
#endif

#endif /* KRR_H_ */
