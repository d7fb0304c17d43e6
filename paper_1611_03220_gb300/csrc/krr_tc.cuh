// Tensor-core (tcgen05) fused kernel-matrix product: state and launchers.
#pragma once
#include <cuda.h>

#include "krr_internal.cuh"

namespace krr {

// One prepared operand set: xh = bf16(sqrt(2c)(x - mu)) (or fp16, f16 set)
// padded to n_pad x kp (K-major, 128-byte rows per 64-element K-block),
// nh = ||xh||^2 and ra = exp2(-nh / 2), with TMA descriptors for 128-row and
// 256-row boxes.
struct TcOperand {
  DevBuf Xa, Xlo, ra, nh;   // Xlo: low BF16 parts of split points (else unused)
  const float* src = nullptr;
  int n = 0, ld = 0, d = 0, kp = 0, n_pad = 0;
  bool split = false;
  bool f16 = false;
  CUtensorMap map_a;
  CUtensorMap map_b;
  CUtensorMap map_a2;       // the low parts (split), else the same as map_a / map_b
  CUtensorMap map_b2;
};

struct TcState {
  TcOperand cols;       // column set (the training points)
  DevBuf mu;            // column mean (FP64, d)
  DevBuf scal;          // small device scratch
  DevBuf w;             // n_pad x kv column weights ra_j v_j
  DevBuf part;          // nchunk x n_pad x kv partial row sums
  DevBuf err;           // device error flag (bounded-wait expiry)
  DevBuf vt;            // 16 x n_pad BF16 ra_j v_jc (two-GEMM variant, k >= 3)
  CUtensorMap map_v;
  TcOperand split;      // split points xh = hi + lo (KRR_BF16X3, d <= 64)
  double split_sigma = 0.0;
  bool split_ready = false;
  TcOperand half;       // FP16-rounded points (KRR_FP16)
  TcOperand rows;       // a row set other than the columns (prediction), in the
                        // format of the product that uses it
  TcOperand poly;       // unscaled, uncentred rounded points of the polynomial kernel
  int poly_fmt = -1;    // their format (0 BF16, 1 split, 2 FP16; -1 none)
  DevBuf mu0;           // d zeros (the polynomial kernel is not shift invariant)
  double half_sigma = 0.0;
  bool half_ready = false;
  int autotune = 0;       // 1: time candidate tile plans per shape (process-wide
                          // cache); 2: the symmetric kernel where it applies
  DevBuf tune_v, tune_q;  // the tuner's scratch right-hand sides and products
  // symmetric product (krr_matvec_sym.cu): per-tile row sums, per-item
  // column sums and the device item list for (n_t, C)
  DevBuf sym_rowpart, sym_colpart, sym_items;
  int sym_items_nt = 0, sym_items_c = 0, sym_n_items = 0;
  double sigma = 0.0;
  bool rows_same = false;
  bool ready = false;
  bool err_zeroed = false;
};

// High-precision product state (krr_matvec_hp.cu): five base-512 fixed-point
// digit slices of the centred, scaled points (BF16, (5 n_pad) x 64), per-row
// (a_hi, a_lo, 2^(E-8)), per-call column records and partial sums.
struct HpState {
  DevBuf mu, slab, slices, rowd, cold, part, err;
  const float* src = nullptr;
  int n = 0, ld = 0, d = 0, n_pad = 0;
  double sigma = 0.0;
  bool ready = false;
  CUtensorMap map_a;
  CUtensorMap map_b;
};

// One persistent launch for the products of many problems (krr_matvec_batch.cu).
constexpr int BATCH_MAX = 64;
struct BatchProb {
  const TcOperand* op;   // the problem's prepared FP16 points (TcState::half)
  const float* V;        // n x 1 right-hand side (device)
  float* Q;              // n x 1 product (device)
  double shift;          // lambda of the problem's system
  const int* run;        // the problem's loop flag: no work while it is 0
};
struct BatchState {
  DevBuf items, table, w, part, err;
  int n_items = 0, nprob = 0;
  std::vector<int> chunks;   // per problem: column chunks of its row tiles
};
// Plans the work list of `probs` (at most BATCH_MAX, FP16 points, d <= 128)
// and allocates the shared buffers; call before a graph capture.
void tc_batch_reserve(BatchState& bs, cudaStream_t st, const std::vector<BatchProb>& probs);
// Enqueues the products of every problem whose run flag is set: the weights,
// the persistent kernel over all problems' (row tile, column chunk) items and
// the chunk sums (three launches).
void tc_batch_matvec(BatchState& bs, cudaStream_t st, const std::vector<BatchProb>& probs);
// Nonzero if a batched launch hit a bounded-wait limit since the reserve.
int tc_batch_error(BatchState& bs, cudaStream_t st);
void tc_batch_release(BatchState& bs);

// Grow a device buffer to at least `bytes` (contents not kept).
void tc_ensure(DevBuf& b, size_t bytes);
// TMA map of a K-major BF16 matrix (rows x row_elems, row_elems a multiple of
// 64), boxes of 64 elements x box_rows rows, 128-byte swizzle.
void tc_make_map_bf16(CUtensorMap* m, const void* base, int rows, int row_elems, int box_rows);

// Symmetric product (k = 1, d <= 64, no split): only tiles I <= J of 128 x 128,
// each exponential serving K_ij and K_ji.  C: row blocks per work item,
// ns: TMA ring stages.
bool sym_supported(const TcOperand& op, int k, int split);
void sym_reserve(TcState& t, cudaStream_t st, const TcOperand& op, int C);
// nepi: epilogue warps, 8 or 16.
void sym_matvec(TcState& t, cudaStream_t st, const TcOperand& op, int f16, int C, int ns,
                int nr, const float* V, int ldv, double shift, float* Q, int ldq, int nepi = 16);

bool hp_supported(int d);
void hp_prepare(HpState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma);
void hp_reserve(HpState& t, cudaStream_t st, int k);
// Q = K(X, X) V + shift V with V, Q in FP64 and K_ij to ~1e-13 relative (d <= 64).
void hp_matvec(HpState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma,
               double shift, const double* V, int k, int ldv, double* Q, int ldq);
void hp_clear_error(HpState& t, cudaStream_t st);
int hp_error(HpState& t, cudaStream_t st);
void hp_release(HpState& t);

// Prepare the operands for the training set X (n x d, ldx) at bandwidth sigma.
void tc_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d, double sigma);
// Also the split operands xh = bf16(u) + bf16(u - bf16(u)) (d <= 64).
void tc_prepare_split(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                      double sigma);
// A row set Xr other than the columns, with the columns' mean and scale, in
// format fmt (0 BF16, 1 split, 2 FP16); the columns must be prepared.
void tc_prepare_rows(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr, int d,
                     double sigma, int fmt);
// Also the FP16-rounded points (same range check as the BF16 set).
void tc_prepare_f16(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                    double sigma);
// Q = K(Xr, Xc) V + shift V through the tensor cores (Xr may differ from Xc
// except with gemm2); with
// `split` the dot products use split points (hi.hi + lo.hi + hi.lo); with
// `f16` the points are rounded to FP16 instead of BF16; with `gemm2` the
// contraction with V runs on the tensor cores on BF16-rounded kernel entries.
void tc_matvec(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr, const float* Xc,
               int nc, int ldxc, int d, double sigma, double shift, const float* V, int k,
               int ldv, float* Q, int ldq, int split = 0, int gemm2 = 0, int f16 = 0);
// Allocate the product's workspace for k right-hand sides (call before a
// graph capture; tc_prepare must have run).  fmt: 0 BF16 points, 1 split
// points, 2 FP16 points.  With autotuning on, this is where an untimed shape
// gets timed (the tuner launches and synchronises, so never during capture).
void tc_reserve(TcState& t, cudaStream_t st, int k, int gemm2 = 0, int fmt = 0);
// The product of the training points split for a PCG loop that forms the
// weights and finishes the chunk sums in its own kernels: ra (n_pad row
// factors), w (n_pad x kv weights, w = ra v) and part (nchunk x n_pad x kv
// chunk sums, q_i = ra_i sum_ch part[ch, i] + shift v_i).  tc_loop_prepare
// prepares the operands and plan outside any capture and returns false when
// the plan is not the full product (the symmetric plan), then tc_loop_product
// enqueues the product kernel alone.
struct TcLoop {
  const float* ra = nullptr;
  float* w = nullptr;
  const float* part = nullptr;
  int n_pad = 0, kv = 0, nchunk = 0;
};
bool tc_loop_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                     double sigma, int k, int split, int f16, TcLoop* out);
void tc_loop_product(TcState& t, cudaStream_t st, int k, int split, int f16);
// Plan selection of the fused product: 0 the fixed rule (default), 1 autotune,
// 2 the symmetric kernel where it applies (k = 1, d <= 64, no split).
void tc_set_autotune(TcState& t, int mode);
// Number of shapes the process has tuned so far.
int tc_tuned_shapes();
// Reset the error flag (enqueued on st).
void tc_clear_error(TcState& t, cudaStream_t st);
// Nonzero if any launch hit a bounded-wait limit since the state was created.
int tc_error(TcState& t, cudaStream_t st);
// Q = P(X, X) V + shift V for the polynomial kernel (gamma x.z + c)^q
// (Section 6) on rounded points (BF16, split or FP16); S = xh_i.xh_j on the
// tensor cores, the power on the FMA pipe.
void tc_poly_matvec(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d,
                    double gamma, double c, int q, double shift, const float* V, int k, int ldv,
                    float* Q, int ldq, int split, int f16);
// The polynomial product's operand in format fmt (0 BF16, 1 split, 2 FP16),
// kept until X or the format changes, and its workspace for k right-hand
// sides (both before a graph capture).
void tc_poly_prepare(TcState& t, cudaStream_t st, const float* X, int n, int ldx, int d, int fmt);
void tc_poly_reserve(TcState& t, cudaStream_t st, int k);
// Q = (D o K(Xr, Xc)) V with D_ij = ||x_i - x_j||^2 / sigma^2 (the derivative
// of K in log sigma) on the rounded points (BF16, split or FP16), any row set.
void tc_dsigma_matvec(TcState& t, cudaStream_t st, const float* Xr, int nr, int ldxr,
                      const float* Xc, int nc, int ldxc, int d, double sigma, const float* V,
                      int k, int ldv, float* Q, int ldq, int split, int f16);
void tc_release(TcState& t);

}  // namespace krr
