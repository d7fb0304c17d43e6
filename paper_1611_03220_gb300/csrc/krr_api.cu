// C ABI entry points, handle and the PCG driver.
//
// Algorithm 1 of the paper, end to end on one GPU:
//   features Z (Section 2.2) -> G = Z^T Z + lambda_p I -> L L^T = G ->
//   factors for the Woodbury apply (Section 3.1) -> PCG on (K + lambda I) c = y
//   with K applied on the fly (the PCG step of Algorithm 1), stopping on the relative
//   residual of every column (Section 5).
// The PCG iteration is captured once per solve into a CUDA graph whose body
// sits under a conditional WHILE node; the loop's last kernel decides on the
// device whether to run again, so an entire solve is one graph launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <type_traits>

#include "krr_internal.cuh"
#include "krr_tc.cuh"

using namespace krr;

struct krr_handle {
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  int device = 0;
  std::string err;
  std::map<std::string, DevBuf> bufs;
  Precond pc;
  CgScalars* sc = nullptr;      // device
  CgScalars* sc_host = nullptr; // pinned mirror
  double* hostd = nullptr;      // pinned scratch (KRR_MAX_RHS * 4 doubles)
  int* info = nullptr;          // device int
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  TcState tc;
  HpState hp;
  BatchState batch;               // the batched product of krr_pcg_solve_batched
  std::vector<TcState> batch_tc;  // operands of krr_kernel_matvec_batched
  DevBuf batch_ones;              // run flags (all 1) of krr_kernel_matvec_batched
  std::vector<krr_handle*> subs;  // per-problem handles of krr_pcg_solve_batched
  // The kernel of the solve in progress: the Gaussian kernel unless a
  // polynomial-kernel solve has set `poly` (products then ignore sigma).
  struct {
    int poly = 0;
    double gamma = 1.0, c = 0.0;
    int q = 1;
    const float* X = nullptr;  // the training points of that solve
    int n = 0, ldx = 0, d = 0;
  } kern;
};

namespace krr {

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

}  // namespace krr

namespace {

bool trace_on() {
  static int on = -1;
  if (on < 0) on = getenv("KRR_TRACE") ? 1 : 0;
  return on == 1;
}
#define KRR_TRACE(...)                   \
  do {                                   \
    if (trace_on()) {                    \
      fprintf(stderr, "[krr] " __VA_ARGS__); \
      fprintf(stderr, "\n");             \
      fflush(stderr);                    \
    }                                    \
  } while (0)

void* ws(krr_handle* h, const std::string& name, size_t bytes) {
  DevBuf& b = h->bufs[name];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      KRR_CUDA(cudaStreamSynchronize(h->stream));
      KRR_CUDA(cudaFree(b.p));
      b.p = nullptr;
      b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{KRR_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + ") for " + name + ": " +
                                  cudaGetErrorString(e)};
    }
    b.bytes = bytes;
  }
  return b.p;
}

template <typename T>
T* wsT(krr_handle* h, const std::string& name, size_t elems) {
  return reinterpret_cast<T*>(ws(h, name, elems * sizeof(T)));
}

void ensure_buf(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{KRR_ENOMEM, std::string("preconditioner allocation: ") + cudaGetErrorString(e)};
  }
  b.bytes = bytes;
}

void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Returns a device copy of a host-or-device buffer of `bytes`.
const void* stage_in(krr_handle* h, const void* p, size_t bytes, const char* name) {
  if (on_device(p)) return p;
  void* d = ws(h, std::string("stage_") + name, bytes);
  KRR_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, h->stream));
  return d;
}

template <typename F>
krr_status guard(krr_handle* h, F&& f) {
  if (!h) return KRR_EINVAL;
  try {
    h->err.clear();
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) KRR_CUDA(cudaSetDevice(h->device));
    krr_status st = f();
    if (cur != h->device) cudaSetDevice(cur);
    return st;
  } catch (const Error& e) {
    h->err = e.msg;
    return e.st;
  } catch (const std::exception& e) {
    h->err = e.what();
    return KRR_ECUDA;
  }
}

double ms_between(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return (double)ms;
}

// --------------------------------------------------------- kernel product --
// Q = K(Xr, Xc) V + shift V in the requested arithmetic; V/Q double for
// FP64/HP, float for FP32/BF16.
// Products of the polynomial kernel (gamma x.z + c)^q: FP64 SIMT for KRR_FP64
// and KRR_HP (the refinement residual), the fused tensor-core kernel on
// rounded points for KRR_BF16, KRR_FP16 and KRR_BF16X3 (training system only).
void poly_dispatch(krr_handle* h, cudaStream_t st, const float* Xr, int nr, int ldxr,
                   const float* Xc, int nc, int ldxc, int d, double shift, const void* V, int k,
                   int ldv, void* Q, int ldq, int prec) {
  const auto& K = h->kern;
  switch (prec) {
    case KRR_FP64:
    case KRR_HP: {
      double* part = wsT<double>(h, "mv_part64", mv_fp64_part_elems(nr, nc, k));
      launch_mv_fp64_poly(st, Xr, nr, ldxr, Xc, nc, ldxc, d, K.gamma, K.c, K.q, shift,
                          (const double*)V, k, ldv, (double*)Q, ldq, part);
      return;
    }
    case KRR_BF16:
    case KRR_FP16:
    case KRR_BF16X3: {
      if (!(Xr == Xc && nr == nc && ldxr == ldxc))
        throw Error{KRR_EUNSUPPORTED, "polynomial tensor-core product: training system only"};
      tc_poly_matvec(h->tc, st, Xc, nc, ldxc, d, K.gamma, K.c, K.q, shift, (const float*)V, k,
                     ldv, (float*)Q, ldq, prec == KRR_BF16X3 ? 1 : 0, prec == KRR_FP16 ? 1 : 0);
      return;
    }
    default:
      throw Error{KRR_EUNSUPPORTED, "polynomial kernel: precision must be KRR_FP64, KRR_HP, "
                                    "KRR_BF16, KRR_FP16 or KRR_BF16X3"};
  }
}

void matvec_dispatch(krr_handle* h, cudaStream_t st, const float* Xr, int nr, int ldxr,
                     const float* Xc, int nc, int ldxc, int d, double sigma, double shift,
                     const void* V, int k, int ldv, void* Q, int ldq, int prec) {
  if (h->kern.poly) {
    poly_dispatch(h, st, Xr, nr, ldxr, Xc, nc, ldxc, d, shift, V, k, ldv, Q, ldq, prec);
    return;
  }
  const bool same = (Xr == Xc && nr == nc && ldxr == ldxc);
  if (prec == KRR_HP && same && hp_supported(d)) {
    hp_matvec(h->hp, st, Xr, nr, ldxr, d, sigma, shift, (const double*)V, k, ldv, (double*)Q, ldq);
    return;
  }
  switch (prec) {
    case KRR_FP64: {
      double* part = wsT<double>(h, "mv_part64", mv_fp64_part_elems(nr, nc, k));
      launch_mv_fp64(st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, shift, (const double*)V, k, ldv,
                     (double*)Q, ldq, part);
      return;
    }
    case KRR_HP: {
      // distinct row and column sets, or d > 64: the SIMT float-float product
      double* part = wsT<double>(h, "hpw_part", mv_hpw_part_elems(nr, nc, k));
      float* nrm_r = wsT<float>(h, "hpw_nr", 2 * (size_t)nr);
      float* nrm_c = wsT<float>(h, "hpw_nc", 2 * (size_t)nc);
      launch_mv_hpw(st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, shift, (const double*)V, k, ldv,
                    (double*)Q, ldq, part, nrm_r, nrm_c, 0);
      return;
    }
    case KRR_FP32: {
      float* part = wsT<float>(h, "mv_part32", mv_fp32_part_elems(nr, nc, k));
      float* nr_ = wsT<float>(h, "mv_nrm_r", (size_t)nr);
      float* nc_ = wsT<float>(h, "mv_nrm_c", (size_t)nc);
      launch_mv_fp32(st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, shift, (const float*)V, k, ldv,
                     (float*)Q, ldq, nr_, nc_, part);
      return;
    }
    case KRR_BF16:
    case KRR_FP16:
    case KRR_BF16X3:
    case KRR_BF16P: {
      tc_matvec(h->tc, st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, shift, (const float*)V, k, ldv,
                (float*)Q, ldq, prec == KRR_BF16X3 ? 1 : 0, prec == KRR_BF16P ? 1 : 0,
                prec == KRR_FP16 ? 1 : 0);
      return;
    }
    default:
      throw Error{KRR_EINVAL, "unknown precision " + std::to_string(prec)};
  }
}

// Allocate the product's workspace ahead of a graph capture (no allocation
// may happen while the loop body is being captured).
void matvec_reserve(krr_handle* h, int n, int k, int prec) {
  if (h->kern.poly) {
    if (prec == KRR_FP64 || prec == KRR_HP) {
      wsT<double>(h, "mv_part64", mv_fp64_part_elems(n, n, k));
    } else {
      const auto& ps = h->kern;
      tc_poly_prepare(h->tc, h->stream, ps.X, ps.n, ps.ldx, ps.d,
                      prec == KRR_BF16X3 ? 1 : (prec == KRR_FP16 ? 2 : 0));
      tc_poly_reserve(h->tc, h->stream, k);
    }
    return;
  }
  switch (prec) {
    case KRR_FP64:
      wsT<double>(h, "mv_part64", mv_fp64_part_elems(n, n, k));
      return;
    case KRR_HP:
      if (h->hp.ready) {
        hp_reserve(h->hp, h->stream, k);
      } else {
        wsT<double>(h, "hpw_part", mv_hpw_part_elems(n, n, k));
        wsT<float>(h, "hpw_nr", 2 * (size_t)n);
        wsT<float>(h, "hpw_nc", 2 * (size_t)n);
      }
      return;
    case KRR_FP32:
      wsT<float>(h, "mv_part32", mv_fp32_part_elems(n, n, k));
      wsT<float>(h, "mv_nrm_r", (size_t)n);
      wsT<float>(h, "mv_nrm_c", (size_t)n);
      return;
    case KRR_BF16:
    case KRR_FP16:
    case KRR_BF16X3:
    case KRR_BF16P:
      tc_reserve(h->tc, h->stream, k, prec == KRR_BF16P ? 1 : 0,
                 prec == KRR_BF16X3 ? 1 : (prec == KRR_FP16 ? 2 : 0));
      return;
    default:
      return;
  }
}

// ------------------------------------------------------------------- PCG --
struct LoopOut {
  int iters[KRR_MAX_RHS];
  double rr[KRR_MAX_RHS];
  double yy[KRR_MAX_RHS];
  double kappa[KRR_MAX_RHS];   // Lanczos estimate of cond(M^-1 A) (0: none)
  int flags;
  int iter;
};

// Eigenvalues of the symmetric tridiagonal (d, e) below x: the Sturm count
// (the number of negative pivots of T - x I).
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double off = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;   // step past an exact zero pivot
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Condition estimate of the preconditioned operator from m PCG steps: the
// Lanczos tridiagonal of CG (diagonal 1/a_0, 1/a_j + b_{j-1}/a_{j-1},
// off-diagonal sqrt(b_j)/a_j) and its extreme eigenvalues by bisection on
// the Sturm count.  0 when fewer than two steps were taken or the estimate
// is not positive.
double lanczos_kappa_est(const std::vector<double>& a, const std::vector<double>& b) {
  const size_t m = a.size();
  if (m < 2) return 0.0;
  std::vector<double> d(m), e(m - 1);
  for (size_t j = 0; j < m; ++j) {
    if (!(a[j] > 0.0)) return 0.0;
    d[j] = 1.0 / a[j] + (j ? b[j - 1] / a[j - 1] : 0.0);
    if (j + 1 < m) e[j] = std::sqrt(std::max(b[j], 0.0)) / a[j];
  }
  double lo = d[0], hi = d[0];
  for (size_t j = 0; j < m; ++j) {
    const double r = (j ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  auto kth = [&](int k) {  // the k-th smallest eigenvalue (1-based)
    double l = lo, u = hi;
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(std::fabs(l), std::fabs(u)); ++it) {
      const double mid = 0.5 * (l + u);
      if (sturm_count(d, e, mid) >= k) u = mid; else l = mid;
    }
    return 0.5 * (l + u);
  };
  const double emin = kth(1), emax = kth((int)m);
  return emin > 0.0 ? emax / emin : 0.0;
}

// One PCG solve's operands: the loop vectors (n x k, ld = k), the right-hand
// side whose norm sets the stopping test, and the two operators.
template <typename T>
struct PcgSpec {
  int n = 0, k = 0;
  const double* Ytol = nullptr;
  int ldy = 0;
  T *x = nullptr, *r = nullptr, *p = nullptr, *z = nullptr, *q = nullptr;
  double tol = 0.0;
  int max_iter = 0;
  std::function<void(cudaStream_t, const T*, T*)> matvec, apply;
  int prec = KRR_FP64;
  // keep the previous solve's last direction (p holds it, in units s times
  // smaller than these) instead of starting from p = z
  bool restart = false;
  ColScale rscale{};
  // the product q = A p is enqueued elsewhere (a batched product shared by
  // several solves) before this loop body runs
  bool skip_matvec = false;
  // fused body (FP32 vectors, the tensor-core product of the training points,
  // the streamed ZL apply): 8 launches an iteration instead of 13
  bool fused = false;
  TcLoop tl{};
  int tc_split = 0, tc_f16 = 0;
  double shift = 0.0;
  T* rn = nullptr;   // the updated residual between the apply's two passes
};

// Everything before the first iteration: ||y||, z0 = M^-1 r0, p0 = z0.
template <typename T>
void pcg_begin(krr_handle* h, const PcgSpec<T>& S) {
  cudaStream_t st = h->stream;
  double* part = wsT<double>(h, "cg_part", cg_part_elems(S.n, S.k));
  double* hist = wsT<double>(h, "cg_hist", (size_t)CG_HIST_CAP * 2 * KRR_MAX_RHS);
  matvec_reserve(h, S.n, S.k, S.prec);
  launch_cg_init<T>(st, h->sc, S.Ytol, S.ldy, S.r, S.n, S.k, S.tol, S.max_iter, part, hist,
                    CG_HIST_CAP);
  if (S.apply)
    S.apply(st, S.r, S.z);
  else
    KRR_CUDA(cudaMemcpyAsync(S.z, S.r, (size_t)S.n * S.k * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (S.restart && 3 * S.k <= KRR_MAX_RHS)
    launch_cg_restart<T>(st, h->sc, S.r, S.z, S.p, S.n, S.k, S.rscale, part);
  else
    launch_cg_rz_first<T>(st, h->sc, S.r, S.z, S.p, S.n, S.k, part);
  if constexpr (std::is_same<T, float>::value) {
    // the fused body starts with the product: its weights from p0
    if (S.fused)
      launch_cg_update_pw<T>(st, h->sc, S.p, S.z, S.n, S.k, 0, S.tl.ra, S.tl.n_pad, S.tl.kv,
                             S.tl.w);
  }
}

// The fused iteration (same arithmetic as pcg_body, in 8 launches):
//   product kernel (weights from the previous iteration) -> chunk sums with
//   p.q and alpha -> Z^T pass with the x, r update and ||r||^2 -> slab sums
//   -> L^-1 -> L^-T -> Z w pass with r.z, beta and the loop test -> p and
//   the next weights.
template <typename T>
void pcg_body_fused(krr_handle* h, const PcgSpec<T>& S, cudaStream_t s2, unsigned long long cond) {
  if constexpr (std::is_same<T, float>::value) {
    double* part = wsT<double>(h, "cg_part", cg_part_elems(S.n, S.k));
    const Precond& pc = h->pc;
    tc_loop_product(h->tc, s2, S.k, S.tc_split, S.tc_f16);
    launch_cg_reduce_alpha<T>(s2, h->sc, S.tl.part, S.tl.nchunk, S.tl.n_pad, S.tl.kv, S.tl.ra,
                              S.shift, S.p, S.q, S.n, S.k, part);
    CgStepArgs<T> f;
    f.sc = h->sc;
    f.X = S.x;
    f.P = S.p;
    f.Q = S.q;
    f.Rn = S.rn;
    f.cpart = part;
    f.cond = cond;
    double* t1 = wsT<double>(h, "ap_t1", (size_t)pc.s * S.k);
    double* t2 = wsT<double>(h, "ap_t2", (size_t)pc.s * S.k);
    double* apart = wsT<double>(h, "ap_part", apply_part_elems(pc.n, pc.s, S.k));
    launch_apply_cg<T>(s2, pc, S.r, S.k, S.z, t1, t2, apart, f);
    launch_cg_update_pw<T>(s2, h->sc, S.p, S.z, S.n, S.k, 1, S.tl.ra, S.tl.n_pad, S.tl.kv,
                           S.tl.w);
  } else {
    throw Error{KRR_EINVAL, "fused PCG body: FP32 vectors only"};
  }
}

// One PCG iteration of Algorithm 1: q = A p, alpha, x and r updates,
// z = M^-1 r, beta and p; the tail kernel decides whether to continue.
// Enqueues only (no allocation), so it can be captured into a graph.
template <typename T>
void pcg_body(krr_handle* h, const PcgSpec<T>& S, cudaStream_t s2, unsigned long long cond) {
  if (S.fused && !S.skip_matvec) {
    pcg_body_fused<T>(h, S, s2, cond);
    return;
  }
  double* part = wsT<double>(h, "cg_part", cg_part_elems(S.n, S.k));
  if (!S.skip_matvec) S.matvec(s2, S.p, S.q);
  launch_cg_alpha<T>(s2, h->sc, S.p, S.q, S.n, S.k, part);
  launch_cg_update_xr<T>(s2, h->sc, S.x, S.r, S.p, S.q, S.n, S.k, part);
  if (S.apply)
    S.apply(s2, S.r, S.z);
  else
    KRR_CUDA(cudaMemcpyAsync(S.z, S.r, (size_t)S.n * S.k * sizeof(T), cudaMemcpyDeviceToDevice, s2));
  launch_cg_rz<T>(s2, h->sc, S.r, S.z, S.n, S.k, part);
  launch_cg_update_p<T>(s2, h->sc, S.p, S.z, S.n, S.k);
  launch_cg_tail(s2, h->sc, cond);
}

// Reads the loop's device scalars back (synchronises the stream).
void pcg_finish(krr_handle* h, int k, LoopOut* out) {
  cudaStream_t st = h->stream;
  KRR_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < k; ++c) {
    out->iters[c] = h->sc_host->iters[c];
    out->rr[c] = h->sc_host->rr[c];
    out->yy[c] = h->sc_host->yy[c];
  }
  out->flags = h->sc_host->flags;
  out->iter = h->sc_host->iter;
  // the condition estimate from the recorded alpha, beta
  const int m = std::min(out->iter, h->sc_host->hist_cap);
  for (int c = 0; c < KRR_MAX_RHS; ++c) out->kappa[c] = 0.0;
  if (m >= 2 && h->sc_host->hist) {
    std::vector<double> hh((size_t)m * 2 * KRR_MAX_RHS);
    KRR_CUDA(cudaMemcpyAsync(hh.data(), h->sc_host->hist, hh.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < k; ++c) {
      const int mc = std::min(out->iters[c], m);
      std::vector<double> a(mc), b(mc);
      for (int j = 0; j < mc; ++j) {
        a[j] = hh[((size_t)j * 2) * KRR_MAX_RHS + c];
        b[j] = hh[((size_t)j * 2 + 1) * KRR_MAX_RHS + c];
      }
      out->kappa[c] = lanczos_kappa_est(a, b);
    }
  }
}

template <typename T>
void pcg_loop(krr_handle* h, const PcgSpec<T>& S, bool use_graph, LoopOut* out, int* matvecs) {
  cudaStream_t st = h->stream;
  pcg_begin<T>(h, S);
  int launched = 0;
  long long body_launches = 0;
  if (S.max_iter > 0) {
    if (use_graph) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      KRR_TRACE("pcg_loop: graph create n=%d k=%d max_iter=%d", S.n, S.k, S.max_iter);
      KRR_CUDA(cudaGraphCreate(&graph, 0));
      try {
        cudaGraphConditionalHandle cond;
        KRR_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams params = {cudaGraphNodeTypeConditional};
        params.conditional.handle = cond;
        params.conditional.type = cudaGraphCondTypeWhile;
        params.conditional.size = 1;
        cudaGraphNode_t node;
        KRR_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &params));
        cudaGraph_t bodyg = params.conditional.phGraph_out[0];
        KRR_CUDA(cudaStreamBeginCaptureToGraph(h->cap, bodyg, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed));
        capture_begin();
        try {
          pcg_body<T>(h, S, h->cap, (unsigned long long)cond);
        } catch (...) {
          capture_end();
          cudaGraph_t tmp;
          cudaStreamEndCapture(h->cap, &tmp);
          cudaGetLastError();
          throw;
        }
        body_launches = capture_end();
        cudaGraph_t captured = nullptr;
        KRR_CUDA(cudaStreamEndCapture(h->cap, &captured));
        KRR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        KRR_CUDA(cudaGraphLaunch(exec, st));
        KRR_TRACE("pcg_loop: launched");
      } catch (...) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        throw;
      }
      KRR_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
      KRR_CUDA(cudaStreamSynchronize(st));
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      launched = h->sc_host->iter;
      add_launches(body_launches * (long long)launched);
    } else {
      // host-driven loop: checks the device scalars every `chk` iterations
      const int chk = 8;
      for (int it = 0; it < S.max_iter; ++it) {
        pcg_body<T>(h, S, st, 0ull);
        ++launched;
        if ((it + 1) % chk == 0 || it + 1 == S.max_iter) {
          KRR_CUDA(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
          KRR_CUDA(cudaStreamSynchronize(st));
          if (!h->sc_host->run) break;
        }
      }
    }
  }
  pcg_finish(h, S.k, out);
  if (matvecs) *matvecs += launched;
}

// Per-column ||a_c||^2 read back to the host.
template <typename T>
void host_colnorm2(krr_handle* h, const T* a, int n, int k, int lda, double* out) {
  double* part = wsT<double>(h, "cg_part", cg_part_elems(n, k));
  double* dout = wsT<double>(h, "colnorm_out", KRR_MAX_RHS);
  unsigned int* ctr = wsT<unsigned int>(h, "colnorm_ctr", 4);
  KRR_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned int), h->stream));
  launch_colnorm2<T>(h->stream, a, n, k, lda, dout, part, ctr);
  KRR_CUDA(cudaMemcpyAsync(h->hostd, dout, k * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KRR_CUDA(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < k; ++c) out[c] = h->hostd[c];
}

// Cholesky of the Gram matrix already in pc.L, then the apply form's factors
// (the rest of Algorithm 1's set-up); z_bf16: storage of pc.Z.
void precond_factor(krr_handle* h, int n, int s, double lambda_p, int form, int z_bf16) {
  cudaStream_t st = h->stream;
  Precond& pc = h->pc;
  launch_cholesky(st, (double*)pc.L.p, s, h->info);
  int info = 0;
  KRR_CUDA(cudaMemcpyAsync(&h->hostd[0], h->info, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  memcpy(&info, &h->hostd[0], sizeof(int));
  if (info != 0)
    throw Error{KRR_ECHOL, "Z^T Z + lambda_p I is not positive definite (pivot " +
                               std::to_string(info - 1) + ")"};
  ensure_buf(pc.Linv, (size_t)s * s * sizeof(double));
  launch_tri_inverse(st, (const double*)pc.L.p, s, (double*)pc.Linv.p,
                     wsT<double>(h, "tri_scratch", tri_inverse_scratch_elems(s)));
  if (form == KRR_APPLY_ZL) {
    ensure_buf(pc.LinvT, (size_t)s * s * sizeof(double));
    launch_transpose_d(st, (const double*)pc.Linv.p, s, (double*)pc.LinvT.p);
    free_buf(pc.U);
  } else {
    ensure_buf(pc.U, (size_t)s * n * sizeof(float));
    launch_form_u(st, (const double*)pc.Linv.p, pc.Z.p, z_bf16, n, s, (float*)pc.U.p);
  }
  if (!pc.err.p) ensure_buf(pc.err, 16);
  KRR_CUDA(cudaMemsetAsync(pc.err.p, 0, 16, st));
  pc.n = n;
  pc.s = s;
  pc.form = form;
  pc.z_bf16 = z_bf16;
  pc.lam_p = lambda_p;
  pc.ready = true;
}

// The exact tensor-core Gram of the fixed-point features in pc.Z (whose
// transpose is in ZT), G' = Zs^T Zs + lambda_p 2^-2e I, and the factors.
void precond_fixed_gram_factor(krr_handle* h, const __nv_bfloat16* ZT, int e, int n, int s,
                               double lambda_p, int form, int* err) {
  cudaStream_t st = h->stream;
  Precond& pc = h->pc;
  ensure_buf(pc.L, (size_t)s * s * sizeof(double));
  int* part = wsT<int>(h, "tcs_part", gram_tc_part_elems(n, s));
  launch_gram_tc(st, ZT, n, s, lambda_p * std::ldexp(1.0, -2 * e), part, (double*)pc.L.p, err);
  precond_factor(h, n, s, lambda_p, form, 2);
  int e_flag = 0;
  KRR_CUDA(cudaMemcpyAsync(&e_flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  KRR_CUDA(cudaStreamSynchronize(st));
  if (e_flag) {
    pc.ready = false;
    throw Error{KRR_ETIMEOUT, "tensor-core set-up: a pipeline wait hit its limit"};
  }
  pc.z_fixed_e = e;
}

void precond_setup_impl(krr_handle* h, const float* Z, int n, int s, int ldz, double lambda_p,
                        int form, int z_format) {
  KRR_REQUIRE(Z && n > 0 && s > 0 && ldz >= s, "precond_setup: bad Z / sizes");
  KRR_REQUIRE(s <= n, "precond_setup: need s <= n");
  KRR_REQUIRE(lambda_p > 0.0 && std::isfinite(lambda_p), "precond_setup: lambda_p must be > 0");
  KRR_REQUIRE(form == KRR_APPLY_ZL || form == KRR_APPLY_U, "precond_setup: bad apply form");
  KRR_REQUIRE(z_format >= KRR_Z_FP32 && z_format <= KRR_Z_FIXED, "precond_setup: bad Z format");
  cudaStream_t st = h->stream;
  Precond& pc = h->pc;
  pc.ready = false;
  pc.z_fixed_e = 0;
  if (z_format == KRR_Z_FIXED) {
    ensure_buf(pc.Z, (size_t)n * s);
    __nv_bfloat16* ZT = wsT<__nv_bfloat16>(
        h, "tcs_zt", (size_t)setup_tc_s_pad(s) * setup_tc_n_pad(n));
    int* scr = wsT<int>(h, "tcs_scr", 4);
    KRR_CUDA(cudaMemsetAsync(scr, 0, 4 * sizeof(int), st));
    const int e = launch_quantize_z(st, Z, n, s, ldz, (signed char*)pc.Z.p, ZT, scr);
    precond_fixed_gram_factor(h, ZT, e, n, s, lambda_p, form, scr + 1);
    return;
  }
  const int z_bf16 = z_format == KRR_Z_BF16 ? 1 : 0;
  const size_t esz = z_bf16 ? 2 : 4;
  ensure_buf(pc.Z, (size_t)n * s * esz);
  launch_copy_z(st, Z, n, s, ldz, pc.Z.p, z_bf16);
  ensure_buf(pc.L, (size_t)s * s * sizeof(double));
  const int nch = gram_chunks(n, s);
  double* part = wsT<double>(h, "gram_part", (size_t)nch * s * s);
  launch_gram(st, pc.Z.p, z_bf16, n, s, lambda_p, (double*)pc.L.p, part, nch);
  precond_factor(h, n, s, lambda_p, form, z_bf16);
}

// Features and preconditioner on the tensor cores in one go (the mixed
// solves' set-up): fixed-point random Fourier features of X straight into
// pc.Z (and their transpose), then the exact Gram and the factors.
void precond_setup_rff_tc(krr_handle* h, const float* Xd, int n, int d, int ldx, const float* Wd,
                          const float* bd, int s, double lambda_p, int form) {
  KRR_REQUIRE(s <= n, "precond_setup: need s <= n");
  KRR_REQUIRE(lambda_p > 0.0 && std::isfinite(lambda_p), "precond_setup: lambda_p must be > 0");
  cudaStream_t st = h->stream;
  Precond& pc = h->pc;
  pc.ready = false;
  pc.z_fixed_e = 0;
  ensure_buf(pc.Z, (size_t)n * s);
  const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s), kp = setup_tc_kp(d);
  __nv_bfloat16* ZT = wsT<__nv_bfloat16>(h, "tcs_zt", (size_t)s_pad * n_pad);
  __nv_bfloat16* Xh = wsT<__nv_bfloat16>(h, "tcs_xh", (size_t)n_pad * kp);
  __nv_bfloat16* Xl = wsT<__nv_bfloat16>(h, "tcs_xl", (size_t)n_pad * kp);
  __nv_bfloat16* Wh = wsT<__nv_bfloat16>(h, "tcs_wh", (size_t)s_pad * kp);
  __nv_bfloat16* Wl = wsT<__nv_bfloat16>(h, "tcs_wl", (size_t)s_pad * kp);
  int* scr = wsT<int>(h, "tcs_scr", 4);
  KRR_CUDA(cudaMemsetAsync(scr, 0, 4 * sizeof(int), st));
  const int e = launch_rff_tc(st, Xd, n, d, ldx, Wd, bd, s, Xh, Xl, Wh, Wl,
                              (signed char*)pc.Z.p, ZT, scr + 1);
  precond_fixed_gram_factor(h, ZT, e, n, s, lambda_p, form, scr + 1);
}

// Nonzero if a streamed apply hit its bounded wait since the set-up.
int precond_error(krr_handle* h) {
  if (!h->pc.err.p) return 0;
  int e = 0;
  KRR_CUDA(cudaMemcpyAsync(&e, h->pc.err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  KRR_CUDA(cudaStreamSynchronize(h->stream));
  return e;
}

template <typename T>
void apply_precond(krr_handle* h, cudaStream_t st, const T* R, int k, int ldr, T* Zo, int ldo) {
  const Precond& pc = h->pc;
  double* t1 = wsT<double>(h, "ap_t1", (size_t)pc.s * k);
  double* t2 = wsT<double>(h, "ap_t2", (size_t)pc.s * k);
  double* part = wsT<double>(h, "ap_part", apply_part_elems(pc.n, pc.s, k));
  launch_apply<T>(st, pc, R, k, ldr, Zo, ldo, t1, t2, part);
}

struct SolveArgs {
  const float* X;
  int n, d, ldx;
  double sigma, lambda;
  const double* Y;
  int k, ldy;
  double* C;
  int ldc;
  krr_opts o;
};

// Plain PCG in element type T with product precision `prec`; FP64 true
// residual restarts when the recursive residual passes but the true one
// does not (up to three times).
template <typename T>
krr_status solve_plain(krr_handle* h, const SolveArgs& a, int prec, krr_report* rep,
                       int* matvecs) {
  cudaStream_t st = h->stream;
  const int n = a.n, k = a.k;
  const size_t nk = (size_t)n * k;
  T* x = wsT<T>(h, "v_x", nk);
  T* r = wsT<T>(h, "v_r", nk);
  T* p = wsT<T>(h, "v_p", nk);
  T* z = wsT<T>(h, "v_z", nk);
  T* q = wsT<T>(h, "v_q", nk);
  double* Yc = wsT<double>(h, "v_y", nk);     // Y packed with ld = k
  double* Rd = wsT<double>(h, "v_rd", nk);    // FP64 true residual
  double* AX = wsT<double>(h, "v_ax", nk);
  ColScale one;
  for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
  launch_convert<double, double>(st, a.Y, n, k, a.ldy, Yc, k, one);
  // initial x and r
  if (a.o.warm_start) {
    double* C0 = wsT<double>(h, "v_c0", nk);
    launch_convert<double, double>(st, a.C, n, k, a.ldc, C0, k, one);
    matvec_dispatch(h, st, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, C0, k, k, AX, k,
                    KRR_FP64);
    ++*matvecs;
    launch_sub_d(st, Yc, k, AX, k, n, k, Rd, k);
    launch_convert<double, T>(st, C0, n, k, k, x, k, one);
    launch_convert<double, T>(st, Rd, n, k, k, r, k, one);
  } else {
    KRR_CUDA(cudaMemsetAsync(x, 0, nk * sizeof(T), st));
    launch_convert<double, T>(st, Yc, n, k, k, r, k, one);
  }
  auto mv = [&](cudaStream_t s2, const T* V, T* Q) {
    matvec_dispatch(h, s2, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, V, k, k, Q, k,
                    prec);
  };
  std::function<void(cudaStream_t, const T*, T*)> ap;
  if (a.o.precond)
    ap = [&](cudaStream_t s2, const T* R, T* Zo) { apply_precond<T>(h, s2, R, k, k, Zo, k); };
  int restarts = 0;
  int total_iters[KRR_MAX_RHS] = {0};
  double kmax[KRR_MAX_RHS] = {0};
  krr_status status = KRR_OK;
  LoopOut lo;
  int remaining = a.o.max_iter;
  for (;;) {
    PcgSpec<T> S;
    S.n = n; S.k = k; S.Ytol = Yc; S.ldy = k;
    S.x = x; S.r = r; S.p = p; S.z = z; S.q = q;
    S.tol = a.o.tol; S.max_iter = remaining; S.matvec = mv; S.apply = ap; S.prec = prec;
    pcg_loop<T>(h, S, a.o.use_graph != 0, &lo, matvecs);
    for (int c = 0; c < k; ++c) {
      total_iters[c] += lo.iters[c];
      kmax[c] = std::max(kmax[c], lo.kappa[c]);
      if (rep) rep->rel_res_rec[c] = lo.yy[c] > 0 ? std::sqrt(lo.rr[c] / lo.yy[c]) : 0.0;
    }
    remaining -= lo.iter;
    if (lo.flags & FLAG_NAN) {
      status = KRR_ENAN;
      break;
    }
    if (lo.flags & FLAG_BREAKDOWN) {
      status = KRR_EBREAKDOWN;
      break;
    }
    // true residual in FP64
    ColScale one2 = one;
    double* xd = wsT<double>(h, "v_xd", nk);
    launch_convert<T, double>(st, x, n, k, k, xd, k, one2);
    matvec_dispatch(h, st, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, xd, k, k, AX, k,
                    prec == KRR_FP64 ? KRR_FP64 : KRR_HP);
    ++*matvecs;
    launch_sub_d(st, Yc, k, AX, k, n, k, Rd, k);
    double rr[KRR_MAX_RHS];
    host_colnorm2<double>(h, Rd, n, k, k, rr);
    bool ok = true;
    for (int c = 0; c < k; ++c) {
      double rel = lo.yy[c] > 0 ? std::sqrt(rr[c] / lo.yy[c]) : 0.0;
      if (rep) rep->rel_res[c] = rel;
      if (rel > a.o.tol) ok = false;
    }
    if (ok) break;
    if (lo.flags & FLAG_CAP || remaining <= 0) {
      status = KRR_ENOTCONV;
      break;
    }
    if (prec != KRR_FP64 || restarts >= 3) {
      // single precision reached its floor: report, do not loop forever
      status = KRR_ENOTCONV;
      break;
    }
    ++restarts;
    launch_convert<double, T>(st, Rd, n, k, k, r, k, one);
  }
  launch_convert<T, double>(st, x, n, k, k, a.C, a.ldc, one);
  if (rep) {
    for (int c = 0; c < k; ++c) {
      rep->iters[c] = total_iters[c];
      rep->kappa[c] = kmax[c];
    }
    rep->outer_steps = restarts;
  }
  return status;
}

// Inner-solve arithmetic of the mixed solve, in the order it is tried: the
// FP16 (or BF16) product, the split-point BF16 product (d <= 64), the HP
// product.
enum InnerLevel { INNER_LOW = 0, INNER_SPLIT = 1, INNER_HP = 2 };

int next_level(int level, int d) {
  if (level == INNER_LOW && d <= 64) return INNER_SPLIT;
  return INNER_HP;
}

// Largest contraction per outer step that keeps the inner arithmetic at its
// level: a split-level solve costs several low-level steps, and when it contracts
// poorly the system is so ill-conditioned that only HP inner solves converge.
double keep_below(int level) { return level == INNER_LOW ? 0.5 : 0.2; }

// Relative tolerance of an inner solve: the FP16/BF16 solve stops at inner_tol,
// or sooner on the last step if the outer test needs less (0.3 tol / rel:
// the rest of the margin is for the product's own error); the more accurate
// ones go as far as the outer test needs (0.5 tol / rel) within what their
// arithmetic can reach.
double inner_tol_for(int level, const krr_opts& o, double rel) {
  if (level == INNER_LOW) return std::max(o.inner_tol, std::min(0.5, 0.3 * o.tol / rel));
  const double want = 0.5 * o.tol / rel;
  return std::min(o.inner_tol, std::max(level == INNER_SPLIT ? 1e-5 : 1e-11, want));
}

// Product of the lowest inner level: FP16 points unless BF16 or split BF16
// points (d <= 64) were asked for (KRR_HP skips the low levels altogether).
int low_precision(const krr_opts& o) {
  if (o.inner_precision == KRR_BF16 || o.inner_precision == KRR_BF16X3) return o.inner_precision;
  return KRR_FP16;
}

const char* level_name(int level) {
  return level == INNER_LOW ? "FP16/BF16" : (level == INNER_SPLIT ? "BF16x3" : "HP");
}

// Operators of an FP64-vector inner solve at the split or HP level: the
// product in KRR_BF16X3 (through FP32 copies of the vectors) or KRR_HP; the
// preconditioner in FP32 arithmetic through FP32 copies (any fixed SPD
// approximation serves as a preconditioner).  Scratch is looked up by name,
// so the first (uncaptured) call allocates it.
void double_inner_ops(krr_handle* h, const float* X, int n, int ldx, int d, double sigma,
                      double lambda, int k, int level, bool precond,
                      std::function<void(cudaStream_t, const double*, double*)>& matvec,
                      std::function<void(cudaStream_t, const double*, double*)>& apply) {
  const size_t nk = (size_t)n * k;
  ColScale one;
  for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
  // allocated here: the loop body may be captured into a graph
  wsT<float>(h, "v_cvin", nk);
  wsT<float>(h, "v_cvout", nk);
  wsT<float>(h, "v_cvr", nk);
  wsT<float>(h, "v_cvz", nk);
  if (level == INNER_SPLIT) {
    matvec = [h, X, n, ldx, d, sigma, lambda, k, nk, one](cudaStream_t s2, const double* V,
                                                          double* Q) {
      float* vf = wsT<float>(h, "v_cvin", nk);
      float* qf = wsT<float>(h, "v_cvout", nk);
      launch_convert<double, float>(s2, V, n, k, k, vf, k, one);
      matvec_dispatch(h, s2, X, n, ldx, X, n, ldx, d, sigma, lambda, vf, k, k, qf, k,
                      KRR_BF16X3);
      launch_convert<float, double>(s2, qf, n, k, k, Q, k, one);
    };
  } else {
    matvec = [h, X, n, ldx, d, sigma, lambda, k](cudaStream_t s2, const double* V, double* Q) {
      matvec_dispatch(h, s2, X, n, ldx, X, n, ldx, d, sigma, lambda, V, k, k, Q, k, KRR_HP);
    };
  }
  apply = nullptr;
  if (precond)
    apply = [h, n, k, nk, one](cudaStream_t s2, const double* R, double* Zo) {
      float* rf = wsT<float>(h, "v_cvr", nk);
      float* zf = wsT<float>(h, "v_cvz", nk);
      launch_convert<double, float>(s2, R, n, k, k, rf, k, one);
      apply_precond<float>(h, s2, rf, k, k, zf, k);
      launch_convert<float, double>(s2, zf, n, k, k, Zo, k, one);
    };
}

// Mixed precision: FP16 (or BF16) tensor-core inner PCG with FP32 vectors;
// outer iterative refinement with the residual in HP arithmetic and FP64
// vectors.
krr_status solve_mixed(krr_handle* h, const SolveArgs& a, krr_report* rep, int* matvecs) {
  cudaStream_t st = h->stream;
  const int n = a.n, k = a.k;
  const size_t nk = (size_t)n * k;
  double* Yc = wsT<double>(h, "v_y", nk);
  double* Cd = wsT<double>(h, "v_cd", nk);
  double* Rd = wsT<double>(h, "v_rd", nk);
  double* AX = wsT<double>(h, "v_ax", nk);
  double* Rs = wsT<double>(h, "v_rs", nk);  // scaled residual (inner tolerance reference)
  double* Cp = wsT<double>(h, "v_cprev", nk);
  double* Rp = wsT<double>(h, "v_rprev", nk);
  ColScale one;
  for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
  launch_convert<double, double>(st, a.Y, n, k, a.ldy, Yc, k, one);
  if (a.o.warm_start) {
    launch_convert<double, double>(st, a.C, n, k, a.ldc, Cd, k, one);
    matvec_dispatch(h, st, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, Cd, k, k, AX, k,
                    KRR_HP);
    ++*matvecs;
    launch_sub_d(st, Yc, k, AX, k, n, k, Rd, k);
  } else {
    KRR_CUDA(cudaMemsetAsync(Cd, 0, nk * sizeof(double), st));
    KRR_CUDA(cudaMemcpyAsync(Rd, Yc, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  double yy[KRR_MAX_RHS];
  host_colnorm2<double>(h, Yc, n, k, k, yy);
  int total_iters[KRR_MAX_RHS] = {0};
  krr_status status = KRR_OK;
  int outer = 0;
  int remaining = a.o.max_iter;
  // the inner arithmetic moves up a level (FP16 -> BF16x3 -> HP) once a
  // correction contracts the residual by less than a half (see batched_mixed)
  int level = a.o.inner_precision == KRR_HP ? INNER_HP : INNER_LOW;
  double rel_prev = 0.0;
  double rel[KRR_MAX_RHS] = {0}, rel_saved[KRR_MAX_RHS] = {0};
  // consecutive low-level inner solves continue the previous search
  // direction (residual replacement) unless a step was taken back
  bool keep_ok = false;
  double norm_prev[KRR_MAX_RHS] = {0};
  double kmax[KRR_MAX_RHS] = {0};
  for (;;) {
    double rr[KRR_MAX_RHS];
    host_colnorm2<double>(h, Rd, n, k, k, rr);
    bool ok = true, finite = true;
    double now = 0.0;
    for (int c = 0; c < k; ++c) {
      rel[c] = yy[c] > 0 ? std::sqrt(rr[c] / yy[c]) : 0.0;
      if (!std::isfinite(rel[c])) finite = false;
      if (!(rel[c] <= a.o.tol)) ok = false;
      now = std::max(now, rel[c]);
    }
    KRR_TRACE("mixed: outer %d rel %.3e (previous %.3e) inner %s", outer, now, rel_prev,
              level_name(level));
    if (finite && ok) break;
    if (outer > 0) {
      if (!finite || !(now < rel_prev)) {
        // the last correction did not help: take it back
        keep_ok = false;
        KRR_CUDA(cudaMemcpyAsync(Cd, Cp, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
        KRR_CUDA(cudaMemcpyAsync(Rd, Rp, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
        host_colnorm2<double>(h, Rd, n, k, k, rr);
        for (int c = 0; c < k; ++c) rel[c] = rel_saved[c];
        finite = true;
        if (level == INNER_HP) {
          status = KRR_ENOTCONV;
          break;
        }
        // a correction that made things worse means the system is far too
        // ill-conditioned for FP32-accurate kernel entries: straight to HP
        level = INNER_HP;
      } else if (now > keep_below(level) * rel_prev && level != INNER_HP) {
        level = next_level(level, a.d);
      }
    }
    if (!finite) {
      status = KRR_ENAN;
      break;
    }
    if (outer >= a.o.max_outer || remaining <= 0) {
      status = KRR_ENOTCONV;
      break;
    }
    ++outer;
    rel_prev = 0.0;
    ColScale sc, inv;
    for (int c = 0; c < KRR_MAX_RHS; ++c) sc.v[c] = inv.v[c] = 0.0;
    for (int c = 0; c < k; ++c) {
      rel_saved[c] = rel[c];
      rel_prev = std::max(rel_prev, rel[c]);
      if (rel[c] > a.o.tol) {
        sc.v[c] = 1.0 / std::sqrt(rr[c]);
        inv.v[c] = std::sqrt(rr[c]);
      }
    }
    KRR_CUDA(cudaMemcpyAsync(Cp, Cd, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
    KRR_CUDA(cudaMemcpyAsync(Rp, Rd, nk * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_convert<double, double>(st, Rd, n, k, k, Rs, k, sc);
    LoopOut lo;
    if (level == INNER_LOW) {
      const int prec = low_precision(a.o);
      PcgSpec<float> S;
      S.n = n; S.k = k; S.Ytol = Rs; S.ldy = k;
      S.x = wsT<float>(h, "v_xf", nk); S.r = wsT<float>(h, "v_rf", nk);
      S.p = wsT<float>(h, "v_pf", nk); S.z = wsT<float>(h, "v_zf", nk);
      S.q = wsT<float>(h, "v_qf", nk);
      S.tol = inner_tol_for(level, a.o, rel_prev); S.max_iter = remaining; S.prec = prec;
      S.matvec = [&, prec](cudaStream_t s2, const float* V, float* Q) {
        matvec_dispatch(h, s2, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, V, k, k, Q,
                        k, prec);
      };
      if (a.o.precond)
        S.apply = [&](cudaStream_t s2, const float* R, float* Zo) {
          apply_precond<float>(h, s2, R, k, k, Zo, k);
        };
      S.restart = keep_ok && a.o.keep_direction != 0;
      for (int c = 0; c < KRR_MAX_RHS; ++c)
        S.rscale.v[c] = (c < k && norm_prev[c] > 0.0 && inv.v[c] > 0.0)
                            ? norm_prev[c] / inv.v[c] : 0.0;
      // the fused body: the plain tensor-core product of the training points
      // and the streamed ZL apply
      if (a.o.fuse_step && a.o.precond && !h->kern.poly && prec != KRR_BF16P &&
          apply_cg_supported(h->pc, n, k) &&
          tc_loop_prepare(h->tc, st, a.X, n, a.ldx, a.d, a.sigma, k, prec == KRR_BF16X3 ? 1 : 0,
                          prec == KRR_FP16 ? 1 : 0, &S.tl)) {
        S.fused = true;
        S.tc_split = prec == KRR_BF16X3 ? 1 : 0;
        S.tc_f16 = prec == KRR_FP16 ? 1 : 0;
        S.shift = a.lambda;
        S.rn = wsT<float>(h, "v_rnf", nk);
      }
      launch_convert<double, float>(st, Rs, n, k, k, S.r, k, one);
      KRR_CUDA(cudaMemsetAsync(S.x, 0, nk * sizeof(float), st));
      pcg_loop<float>(h, S, a.o.use_graph != 0, &lo, matvecs);
      if (!(lo.flags & FLAG_NAN)) launch_axpy_d<float>(st, S.x, n, k, k, Cd, k, inv);
      keep_ok = !(lo.flags & (FLAG_NAN | FLAG_BREAKDOWN));
      for (int c = 0; c < KRR_MAX_RHS; ++c) norm_prev[c] = inv.v[c];
    } else {
      keep_ok = false;
      PcgSpec<double> S;
      S.n = n; S.k = k; S.Ytol = Rs; S.ldy = k;
      S.x = wsT<double>(h, "v_x", nk); S.r = wsT<double>(h, "v_r", nk);
      S.p = wsT<double>(h, "v_p", nk); S.z = wsT<double>(h, "v_z", nk);
      S.q = wsT<double>(h, "v_q", nk);
      S.tol = inner_tol_for(level, a.o, rel_prev);
      S.max_iter = remaining;
      S.prec = level == INNER_SPLIT ? KRR_BF16X3 : KRR_HP;
      if (level == INNER_SPLIT && !h->kern.poly)
        tc_prepare_split(h->tc, st, a.X, n, a.ldx, a.d, a.sigma);
      double_inner_ops(h, a.X, n, a.ldx, a.d, a.sigma, a.lambda, k, level, a.o.precond != 0,
                       S.matvec, S.apply);
      launch_convert<double, double>(st, Rs, n, k, k, S.r, k, one);
      KRR_CUDA(cudaMemsetAsync(S.x, 0, nk * sizeof(double), st));
      pcg_loop<double>(h, S, a.o.use_graph != 0, &lo, matvecs);
      if (!(lo.flags & FLAG_NAN)) launch_axpy_d<double>(st, S.x, n, k, k, Cd, k, inv);
    }
    for (int c = 0; c < k; ++c) {
      total_iters[c] += lo.iters[c];
      kmax[c] = std::max(kmax[c], lo.kappa[c]);
      // the inner system is r / ||r||: its recursive residual in units of ||y||
      if (rep)
        rep->rel_res_rec[c] =
            (lo.yy[c] > 0 ? std::sqrt(lo.rr[c] / lo.yy[c]) : 0.0) * rel_saved[c];
    }
    remaining -= lo.iter;
    KRR_TRACE("mixed: inner solve %d iterations, flags %d", lo.iter, lo.flags);
    // a NaN in the inner solve leaves Cd unchanged; the next pass takes the
    // correction back and switches to the HP inner solve
    matvec_dispatch(h, st, a.X, n, a.ldx, a.X, n, a.ldx, a.d, a.sigma, a.lambda, Cd, k, k, AX, k,
                    KRR_HP);
    ++*matvecs;
    launch_sub_d(st, Yc, k, AX, k, n, k, Rd, k);
  }
  if (rep)
    for (int c = 0; c < k; ++c) rep->rel_res[c] = rel[c];
  launch_convert<double, double>(st, Cd, n, k, k, a.C, a.ldc, one);
  if (rep) {
    for (int c = 0; c < k; ++c) {
      rep->iters[c] = total_iters[c];
      rep->kappa[c] = kmax[c];
    }
    rep->outer_steps = outer;
  }
  return status;
}

void check_solve_args(const krr_opts& o, int n, int d, int ldx, double sigma, double lambda,
                      const float* W, const float* b, int s, int k, int ldy, int ldc) {
  KRR_REQUIRE(n > 0 && d > 0 && k >= 1 && k <= KRR_MAX_RHS, "pcg_solve: bad sizes");
  KRR_REQUIRE(ldx >= d && ldy >= k && ldc >= k, "pcg_solve: leading dimension too small");
  KRR_REQUIRE(sigma > 0.0 && std::isfinite(sigma), "pcg_solve: sigma must be > 0");
  KRR_REQUIRE(lambda > 0.0 && std::isfinite(lambda), "pcg_solve: lambda must be > 0");
  KRR_REQUIRE(o.tol > 0.0 && o.max_iter >= 0, "pcg_solve: bad tol / max_iter");
  KRR_REQUIRE(o.precision == KRR_FP64 || o.precision == KRR_FP32 || o.precision == KRR_MIXED,
              "pcg_solve: precision must be KRR_FP64, KRR_FP32 or KRR_MIXED");
  KRR_REQUIRE(o.precond >= 0 && o.precond <= 2, "pcg_solve: precond must be 0, 1 or 2");
  if (o.precond == 1) {
    KRR_REQUIRE(W && b && s > 0 && s <= n, "pcg_solve: preconditioner needs W, b and 0 < s <= n");
  }
  if (o.precision == KRR_MIXED) {
    KRR_REQUIRE(o.inner_tol > 0.0 && o.inner_tol < 1.0, "pcg_solve: inner_tol in (0, 1)");
    KRR_REQUIRE(o.inner_precision == 0 || o.inner_precision == KRR_FP16 ||
                    o.inner_precision == KRR_BF16 || o.inner_precision == KRR_BF16X3 ||
                    o.inner_precision == KRR_HP,
                "pcg_solve: inner_precision must be 0, KRR_FP16, KRR_BF16, KRR_BF16X3 or KRR_HP");
  }
}

// The set-up of Algorithm 1 on device-resident operands: RFF features and the
// preconditioner factors; for the mixed solve also the FP16 (or BF16) and HP
// operands.
void setup_impl(krr_handle* h, const float* Xd, int n, int d, int ldx, double sigma,
                double lambda, const float* Wd, const float* bd, int s, const krr_opts& o) {
  cudaStream_t st = h->stream;
  if (o.precond == 2)
    KRR_REQUIRE(h->pc.ready && h->pc.n == n,
                "pcg_solve: precond = 2 needs a preconditioner set up for these n points");
  if (o.precond == 1) {
    const int zf = o.z_format < 0 ? (o.precision == KRR_MIXED ? KRR_Z_FIXED : KRR_Z_FP32)
                                : o.z_format;
    const double lp = o.lambda_p > 0.0 ? o.lambda_p : lambda;
    if (zf == KRR_Z_FIXED) {
      precond_setup_rff_tc(h, Xd, n, d, ldx, Wd, bd, s, lp, o.apply_form);
    } else {
      float* Z = wsT<float>(h, "rff_Z", (size_t)n * s);
      launch_rff(st, Xd, n, d, ldx, Wd, bd, s, Z, s);
      precond_setup_impl(h, Z, n, s, s, lp, o.apply_form, zf);
    }
  }
  if (o.precision == KRR_MIXED) {
    if (low_precision(o) == KRR_FP16)
      tc_prepare_f16(h->tc, st, Xd, n, ldx, d, sigma);
    else if (low_precision(o) == KRR_BF16X3)
      tc_prepare_split(h->tc, st, Xd, n, ldx, d, sigma);
    else
      tc_prepare(h->tc, st, Xd, n, ldx, d, sigma);
    tc_clear_error(h->tc, st);
    if (hp_supported(d)) {
      hp_prepare(h->hp, st, Xd, n, ldx, d, sigma);
      hp_clear_error(h->hp, st);
    }
  }
}

// Algorithm 1 on device-resident operands: features and preconditioner
// (lines 5-7), then PCG in the requested arithmetic.  Records `ev_setup`
// once the set-up work is enqueued (null: not recorded).
krr_status solve_impl(krr_handle* h, const float* Xd, int n, int d, int ldx, double sigma,
                      double lambda, const float* Wd, const float* bd, int s, const double* Yd,
                      int k, int ldy, double* Cd, int ldc, const krr_opts& o, krr_report* rep,
                      int* matvecs, cudaEvent_t ev_setup) {
  KRR_TRACE("pcg_solve: n=%d d=%d k=%d s=%d prec=%d graph=%d", n, d, k, s, o.precision,
            o.use_graph);
  setup_impl(h, Xd, n, d, ldx, sigma, lambda, Wd, bd, s, o);
  cudaStream_t st = h->stream;
  if (ev_setup) KRR_CUDA(cudaEventRecord(ev_setup, st));
  KRR_TRACE("pcg_solve: setup done");
  SolveArgs a{Xd, n, d, ldx, sigma, lambda, Yd, k, ldy, Cd, ldc, o};
  krr_status status;
  if (o.precision == KRR_FP64)
    status = solve_plain<double>(h, a, KRR_FP64, rep, matvecs);
  else if (o.precision == KRR_FP32)
    status = solve_plain<float>(h, a, KRR_FP32, rep, matvecs);
  else
    status = solve_mixed(h, a, rep, matvecs);
  if (o.precision == KRR_MIXED && (tc_error(h->tc, st) || hp_error(h->hp, st)))
    status = KRR_ETIMEOUT;
  if (o.precond && precond_error(h)) status = KRR_ETIMEOUT;
  return status;
}

// (D o K)(Xr, Xc) V: FP64 (direct differences) or HP (float-float SIMT).
void dsigma_dispatch(krr_handle* h, cudaStream_t st, const float* Xr, int nr, int ldxr,
                     const float* Xc, int nc, int ldxc, int d, double sigma, const double* V,
                     int k, int ldv, double* Q, int ldq, int prec) {
  if (prec == KRR_FP16 || prec == KRR_BF16 || prec == KRR_BF16X3) {
    // tensor-core derivative product on rounded points: FP32 in and out
    ColScale one;
    for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
    float* Vf = wsT<float>(h, "ds_vf", (size_t)nc * k);
    float* Qf = wsT<float>(h, "ds_qf", (size_t)nr * k);
    launch_convert<double, float>(st, V, nc, k, ldv, Vf, k, one);
    tc_dsigma_matvec(h->tc, st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, Vf, k, k, Qf, k,
                     prec == KRR_BF16X3 ? 1 : 0, prec == KRR_FP16 ? 1 : 0);
    launch_convert<float, double>(st, Qf, nr, k, k, Q, ldq, one);
    return;
  }
  if (prec == KRR_FP64) {
    double* part = wsT<double>(h, "mv_part64", mv_fp64_part_elems(nr, nc, k));
    launch_mv_fp64(st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, 0.0, V, k, ldv, Q, ldq, part, 1);
    return;
  }
  double* part = wsT<double>(h, "hpw_part", mv_hpw_part_elems(nr, nc, k));
  float* nrm_r = wsT<float>(h, "hpw_nr", 2 * (size_t)nr);
  float* nrm_c = wsT<float>(h, "hpw_nc", 2 * (size_t)nc);
  launch_mv_hpw(st, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, 0.0, V, k, ldv, Q, ldq, part, nrm_r,
                nrm_c, 1);
}

// sum_{i, c} A[i, c] B[i, c] read back to the host.
double host_dot(krr_handle* h, const double* A, int lda, const double* B, int ldb, int n, int k) {
  double* part = wsT<double>(h, "cg_part", cg_part_elems(n, k));
  double* dout = wsT<double>(h, "dot_out", 1);
  unsigned int* ctr = wsT<unsigned int>(h, "dot_ctr", 4);
  KRR_CUDA(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned int), h->stream));
  launch_dot_d(h->stream, A, lda, B, ldb, n, k, dout, part, ctr);
  KRR_CUDA(cudaMemcpyAsync(h->hostd, dout, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KRR_CUDA(cudaStreamSynchronize(h->stream));
  return h->hostd[0];
}

// ---------------------------------------------------------- batched solve --
// Captures what `f` enqueues on the handle's capture stream into graph `g`
// after the nodes `deps`; returns the number of kernel launches captured.
template <typename F>
long long capture_into(krr_handle* h, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                       F&& f) {
  KRR_CUDA(cudaStreamBeginCaptureToGraph(h->cap, g, deps, nullptr, ndeps,
                                         cudaStreamCaptureModeRelaxed));
  capture_begin();
  try {
    f(h->cap);
  } catch (...) {
    capture_end();
    cudaGraph_t tmp;
    cudaStreamEndCapture(h->cap, &tmp);
    cudaGetLastError();
    throw;
  }
  long long n = capture_end();
  cudaGraph_t out = nullptr;
  KRR_CUDA(cudaStreamEndCapture(h->cap, &out));
  return n;
}

// One solve of a lockstep batch: its handle (workspace, scalars, factors,
// product state) and its loop body.
struct BatchEntry {
  krr_handle* sub = nullptr;
  std::function<void(cudaStream_t)> body;
  long long body_launches = 0;
};

// Runs the loop bodies of independent PCG solves in lockstep in one graph
// launch.  Graph: WHILE { gate -> IF_0 { body_0 } ... IF_{m-1} { body_{m-1} }
// -> tail }.  The gate sets IF_i from solve i's `run` flag, so a finished
// solve launches nothing; the IF nodes have no edges between them, so the
// graph executor may run the solves' kernels concurrently; the tail keeps
// the loop going while any solve runs.  pcg_begin must have run for every
// entry.
void pcg_loop_batched(krr_handle* h, std::vector<BatchEntry>& E,
                      const std::function<void(cudaStream_t)>& pre = nullptr) {
  const int ne = (int)E.size();
  if (ne == 0) return;
  cudaStream_t st = h->stream;
  CgScalars** d_scs = wsT<CgScalars*>(h, "bt_scs", ne);
  unsigned long long* d_cond = wsT<unsigned long long>(h, "bt_cond", ne);
  std::vector<CgScalars*> scs(ne);
  std::vector<unsigned long long> conds(ne);
  for (int i = 0; i < ne; ++i) scs[i] = E[i].sub->sc;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  KRR_CUDA(cudaGraphCreate(&graph, 0));
  long long fixed = 0;
  try {
    cudaGraphConditionalHandle wcond;
    KRR_CUDA(cudaGraphConditionalHandleCreate(&wcond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
    wp.conditional.handle = wcond;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    KRR_CUDA(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    for (int i = 0; i < ne; ++i) {
      cudaGraphConditionalHandle c;
      KRR_CUDA(cudaGraphConditionalHandleCreate(&c, body, 0, 0));
      conds[i] = (unsigned long long)c;
    }
    KRR_CUDA(cudaMemcpyAsync(d_scs, scs.data(), ne * sizeof(CgScalars*), cudaMemcpyHostToDevice,
                             st));
    KRR_CUDA(cudaMemcpyAsync(d_cond, conds.data(), ne * sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, st));
    // the gate, then the products shared by several solves (one launch
    // sequence over all their problems), before any solve's own body
    fixed += capture_into(h, body, nullptr, 0, [&](cudaStream_t cs) {
      launch_batch_gate(cs, d_scs, d_cond, ne);
      if (pre) pre(cs);
    });
    size_t nn = 0;
    KRR_CUDA(cudaGraphGetNodes(body, nullptr, &nn));
    std::vector<cudaGraphNode_t> heads(nn);
    KRR_CUDA(cudaGraphGetNodes(body, heads.data(), &nn));
    cudaGraphNode_t gate = nullptr;   // the chain's last node
    for (cudaGraphNode_t nd : heads) {
      size_t nd_out = 0;
      KRR_CUDA(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out));
      if (nd_out == 0) gate = nd;
    }
    KRR_REQUIRE(nn >= 1 && gate, "batched loop: unexpected gate graph");
    std::vector<cudaGraphNode_t> ifn(ne);
    for (int i = 0; i < ne; ++i) {
      cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
      ip.conditional.handle = (cudaGraphConditionalHandle)conds[i];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      KRR_CUDA(cudaGraphAddNode(&ifn[i], body, &gate, nullptr, 1, &ip));
      E[i].body_launches =
          capture_into(h, ip.conditional.phGraph_out[0], nullptr, 0, E[i].body);
    }
    fixed += capture_into(h, body, ifn.data(), ifn.size(), [&](cudaStream_t cs) {
      launch_batch_tail(cs, d_scs, ne, (unsigned long long)wcond);
    });
    KRR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    KRR_CUDA(cudaGraphLaunch(exec, st));
    KRR_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    throw;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  int rounds = 0;
  for (int i = 0; i < ne; ++i) {
    krr_handle* g = E[i].sub;
    KRR_CUDA(cudaMemcpyAsync(g->sc_host, g->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
  }
  KRR_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < ne; ++i) {
    const int it = E[i].sub->sc_host->iter;
    rounds = std::max(rounds, it);
    add_launches(E[i].body_launches * (long long)it);
  }
  add_launches(fixed * (long long)rounds);
}

// A problem of krr_pcg_solve_batched with its device operands and progress.
struct BItem {
  int idx = 0;                   // position in the caller's array
  krr_handle* sub = nullptr;
  const float* X = nullptr;
  int n = 0, d = 0, ldx = 0, k = 0, ldy = 0, ldc = 0, s = 0;
  double sigma = 0.0, lambda = 0.0;
  const double* Y = nullptr;
  double* C = nullptr;           // device result (the caller's or a staging copy)
  double* C_user = nullptr;
  bool c_host = false;
  bool done = false;
  krr_status status = KRR_OK;
  int matvecs = 0, outer = 0, remaining = 0;
  int iters[KRR_MAX_RHS] = {0};
  double rel[KRR_MAX_RHS] = {0};
  double yy[KRR_MAX_RHS] = {0};
  ColScale inv;
  // mixed precision: the inner arithmetic moves up a level (FP16 -> BF16x3
  // -> HP) when a correction contracts the residual by less than a half
  int level = INNER_LOW;
  double rel_prev = 0.0;
  double rel_saved[KRR_MAX_RHS] = {0};
  double kappa[KRR_MAX_RHS] = {0};   // largest condition estimate over its loops
  double rrec[KRR_MAX_RHS] = {0};    // last loop's recursive residual (units of ||y||)
};

double max_rel(const BItem& it) {
  double m = 0.0;
  for (int c = 0; c < it.k; ++c) m = std::max(m, it.rel[c]);
  return m;
}

ColScale ones() {
  ColScale one;
  for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
  return one;
}

template <typename T>
PcgSpec<T> item_spec(BItem& it, const double* Ytol, double tol, int prec, bool precond) {
  krr_handle* g = it.sub;
  const size_t nk = (size_t)it.n * it.k;
  PcgSpec<T> S;
  S.n = it.n;
  S.k = it.k;
  S.Ytol = Ytol;
  S.ldy = it.k;
  const bool f = sizeof(T) == 4;
  S.x = wsT<T>(g, f ? "v_xf" : "v_x", nk);
  S.r = wsT<T>(g, f ? "v_rf" : "v_r", nk);
  S.p = wsT<T>(g, f ? "v_pf" : "v_p", nk);
  S.z = wsT<T>(g, f ? "v_zf" : "v_z", nk);
  S.q = wsT<T>(g, f ? "v_qf" : "v_q", nk);
  S.tol = tol;
  S.max_iter = it.remaining;
  S.prec = prec;
  const float* X = it.X;
  const int n = it.n, ldx = it.ldx, d = it.d, k = it.k;
  const double sigma = it.sigma, lambda = it.lambda;
  S.matvec = [g, X, n, ldx, d, sigma, lambda, k, prec](cudaStream_t s2, const T* V, T* Q) {
    matvec_dispatch(g, s2, X, n, ldx, X, n, ldx, d, sigma, lambda, V, k, k, Q, k, prec);
  };
  if (precond)
    S.apply = [g, k](cudaStream_t s2, const T* R, T* Zo) { apply_precond<T>(g, s2, R, k, k, Zo, k); };
  return S;
}

// Per-column relative residual ||Rd_c|| / ||y_c|| of an item (host read).
bool item_converged(BItem& it, const double* Rd, double tol, double* rr) {
  host_colnorm2<double>(it.sub, Rd, it.n, it.k, it.k, rr);
  bool ok = true;
  for (int c = 0; c < it.k; ++c) {
    double rel = it.yy[c] > 0 ? std::sqrt(rr[c] / it.yy[c]) : 0.0;
    it.rel[c] = rel;
    if (!std::isfinite(rel)) it.status = KRR_ENAN;
    if (!(rel <= tol)) ok = false;
  }
  return ok;
}

// Plain PCG (FP64 or FP32 vectors) for every item in lockstep; FP64 true
// residual after each round, FP64 items restart from it up to three times.
template <typename T>
void batched_plain(krr_handle* h, std::vector<BItem>& B, const krr_opts& o, int prec) {
  const ColScale one = ones();
  for (BItem& it : B) {
    krr_handle* g = it.sub;
    const size_t nk = (size_t)it.n * it.k;
    double* Yc = wsT<double>(g, "v_y", nk);
    launch_convert<double, double>(g->stream, it.Y, it.n, it.k, it.ldy, Yc, it.k, one);
    host_colnorm2<double>(g, Yc, it.n, it.k, it.k, it.yy);
    PcgSpec<T> S = item_spec<T>(it, Yc, o.tol, prec, o.precond != 0);
    KRR_CUDA(cudaMemsetAsync(S.x, 0, nk * sizeof(T), g->stream));
    launch_convert<double, T>(g->stream, Yc, it.n, it.k, it.k, S.r, it.k, one);
    it.remaining = o.max_iter;
  }
  std::vector<bool> pending(B.size(), true);
  for (;;) {
    std::vector<BatchEntry> E;
    std::vector<int> act;
    for (size_t i = 0; i < B.size(); ++i) {
      BItem& it = B[i];
      if (it.done || !pending[i]) continue;
      double* Yc = wsT<double>(it.sub, "v_y", (size_t)it.n * it.k);
      PcgSpec<T> S = item_spec<T>(it, Yc, o.tol, prec, o.precond != 0);
      pcg_begin<T>(it.sub, S);
      krr_handle* g = it.sub;
      E.push_back(BatchEntry{g, [g, S](cudaStream_t cs) { pcg_body<T>(g, S, cs, 0ull); }, 0});
      act.push_back((int)i);
    }
    if (E.empty()) break;
    if (o.max_iter > 0) pcg_loop_batched(h, E);
    for (int i : act) {
      BItem& it = B[i];
      krr_handle* g = it.sub;
      pending[i] = false;
      LoopOut lo;
      pcg_finish(g, it.k, &lo);
      for (int c = 0; c < it.k; ++c) {
        it.iters[c] += lo.iters[c];
        it.kappa[c] = std::max(it.kappa[c], lo.kappa[c]);
        it.rrec[c] = lo.yy[c] > 0 ? std::sqrt(lo.rr[c] / lo.yy[c]) : 0.0;
      }
      it.remaining -= lo.iter;
      it.matvecs += lo.iter;
      if (lo.flags & FLAG_NAN) {
        it.status = KRR_ENAN;
        it.done = true;
        continue;
      }
      if (lo.flags & FLAG_BREAKDOWN) {
        it.status = KRR_EBREAKDOWN;
        it.done = true;
        continue;
      }
      const size_t nk = (size_t)it.n * it.k;
      double* Yc = wsT<double>(g, "v_y", nk);
      double* xd = wsT<double>(g, "v_xd", nk);
      double* AX = wsT<double>(g, "v_ax", nk);
      double* Rd = wsT<double>(g, "v_rd", nk);
      PcgSpec<T> S = item_spec<T>(it, Yc, o.tol, prec, o.precond != 0);
      launch_convert<T, double>(g->stream, S.x, it.n, it.k, it.k, xd, it.k, one);
      matvec_dispatch(g, g->stream, it.X, it.n, it.ldx, it.X, it.n, it.ldx, it.d, it.sigma,
                      it.lambda, xd, it.k, it.k, AX, it.k, prec == KRR_FP64 ? KRR_FP64 : KRR_HP);
      ++it.matvecs;
      launch_sub_d(g->stream, Yc, it.k, AX, it.k, it.n, it.k, Rd, it.k);
      double rr[KRR_MAX_RHS];
      if (item_converged(it, Rd, o.tol, rr) && it.status == KRR_OK) {
        it.done = true;
      } else if (it.status != KRR_OK || (lo.flags & FLAG_CAP) || it.remaining <= 0 ||
                 prec != KRR_FP64 || it.outer >= 3) {
        if (it.status == KRR_OK) it.status = KRR_ENOTCONV;
        it.done = true;
      } else {
        ++it.outer;
        launch_convert<double, T>(g->stream, Rd, it.n, it.k, it.k, S.r, it.k, one);
        pending[i] = true;
      }
    }
  }
  for (BItem& it : B) {
    PcgSpec<T> S = item_spec<T>(it, nullptr, o.tol, prec, false);
    launch_convert<T, double>(it.sub->stream, S.x, it.n, it.k, it.k, it.C, it.ldc, one);
  }
}

// Mixed precision for every item: rounds of lockstep inner PCG on the scaled
// residuals, each followed by the HP residual of every item.  The inner
// product is the BF16 tensor-core product; an item whose BF16 correction
// contracts its residual by less than a half (the BF16 kernel of the
// rounded points is too far from K for its lambda) discards a correction
// that made things worse and continues with inner solves on the HP product
// in FP64 vectors, run to the accuracy the outer test needs.
void batched_mixed(krr_handle* h, std::vector<BItem>& B, const krr_opts& o) {
  const ColScale one = ones();
  for (BItem& it : B) {
    krr_handle* g = it.sub;
    if (o.inner_precision == KRR_HP) it.level = INNER_HP;
    const size_t nk = (size_t)it.n * it.k;
    double* Yc = wsT<double>(g, "v_y", nk);
    double* Cd = wsT<double>(g, "v_cd", nk);
    double* Rd = wsT<double>(g, "v_rd", nk);
    wsT<double>(g, "v_ax", nk);
    wsT<double>(g, "v_rs", nk);
    wsT<double>(g, "v_cprev", nk);
    wsT<double>(g, "v_rprev", nk);
    launch_convert<double, double>(g->stream, it.Y, it.n, it.k, it.ldy, Yc, it.k, one);
    KRR_CUDA(cudaMemsetAsync(Cd, 0, nk * sizeof(double), g->stream));
    KRR_CUDA(cudaMemcpyAsync(Rd, Yc, nk * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    host_colnorm2<double>(g, Yc, it.n, it.k, it.k, it.yy);
    it.remaining = o.max_iter;
  }
  for (;;) {
    std::vector<BatchEntry> E;
    std::vector<int> act;
    // the FP16-point products of the low-level solves (one right-hand side,
    // d <= 128) run as one persistent launch over all their problems
    std::vector<BatchProb> bp;
    const bool can_batch = o.batch_product != 0 && low_precision(o) == KRR_FP16;
    for (size_t i = 0; i < B.size(); ++i) {
      BItem& it = B[i];
      if (it.done) continue;
      krr_handle* g = it.sub;
      const size_t nk = (size_t)it.n * it.k;
      double* Cd = wsT<double>(g, "v_cd", nk);
      double* Rd = wsT<double>(g, "v_rd", nk);
      double* Rs = wsT<double>(g, "v_rs", nk);
      double* Cp = wsT<double>(g, "v_cprev", nk);
      double* Rp = wsT<double>(g, "v_rprev", nk);
      double rr[KRR_MAX_RHS];
      const bool ok = item_converged(it, Rd, o.tol, rr);
      if (it.status == KRR_OK && ok) {
        it.done = true;
        continue;
      }
      if (it.outer > 0) {
        const double now = max_rel(it);
        if (!(now < it.rel_prev)) {
          // the last correction did not help: take it back
          KRR_CUDA(cudaMemcpyAsync(Cd, Cp, nk * sizeof(double), cudaMemcpyDeviceToDevice,
                                   g->stream));
          KRR_CUDA(cudaMemcpyAsync(Rd, Rp, nk * sizeof(double), cudaMemcpyDeviceToDevice,
                                   g->stream));
          for (int c = 0; c < it.k; ++c) it.rel[c] = it.rel_saved[c];
          host_colnorm2<double>(g, Rd, it.n, it.k, it.k, rr);
          it.status = KRR_OK;
          if (it.level == INNER_HP) {
            // HP inner solves no longer help: the HP residual's accuracy floor
            it.status = KRR_ENOTCONV;
            it.done = true;
            continue;
          }
          // worse, not just slow: straight to HP (see solve_mixed)
          it.level = INNER_HP;
        } else if (now > keep_below(it.level) * it.rel_prev && it.level != INNER_HP) {
          it.level = next_level(it.level, it.d);
        }
      }
      if (it.status != KRR_OK) {
        it.done = true;
        continue;
      }
      if (it.outer >= o.max_outer || it.remaining <= 0) {
        it.status = KRR_ENOTCONV;
        it.done = true;
        continue;
      }
      ++it.outer;
      it.rel_prev = max_rel(it);
      for (int c = 0; c < it.k; ++c) it.rel_saved[c] = it.rel[c];
      KRR_CUDA(cudaMemcpyAsync(Cp, Cd, nk * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      KRR_CUDA(cudaMemcpyAsync(Rp, Rd, nk * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      ColScale sc;
      for (int c = 0; c < KRR_MAX_RHS; ++c) sc.v[c] = it.inv.v[c] = 0.0;
      for (int c = 0; c < it.k; ++c)
        if (it.rel[c] > o.tol) {
          sc.v[c] = 1.0 / std::sqrt(rr[c]);
          it.inv.v[c] = std::sqrt(rr[c]);
        }
      launch_convert<double, double>(g->stream, Rd, it.n, it.k, it.k, Rs, it.k, sc);
      if (it.level == INNER_LOW) {
        PcgSpec<float> S =
            item_spec<float>(it, Rs, inner_tol_for(INNER_LOW, o, it.rel_prev), low_precision(o),
                             o.precond != 0);
        launch_convert<double, float>(g->stream, Rs, it.n, it.k, it.k, S.r, it.k, one);
        KRR_CUDA(cudaMemsetAsync(S.x, 0, nk * sizeof(float), g->stream));
        pcg_begin<float>(g, S);
        if (can_batch && it.k == 1 && it.d <= 128 && (int)bp.size() < BATCH_MAX &&
            g->tc.half_ready) {
          S.skip_matvec = true;
          bp.push_back(BatchProb{&g->tc.half, S.p, S.q, it.lambda, &g->sc->run});
        }
        E.push_back(BatchEntry{g, [g, S](cudaStream_t cs) { pcg_body<float>(g, S, cs, 0ull); }, 0});
      } else {
        // FP64 vectors; the split or HP product
        if (it.level == INNER_SPLIT)
          tc_prepare_split(g->tc, g->stream, it.X, it.n, it.ldx, it.d, it.sigma);
        PcgSpec<double> S = item_spec<double>(it, Rs, inner_tol_for(it.level, o, it.rel_prev),
                                              it.level == INNER_SPLIT ? KRR_BF16X3 : KRR_HP,
                                              false);
        double_inner_ops(g, it.X, it.n, it.ldx, it.d, it.sigma, it.lambda, it.k, it.level,
                         o.precond != 0, S.matvec, S.apply);
        launch_convert<double, double>(g->stream, Rs, it.n, it.k, it.k, S.r, it.k, one);
        KRR_CUDA(cudaMemsetAsync(S.x, 0, nk * sizeof(double), g->stream));
        pcg_begin<double>(g, S);
        E.push_back(
            BatchEntry{g, [g, S](cudaStream_t cs) { pcg_body<double>(g, S, cs, 0ull); }, 0});
      }
      act.push_back((int)i);
    }
    if (E.empty()) break;
    if (!bp.empty()) {
      tc_batch_reserve(h->batch, h->stream, bp);   // the sub-handles share h's stream
      pcg_loop_batched(h, E, [&](cudaStream_t cs) { tc_batch_matvec(h->batch, cs, bp); });
      if (tc_batch_error(h->batch, h->stream))
        for (int i : act) B[i].status = KRR_ETIMEOUT;
    } else {
      pcg_loop_batched(h, E);
    }
    for (int i : act) {
      BItem& it = B[i];
      krr_handle* g = it.sub;
      LoopOut lo;
      pcg_finish(g, it.k, &lo);
      for (int c = 0; c < it.k; ++c) {
        it.iters[c] += lo.iters[c];
        it.kappa[c] = std::max(it.kappa[c], lo.kappa[c]);
        it.rrec[c] = (lo.yy[c] > 0 ? std::sqrt(lo.rr[c] / lo.yy[c]) : 0.0) * it.rel_saved[c];
      }
      it.remaining -= lo.iter;
      it.matvecs += lo.iter;
      const size_t nk = (size_t)it.n * it.k;
      double* Yc = wsT<double>(g, "v_y", nk);
      double* Cd = wsT<double>(g, "v_cd", nk);
      double* Rd = wsT<double>(g, "v_rd", nk);
      double* AX = wsT<double>(g, "v_ax", nk);
      // a NaN in the inner solve leaves Cd unchanged; the next round takes
      // the correction back and moves the inner arithmetic up a level
      if (!(lo.flags & FLAG_NAN)) {
        if (it.level != INNER_LOW)
          launch_axpy_d<double>(g->stream, wsT<double>(g, "v_x", nk), it.n, it.k, it.k, Cd, it.k,
                                it.inv);
        else
          launch_axpy_d<float>(g->stream, wsT<float>(g, "v_xf", nk), it.n, it.k, it.k, Cd, it.k,
                               it.inv);
      }
      matvec_dispatch(g, g->stream, it.X, it.n, it.ldx, it.X, it.n, it.ldx, it.d, it.sigma,
                      it.lambda, Cd, it.k, it.k, AX, it.k, KRR_HP);
      ++it.matvecs;
      launch_sub_d(g->stream, Yc, it.k, AX, it.k, it.n, it.k, Rd, it.k);
    }
  }
  for (BItem& it : B) {
    krr_handle* g = it.sub;
    const size_t nk = (size_t)it.n * it.k;
    double* Cd = wsT<double>(g, "v_cd", nk);
    launch_convert<double, double>(g->stream, Cd, it.n, it.k, it.k, it.C, it.ldc, one);
    if (tc_error(g->tc, g->stream) || hp_error(g->hp, g->stream) || precond_error(g)) {
      it.status = KRR_ETIMEOUT;
    }
  }
}

}  // namespace

// ======================================================================= ABI
extern "C" {

krr_status krr_set_autotune(krr_handle* h, int on, int* shapes) {
  if (!h || on < 0 || on > 3) return KRR_EINVAL;
  tc_set_autotune(h->tc, on);
  for (krr_handle* sub : h->subs) tc_set_autotune(sub->tc, on);
  if (shapes) *shapes = tc_tuned_shapes();
  return KRR_OK;
}

void krr_default_opts(krr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->max_iter = 1000;
  o->lambda_p = 0.0;
  o->precond = 1;
  o->precision = KRR_FP64;
  o->apply_form = KRR_APPLY_ZL;
  o->use_graph = 1;
  o->inner_tol = 3e-2;
  o->max_outer = 30;
  o->z_format = -1;
  o->batch_product = 1;
  o->warm_start = 0;
  o->inner_precision = KRR_FP16;
  o->keep_direction = 0;
  o->fuse_step = 1;
}

const char* krr_status_string(krr_status s) {
  switch (s) {
    case KRR_OK: return "ok";
    case KRR_EINVAL: return "invalid argument";
    case KRR_ENOMEM: return "out of device memory";
    case KRR_ECUDA: return "CUDA error";
    case KRR_ECHOL: return "preconditioner Gram matrix not positive definite";
    case KRR_ENOTCONV: return "not converged";
    case KRR_EBREAKDOWN: return "CG breakdown";
    case KRR_ENAN: return "NaN or Inf";
    case KRR_ETIMEOUT: return "device loop iteration cap";
    case KRR_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

krr_status krr_create(krr_handle** out, void* stream) {
  if (!out) return KRR_EINVAL;
  *out = nullptr;
  krr_handle* h = new (std::nothrow) krr_handle();
  if (!h) return KRR_ENOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&h->sc, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMemset(h->sc, 0, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&h->sc_host, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&h->hostd, KRR_MAX_RHS * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->info, sizeof(int));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    krr_destroy(h);
    return e == cudaErrorMemoryAllocation ? KRR_ENOMEM : KRR_ECUDA;
  }
  h->stream = (cudaStream_t)stream;
  *out = h;
  return KRR_OK;
}

krr_status krr_destroy(krr_handle* h) {
  if (!h) return KRR_EINVAL;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->bufs) free_buf(kv.second);
  free_buf(h->pc.Z);
  free_buf(h->pc.L);
  free_buf(h->pc.Linv);
  free_buf(h->pc.LinvT);
  free_buf(h->pc.U);
  free_buf(h->pc.err);
  for (krr_handle* sub : h->subs) krr_destroy(sub);
  h->subs.clear();
  tc_release(h->tc);
  hp_release(h->hp);
  tc_batch_release(h->batch);
  for (TcState& t : h->batch_tc) tc_release(t);
  if (h->batch_ones.p) cudaFree(h->batch_ones.p);
  if (h->sc) cudaFree(h->sc);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->hostd) cudaFreeHost(h->hostd);
  if (h->info) cudaFree(h->info);
  for (auto ev : h->ev)
    if (ev) cudaEventDestroy(ev);
  if (h->cap) cudaStreamDestroy(h->cap);
  cudaSetDevice(cur);
  delete h;
  return KRR_OK;
}

krr_status krr_set_stream(krr_handle* h, void* stream) {
  if (!h) return KRR_EINVAL;
  h->stream = (cudaStream_t)stream;
  return KRR_OK;
}

const char* krr_last_error(const krr_handle* h) { return h ? h->err.c_str() : "null handle"; }

krr_status krr_rff_features(krr_handle* h, const float* X, int n, int d, int ldx, const float* W,
                            const float* b, int s, float* Z, int ldz) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(X && W && b && Z, "rff_features: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && s > 0, "rff_features: sizes must be positive");
    KRR_REQUIRE(ldx >= d && ldz >= s, "rff_features: leading dimension too small");
    launch_rff(h->stream, X, n, d, ldx, W, b, s, Z, ldz);
    return KRR_OK;
  });
}

krr_status krr_rff_features_fixed(krr_handle* h, const float* X, int n, int d, int ldx,
                                  const float* W, const float* b, int s, signed char* Zq, int ldz,
                                  int* e_out) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(X && W && b && Zq && e_out, "rff_features_fixed: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && s > 0, "rff_features_fixed: sizes must be positive");
    KRR_REQUIRE(ldx >= d && ldz >= s, "rff_features_fixed: leading dimension too small");
    cudaStream_t st = h->stream;
    const int n_pad = setup_tc_n_pad(n), s_pad = setup_tc_s_pad(s), kp = setup_tc_kp(d);
    __nv_bfloat16* ZT = wsT<__nv_bfloat16>(h, "tcs_zt", (size_t)s_pad * n_pad);
    __nv_bfloat16* Xh = wsT<__nv_bfloat16>(h, "tcs_xh", (size_t)n_pad * kp);
    __nv_bfloat16* Xl = wsT<__nv_bfloat16>(h, "tcs_xl", (size_t)n_pad * kp);
    __nv_bfloat16* Wh = wsT<__nv_bfloat16>(h, "tcs_wh", (size_t)s_pad * kp);
    __nv_bfloat16* Wl = wsT<__nv_bfloat16>(h, "tcs_wl", (size_t)s_pad * kp);
    signed char* Zo = ldz == s ? Zq : wsT<signed char>(h, "tcs_zout", (size_t)n * s);
    int* scr = wsT<int>(h, "tcs_scr", 4);
    KRR_CUDA(cudaMemsetAsync(scr, 0, 4 * sizeof(int), st));
    *e_out = launch_rff_tc(st, X, n, d, ldx, W, b, s, Xh, Xl, Wh, Wl, Zo, ZT, scr + 1);
    if (ldz != s)
      KRR_CUDA(cudaMemcpy2DAsync(Zq, (size_t)ldz, Zo, (size_t)s, (size_t)s, n,
                                 cudaMemcpyDeviceToDevice, st));
    int flag = 0;
    KRR_CUDA(cudaMemcpyAsync(&flag, scr + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaStreamSynchronize(st));
    if (flag) throw Error{KRR_ETIMEOUT, "rff_features_fixed: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

krr_status krr_kernel_matvec(krr_handle* h, const float* Xr, int nr, int ldxr, const float* Xc,
                             int nc, int ldxc, int d, double sigma, double shift, const void* V,
                             int k, int ldv, void* Q, int ldq, int precision) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Xr && Xc && V && Q, "kernel_matvec: null pointer");
    KRR_REQUIRE(nr > 0 && nc > 0 && d > 0, "kernel_matvec: sizes must be positive");
    KRR_REQUIRE(k >= 1 && k <= KRR_MAX_RHS, "kernel_matvec: need 1 <= k <= KRR_MAX_RHS");
    KRR_REQUIRE(ldxr >= d && ldxc >= d && ldv >= k && ldq >= k,
                "kernel_matvec: leading dimension too small");
    KRR_REQUIRE(sigma > 0.0 && std::isfinite(sigma), "kernel_matvec: sigma must be > 0");
    KRR_REQUIRE(shift == 0.0 || nr == nc, "kernel_matvec: shift needs a square product");
    KRR_REQUIRE(precision == KRR_FP64 || precision == KRR_FP32 || precision == KRR_BF16 ||
                    precision == KRR_HP || precision == KRR_BF16X3 || precision == KRR_BF16P ||
                    precision == KRR_FP16,
                "kernel_matvec: bad precision");
    matvec_dispatch(h, h->stream, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, shift, V, k, ldv, Q, ldq,
                    precision);
    if (((precision == KRR_BF16 || precision == KRR_BF16X3 || precision == KRR_BF16P ||
          precision == KRR_FP16) &&
         tc_error(h->tc, h->stream)) ||
        (precision == KRR_HP && hp_error(h->hp, h->stream)))
      throw Error{KRR_ETIMEOUT, "tensor-core product: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

krr_status krr_precond_setup(krr_handle* h, const float* Z, int n, int s, int ldz,
                             double lambda_p, int apply_form, int z_format) {
  return guard(h, [&]() -> krr_status {
    precond_setup_impl(h, Z, n, s, ldz, lambda_p, apply_form, z_format);
    return KRR_OK;
  });
}

krr_status krr_precond_apply(krr_handle* h, const double* R, int k, int ldr, double* Zout,
                             int ldo) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(h->pc.ready, "precond_apply: call krr_precond_setup first");
    KRR_REQUIRE(R && Zout, "precond_apply: null pointer");
    KRR_REQUIRE(k >= 1 && k <= KRR_MAX_RHS && ldr >= k && ldo >= k, "precond_apply: bad k / ld");
    apply_precond<double>(h, h->stream, R, k, ldr, Zout, ldo);
    return KRR_OK;
  });
}

krr_status krr_pcg_solve(krr_handle* h, const float* X, int n, int d, int ldx, double sigma,
                         double lambda, const float* W, const float* b, int s, const double* Y,
                         int k, int ldy, double* C, int ldc, const krr_opts* opts,
                         krr_report* rep) {
  return guard(h, [&]() -> krr_status {
    krr_opts o;
    if (opts)
      o = *opts;
    else
      krr_default_opts(&o);
    KRR_REQUIRE(X && Y && C, "pcg_solve: null pointer");
    check_solve_args(o, n, d, ldx, sigma, lambda, W, b, s, k, ldy, ldc);
    if (rep) {
      memset(rep, 0, sizeof(*rep));
      rep->k = k;
    }
    cudaStream_t st = h->stream;
    KRR_CUDA(cudaEventRecord(h->ev[0], st));
    // stage host inputs
    const bool c_host = !on_device(C);
    const float* Xd = (const float*)stage_in(h, X, (size_t)n * ldx * sizeof(float), "X");
    const double* Yd = (const double*)stage_in(h, Y, (size_t)n * ldy * sizeof(double), "Y");
    double* Cd = C;
    if (c_host) {
      Cd = wsT<double>(h, "stage_C", (size_t)n * ldc);
      if (o.warm_start)
        KRR_CUDA(cudaMemcpyAsync(Cd, C, (size_t)n * ldc * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    int matvecs = 0;
    const float* Wd = nullptr;
    const float* bd = nullptr;
    if (o.precond == 1) {
      Wd = (const float*)stage_in(h, W, (size_t)d * s * sizeof(float), "W");
      bd = (const float*)stage_in(h, b, (size_t)s * sizeof(float), "b");
    }
    krr_status status = solve_impl(h, Xd, n, d, ldx, sigma, lambda, Wd, bd, s, Yd, k, ldy, Cd,
                                   ldc, o, rep, &matvecs, h->ev[1]);
    if (c_host)
      KRR_CUDA(cudaMemcpyAsync(C, Cd, (size_t)n * ldc * sizeof(double), cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaEventRecord(h->ev[2], st));
    KRR_CUDA(cudaEventSynchronize(h->ev[2]));
    if (rep) {
      rep->status = status;
      rep->matvecs = matvecs;
      rep->ms_setup = ms_between(h->ev[0], h->ev[1]);
      rep->ms_solve = ms_between(h->ev[1], h->ev[2]);
      rep->ms_total = ms_between(h->ev[0], h->ev[2]);
    }
    if (status != KRR_OK) h->err = krr_status_string(status);
    return status;
  });
}

krr_status krr_pcg_solve_batched(krr_handle* h, const krr_problem* probs, int nprob,
                                 const krr_opts* opts, krr_report* reps) {
  return guard(h, [&]() -> krr_status {
    krr_opts o;
    if (opts)
      o = *opts;
    else
      krr_default_opts(&o);
    KRR_REQUIRE(probs && nprob > 0, "pcg_solve_batched: need nprob > 0 problems");
    KRR_REQUIRE(!o.warm_start, "pcg_solve_batched: warm_start is not supported");
    for (int i = 0; i < nprob; ++i) {
      const krr_problem& p = probs[i];
      KRR_REQUIRE(p.X && p.Y && p.C, "pcg_solve_batched: null pointer in problem " +
                                         std::to_string(i));
      check_solve_args(o, p.n, p.d, p.ldx, p.sigma, p.lambda, p.W, p.b, p.s, p.k, p.ldy, p.ldc);
    }
    cudaStream_t st = h->stream;
    while ((int)h->subs.size() < nprob) {
      krr_handle* sub = nullptr;
      krr_status cs = krr_create(&sub, (void*)st);
      if (cs != KRR_OK) throw Error{cs, "pcg_solve_batched: could not create a problem handle"};
      h->subs.push_back(sub);
    }
    for (krr_handle* sub : h->subs) tc_set_autotune(sub->tc, h->tc.autotune);
    KRR_CUDA(cudaEventRecord(h->ev[0], st));
    // largest problems first: their graph branches are issued first
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const double wa = (double)probs[a].n * probs[a].n * (probs[a].d + probs[a].k);
      const double wb = (double)probs[b].n * probs[b].n * (probs[b].d + probs[b].k);
      return wa > wb;
    });
    std::vector<BItem> B(nprob);
    for (int j = 0; j < nprob; ++j) {
      const int i = order[j];
      const krr_problem& p = probs[i];
      BItem& it = B[j];
      krr_handle* g = h->subs[j];
      g->stream = st;
      g->err.clear();
      it.idx = i;
      it.sub = g;
      it.n = p.n;
      it.d = p.d;
      it.ldx = p.ldx;
      it.k = p.k;
      it.ldy = p.ldy;
      it.ldc = p.ldc;
      it.s = p.s;
      it.sigma = p.sigma;
      it.lambda = p.lambda;
      it.X = (const float*)stage_in(g, p.X, (size_t)p.n * p.ldx * sizeof(float), "X");
      it.Y = (const double*)stage_in(g, p.Y, (size_t)p.n * p.ldy * sizeof(double), "Y");
      it.C_user = p.C;
      it.c_host = !on_device(p.C);
      it.C = it.c_host ? wsT<double>(g, "stage_C", (size_t)p.n * p.ldc) : p.C;
      const float* Wd = nullptr;
      const float* bd = nullptr;
      KRR_REQUIRE(o.precond != 2, "pcg_solve_batched: precond must be 0 or 1");
      if (o.precond) {
        Wd = (const float*)stage_in(g, p.W, (size_t)p.d * p.s * sizeof(float), "W");
        bd = (const float*)stage_in(g, p.b, (size_t)p.s * sizeof(float), "b");
      }
      setup_impl(g, it.X, p.n, p.d, p.ldx, p.sigma, p.lambda, Wd, bd, p.s, o);
    }
    KRR_CUDA(cudaEventRecord(h->ev[1], st));
    if (o.precision == KRR_FP64)
      batched_plain<double>(h, B, o, KRR_FP64);
    else if (o.precision == KRR_FP32)
      batched_plain<float>(h, B, o, KRR_FP32);
    else
      batched_mixed(h, B, o);
    for (BItem& it : B)
      if (it.c_host)
        KRR_CUDA(cudaMemcpyAsync(it.C_user, it.C, (size_t)it.n * it.ldc * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaEventRecord(h->ev[2], st));
    KRR_CUDA(cudaEventSynchronize(h->ev[2]));
    krr_status first = KRR_OK;
    std::vector<krr_status> by_idx(nprob, KRR_OK);
    for (BItem& it : B) by_idx[it.idx] = it.status;
    for (int i = 0; i < nprob; ++i)
      if (by_idx[i] != KRR_OK) {
        first = by_idx[i];
        break;
      }
    if (reps) {
      const double ms_setup = ms_between(h->ev[0], h->ev[1]);
      const double ms_solve = ms_between(h->ev[1], h->ev[2]);
      const double ms_total = ms_between(h->ev[0], h->ev[2]);
      for (BItem& it : B) {
        krr_report& r = reps[it.idx];
        memset(&r, 0, sizeof(r));
        r.status = it.status;
        r.k = it.k;
        for (int c = 0; c < it.k; ++c) {
          r.iters[c] = it.iters[c];
          r.rel_res[c] = it.rel[c];
          r.kappa[c] = it.kappa[c];
          r.rel_res_rec[c] = it.rrec[c];
        }
        r.outer_steps = it.outer;
        r.matvecs = it.matvecs;
        r.ms_setup = ms_setup;
        r.ms_solve = ms_solve;
        r.ms_total = ms_total;
      }
    }
    if (first != KRR_OK) h->err = krr_status_string(first);
    return first;
  });
}

krr_status krr_predict(krr_handle* h, const float* Xtr, int n, int ldxtr, const float* Xte, int m,
                       int ldxte, int d, double sigma, const double* C, int k, int ldc, double* F,
                       int ldf, int precision) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Xtr && Xte && C && F, "predict: null pointer");
    KRR_REQUIRE(n > 0 && m > 0 && d > 0 && k >= 1 && k <= KRR_MAX_RHS, "predict: bad sizes");
    KRR_REQUIRE(ldxtr >= d && ldxte >= d && ldc >= k && ldf >= k, "predict: bad leading dims");
    KRR_REQUIRE(sigma > 0.0 && std::isfinite(sigma), "predict: sigma must be > 0");
    KRR_REQUIRE(precision == KRR_FP64 || precision == KRR_HP || precision == KRR_FP32 ||
                    precision == KRR_FP16 || precision == KRR_BF16 || precision == KRR_BF16X3,
                "predict: bad precision");
    cudaStream_t st = h->stream;
    const float* Xtr_d = (const float*)stage_in(h, Xtr, (size_t)n * ldxtr * sizeof(float), "pXtr");
    const float* Xte_d = (const float*)stage_in(h, Xte, (size_t)m * ldxte * sizeof(float), "pXte");
    const double* C_d = (const double*)stage_in(h, C, (size_t)n * ldc * sizeof(double), "pC");
    const bool f_host = !on_device(F);
    double* F_d = f_host ? wsT<double>(h, "pF", (size_t)m * ldf) : F;
    if (precision != KRR_FP64 && precision != KRR_HP) {
      // FP32 SIMT or a tensor-core product on rounded points: FP32 in and out
      ColScale one;
      for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
      float* Cf = wsT<float>(h, "pr_cf", (size_t)n * k);
      float* Ff = wsT<float>(h, "pr_ff", (size_t)m * k);
      launch_convert<double, float>(st, C_d, n, k, ldc, Cf, k, one);
      matvec_dispatch(h, st, Xte_d, m, ldxte, Xtr_d, n, ldxtr, d, sigma, 0.0, Cf, k, k, Ff, k,
                      precision);
      launch_convert<float, double>(st, Ff, m, k, k, F_d, ldf, one);
      if (precision != KRR_FP32 && tc_error(h->tc, st))
        throw Error{KRR_ETIMEOUT, "tensor-core product: a pipeline wait hit its limit"};
    } else {
      matvec_dispatch(h, st, Xte_d, m, ldxte, Xtr_d, n, ldxtr, d, sigma, 0.0, C_d, k, ldc, F_d,
                      ldf, precision);
    }
    if (f_host) {
      KRR_CUDA(cudaMemcpyAsync(F, F_d, (size_t)m * ldf * sizeof(double), cudaMemcpyDeviceToHost, st));
      KRR_CUDA(cudaStreamSynchronize(st));
    }
    return KRR_OK;
  });
}

krr_status krr_rfm_fit(krr_handle* h, const float* X, int n, int d, int ldx, const float* W,
                       const float* b, int s, double lambda, const double* Y, int k, int ldy,
                       double* Wf, int ldw) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(X && W && b && Y && Wf, "rfm_fit: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && s > 0 && k >= 1 && k <= KRR_MAX_RHS, "rfm_fit: bad sizes");
    KRR_REQUIRE(ldx >= d && ldy >= k && ldw >= k, "rfm_fit: bad leading dims");
    KRR_REQUIRE(lambda > 0.0 && std::isfinite(lambda), "rfm_fit: lambda must be > 0");
    KRR_REQUIRE(s <= n, "rfm_fit: need s <= n (the preconditioner set-up's Gram path)");
    cudaStream_t st = h->stream;
    const float* Xd = (const float*)stage_in(h, X, (size_t)n * ldx * sizeof(float), "X");
    const float* Wd = (const float*)stage_in(h, W, (size_t)d * s * sizeof(float), "W");
    const float* bd = (const float*)stage_in(h, b, (size_t)s * sizeof(float), "b");
    const double* Yd = (const double*)stage_in(h, Y, (size_t)n * ldy * sizeof(double), "Y");
    // features, then the preconditioner set-up with lambda_p = lambda (FP32 Z):
    // G = Z^T Z + lambda I, L L^T = G, L^-1
    float* Z = wsT<float>(h, "rff_Z", (size_t)n * s);
    launch_rff(st, Xd, n, d, ldx, Wd, bd, s, Z, s);
    precond_setup_impl(h, Z, n, s, s, lambda, KRR_APPLY_ZL, 0);
    double* t1 = wsT<double>(h, "ap_t1", (size_t)s * k);
    double* t2 = wsT<double>(h, "ap_t2", (size_t)s * k);
    double* part = wsT<double>(h, "ap_part", apply_part_elems(n, s, k));
    launch_ginv_zt(st, h->pc, Yd, k, ldy, t1, t2, part);
    ColScale one;
    for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
    const bool w_host = !on_device(Wf);
    double* Wd_out = w_host ? wsT<double>(h, "rfm_w", (size_t)s * ldw) : Wf;
    launch_convert<double, double>(st, t1, s, k, k, Wd_out, ldw, one);
    if (w_host)
      KRR_CUDA(cudaMemcpyAsync(Wf, Wd_out, (size_t)s * ldw * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    if (precond_error(h)) throw Error{KRR_ETIMEOUT, "rfm_fit: a streamed pass hit its wait limit"};
    return KRR_OK;
  });
}

krr_status krr_rfm_predict(krr_handle* h, const float* Xte, int m, int d, int ldx,
                           const float* W, const float* b, int s, const double* Wf, int k,
                           int ldw, double* F, int ldf) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Xte && W && b && Wf && F, "rfm_predict: null pointer");
    KRR_REQUIRE(m > 0 && d > 0 && s > 0 && k >= 1 && k <= KRR_MAX_RHS, "rfm_predict: bad sizes");
    KRR_REQUIRE(ldx >= d && ldw >= k && ldf >= k, "rfm_predict: bad leading dims");
    cudaStream_t st = h->stream;
    const float* Xd = (const float*)stage_in(h, Xte, (size_t)m * ldx * sizeof(float), "rXte");
    const float* Wd = (const float*)stage_in(h, W, (size_t)d * s * sizeof(float), "W");
    const float* bd = (const float*)stage_in(h, b, (size_t)s * sizeof(float), "b");
    const double* wd = (const double*)stage_in(h, Wf, (size_t)s * ldw * sizeof(double), "rW");
    ColScale one;
    for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
    double* wc = wsT<double>(h, "rfm_wc", (size_t)s * k);
    launch_convert<double, double>(st, wd, s, k, ldw, wc, k, one);
    float* Zte = wsT<float>(h, "rfm_Zte", (size_t)m * s);
    launch_rff(st, Xd, m, d, ldx, Wd, bd, s, Zte, s);
    const bool f_host = !on_device(F);
    double* Fd = f_host ? wsT<double>(h, "rfm_F", (size_t)m * ldf) : F;
    launch_feature_gemv(st, Zte, m, s, wc, k, Fd, ldf);
    if (f_host) {
      KRR_CUDA(cudaMemcpyAsync(F, Fd, (size_t)m * ldf * sizeof(double), cudaMemcpyDeviceToHost, st));
      KRR_CUDA(cudaStreamSynchronize(st));
    }
    return KRR_OK;
  });
}

krr_status krr_kernel_dsigma_matvec(krr_handle* h, const float* Xr, int nr, int ldxr,
                                    const float* Xc, int nc, int ldxc, int d, double sigma,
                                    const double* V, int k, int ldv, double* Q, int ldq,
                                    int precision) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Xr && Xc && V && Q, "kernel_dsigma_matvec: null pointer");
    KRR_REQUIRE(nr > 0 && nc > 0 && d > 0, "kernel_dsigma_matvec: sizes must be positive");
    KRR_REQUIRE(k >= 1 && k <= KRR_MAX_RHS, "kernel_dsigma_matvec: need 1 <= k <= KRR_MAX_RHS");
    KRR_REQUIRE(ldxr >= d && ldxc >= d && ldv >= k && ldq >= k,
                "kernel_dsigma_matvec: leading dimension too small");
    KRR_REQUIRE(sigma > 0.0 && std::isfinite(sigma), "kernel_dsigma_matvec: sigma must be > 0");
    KRR_REQUIRE(precision == KRR_FP64 || precision == KRR_HP || precision == KRR_FP16 ||
                    precision == KRR_BF16 || precision == KRR_BF16X3,
                "kernel_dsigma_matvec: precision must be KRR_FP64, KRR_HP, KRR_FP16, KRR_BF16 "
                "or KRR_BF16X3");
    dsigma_dispatch(h, h->stream, Xr, nr, ldxr, Xc, nc, ldxc, d, sigma, V, k, ldv, Q, ldq,
                    precision);
    if ((precision == KRR_FP16 || precision == KRR_BF16 || precision == KRR_BF16X3) &&
        tc_error(h->tc, h->stream))
      throw Error{KRR_ETIMEOUT, "tensor-core product: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

krr_status krr_hypergrad(krr_handle* h, const float* X, int n, int d, int ldx, const float* Xte,
                         int m, int ldxte, double sigma, double lambda, const float* W,
                         const float* b, int s, const double* C, int ldc, const double* GF, int k,
                         int ldg, const krr_opts* opts, double* grad, double* Wadj, int ldw,
                         krr_report* rep) {
  return guard(h, [&]() -> krr_status {
    krr_opts o;
    if (opts)
      o = *opts;
    else
      krr_default_opts(&o);
    KRR_REQUIRE(X && Xte && C && GF && grad, "hypergrad: null pointer");
    KRR_REQUIRE(m > 0 && ldxte >= d && ldg >= k, "hypergrad: bad held-out sizes");
    KRR_REQUIRE(!Wadj || ldw >= k, "hypergrad: ldw too small");
    KRR_REQUIRE(!o.warm_start, "hypergrad: warm_start is not supported for the adjoint solve");
    check_solve_args(o, n, d, ldx, sigma, lambda, W, b, s, k, ldc, ldc);
    if (rep) {
      memset(rep, 0, sizeof(*rep));
      rep->k = k;
    }
    cudaStream_t st = h->stream;
    KRR_CUDA(cudaEventRecord(h->ev[0], st));
    const float* Xd = (const float*)stage_in(h, X, (size_t)n * ldx * sizeof(float), "X");
    const float* Xted = (const float*)stage_in(h, Xte, (size_t)m * ldxte * sizeof(float), "hXte");
    const double* Cd = (const double*)stage_in(h, C, (size_t)n * ldc * sizeof(double), "hC");
    const double* Gd = (const double*)stage_in(h, GF, (size_t)m * ldg * sizeof(double), "hG");
    const float* Wd = nullptr;
    const float* bd = nullptr;
    if (o.precond == 1) {
      Wd = (const float*)stage_in(h, W, (size_t)d * s * sizeof(float), "W");
      bd = (const float*)stage_in(h, b, (size_t)s * sizeof(float), "b");
    }
    const size_t nk = (size_t)n * k, mk = (size_t)m * k;
    double* gbar = wsT<double>(h, "hg_gbar", nk);
    double* wadj = wsT<double>(h, "hg_w", nk);
    double* t_tr = wsT<double>(h, "hg_ttr", nk);
    double* t_te = wsT<double>(h, "hg_tte", mk);
    // gbar = K(X, Xte) g_f: the held-out gradient pulled back to the training points
    matvec_dispatch(h, st, Xd, n, ldx, Xted, m, ldxte, d, sigma, 0.0, Gd, k, ldg, gbar, k,
                    KRR_HP);
    // adjoint system (K + lambda I) w = gbar, the same operator as Eq. (1)
    int matvecs = 1;
    krr_status status = solve_impl(h, Xd, n, d, ldx, sigma, lambda, Wd, bd, s, gbar, k, k, wadj,
                                   k, o, rep, &matvecs, h->ev[1]);
    // (D_te o K_te) c and (D o K) c, then the three contractions
    dsigma_dispatch(h, st, Xted, m, ldxte, Xd, n, ldx, d, sigma, Cd, k, ldc, t_te, k, KRR_HP);
    dsigma_dispatch(h, st, Xd, n, ldx, Xd, n, ldx, d, sigma, Cd, k, ldc, t_tr, k, KRR_HP);
    matvecs += 2;
    const double w_c = host_dot(h, wadj, k, Cd, ldc, n, k);
    const double g_t = host_dot(h, Gd, ldg, t_te, k, m, k);
    const double w_t = host_dot(h, wadj, k, t_tr, k, n, k);
    grad[0] = g_t - w_t;
    grad[1] = -lambda * w_c;
    if (Wadj) {
      if (on_device(Wadj)) {
        KRR_CUDA(cudaMemcpy2DAsync(Wadj, (size_t)ldw * sizeof(double), wadj, k * sizeof(double),
                                   k * sizeof(double), n, cudaMemcpyDeviceToDevice, st));
      } else {
        KRR_CUDA(cudaMemcpy2DAsync(Wadj, (size_t)ldw * sizeof(double), wadj, k * sizeof(double),
                                   k * sizeof(double), n, cudaMemcpyDeviceToHost, st));
      }
    }
    KRR_CUDA(cudaEventRecord(h->ev[2], st));
    KRR_CUDA(cudaEventSynchronize(h->ev[2]));
    if (rep) {
      rep->status = status;
      rep->matvecs = matvecs;
      rep->ms_setup = ms_between(h->ev[0], h->ev[1]);
      rep->ms_solve = ms_between(h->ev[1], h->ev[2]);
      rep->ms_total = ms_between(h->ev[0], h->ev[2]);
    }
    if (status != KRR_OK) h->err = krr_status_string(status);
    return status;
  });
}

}  // extern "C"

extern "C" krr_status krr_bench_ex2(krr_handle* h, int iters, double* ex2_per_s, double* ms) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(iters > 0 && ex2_per_s, "bench_ex2: iters > 0 and an output pointer");
    *ex2_per_s = bench_ex2(h->stream, iters, ms);
    return KRR_OK;
  });
}

extern "C" krr_status krr_bench_ex2_mix(krr_handle* h, int iters, int fma_per_32,
                                        double* exp2_per_s, double* ms) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(iters > 0 && exp2_per_s, "bench_ex2_mix: iters > 0 and an output pointer");
    KRR_REQUIRE(fma_per_32 == 0 || fma_per_32 == 2 || fma_per_32 == 4 || fma_per_32 == 6 ||
                    fma_per_32 == 8 || fma_per_32 == 10 || fma_per_32 == 12 ||
                    fma_per_32 == 16 || fma_per_32 == 32,
                "bench_ex2_mix: fma_per_32 must be one of 0 2 4 6 8 10 12 16 32");
    *exp2_per_s = bench_ex2_mix(h->stream, iters, fma_per_32, ms);
    return KRR_OK;
  });
}

// ------------------------------------------------ polynomial kernel ------
namespace {

// The TensorSketch tables, checked on the host (every hash in [0, s), every
// sign +-1: an out-of-range hash would address outside the sketch) and
// staged on the device.
void stage_sketch_tables(krr_handle* h, const int* hash, const signed char* sign, int q, int dd,
                         int s, const int** hd, const signed char** sd) {
  const size_t m = (size_t)q * dd;
  std::vector<int> hh(m);
  std::vector<signed char> sh(m);
  KRR_CUDA(cudaMemcpy(hh.data(), hash, m * sizeof(int), cudaMemcpyDefault));
  KRR_CUDA(cudaMemcpy(sh.data(), sign, m, cudaMemcpyDefault));
  for (size_t i = 0; i < m; ++i) {
    KRR_REQUIRE(hh[i] >= 0 && hh[i] < s, "tensorsketch: hash values must lie in [0, s)");
    KRR_REQUIRE(sh[i] == 1 || sh[i] == -1, "tensorsketch: signs must be +1 or -1");
  }
  *hd = (const int*)stage_in(h, hash, m * sizeof(int), "ts_hash");
  *sd = (const signed char*)stage_in(h, sign, m, "ts_sign");
}

// Makes the handle's products the polynomial kernel's for one call.
struct PolyKernelScope {
  krr_handle* h;
  PolyKernelScope(krr_handle* hh, double gamma, double c, int q, const float* X, int n, int ldx,
                  int d)
      : h(hh) {
    h->kern.poly = 1;
    h->kern.gamma = gamma;
    h->kern.c = c;
    h->kern.q = q;
    h->kern.X = X;
    h->kern.n = n;
    h->kern.ldx = ldx;
    h->kern.d = d;
  }
  ~PolyKernelScope() { h->kern.poly = 0; }
};

void check_poly(double gamma, double c, int q) {
  KRR_REQUIRE(gamma > 0.0 && std::isfinite(gamma), "polynomial kernel: gamma must be > 0");
  KRR_REQUIRE(c >= 0.0 && std::isfinite(c), "polynomial kernel: c must be >= 0");
  KRR_REQUIRE(q >= 1 && q <= 8, "polynomial kernel: need 1 <= q <= 8");
}

}  // namespace

extern "C" krr_status krr_tensorsketch_features(krr_handle* h, const float* X, int n, int d,
                                                int ldx, const int* hash,
                                                const signed char* sign, int q, int s,
                                                double gamma, double c, float* Z, int ldz) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(X && hash && sign && Z, "tensorsketch: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && s > 0 && ldx >= d && ldz >= s, "tensorsketch: bad sizes");
    check_poly(gamma, c, q);
    const int dd = d + (c > 0.0 ? 1 : 0);
    const int* hd = nullptr;
    const signed char* sd = nullptr;
    stage_sketch_tables(h, hash, sign, q, dd, s, &hd, &sd);
    launch_tensorsketch(h->stream, X, n, d, ldx, hd, sd, q, s, gamma, c, Z, ldz);
    return KRR_OK;
  });
}

extern "C" krr_status krr_kernel_matvec_poly(krr_handle* h, const float* Xr, int nr, int ldxr,
                                             const float* Xc, int nc, int ldxc, int d,
                                             double gamma, double c, int q, double shift,
                                             const void* V, int k, int ldv, void* Q, int ldq,
                                             int precision) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Xr && Xc && V && Q, "kernel_matvec_poly: null pointer");
    KRR_REQUIRE(nr > 0 && nc > 0 && d > 0 && k >= 1 && k <= KRR_MAX_RHS,
                "kernel_matvec_poly: bad sizes");
    KRR_REQUIRE(ldxr >= d && ldxc >= d && ldv >= k && ldq >= k,
                "kernel_matvec_poly: leading dimension too small");
    KRR_REQUIRE(shift == 0.0 || nr == nc, "kernel_matvec_poly: shift needs a square product");
    KRR_REQUIRE(precision == KRR_FP64 || precision == KRR_BF16 || precision == KRR_FP16 ||
                    precision == KRR_BF16X3,
                "kernel_matvec_poly: precision must be KRR_FP64, KRR_BF16, KRR_FP16 or "
                "KRR_BF16X3");
    check_poly(gamma, c, q);
    PolyKernelScope scope(h, gamma, c, q, Xc, nc, ldxc, d);
    matvec_dispatch(h, h->stream, Xr, nr, ldxr, Xc, nc, ldxc, d, 1.0, shift, V, k, ldv, Q, ldq,
                    precision);
    if (precision != KRR_FP64 && tc_error(h->tc, h->stream))
      throw Error{KRR_ETIMEOUT, "tensor-core product: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

extern "C" krr_status krr_poly_pcg_solve(krr_handle* h, const float* X, int n, int d, int ldx,
                                         double gamma, double c, int q, double lambda,
                                         const int* hash, const signed char* sign, int s,
                                         const double* Y, int k, int ldy, double* C, int ldc,
                                         const krr_opts* opts, krr_report* rep) {
  return guard(h, [&]() -> krr_status {
    krr_opts o;
    if (opts)
      o = *opts;
    else
      krr_default_opts(&o);
    KRR_REQUIRE(X && Y && C, "poly_pcg_solve: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && k >= 1 && k <= KRR_MAX_RHS, "poly_pcg_solve: bad sizes");
    KRR_REQUIRE(ldx >= d && ldy >= k && ldc >= k, "poly_pcg_solve: leading dimension too small");
    KRR_REQUIRE(lambda > 0.0 && std::isfinite(lambda), "poly_pcg_solve: lambda must be > 0");
    KRR_REQUIRE(o.tol > 0.0 && o.max_iter >= 0, "poly_pcg_solve: bad tol / max_iter");
    KRR_REQUIRE(o.precision == KRR_FP64 || o.precision == KRR_MIXED,
                "poly_pcg_solve: precision must be KRR_FP64 or KRR_MIXED");
    if (o.precision == KRR_MIXED) {
      KRR_REQUIRE(o.inner_tol > 0.0 && o.inner_tol < 1.0, "poly_pcg_solve: inner_tol in (0, 1)");
      KRR_REQUIRE(o.inner_precision == 0 || o.inner_precision == KRR_FP16 ||
                      o.inner_precision == KRR_BF16 || o.inner_precision == KRR_BF16X3 ||
                    o.inner_precision == KRR_HP,
                  "poly_pcg_solve: inner_precision must be 0, KRR_FP16, KRR_BF16, KRR_BF16X3 or KRR_HP");
    }
    check_poly(gamma, c, q);
    KRR_REQUIRE(o.precond >= 0 && o.precond <= 2, "poly_pcg_solve: precond must be 0, 1 or 2");
    if (o.precond == 1)
      KRR_REQUIRE(hash && sign && s > 0 && s <= n,
                  "poly_pcg_solve: the preconditioner needs hash, sign and 0 < s <= n");
    if (o.precond == 2)
      KRR_REQUIRE(h->pc.ready && h->pc.n == n,
                  "poly_pcg_solve: precond = 2 needs a preconditioner set up for these n points");
    if (rep) {
      memset(rep, 0, sizeof(*rep));
      rep->k = k;
    }
    cudaStream_t st = h->stream;
    KRR_CUDA(cudaEventRecord(h->ev[0], st));
    const bool c_host = !on_device(C);
    const float* Xd = (const float*)stage_in(h, X, (size_t)n * ldx * sizeof(float), "X");
    const double* Yd = (const double*)stage_in(h, Y, (size_t)n * ldy * sizeof(double), "Y");
    double* Cd = C;
    if (c_host) {
      Cd = wsT<double>(h, "stage_C", (size_t)n * ldc);
      if (o.warm_start)
        KRR_CUDA(cudaMemcpyAsync(Cd, C, (size_t)n * ldc * sizeof(double), cudaMemcpyHostToDevice,
                                 st));
    }
    PolyKernelScope scope(h, gamma, c, q, Xd, n, ldx, d);
    if (o.precond == 1) {
      // Algorithm 1 with TensorSketch features (Section 2.2) for the preconditioner
      const int dd = d + (c > 0.0 ? 1 : 0);
      const int* hd = nullptr;
      const signed char* sd = nullptr;
      stage_sketch_tables(h, hash, sign, q, dd, s, &hd, &sd);
      float* Z = wsT<float>(h, "ts_Z", (size_t)n * s);
      launch_tensorsketch(st, Xd, n, d, ldx, hd, sd, q, s, gamma, c, Z, s);
      const int zf = o.z_format < 0 ? (o.precision == KRR_MIXED ? KRR_Z_FIXED : KRR_Z_FP32)
                                    : o.z_format;
      const double lp = o.lambda_p > 0.0 ? o.lambda_p : lambda;
      precond_setup_impl(h, Z, n, s, s, lp, o.apply_form, zf);
    }
    KRR_CUDA(cudaEventRecord(h->ev[1], st));
    int matvecs = 0;
    SolveArgs a{Xd, n, d, ldx, 1.0, lambda, Yd, k, ldy, Cd, ldc, o};
    krr_status status = o.precision == KRR_FP64 ? solve_plain<double>(h, a, KRR_FP64, rep, &matvecs)
                                                : solve_mixed(h, a, rep, &matvecs);
    if (o.precision == KRR_MIXED && tc_error(h->tc, st)) status = KRR_ETIMEOUT;
    if (o.precond && precond_error(h)) status = KRR_ETIMEOUT;
    if (c_host)
      KRR_CUDA(cudaMemcpyAsync(C, Cd, (size_t)n * ldc * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    KRR_CUDA(cudaEventRecord(h->ev[2], st));
    KRR_CUDA(cudaEventSynchronize(h->ev[2]));
    if (rep) {
      rep->status = status;
      rep->matvecs = matvecs;
      rep->ms_setup = ms_between(h->ev[0], h->ev[1]);
      rep->ms_solve = ms_between(h->ev[1], h->ev[2]);
      rep->ms_total = ms_between(h->ev[0], h->ev[2]);
    }
    if (status != KRR_OK) h->err = krr_status_string(status);
    return status;
  });
}

// ------------------------------------------- multiple-level sketching ---
extern "C" krr_status krr_multilevel_features(krr_handle* h, const float* Z1, int n, int s1,
                                              int ldz1, const signed char* signs, int m,
                                              const int* rows, int s2, const float* G, int s3,
                                              float* Z3, int ldz3) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(Z1 && signs && rows && G && Z3, "multilevel_features: null pointer");
    KRR_REQUIRE(n > 0 && s1 > 0 && s2 > 0 && s3 > 0 && ldz1 >= s1 && ldz3 >= s3,
                "multilevel_features: bad sizes");
    KRR_REQUIRE(m >= s1 && m > 0 && (m & (m - 1)) == 0 && m <= 32768,
                "multilevel_features: m must be a power of two, s1 <= m <= 32768");
    KRR_REQUIRE(s2 <= m && s3 <= s2, "multilevel_features: need s3 <= s2 <= m");
    // the signs and the sampled rows, checked on the host: a row index out of
    // range would read outside the transform's buffer
    std::vector<signed char> sg(m);
    std::vector<int> rw(s2);
    KRR_CUDA(cudaMemcpy(sg.data(), signs, (size_t)m, cudaMemcpyDefault));
    KRR_CUDA(cudaMemcpy(rw.data(), rows, (size_t)s2 * sizeof(int), cudaMemcpyDefault));
    for (int j = 0; j < m; ++j)
      KRR_REQUIRE(sg[j] == 1 || sg[j] == -1, "multilevel_features: signs must be +1 or -1");
    for (int k = 0; k < s2; ++k)
      KRR_REQUIRE(rw[k] >= 0 && rw[k] < m, "multilevel_features: rows must lie in [0, m)");
    cudaStream_t st = h->stream;
    const signed char* sd = (const signed char*)stage_in(h, signs, (size_t)m, "ml_signs");
    const int* rd = (const int*)stage_in(h, rows, (size_t)s2 * sizeof(int), "ml_rows");
    float* Z2 = wsT<float>(h, "ml_Z2", (size_t)n * s2);
    launch_srht(st, Z1, n, s1, ldz1, sd, m, rd, s2, Z2, s2);
    const int kp = setup_tc_kp(s2);
    __nv_bfloat16* Ah = wsT<__nv_bfloat16>(h, "ml_ah", (size_t)setup_tc_n_pad(n) * kp);
    __nv_bfloat16* Al = wsT<__nv_bfloat16>(h, "ml_al", (size_t)setup_tc_n_pad(n) * kp);
    __nv_bfloat16* Bh = wsT<__nv_bfloat16>(h, "ml_bh", (size_t)setup_tc_s_pad(s3) * kp);
    __nv_bfloat16* Bl = wsT<__nv_bfloat16>(h, "ml_bl", (size_t)setup_tc_s_pad(s3) * kp);
    int* err = wsT<int>(h, "ml_err", 4);
    KRR_CUDA(cudaMemsetAsync(err, 0, 4 * sizeof(int), st));
    launch_gemm_tc_f32(st, Z2, n, s2, s2, G, s3, s2, (float)(1.0 / std::sqrt((double)s3)), Z3,
                       ldz3, Ah, Al, Bh, Bl, err);
    int flag = 0;
    KRR_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KRR_CUDA(cudaStreamSynchronize(st));
    if (flag) throw Error{KRR_ETIMEOUT, "multilevel_features: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

// ------------------------------------------------ adaptive sketch size ---
extern "C" krr_status krr_precond_setup_adaptive(
    krr_handle* h, const float* X, int n, int d, int ldx, double sigma, double lambda,
    const float* W, const float* b, int s_max, int s0, const double* x0, int power_iters,
    int ns_iters, int product_precision, double lambda_p, int apply_form, int z_format,
    int* s_out, double* estimates, int* tests_out) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(X && W && b && x0 && s_out, "precond_setup_adaptive: null pointer");
    KRR_REQUIRE(n > 0 && d > 0 && ldx >= d && s0 > 0 && s0 <= s_max && s_max <= n,
                "precond_setup_adaptive: need 0 < s0 <= s_max <= n");
    KRR_REQUIRE(sigma > 0.0 && lambda > 0.0 && std::isfinite(sigma) && std::isfinite(lambda),
                "precond_setup_adaptive: sigma and lambda must be > 0");
    KRR_REQUIRE(power_iters >= 1 && ns_iters >= 1, "precond_setup_adaptive: iteration counts");
    KRR_REQUIRE(product_precision == KRR_FP64 || product_precision == KRR_HP ||
                    product_precision == KRR_FP16,
                "precond_setup_adaptive: products in KRR_FP64, KRR_HP or KRR_FP16");
    cudaStream_t st = h->stream;
    const float* Xd = (const float*)stage_in(h, X, (size_t)n * ldx * sizeof(float), "X");
    const float* Wd = (const float*)stage_in(h, W, (size_t)d * s_max * sizeof(float), "ad_Wmax");
    const float* bd = (const float*)stage_in(h, b, (size_t)s_max * sizeof(float), "b");
    const double* x0d = (const double*)stage_in(h, x0, (size_t)n * sizeof(double), "ad_x0");
    double* xv = wsT<double>(h, "ad_x", n);
    double* yv = wsT<double>(h, "ad_y", n);
    double* wv = wsT<double>(h, "ad_w", n);
    float* vf = wsT<float>(h, "ad_vf", n);
    float* qf = wsT<float>(h, "ad_qf", n);
    ColScale one;
    for (int c = 0; c < KRR_MAX_RHS; ++c) one.v[c] = 1.0;
    const double tau = 0.05 * lambda, bound = 0.1 * lambda;
    int s = s0, tests = 0;
    float* Z = nullptr;
    for (;;) {
      float* Wc = wsT<float>(h, "ad_W", (size_t)d * s);
      KRR_CUDA(cudaMemcpy2DAsync(Wc, (size_t)s * sizeof(float), Wd, (size_t)s_max * sizeof(float),
                                 (size_t)s * sizeof(float), d, cudaMemcpyDeviceToDevice, st));
      Z = wsT<float>(h, "ad_Z", (size_t)n * s);
      launch_rff(st, Xd, n, d, ldx, Wc, bd, s, Z, s);
      double* G = wsT<double>(h, "ad_G", (size_t)s * s);
      const int nch = gram_chunks(n, s);
      double* part = wsT<double>(h, "gram_part", (size_t)nch * s * s);
      launch_gram(st, Z, 0, n, s, 0.0, G, part, nch);
      double* work = wsT<double>(h, "ad_work", adaptive_work_elems(n, s));
      adaptive_projector(st, G, s, tau, ns_iters, work, h->info, (int*)h->hostd);
      // power iteration on (I - P) K (I - P) from x0
      KRR_CUDA(cudaMemcpyAsync(xv, x0d, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      double nrm = 0.0;
      host_colnorm2<double>(h, xv, n, 1, 1, &nrm);
      KRR_REQUIRE(nrm > 0.0, "precond_setup_adaptive: x0 is zero");
      launch_scale_d(st, xv, n, 1.0 / std::sqrt(nrm));
      double est = 0.0;
      for (int it = 0; it < power_iters; ++it) {
        apply_i_minus_p(st, Z, n, s, work, xv, yv);
        if (product_precision == KRR_FP16) {
          launch_convert<double, float>(st, yv, n, 1, 1, vf, 1, one);
          matvec_dispatch(h, st, Xd, n, ldx, Xd, n, ldx, d, sigma, 0.0, vf, 1, 1, qf, 1,
                          KRR_FP16);
          launch_convert<float, double>(st, qf, n, 1, 1, wv, 1, one);
        } else {
          matvec_dispatch(h, st, Xd, n, ldx, Xd, n, ldx, d, sigma, 0.0, yv, 1, 1, wv, 1,
                          product_precision);
        }
        apply_i_minus_p(st, Z, n, s, work, wv, yv);
        est = host_dot(h, xv, 1, yv, 1, n, 1);
        double nw = 0.0;
        host_colnorm2<double>(h, yv, n, 1, 1, &nw);
        if (!(nw > 0.0)) {
          est = 0.0;
          break;
        }
        KRR_CUDA(cudaMemcpyAsync(xv, yv, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        launch_scale_d(st, xv, n, 1.0 / std::sqrt(nw));
      }
      if (estimates) estimates[tests] = est;
      ++tests;
      KRR_TRACE("adaptive: s=%d ||(I-P)K(I-P)|| ~ %.3e (bound %.3e)", s, est, bound);
      if (est <= bound || s >= s_max) break;
      s = std::min(2 * s, s_max);
    }
    *s_out = s;
    if (tests_out) *tests_out = tests;
    const double lp = lambda_p > 0.0 ? lambda_p : lambda;
    precond_setup_impl(h, Z, n, s, s, lp, apply_form, z_format < 0 ? KRR_Z_FP32 : z_format);
    return KRR_OK;
  });
}

// ------------------------------------------------ batched kernel products ---
extern "C" krr_status krr_kernel_matvec_batched(krr_handle* h, const krr_matvec_problem* probs,
                                                int count) {
  return guard(h, [&]() -> krr_status {
    KRR_REQUIRE(probs && count >= 1 && count <= BATCH_MAX,
                "kernel_matvec_batched: 1 <= count <= 64 problems");
    for (int i = 0; i < count; ++i) {
      const krr_matvec_problem& q = probs[i];
      KRR_REQUIRE(q.X && q.V && q.Q, "kernel_matvec_batched: null pointer");
      KRR_REQUIRE(q.n > 0 && q.d > 0 && q.d <= 128 && q.ldx >= q.d,
                  "kernel_matvec_batched: need n > 0 and 0 < d <= 128");
      KRR_REQUIRE(q.sigma > 0.0 && std::isfinite(q.sigma), "kernel_matvec_batched: sigma > 0");
    }
    cudaStream_t st = h->stream;
    if ((int)h->batch_tc.size() < count) h->batch_tc.resize(count);
    if (!h->batch_ones.p) {
      ensure_buf(h->batch_ones, sizeof(int));
      const int one = 1;
      KRR_CUDA(cudaMemcpy(h->batch_ones.p, &one, sizeof(int), cudaMemcpyHostToDevice));
    }
    std::vector<BatchProb> bp(count);
    for (int i = 0; i < count; ++i) {
      const krr_matvec_problem& q = probs[i];
      tc_prepare_f16(h->batch_tc[i], st, q.X, q.n, q.ldx, q.d, q.sigma);
      bp[i] = BatchProb{&h->batch_tc[i].half, q.V, q.Q, q.shift, (const int*)h->batch_ones.p};
    }
    tc_batch_reserve(h->batch, st, bp);
    tc_batch_matvec(h->batch, st, bp);
    if (tc_batch_error(h->batch, st))
      throw Error{KRR_ETIMEOUT, "batched product: a pipeline wait hit its limit"};
    return KRR_OK;
  });
}

