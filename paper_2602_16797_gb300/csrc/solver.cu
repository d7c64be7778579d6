// Host driver of one RLOBPCG solve (Algorithm 2 of arXiv 2602.16797) on the GPU.
//
// The plan owns every device buffer of a solve; solve() issues the kernels of sketch.cu,
// factor.cu, gram.cu / gram_tc.cu and small.cu on the plan's stream. Per iteration it copies
// back only the b residual norms and b Ritz values the host-side stopping rule (Sec. 2.1) needs,
// asynchronously into a pinned history; the host waits for the GPU only on the iterations where
// the rule is tested (every check_every iterations), so it queues the iterations in between.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "engine.h"
#include "split.cuh"

namespace rl {

// kernels and launchers defined in the other translation units
int sketch_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int d, int zeta, uint64_t seed,
                    int sketch_prec, void* SA, cudaStream_t st);
size_t factor_workspace_bytes(int64_t d, int64_t n, size_t esz);
size_t refine_workspace_bytes(int64_t d, int64_t n, int dtype);
template <class T>
int factor_refine_impl(T* SA, int d, int n, T* Rout, T* Rout_r, double* sigma, T* Vt, T* Rinv_r, T* Rinv_c,
                       void* work, size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err);
template <class S>
int factor_impl(S* SA, int d, int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c, void* work,
                size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err);
template <class T>
int fill_random_launch(T* Z, int64_t rows, int q, int64_t ld, uint64_t seed, cudaStream_t st);
template <class T>
int small_gemm_launch(const T* In, int64_t ldi, int q, const T* K, int ldk, int b, T* Out, int64_t ldo, int64_t rows,
                      cudaStream_t st);
template <class T, class S>
int trimul_launch(const S* L, int n, const T* X, int64_t ldx, int q, T* Y, int64_t ldy, int lower, int conj_l,
                  cudaStream_t st);
size_t gram_workspace_bytes(int64_t m, int64_t n, int b, int dtype);
int gram_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b, int64_t ldw,
                  void* AW, int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes, int resid_mode,
                  int* err, cudaStream_t st);
size_t split_prep_bytes(int64_t m, int64_t n);
size_t split_work_bytes(int64_t m, int64_t n, int b);
int split_prepare(const double* A, int64_t m, int64_t n, int64_t lda, void* prep, size_t prep_bytes, int* err,
                  cudaStream_t st);
int split_gram(const void* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw, double* AW, int64_t ldaw,
               double* G, int64_t ldg, void* work, size_t work_bytes, int flags, int* err, cudaEvent_t mid,
               cudaStream_t st);
size_t split_work_bytes_c128(int64_t m, int64_t n, int b);
int split_gram_c128(const void* prep, int64_t m, int64_t n, const cd* W, int b, int64_t ldw, cd* AW, int64_t ldaw,
                    cd* G, int64_t ldg, void* work, size_t work_bytes, int flags, int* err, cudaEvent_t mid,
                    cudaStream_t st);
size_t tsqr_workspace_bytes(int64_t m, int c, size_t esz);
template <class T>
int tsqr_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st);
template <class T>
int tsqr_split_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st,
                    cudaStream_t mst, cudaEvent_t lvl_done);
int tsqr_merge1_ctas(int64_t m, int c, size_t esz);
template <class T>
int rr_small_launch(const T* Rt, int c, int b, double* theta, T* K, size_t k_cap, int* info, cudaStream_t st);
template <class T>
int update_launch(T* Tb, int64_t n, T* ATb, int64_t m, T* GTb, int64_t ld, int c, int b, const T* K, cudaStream_t st);
template <class T>
int residual_launch(const T* Tb, const T* Gb, int n, int b, int64_t ld, const double* theta_s, T* Res,
                    double* res_norm, T* Rs, int* err, cudaStream_t st);
template <class T, class S>
int precond_launch(const S* Rinv_r, const S* Rinv_c, int n, int b, const T* Rs, T* Y, T* Tb, int64_t ld, int wo,
                   cudaStream_t st);
template <class T>
int bcgs2_orth_launch(T* Tb, int n, int b, int64_t ld, int wo, int nx, T* E, int passes, cudaStream_t st,
                      const split::WDigits* wd, int* err, bool* digits_done, void* coop, size_t coop_bytes,
                      int svqb, const T* Dl = nullptr, int nl = 0, int64_t ldl = 0);
size_t bcgs2_coop_bytes(int64_t n, int qmax, int b, size_t esz);
template <class T>
int gather_cols_launch(T* buf, int64_t rows, int64_t ld, const int* src, const int* dst, int cnt, cudaStream_t st);
int colnorm_parts(int64_t m);
template <class T>
int colnorm2_launch(const T* A, int64_t m, int n, int64_t lda, double* part, double* out, cudaStream_t st);
template <class T>
int scale_rows_launch(const T* Rs, int n, int b, const double* d2, T* Tb, int64_t ld, int wo, cudaStream_t st);
template <class T>
int copy_cols_launch(const T* src, int64_t lds, int so, T* dst, int64_t ldd, int dof, int64_t rows, int w,
                     cudaStream_t st);
split::WDigits split_w_digits(void* work, int64_t m, int64_t n, int b);
template <class S, class T>
int take_start_launch(const S* Vt, int n, int b, T* Tb, int64_t ld, cudaStream_t st);
template <class T>
int outputs_launch(const T* Tb, const T* ATb, int64_t n, int64_t m, int b, int k, int64_t ld, const double* theta_s,
                   const double* res_norm, double* sigma, T* Vout, T* Uout, double* resid, cudaStream_t st);
template <class T>
int nonfinite_scan_launch(const T* A, int64_t m, int n, int64_t lda, int* err, cudaStream_t st);

}  // namespace rl

using namespace rl;

struct rlobpcg_plan_s {
  // rlobpcg_solve_async: the solve runs on this host thread until rlobpcg_solve_wait joins it
  std::thread async_th;
  bool async_busy = false;
  int async_rc = 0;
  std::string async_err;
  int64_t m = 0, n = 0;
  int k = 0, b = 0, d = 0, dtype = 0;
  rlobpcg_opts opts{};
  cudaStream_t st = nullptr;
  size_t esz = 8, ssz = 8;  // element sizes of the state (T) and of the sketch side (S)
  // device buffers
  void* A_dev = nullptr;    // plan-owned copy of a host A (allocated on first use)
  size_t A_dev_bytes = 0;
  void* SA = nullptr;
  double* sk_sigma = nullptr;
  void* Vt = nullptr;
  void* Rinv_r = nullptr;
  void* Rinv_c = nullptr;
  void* R_c = nullptr;      // R column-major
  void* R_r = nullptr;      // R row-major
  void* Zb = nullptr;       // n x qmax blocks of the start-block / Sigma~(1,1) iterations
  void* Yb = nullptr;
  int qmax = 0;
  size_t K_cap = 0;         // elements of K
  void* fwork = nullptr;
  size_t fwork_bytes = 0;
  void* Tb = nullptr;
  void* ATb = nullptr;
  void* GTb = nullptr;
  void* E = nullptr;
  void* Res = nullptr;
  void* Rs = nullptr;
  void* Y = nullptr;
  void* Rt = nullptr;
  void* K = nullptr;
  double* theta = nullptr;
  double* res_norm = nullptr;
  int* err = nullptr;
  int* info = nullptr;
  void* gwork = nullptr;
  size_t gwork_bytes = 0;
  bool split = false;       // Gram products on the tensor cores (split-bf16)
  bool csplit = false;      // ... of complex A, through its real view (W digits formed per pass)
  void* sprep = nullptr;    // digits of A (split once per solve)
  size_t sprep_bytes = 0;
  void* swork = nullptr;
  size_t swork_bytes = 0;
  void* twork = nullptr;
  size_t twork_bytes = 0;
  void* coop = nullptr;     // global scratch of the cooperative BCGS2 + Orth kernel
  size_t coop_bytes = 0;
  void* cn2 = nullptr;      // squared column norms of A (diagonal preconditioner)
  void* cnpart = nullptr;   // their per-block partial sums
  void* VL = nullptr;       // locked columns of V (n x b) and of A V (m x b), with locking
  void* AVL = nullptr;
  cudaEvent_t ev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // Split Gram path: the TSQR merges and the Rayleigh-Ritz SVD of an iteration run on st2 beside
  // the second split product, which leaves them the SMs they need (ev_lvl: TSQR level done on st;
  // ev_rr: the SVD done on st2)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_lvl = nullptr, ev_rr = nullptr;
  // Per-iteration Gram timing events (4 per slot, a ring) and the pinned history of residual
  // norms and Ritz values, copied asynchronously; the host synchronises only to test the stop rule.
  std::vector<cudaEvent_t> gev;
  double* hist_h = nullptr;
  int hist_slots = 0;
  std::vector<void*> owned;
  size_t bytes = 0;          // device bytes owned by the plan (excluding a host-A copy)
  // history of the last solve: per iteration t = 0 .. iters, the b Ritz values (the b smallest,
  // descending; t = 0 is the start block's Rayleigh-Ritz) and the b residual column norms
  std::vector<double> last_theta, last_res;
  int last_rows = 0;
};

namespace {

// Plan memory is stream-ordered (cudaMallocAsync on the plan's stream, from the device's default
// pool): creating and destroying plans does not synchronise the device, which matters when a
// server creates one plan per request while other solves run.
int dev_alloc(rlobpcg_plan_s* p, void** out, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaMallocAsync(out, bytes, p->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(cudaGetErrorString(e), __FILE__, __LINE__);
    return RLOBPCG_ERR_OOM;
  }
  p->owned.push_back(*out);
  p->bytes += bytes;
  return RLOBPCG_OK;
}

void free_plan(rlobpcg_plan_s* p) {
  for (void* q : p->owned) cudaFreeAsync(q, p->st);
  p->owned.clear();
  if (p->A_dev) cudaFreeAsync(p->A_dev, p->st);
  p->A_dev = nullptr;
  cudaStreamSynchronize(p->st);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->gev)
    if (e) cudaEventDestroy(e);
  p->gev.clear();
  if (p->st2) {
    cudaStreamSynchronize(p->st2);
    cudaStreamDestroy(p->st2);
    p->st2 = nullptr;
  }
  if (p->ev_lvl) cudaEventDestroy(p->ev_lvl);
  if (p->ev_rr) cudaEventDestroy(p->ev_rr);
  p->ev_lvl = p->ev_rr = nullptr;
  if (p->hist_h) cudaFreeHost(p->hist_h);
  p->hist_h = nullptr;
}

constexpr int kRing = 16;   // slots of per-iteration timing events

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stopping rule of Sec. 2.1 (Alg. 1 / Alg. 2): tolerance on max_j ||R(:,j)|| against
// Sigma~(1,1)^2 tau, plus (optionally) the two stagnation checks for every column. History
// that does not exist yet is +inf, so comparisons with it are false.
struct StopRule {
  std::vector<std::vector<double>> r, th;  // index t = 0 .. i+1
  bool check(int i, double sigma11, double tau, bool stag) const {
    const double inf = std::numeric_limits<double>::infinity();
    auto rv = [&](int t, int j) { return t >= 0 ? r[t][j] : inf; };
    auto tv = [&](int t, int j) { return t >= 0 ? th[t][j] : inf; };
    const int b = (int)r[i + 1].size();
    double mx = 0;
    for (int j = 0; j < b; ++j) mx = std::max(mx, r[i + 1][j]);
    if (!(mx <= sigma11 * sigma11 * tau)) return false;
    if (!stag) return true;
    for (int j = 0; j < b; ++j) {
      if (!(1.1 * rv(i + 1, j) >= rv(i - 4, j))) return false;
      const double lhs = 1.1 * (tv(i - 4, j) - tv(i + 1, j)) / tv(i + 1, j);
      const double rhs = (tv(i - 9, j) - tv(i - 4, j)) / tv(i - 4, j);
      if (!(lhs >= rhs)) return false;
    }
    return true;
  }
};

// One Gram pass: AW = A W and G = A^H AW (resid_mode: G = A^H AW for the given AW), on the FP64
// CUDA cores or, for plans with gram_split, on the tensor cores from the digits of A. phase: 0,
// or split::SPLIT_FIRST_ONLY / SPLIT_SECOND_ONLY (with reserved SMs) to run the split path's two
// products as separate launches.
template <class T>
int gram_pass(rlobpcg_plan_s* p, const T* A, int64_t lda, const T* W, T* AW, T* G, int resid_mode,
              cudaEvent_t mid = nullptr, bool w_ready = false, int bw = 0, int phase = 0) {
  const int64_t ld = 3 * p->b;
  if (bw <= 0) bw = p->b;   // block width (the active columns with locking)
  if (p->csplit)
    return split_gram_c128(p->sprep, p->m, p->n, (const cd*)W, bw, ld, (cd*)AW, ld, (cd*)G, ld, p->swork,
                           p->swork_bytes, (resid_mode ? split::SPLIT_RESID : 0) | phase, p->err, mid, p->st);
  if (p->split)
    return split_gram(p->sprep, p->m, p->n, (const double*)W, bw, ld, (double*)AW, ld, (double*)G, ld, p->swork,
                      p->swork_bytes,
                      (resid_mode ? split::SPLIT_RESID : 0) | (w_ready ? split::SPLIT_W_READY : 0) | phase, p->err,
                      mid, p->st);
  return gram_dispatch(A, p->m, p->n, lda, p->dtype, W, bw, ld, AW, ld, G, ld, p->gwork, p->gwork_bytes, resid_mode,
                       p->err, p->st);
}

// State of one solve carried between its phases (set-up, iterations, outputs), so that a batch
// of solves can run the set-up and output phases per solve around one batched iteration loop.
struct SolveRun {
  double tau = 0;
  double sigma11 = 0;
  std::vector<double> theta0;
  StopRule hist;
  int herr = 0;
  long launches0 = 0;
  double gram_ms = 0, gram_ab_ms = 0, gram_atb_ms = 0;
  int gram_passes = 0;
  int sweeps = 0;
  int it = 0, stop = 0, matvecs = 0, nx = 0;
  const double* theta_s = nullptr;
  split::WDigits wd{};
  bool w_ready = false;
};

template <class T, class S>
int setup_impl(rlobpcg_plan_s* p, const T* A, int64_t lda, SolveRun& r, double tau_in) {
  cudaStream_t st = p->st;
  const int64_t m = p->m;
  const int n = (int)p->n, b = p->b, k = p->k, d = p->d;
  const int64_t ld = 3 * b;
  T* Tb = (T*)p->Tb;
  T* ATb = (T*)p->ATb;
  T* GTb = (T*)p->GTb;
  double& tau = r.tau;
  double& sigma11 = r.sigma11;
  std::vector<double>& theta0 = r.theta0;
  StopRule& hist = r.hist;
  int& herr = r.herr;
  double& gram_ms = r.gram_ms;
  double& gram_ab_ms = r.gram_ab_ms;
  double& gram_atb_ms = r.gram_atb_ms;
  int& gram_passes = r.gram_passes;
  int& sweeps = r.sweeps;
  int& it = r.it;
  int& stop = r.stop;
  int& matvecs = r.matvecs;
  int& nx = r.nx;
  const double*& theta_s = r.theta_s;
  split::WDigits& wd = r.wd;
  const bool rwd = p->split && !p->csplit;   // BCGS2 writes the W digits of the real split pass
  bool& w_ready = r.w_ready;
  (void)tau; (void)sigma11; (void)theta0; (void)hist; (void)herr; (void)gram_ms; (void)gram_ab_ms;
  (void)gram_atb_ms; (void)gram_passes; (void)sweeps; (void)it; (void)stop; (void)matvecs; (void)nx;
  (void)theta_s; (void)wd; (void)rwd; (void)w_ready; (void)A; (void)lda; (void)Tb; (void)ATb; (void)GTb; (void)m; (void)n;
  (void)k; (void)d; (void)ld; (void)st;
  r = SolveRun{};
  r.tau = tau_in;
  r.launches0 = launch_count();
  RL_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), st));
  RL_CUDA(cudaMemsetAsync(p->info, 0, 2 * sizeof(int), st));
  RL_CUDA(cudaEventRecord(p->ev[0], st));
  if (p->split) {
    // the split of A (constant through the solve) also flags NaN and infinity
    RL_CUDA(cudaEventRecord(p->ev[8], st));
    // complex A: the split of its real view (m x 2n, leading dimension 2 lda)
    const int64_t f = p->csplit ? 2 : 1;
    RL_TRY(split_prepare((const double*)A, m, f * n, f * lda, p->sprep, p->sprep_bytes, p->err, st));
    RL_CUDA(cudaEventRecord(p->ev[9], st));
  } else {
    RL_TRY(nonfinite_scan_launch<T>(A, m, n, lda, p->err, st));
  }
  RL_CUDA(cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));

  // squared column norms of A for the diagonal preconditioner (one pass over A)
  if (p->opts.precond == RLOBPCG_PRECOND_DIAG)
    RL_TRY(colnorm2_launch<T>(A, m, n, lda, (double*)p->cnpart, (double*)p->cn2, st));

  // Sketch and factorise (the first steps of Alg. 2)
  // the refined form keeps SA in FP64; its QR input is rounded to FP32 inside the factor step
  const bool refine = p->opts.sketch_prec == RLOBPCG_SKETCH_F32_REFINE;
  RL_TRY(sketch_dispatch(A, m, n, lda, p->dtype, d, p->opts.zeta, p->opts.seed,
                         refine ? RLOBPCG_SKETCH_F64 : p->opts.sketch_prec, p->SA, st));
  RL_CUDA(cudaEventRecord(p->ev[1], st));
  const bool exact = p->opts.exact_sketch_svd != 0;
  if constexpr (std::is_same<S, T>::value) {
    if (refine)
      RL_TRY(factor_refine_impl<S>((S*)p->SA, d, n, (S*)p->R_c, (S*)p->R_r, p->sk_sigma, (S*)p->Vt, (S*)p->Rinv_r,
                                   (S*)p->Rinv_c, p->fwork, p->fwork_bytes, st, &sweeps, exact, p->err));
  }
  if (!refine)
    RL_TRY(factor_impl<S>((S*)p->SA, d, n, (S*)p->R_c, (S*)p->R_r, p->sk_sigma, (S*)p->Vt, (S*)p->Rinv_r,
                          (S*)p->Rinv_c, p->fwork, p->fwork_bytes, st, &sweeps, exact, p->err));
  if (exact) {
    RL_CUDA(cudaMemcpyAsync(&sigma11, p->sk_sigma, sizeof(double), cudaMemcpyDeviceToHost, st));
    // Sketch-and-solve start V~(:, n-b+1:n) (Alg. 2)
    RL_TRY((take_start_launch<S, T>((const S*)p->Vt, n, b, Tb, ld, st)));
  } else {
    // Only the two parts of SVD(SA) = SVD(R) the method uses. Sigma~(1,1): block power iteration
    // Z <- Orth(R^H R Z), then the largest singular value of R Z by TSQR + Jacobi.
    T* Z = (T*)p->Zb;
    T* Y = (T*)p->Yb;
    const int qt = std::min(n, std::min(8, p->qmax));
    RL_TRY(fill_random_launch<T>(Z, n, qt, qt, p->opts.seed ^ 0x243F6A8885A308D3ull, st));
    for (int it = 0; it < 8; ++it) {
      RL_TRY((trimul_launch<T, S>((const S*)p->R_r, n, Z, qt, qt, Y, qt, 0, 0, st)));
      RL_TRY((trimul_launch<T, S>((const S*)p->R_c, n, Y, qt, qt, Z, qt, 1, 1, st)));
      RL_TRY(bcgs2_orth_launch<T>(Z, n, qt, qt, 0, 0, (T*)p->E, 0, st, nullptr, p->err, nullptr, p->coop, p->coop_bytes, 0));
    }
    RL_TRY((trimul_launch<T, S>((const S*)p->R_r, n, Z, qt, qt, Y, qt, 0, 0, st)));
    RL_TRY(tsqr_impl<T>(Y, n, qt, qt, (T*)p->Rt, p->twork, p->twork_bytes, st));
    RL_TRY(rr_small_launch<T>((const T*)p->Rt, qt, qt, p->theta, (T*)p->K, p->K_cap, p->info, st));
    RL_CUDA(cudaMemcpyAsync(&sigma11, p->theta, sizeof(double), cudaMemcpyDeviceToHost, st));
    // Start block V~(:, n-b+1:n): block inverse iteration Z <- Orth((R^H R)^{-1} Z) with the
    // oversampled block q = min(n, 2b + 4), then Rayleigh-Ritz on R Z (its b smallest).
    const int q = p->qmax;
    RL_TRY(fill_random_launch<T>(Z, n, q, q, p->opts.seed ^ 0x13198A2E03707344ull, st));
    for (int it = 0; it < 3; ++it) {
      RL_TRY((trimul_launch<T, S>((const S*)p->Rinv_c, n, Z, q, q, Y, q, 1, 1, st)));
      RL_TRY((trimul_launch<T, S>((const S*)p->Rinv_r, n, Y, q, q, Z, q, 0, 0, st)));
      RL_TRY(bcgs2_orth_launch<T>(Z, n, q, q, 0, 0, (T*)p->E, 0, st, nullptr, p->err, nullptr, p->coop, p->coop_bytes, 0));
    }
    RL_TRY((trimul_launch<T, S>((const S*)p->R_r, n, Z, q, q, Y, q, 0, 0, st)));
    RL_TRY(tsqr_impl<T>(Y, n, q, q, (T*)p->Rt, p->twork, p->twork_bytes, st));
    RL_TRY(rr_small_launch<T>((const T*)p->Rt, q, b, p->theta, (T*)p->K, p->K_cap, p->info, st));
    RL_TRY(small_gemm_launch<T>(Z, q, q, (const T*)p->K, 2 * b, b, Tb, ld, n, st));
  }
  RL_CUDA(cudaStreamSynchronize(st));
  if (herr & DEV_ERR_NONFINITE) return RLOBPCG_ERR_NONFINITE;

  // Sketch-and-solve start and the initial Rayleigh-Ritz step (Alg. 2)
  if (rwd) wd = split_w_digits(p->swork, m, n, b);
  RL_TRY(bcgs2_orth_launch<T>(Tb, n, b, ld, 0, 0, (T*)p->E, 0, st, rwd ? &wd : nullptr, p->err, &w_ready,
                              p->coop, p->coop_bytes, 0));
  RL_TRY(gram_pass<T>(p, A, lda, Tb, ATb, GTb, 0, nullptr, w_ready));
  RL_TRY(tsqr_impl<T>(ATb, m, b, ld, (T*)p->Rt, p->twork, p->twork_bytes, st));
  RL_TRY(rr_small_launch<T>((const T*)p->Rt, b, b, p->theta, (T*)p->K, p->K_cap, p->info, st));
  RL_TRY(update_launch<T>(Tb, n, ATb, m, GTb, ld, b, b, (const T*)p->K, st));
  RL_TRY((residual_launch<T>(Tb, GTb, n, b, ld, p->theta, (T*)p->Res, p->res_norm, (T*)p->Rs, p->err, st)));
  RL_CUDA(cudaEventRecord(p->ev[2], st));

  theta0.assign(b, 0.0);
  {
    std::vector<double> hr(b);
    RL_CUDA(cudaMemcpyAsync(hr.data(), p->res_norm, b * sizeof(double), cudaMemcpyDeviceToHost, st));
    RL_CUDA(cudaMemcpyAsync(theta0.data(), p->theta, b * sizeof(double), cudaMemcpyDeviceToHost, st));
    RL_CUDA(cudaStreamSynchronize(st));
    hist.r.push_back(hr);
    hist.th.push_back(std::vector<double>(b, std::numeric_limits<double>::infinity()));
  }

  return RLOBPCG_OK;
}

template <class T, class S>
int loop_impl(rlobpcg_plan_s* p, const T* A, int64_t lda, SolveRun& r) {
  cudaStream_t st = p->st;
  const int64_t m = p->m;
  const int n = (int)p->n, b = p->b, k = p->k, d = p->d;
  const int64_t ld = 3 * b;
  T* Tb = (T*)p->Tb;
  T* ATb = (T*)p->ATb;
  T* GTb = (T*)p->GTb;
  double& tau = r.tau;
  double& sigma11 = r.sigma11;
  std::vector<double>& theta0 = r.theta0;
  StopRule& hist = r.hist;
  int& herr = r.herr;
  double& gram_ms = r.gram_ms;
  double& gram_ab_ms = r.gram_ab_ms;
  double& gram_atb_ms = r.gram_atb_ms;
  int& gram_passes = r.gram_passes;
  int& sweeps = r.sweeps;
  int& it = r.it;
  int& stop = r.stop;
  int& matvecs = r.matvecs;
  int& nx = r.nx;
  const double*& theta_s = r.theta_s;
  split::WDigits& wd = r.wd;
  const bool rwd = p->split && !p->csplit;   // BCGS2 writes the W digits of the real split pass
  bool& w_ready = r.w_ready;
  (void)tau; (void)sigma11; (void)theta0; (void)hist; (void)herr; (void)gram_ms; (void)gram_ab_ms;
  (void)gram_atb_ms; (void)gram_passes; (void)sweeps; (void)it; (void)stop; (void)matvecs; (void)nx;
  (void)theta_s; (void)wd; (void)rwd; (void)w_ready; (void)A; (void)lda; (void)Tb; (void)ATb; (void)GTb; (void)m; (void)n;
  (void)k; (void)d; (void)ld; (void)st;
  const int fixed = p->opts.fixed_iters;
  const int max_iter = fixed > 0 ? fixed : p->opts.max_iter;
  const bool stag = p->opts.use_stagnation != 0;
  const int check_every = std::max(1, p->opts.check_every);
  const int refresh = p->opts.residual_refresh_every;
  nx = 0; it = 0; stop = fixed > 0 ? RLOBPCG_STOP_FIXED : RLOBPCG_STOP_MAX_ITER;
  matvecs = b;
  theta_s = p->theta;
  int drained = 0;   // iterations whose history and timings the host has read
  // the Gram pass of one iteration: e[0] -> e[2] on the FP64 path; on the split path the first
  // product e[0] -> e[1] and the second e[3] -> e[2] (the TSQR level runs between them)
  auto gram_time = [&](cudaEvent_t* e) -> int {
    float gms = 0;
    ++gram_passes;
    if (!p->split) {
      RL_CUDA(cudaEventElapsedTime(&gms, e[0], e[2]));
      gram_ms += gms;
      return RLOBPCG_OK;
    }
    RL_CUDA(cudaEventElapsedTime(&gms, e[0], e[1]));
    gram_ab_ms += gms;
    gram_ms += gms;
    RL_CUDA(cudaEventElapsedTime(&gms, e[3], e[2]));
    gram_atb_ms += gms;
    gram_ms += gms;
    return RLOBPCG_OK;
  };
  auto drain = [&](int upto) -> int {
    for (int t = drained; t < upto; ++t) {
      const double* slot = p->hist_h + (size_t)(t + 1) * 2 * b;
      hist.r.emplace_back(slot, slot + b);
      hist.th.emplace_back(slot + b, slot + 2 * b);
      RL_TRY(gram_time(&p->gev[(size_t)(t % kRing) * 4]));
    }
    drained = upto;
    return RLOBPCG_OK;
  };
  // Locking (Sec. 2.3): the active columns sit at [0, a) (V), [a, 2a) (W), [2a, 3a) (X) of the
  // state (row-major, ld 3b); locked columns move to VL / AVL, keep their Ritz value and residual
  // norm (frozen in the history, which stays indexed by the original column slot), and W is
  // made orthogonal to them as well. Without locking a = b throughout.
  const bool locking = p->opts.locking != 0;
  int a = b, nl = 0;
  std::vector<int> slot_of(b), lslot;
  for (int j = 0; j < b; ++j) slot_of[j] = j;
  std::vector<double> th_cur(b, 0.0), r_cur = hist.r[0], thL, rL;
  for (int j = 0; j < b; ++j) th_cur[j] = theta0[j];
  T* VL = (T*)p->VL;
  T* AVL = (T*)p->AVL;
  for (int i = 0; i < max_iter; ++i) {
    // W = P (P^* R_i), then BCGS2 against [V X] (and the locked columns) and Orth
    if (p->opts.precond == RLOBPCG_PRECOND_SKETCH)
      RL_TRY((precond_launch<T, S>((const S*)p->Rinv_r, (const S*)p->Rinv_c, n, a, (const T*)p->Rs, (T*)p->Y, Tb, ld,
                                   a, st)));
    else   // W = D^2 Rs with D = diag(||A(:, i)||^{-1}), or W = Rs
      RL_TRY(scale_rows_launch<T>((const T*)p->Rs, n, a, p->opts.precond == RLOBPCG_PRECOND_DIAG ? (const double*)p->cn2
                                                                                                  : nullptr,
                                  Tb, ld, a, st));
    RL_TRY(bcgs2_orth_launch<T>(Tb, n, a, ld, a, nx, (T*)p->E, 2, st, rwd ? &wd : nullptr, p->err, &w_ready,
                                p->coop, p->coop_bytes, p->opts.orth_mode, VL, nl, b));
    const int c = 2 * a + nx;
    cudaEvent_t* e = &p->gev[(size_t)(i % kRing) * 4];
    RL_CUDA(cudaEventRecord(e[0], st));
    if (p->split) {
      // A W, then the TSQR level of A_T = [A_V A_W A_X] over all SMs. The Rayleigh-Ritz step
      // needs only A_T, so the TSQR merges and the SVD of R_T (chains of small single-CTA
      // kernels) run on st2 while A^H (A W) runs on st on all but the SMs they need: a split
      // kernel's CTA fills its SM's register file on two sub-partitions, so nothing else is ever
      // placed beside it, and reserving the SMs is what lets the two run at the same time.
      RL_TRY(gram_pass<T>(p, A, lda, Tb + a, ATb + a, GTb + a, 0, e[1], w_ready, a, split::SPLIT_FIRST_ONLY));
      RL_TRY(tsqr_split_impl<T>(ATb, m, c, ld, (T*)p->Rt, p->twork, p->twork_bytes, st, p->st2, p->ev_lvl));
      RL_TRY(rr_small_launch<T>((const T*)p->Rt, c, a, p->theta, (T*)p->K, p->K_cap, p->info, p->st2));
      RL_CUDA(cudaEventRecord(p->ev_rr, p->st2));
      // SMs left to the side chain: one per CTA of the first merge level, all of which launch at
      // once (with fewer, they take SMs that the second product then waits for). A function of
      // the shape only, so that the order of the partial sums, and the results, do not depend on
      // timing.
      const int reserve = std::max(1, tsqr_merge1_ctas(m, c, sizeof(T)));
      RL_CUDA(cudaEventRecord(e[3], st));
      RL_TRY(gram_pass<T>(p, A, lda, Tb + a, ATb + a, GTb + a, 0, nullptr, w_ready, a,
                          split::SPLIT_SECOND_ONLY | split::split_reserve_flag(reserve)));
      RL_CUDA(cudaEventRecord(e[2], st));
      RL_CUDA(cudaStreamWaitEvent(st, p->ev_rr, 0));
    } else {
      RL_TRY(gram_pass<T>(p, A, lda, Tb + a, ATb + a, GTb + a, 0, nullptr, w_ready, a));
      RL_CUDA(cudaEventRecord(e[2], st));
      // Rayleigh-Ritz by SVD of A_T (TSQR + Jacobi of R_T)
      RL_TRY(tsqr_impl<T>(ATb, m, c, ld, (T*)p->Rt, p->twork, p->twork_bytes, st));
      RL_TRY(rr_small_launch<T>((const T*)p->Rt, c, a, p->theta, (T*)p->K, p->K_cap, p->info, st));
    }
    matvecs += a;
    theta_s = p->theta + (c - a);
    RL_TRY(update_launch<T>(Tb, n, ATb, m, GTb, ld, c, a, (const T*)p->K, st));
    if (refresh > 0 && (i + 1) % refresh == 0) {
      RL_TRY(gram_pass<T>(p, A, lda, nullptr, ATb, GTb, 1, nullptr, false, a));
      matvecs += a;
    }
    RL_TRY((residual_launch<T>(Tb, GTb, n, a, ld, theta_s, (T*)p->Res, p->res_norm, (T*)p->Rs, p->err, st)));
    double* slot = p->hist_h + (size_t)(i + 1) * 2 * b;
    RL_CUDA(cudaMemcpyAsync(slot, p->res_norm, a * sizeof(double), cudaMemcpyDeviceToHost, st));
    RL_CUDA(cudaMemcpyAsync(slot + b, theta_s, a * sizeof(double), cudaMemcpyDeviceToHost, st));
    it = i + 1;
    nx = a;
    const bool check = fixed <= 0 && i % check_every == 0;
    if (!locking) {
      if (check || i + 1 == max_iter || i + 1 - drained >= kRing - 1) {
        RL_CUDA(cudaStreamSynchronize(st));
        RL_TRY(drain(i + 1));
        if (check && hist.check(i, sigma11, tau, stag)) {
          stop = RLOBPCG_STOP_CONVERGED;
          break;
        }
      }
      continue;
    }
    // locking: every iteration, the history row in slot order (locked slots frozen), then the
    // stop rule and the columns that met the tolerance
    RL_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < a; ++q) {
      r_cur[slot_of[q]] = slot[q];
      th_cur[slot_of[q]] = slot[b + q];
    }
    hist.r.push_back(r_cur);
    hist.th.push_back(th_cur);
    RL_TRY(gram_time(e));
    drained = i + 1;
    if (check && hist.check(i, sigma11, tau, stag)) {
      stop = RLOBPCG_STOP_CONVERGED;
      break;
    }
    std::vector<int> keep, lock;
    for (int q = 0; q < a; ++q) (slot[q] <= sigma11 * sigma11 * tau ? lock : keep).push_back(q);
    if (lock.empty()) continue;
    for (int q : lock) {
      RL_TRY(copy_cols_launch<T>(Tb, ld, q, VL, b, nl, n, 1, st));
      RL_TRY(copy_cols_launch<T>(ATb, ld, q, AVL, b, nl, m, 1, st));
      thL.push_back(slot[b + q]);
      rL.push_back(slot[q]);
      lslot.push_back(slot_of[q]);
      ++nl;
    }
    const int an = (int)keep.size();
    {
      std::vector<int> src, dst;
      for (int t = 0; t < an; ++t) {
        src.push_back(keep[t]);
        dst.push_back(t);
        src.push_back(2 * a + keep[t]);
        dst.push_back(2 * an + t);
      }
      RL_TRY(gather_cols_launch<T>(Tb, n, ld, src.data(), dst.data(), (int)src.size(), st));
      RL_TRY(gather_cols_launch<T>(ATb, m, ld, src.data(), dst.data(), (int)src.size(), st));
      RL_TRY(gather_cols_launch<T>(GTb, n, ld, src.data(), dst.data(), (int)src.size(), st));
    }
    std::vector<int> so(an);
    std::vector<double> thk(an);
    for (int t = 0; t < an; ++t) {
      so[t] = slot_of[keep[t]];
      thk[t] = slot[b + keep[t]];
    }
    slot_of = so;
    a = an;
    nx = a;
    if (a == 0) {   // every column locked: the solve ends (also in fixed-iteration mode)
      if (fixed <= 0) stop = RLOBPCG_STOP_CONVERGED;
      break;
    }
    if (rwd) wd = split_w_digits(p->swork, m, n, a);
    w_ready = false;
    // the residual of the kept columns in the compacted layout (the preconditioner's input)
    RL_CUDA(cudaMemcpyAsync(p->theta, thk.data(), a * sizeof(double), cudaMemcpyHostToDevice, st));
    RL_TRY((residual_launch<T>(Tb, GTb, n, a, ld, p->theta, (T*)p->Res, p->res_norm, (T*)p->Rs, p->err, st)));
    theta_s = p->theta;
    RL_CUDA(cudaStreamSynchronize(st));   // thk lives on the host stack
  }
  if (locking) {
    // outputs in slot-independent order: the active columns, then the locked ones, sorted by
    // descending Ritz value (the order outputs_launch expects)
    std::vector<double> thA(a), rA(a);
    if (a > 0) {
      RL_CUDA(cudaMemcpyAsync(thA.data(), theta_s, a * sizeof(double), cudaMemcpyDeviceToHost, st));
      RL_CUDA(cudaMemcpyAsync(rA.data(), p->res_norm, a * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (nl > 0) {
      RL_TRY(copy_cols_launch<T>(VL, b, 0, Tb, ld, a, n, nl, st));
      RL_TRY(copy_cols_launch<T>(AVL, b, 0, ATb, ld, a, m, nl, st));
    }
    RL_CUDA(cudaStreamSynchronize(st));
    std::vector<double> thAll(thA), rAll(rA);
    thAll.insert(thAll.end(), thL.begin(), thL.end());
    rAll.insert(rAll.end(), rL.begin(), rL.end());
    std::vector<int> perm(b), dst(b);
    for (int j = 0; j < b; ++j) { perm[j] = j; dst[j] = j; }
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return thAll[x] > thAll[y]; });
    std::vector<double> ths(b), rs(b);
    for (int j = 0; j < b; ++j) { ths[j] = thAll[perm[j]]; rs[j] = rAll[perm[j]]; }
    RL_TRY(gather_cols_launch<T>(Tb, n, ld, perm.data(), dst.data(), b, st));
    RL_TRY(gather_cols_launch<T>(ATb, m, ld, perm.data(), dst.data(), b, st));
    RL_CUDA(cudaMemcpyAsync(p->theta, ths.data(), b * sizeof(double), cudaMemcpyHostToDevice, st));
    RL_CUDA(cudaMemcpyAsync(p->res_norm, rs.data(), b * sizeof(double), cudaMemcpyHostToDevice, st));
    RL_CUDA(cudaStreamSynchronize(st));
    theta_s = p->theta;
  }
  return RLOBPCG_OK;
}

template <class T, class S>
int finish_impl(rlobpcg_plan_s* p, const T* A, int64_t lda, SolveRun& r, double* sigma, T* Vout, T* Uout,
                double* resid, rlobpcg_info* info) {
  cudaStream_t st = p->st;
  const int64_t m = p->m;
  const int n = (int)p->n, b = p->b, k = p->k, d = p->d;
  const int64_t ld = 3 * b;
  T* Tb = (T*)p->Tb;
  T* ATb = (T*)p->ATb;
  T* GTb = (T*)p->GTb;
  double& tau = r.tau;
  double& sigma11 = r.sigma11;
  std::vector<double>& theta0 = r.theta0;
  StopRule& hist = r.hist;
  int& herr = r.herr;
  double& gram_ms = r.gram_ms;
  double& gram_ab_ms = r.gram_ab_ms;
  double& gram_atb_ms = r.gram_atb_ms;
  int& gram_passes = r.gram_passes;
  int& sweeps = r.sweeps;
  int& it = r.it;
  int& stop = r.stop;
  int& matvecs = r.matvecs;
  int& nx = r.nx;
  const double*& theta_s = r.theta_s;
  split::WDigits& wd = r.wd;
  const bool rwd = p->split && !p->csplit;   // BCGS2 writes the W digits of the real split pass
  bool& w_ready = r.w_ready;
  (void)tau; (void)sigma11; (void)theta0; (void)hist; (void)herr; (void)gram_ms; (void)gram_ab_ms;
  (void)gram_atb_ms; (void)gram_passes; (void)sweeps; (void)it; (void)stop; (void)matvecs; (void)nx;
  (void)theta_s; (void)wd; (void)rwd; (void)w_ready; (void)A; (void)lda; (void)Tb; (void)ATb; (void)GTb; (void)m; (void)n;
  (void)k; (void)d; (void)ld; (void)st;
  RL_CUDA(cudaEventRecord(p->ev[3], st));
  // keep the history for rlobpcg_history (row 0: the start block's Ritz values)
  p->last_rows = (int)hist.r.size();
  p->last_theta.assign((size_t)p->last_rows * b, 0.0);
  p->last_res.assign((size_t)p->last_rows * b, 0.0);
  for (int t = 0; t < p->last_rows; ++t)
    for (int j = 0; j < b; ++j) {
      p->last_res[(size_t)t * b + j] = hist.r[t][j];
      p->last_theta[(size_t)t * b + j] = t == 0 ? theta0[j] : hist.th[t][j];
    }
  // outputs (ascending sigma): staged in plan scratch, then copied to host or device pointers
  {
    double* sig_stage = p->res_norm + b;   // k doubles after the b norms
    double* res_stage = sig_stage + k;
    T* V_stage = (T*)p->E;                  // n x k fits in the n x b scratch
    T* U_dev = (Uout && is_device_ptr(Uout)) ? Uout : nullptr;
    RL_TRY(outputs_launch<T>(Tb, ATb, n, m, b, k, ld, theta_s, p->res_norm, sig_stage, V_stage, U_dev, res_stage, st));
    RL_CUDA(cudaMemcpyAsync(sigma, sig_stage, k * sizeof(double), cudaMemcpyDefault, st));
    if (resid) RL_CUDA(cudaMemcpyAsync(resid, res_stage, k * sizeof(double), cudaMemcpyDefault, st));
    RL_CUDA(cudaMemcpyAsync(Vout, V_stage, (size_t)n * k * sizeof(T), cudaMemcpyDefault, st));
    if (Uout && !U_dev) {
      // host U: a temporary device array (the only allocation of solve() besides a host A copy)
      T* Ud = nullptr;
      RL_CUDA(cudaMallocAsync((void**)&Ud, (size_t)m * k * sizeof(T), st));
      RL_TRY(outputs_launch<T>(Tb, ATb, n, m, b, k, ld, theta_s, p->res_norm, sig_stage, V_stage, Ud, res_stage, st));
      RL_CUDA(cudaMemcpyAsync(Uout, Ud, (size_t)m * k * sizeof(T), cudaMemcpyDeviceToHost, st));
      RL_CUDA(cudaFreeAsync(Ud, st));
    }
  }
  RL_CUDA(cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  int rr_stats[2] = {0, 0};
  RL_CUDA(cudaMemcpyAsync(rr_stats, p->info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  RL_CUDA(cudaEventRecord(p->ev[4], st));
  RL_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->iters = it;
    info->matvecs = matvecs;
    info->stop_reason = stop;
    info->block = b;
    info->sigma11 = sigma11;
    float ms = 0;
    cudaEventElapsedTime(&ms, p->ev[p->split ? 9 : 0], p->ev[1]); info->ms_sketch = ms;   // split of A excluded
    cudaEventElapsedTime(&ms, p->ev[1], p->ev[2]); info->ms_factor = ms;
    cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]); info->ms_iterate = ms;
    cudaEventElapsedTime(&ms, p->ev[0], p->ev[4]); info->ms_total = ms;
    info->ms_gram = gram_ms;
    info->gram_passes = gram_passes;
    info->kernel_launches = (int)(launch_count() - r.launches0);
    info->jacobi_sweeps = sweeps;
    info->rr_sweeps = rr_stats[0];
    info->rr_calls = rr_stats[1];
    info->ms_gram_ab = gram_ab_ms;
    info->ms_gram_atb = gram_atb_ms;
    info->ms_split_a = 0;
    if (p->split) {
      cudaEventElapsedTime(&ms, p->ev[8], p->ev[9]);
      info->ms_split_a = ms;
    }
  }
  if (dev_err_status(herr) != RLOBPCG_OK) return dev_err_status(herr);
  return stop == RLOBPCG_STOP_MAX_ITER ? RLOBPCG_NOT_CONVERGED : RLOBPCG_OK;
}

template <class T, class S>
int solve_impl(rlobpcg_plan_s* p, const T* A, int64_t lda, double tau, double* sigma, T* Vout, T* Uout,
               double* resid, rlobpcg_info* info) {
  SolveRun r;
  RL_TRY((setup_impl<T, S>(p, A, lda, r, tau)));
  RL_TRY((loop_impl<T, S>(p, A, lda, r)));
  return finish_impl<T, S>(p, A, lda, r, sigma, Vout, Uout, resid, info);
}

}  // namespace

extern "C" int rlobpcg_default_opts(rlobpcg_opts* o) {
  if (!o) return RLOBPCG_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->seed = 0;
  o->d = 0;
  o->zeta = 8;
  o->block = 0;
  o->max_iter = 0;
  o->check_every = 0;
  o->use_stagnation = 1;
  o->sketch_prec = RLOBPCG_SKETCH_F64;
  o->fixed_iters = 0;
  o->residual_refresh_every = 0;
  o->gram_split = 1;
  o->tau = -1.0;
  o->orth_mode = RLOBPCG_ORTH_HOUSEHOLDER;
  o->locking = 0;
  o->precond = RLOBPCG_PRECOND_SKETCH;
  return RLOBPCG_OK;
}

namespace {

// Validate the plan arguments and fill the resolved options; returns 0 or INVALID_ARG.
int resolve_plan_args(int64_t m, int64_t n, int k, int dtype, const rlobpcg_opts* opts, rlobpcg_opts* o, int* b_out,
                      int64_t* d_out) {
  if (opts) *o = *opts; else rlobpcg_default_opts(o);
  if (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128) return RLOBPCG_ERR_INVALID_ARG;
  const int b = o->block > 0 ? o->block : k;
  const int64_t d = o->d > 0 ? o->d : 4 * n;
  if (k < 1 || b < k || 3 * (int64_t)b > n || n > m || o->zeta < 1 || d < n || d < o->zeta || b > 21 ||
      n > (1 << 20) || (o->sketch_prec != RLOBPCG_SKETCH_F64 && o->sketch_prec != RLOBPCG_SKETCH_F32 &&
                        o->sketch_prec != RLOBPCG_SKETCH_F32_REFINE) ||
      (o->orth_mode != RLOBPCG_ORTH_HOUSEHOLDER && o->orth_mode != RLOBPCG_ORTH_SVQB) ||
      (o->locking != 0 && o->locking != 1) ||
      (o->precond != RLOBPCG_PRECOND_SKETCH && o->precond != RLOBPCG_PRECOND_DIAG &&
       o->precond != RLOBPCG_PRECOND_NONE)) {
    set_last_error("invalid plan arguments (need 1 <= k <= b <= 21, 3b <= n <= m, n <= d, zeta <= d, a known sketch precision and orth_mode, locking 0 or 1)", __FILE__, __LINE__);
    return RLOBPCG_ERR_INVALID_ARG;
  }
  if (o->max_iter <= 0) o->max_iter = (b == 1) ? 200 : 100;
  if (o->check_every <= 0) o->check_every = o->use_stagnation ? 5 : 1;
  if (!(o->tau >= 0)) o->tau = 2.0 * sqrt((double)n) * ldexp(1.0, -52);
  *b_out = b;
  *d_out = d;
  return RLOBPCG_OK;
}

// real FP64 with b <= 24; complex128 (its real view, block width 2b) with b <= 12
bool uses_split(const rlobpcg_opts& o, int dtype, int b) {
  return o.gram_split && ((dtype == RLOBPCG_F64 && b <= 24) || (dtype == RLOBPCG_C128 && 2 * b <= 24));
}

// Every device buffer of a plan, in one place: with p == nullptr only the bytes are summed.
struct PlanAlloc {
  rlobpcg_plan_s* p;
  size_t total = 0;
  int operator()(void** slot, size_t bytes) {
    bytes = (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
    if (!p) { total += bytes; return RLOBPCG_OK; }
    return dev_alloc(p, slot, bytes);
  }
};

int plan_buffers(PlanAlloc& A_, rlobpcg_plan_s* p, int64_t m, int64_t n, int b, int64_t d, int k, int dtype,
                 const rlobpcg_opts& o, size_t* K_cap_out, int* qmax_out, size_t* gwork, size_t* twork,
                 size_t* fwork) {
  const bool cplx = dtype == RLOBPCG_C128;
  const bool f32 = o.sketch_prec == RLOBPCG_SKETCH_F32;
  const size_t esz = cplx ? 16 : 8;
  const size_t ssz = (cplx ? 2 : 1) * (f32 ? 4 : 8);
  const int64_t ld = 3 * b;
  void* dummy = nullptr;
  auto slot = [&](void* rlobpcg_plan_s::*member) -> void** { return p ? &(p->*member) : &dummy; };
  int rc;
#define RL_B(member, bytes) do { rc = A_(slot(&rlobpcg_plan_s::member), (bytes)); if (rc) return rc; } while (0)
  RL_B(SA, (size_t)d * n * ssz);
  RL_B(Vt, (size_t)n * n * ssz);
  RL_B(Rinv_r, (size_t)n * n * ssz);
  RL_B(Rinv_c, (size_t)n * n * ssz);
  RL_B(R_c, (size_t)n * n * ssz);
  RL_B(R_r, (size_t)n * n * ssz);
  const int qmax = (int)std::min<int64_t>(n, 2 * b + 4);
  const int64_t cmax = std::max<int64_t>(ld, qmax);
  RL_B(Zb, (size_t)n * qmax * esz);
  RL_B(Yb, (size_t)n * qmax * esz);
  *fwork = o.sketch_prec == RLOBPCG_SKETCH_F32_REFINE ? refine_workspace_bytes(d, n, dtype)
                                                     : factor_workspace_bytes(d, n, ssz);
  RL_B(fwork, *fwork);
  RL_B(Tb, (size_t)n * ld * esz);
  RL_B(ATb, (size_t)m * ld * esz);
  RL_B(GTb, (size_t)n * ld * esz);
  RL_B(E, (size_t)n * cmax * esz);
  RL_B(Res, (size_t)n * b * esz);
  RL_B(Rs, (size_t)n * b * esz);
  RL_B(Y, (size_t)std::max<int64_t>(n * b, 64) * esz);
  RL_B(Rt, (size_t)cmax * cmax * esz);
  // coefficient blocks c x 2b of every Rayleigh-Ritz step, including the qt x 2qt block (qt <= 8)
  // of the Sigma~(1,1) estimate
  *K_cap_out = (size_t)cmax * 2 * std::max<int64_t>(b, 8);
  RL_B(K, *K_cap_out * esz);
  {
    void** sl = p ? (void**)&p->theta : &dummy;
    rc = A_(sl, (size_t)cmax * sizeof(double)); if (rc) return rc;
    sl = p ? (void**)&p->sk_sigma : &dummy;
    rc = A_(sl, (size_t)n * sizeof(double)); if (rc) return rc;
    sl = p ? (void**)&p->res_norm : &dummy;
    rc = A_(sl, (size_t)(b + 2 * k + 8) * sizeof(double)); if (rc) return rc;
    sl = p ? (void**)&p->err : &dummy;
    rc = A_(sl, 64); if (rc) return rc;
    sl = p ? (void**)&p->info : &dummy;
    rc = A_(sl, 64); if (rc) return rc;
  }
  if (uses_split(o, dtype, b)) {
    const bool cx = dtype == RLOBPCG_C128;
    const size_t sp = split_prep_bytes(m, cx ? 2 * n : n);
    const size_t sw = cx ? split_work_bytes_c128(m, n, b) : split_work_bytes(m, n, b);
    if (sp == 0 || sw == 0) return RLOBPCG_ERR_INVALID_ARG;
    RL_B(sprep, sp);
    RL_B(swork, sw);
    if (p) { p->split = true; p->csplit = cx; p->sprep_bytes = sp; p->swork_bytes = sw; }
    *gwork = 0;
  } else {
    *gwork = gram_workspace_bytes(m, n, b, dtype);
    if (*gwork == 0) {
      set_last_error("Gram kernel: n*b too large for on-chip accumulation", __FILE__, __LINE__);
      return RLOBPCG_ERR_UNSUPPORTED;
    }
    RL_B(gwork, *gwork);
  }
  *twork = std::max(tsqr_workspace_bytes(m, (int)ld, esz), tsqr_workspace_bytes(n, qmax, esz));
  RL_B(twork, *twork);
  if (o.precond == RLOBPCG_PRECOND_DIAG) {
    RL_B(cn2, (size_t)n * sizeof(double));
    RL_B(cnpart, (size_t)colnorm_parts(m) * n * sizeof(double));
  }
  if (o.locking) {
    RL_B(VL, (size_t)n * b * esz);
    RL_B(AVL, (size_t)m * b * esz);
  }
  {
    const size_t cb = bcgs2_coop_bytes(n, (int)std::max<int64_t>(ld, qmax) + b, std::max(b, qmax), esz);
    RL_B(coop, cb);
    if (p) p->coop_bytes = cb;
  }
#undef RL_B
  *qmax_out = qmax;
  return RLOBPCG_OK;
}

}  // namespace

extern "C" size_t rlobpcg_plan_workspace_size(int64_t m, int64_t n, int k, int dtype, const rlobpcg_opts* opts) {
  rlobpcg_opts o;
  int b = 0;
  int64_t d = 0;
  if (resolve_plan_args(m, n, k, dtype, opts, &o, &b, &d)) return 0;
  PlanAlloc dry{nullptr};
  size_t kc, gw, tw, fw;
  int qm;
  if (plan_buffers(dry, nullptr, m, n, b, d, k, dtype, o, &kc, &qm, &gw, &tw, &fw)) return 0;
  return dry.total;
}

extern "C" int rlobpcg_plan(rlobpcg_plan_t* out, int64_t m, int64_t n, int k, int dtype, const rlobpcg_opts* opts,
                            void* stream) {
  if (!out) return RLOBPCG_ERR_INVALID_ARG;
  *out = nullptr;
  rlobpcg_opts o;
  int b = 0;
  int64_t d = 0;
  int rc = resolve_plan_args(m, n, k, dtype, opts, &o, &b, &d);
  if (rc) return rc;
  auto* p = new rlobpcg_plan_s();
  p->m = m; p->n = n; p->k = k; p->b = b; p->d = (int)d; p->dtype = dtype;
  p->st = (cudaStream_t)stream;
  p->opts = o;
  const bool cplx = dtype == RLOBPCG_C128;
  p->esz = cplx ? 16 : 8;
  p->ssz = (cplx ? 2 : 1) * (o.sketch_prec == RLOBPCG_SKETCH_F32 ? 4 : 8);
  PlanAlloc alloc{p};
  rc = plan_buffers(alloc, p, m, n, b, d, k, dtype, o, &p->K_cap, &p->qmax, &p->gwork_bytes, &p->twork_bytes,
                    &p->fwork_bytes);
  if (rc) { free_plan(p); delete p; return rc; }
  for (auto& e : p->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) { free_plan(p); delete p; return RLOBPCG_ERR_CUDA; }
  }
  p->gev.assign((size_t)kRing * 4, nullptr);
  for (auto& e : p->gev) {
    if (cudaEventCreate(&e) != cudaSuccess) { free_plan(p); delete p; return RLOBPCG_ERR_CUDA; }
  }
  if (p->split) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&p->st2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_lvl, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_rr, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("plan: side stream of the split Gram path", __FILE__, __LINE__);
      free_plan(p);
      delete p;
      return RLOBPCG_ERR_CUDA;
    }
  }
  {
    const int iters = std::max(o.max_iter, o.fixed_iters);
    p->hist_slots = iters + 2;
    if (cudaMallocHost((void**)&p->hist_h, (size_t)p->hist_slots * 2 * b * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("plan: pinned host buffer for the stop-rule history", __FILE__, __LINE__);
      free_plan(p);
      delete p;
      return RLOBPCG_ERR_CUDA;
    }
  }
  *out = p;
  return RLOBPCG_OK;
}

static int async_in_flight(rlobpcg_plan_t p) {
  rl::set_last_error("the plan has an asynchronous solve in flight: call rlobpcg_solve_wait first", __FILE__, __LINE__);
  (void)p;
  return RLOBPCG_ERR_INVALID_ARG;
}

static int solve_entry(rlobpcg_plan_t p, const void* A, int64_t lda, double tol, double* sigma, void* V, void* U,
                       double* resid, rlobpcg_info* info);

extern "C" int rlobpcg_solve(rlobpcg_plan_t p, const void* A, int64_t lda, double tol, double* sigma, void* V, void* U,
                             double* resid, rlobpcg_info* info) {
  if (p && p->async_busy) return async_in_flight(p);
  return solve_entry(p, A, lda, tol, sigma, V, U, resid, info);
}

extern "C" int rlobpcg_solve_async(rlobpcg_plan_t p, const void* A, int64_t lda, double tol, double* sigma, void* V,
                                   void* U, double* resid, rlobpcg_info* info) {
  if (!p || !A || !sigma || !V || lda < p->n) return RLOBPCG_ERR_INVALID_ARG;
  if (p->async_busy) return async_in_flight(p);
  int dev = 0;
  RL_CUDA(cudaGetDevice(&dev));
  p->async_rc = 0;
  p->async_err.clear();
  try {
    p->async_th = std::thread([=]() {
      // the solve's launches go to the plan's stream from this thread, on the caller's device
      int rc = cudaSetDevice(dev) == cudaSuccess ? RLOBPCG_OK : RLOBPCG_ERR_CUDA;
      if (rc == RLOBPCG_OK) rc = solve_entry(p, A, lda, tol, sigma, V, U, resid, info);
      else rl::set_last_error("rlobpcg_solve_async: cudaSetDevice failed on the solve thread", __FILE__, __LINE__);
      p->async_rc = rc;
      if (rc < 0) p->async_err = rlobpcg_last_error();
    });
  } catch (...) {
    rl::set_last_error("rlobpcg_solve_async: could not start the solve thread", __FILE__, __LINE__);
    return RLOBPCG_ERR_OOM;
  }
  p->async_busy = true;
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_solve_wait(rlobpcg_plan_t p) {
  if (!p || !p->async_busy) return RLOBPCG_ERR_INVALID_ARG;
  p->async_th.join();
  p->async_busy = false;
  if (p->async_rc < 0) rl::set_last_error_text(p->async_err.c_str());
  return p->async_rc;
}

static int solve_entry(rlobpcg_plan_t p, const void* A, int64_t lda, double tol, double* sigma, void* V, void* U,
                       double* resid, rlobpcg_info* info) {
  if (!p || !A || !sigma || !V || lda < p->n) return RLOBPCG_ERR_INVALID_ARG;
  const double tau = tol >= 0 ? tol : p->opts.tau;
  const void* Ause = A;
  int64_t ldause = lda;
  cudaEvent_t h0 = nullptr, h1 = nullptr;
  const bool host_A = !is_device_ptr(A);
  if (host_A) {
    // host input: copy into a plan-owned device buffer (compact, lda = n)
    const size_t bytes = (size_t)p->m * p->n * p->esz;
    if (p->A_dev_bytes < bytes) {
      if (p->A_dev) cudaFreeAsync(p->A_dev, p->st);
      p->A_dev = nullptr;
      p->A_dev_bytes = 0;
      if (cudaMallocAsync(&p->A_dev, bytes, p->st) != cudaSuccess) { cudaGetLastError(); return RLOBPCG_ERR_OOM; }
      p->A_dev_bytes = bytes;
    }
    RL_CUDA(cudaEventCreate(&h0));
    RL_CUDA(cudaEventCreate(&h1));
    RL_CUDA(cudaEventRecord(h0, p->st));
    RL_CUDA(cudaMemcpy2DAsync(p->A_dev, p->n * p->esz, A, lda * p->esz, p->n * p->esz, p->m, cudaMemcpyHostToDevice, p->st));
    Ause = p->A_dev;
    ldause = p->n;
  }
  int rc;
  const bool f32 = p->opts.sketch_prec == RLOBPCG_SKETCH_F32;
  if (p->dtype == RLOBPCG_F64) {
    rc = f32 ? solve_impl<double, float>(p, (const double*)Ause, ldause, tau, sigma, (double*)V, (double*)U, resid, info)
             : solve_impl<double, double>(p, (const double*)Ause, ldause, tau, sigma, (double*)V, (double*)U, resid, info);
  } else {
    rc = f32 ? solve_impl<cd, cf>(p, (const cd*)Ause, ldause, tau, sigma, (cd*)V, (cd*)U, resid, info)
             : solve_impl<cd, cd>(p, (const cd*)Ause, ldause, tau, sigma, (cd*)V, (cd*)U, resid, info);
  }
  if (host_A) {
    cudaEventRecord(h1, p->st);
    cudaEventSynchronize(h1);
    if (info && rc >= 0) { float ms = 0; cudaEventElapsedTime(&ms, h0, h1); info->ms_total = ms; }
    cudaEventDestroy(h0);
    cudaEventDestroy(h1);
  }
  return rc;
}

extern "C" int rlobpcg_plan_destroy(rlobpcg_plan_t p) {
  if (!p) return RLOBPCG_OK;
  if (p->async_busy) {   // a solve still in flight finishes first
    p->async_th.join();
    p->async_busy = false;
  }
  cudaStreamSynchronize(p->st);
  free_plan(p);
  delete p;
  return RLOBPCG_OK;
}

extern "C" size_t rlobpcg_plan_device_bytes(rlobpcg_plan_t p) { return p ? p->bytes : 0; }

extern "C" int rlobpcg_history(rlobpcg_plan_t p, double* theta, double* resnorm, int cap_rows, int* rows, int* block) {
  if (!p || !rows || cap_rows < 0) return RLOBPCG_ERR_INVALID_ARG;
  if (p->async_busy) return async_in_flight(p);
  *rows = p->last_rows;
  if (block) *block = p->b;
  const int n = std::min(cap_rows, p->last_rows);
  if (theta) memcpy(theta, p->last_theta.data(), (size_t)n * p->b * sizeof(double));
  if (resnorm) memcpy(resnorm, p->last_res.data(), (size_t)n * p->b * sizeof(double));
  return RLOBPCG_OK;
}

// =================================================================================================
// Batched solves: many small solves iterate together (Alg. 2 per solve; the iterations of all of
// them run as two persistent kernels per iteration, replayed from a captured CUDA graph). Each
// solve's set-up (sketch, factor, start block, first Rayleigh-Ritz step) and outputs use its own
// plan and stream, exactly as rlobpcg_solve does.
// =================================================================================================
namespace {

struct TileChoice {
  int trows = 0, rt = 0;
};
std::mutex g_tile_mu;
std::map<std::pair<int, int>, TileChoice> g_tile_table;

int n_class(int n) {
  int c = 32;
  while (c < n) c *= 2;
  return c;
}

// Candidate tile shapes for one (n class, b): every (trows, rt) whose shared memory fits.
std::vector<TileChoice> tile_candidates(int nc, int b, size_t static_tile) {
  std::vector<TileChoice> out;
  for (int trows : {256, 512, 1024, 2048})
    for (int rt : {8, 16}) {
      const size_t sm = batch::tile_smem_bytes(nc * b, batch::abuf_need(nc, b, rt), rt);
      if (sm + static_tile <= max_smem_optin()) out.push_back({trows, rt});
    }
  return out;
}

struct DevArena {   // one stream-ordered allocation carved into pieces
  char* base = nullptr;
  size_t used = 0, cap = 0;
  std::vector<std::pair<void**, size_t>> req;
  void want(void** p, size_t bytes) { req.push_back({p, (bytes + 255) & ~(size_t)255}); cap += (bytes + 255) & ~(size_t)255; }
  int alloc(cudaStream_t st) {
    if (cap == 0) cap = 256;
    if (cudaMallocAsync((void**)&base, cap, st) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("batch: device workspace", __FILE__, __LINE__);
      return RLOBPCG_ERR_OOM;
    }
    for (auto& r : req) {
      *r.first = base + used;
      used += r.second;
    }
    return RLOBPCG_OK;
  }
  void release(cudaStream_t st) {
    if (base) cudaFreeAsync(base, st);
    base = nullptr;
  }
};

// The autotuner: times the tile kernel (one full iteration of the Gram, the local factors, the
// reductions and the Rayleigh-Ritz tails) on synthetic solves of the class, for every candidate,
// and keeps the fastest. Results depend on the tile shape (it fixes the summation order), so the
// choice is made once per process and class and then used for every solve of that class.
int tune_class(int nc, int b, cudaStream_t st, TileChoice* out) {
  size_t s_pre = 0, s_tile = 0;
  RL_TRY(batch::static_smem_bytes(&s_pre, &s_tile));
  const std::vector<TileChoice> cand = tile_candidates(nc, b, s_tile);
  if (cand.empty()) {
    set_last_error("batch: no tile shape fits shared memory for this n", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  constexpr int NS = 4;
  const int64_t m = 16384;
  const int n = nc, C = 3 * b;
  const int tmax = (int)((m + 255) / 256), gmax = (tmax + batch::GS - 1) / batch::GS;
  DevArena ar;
  double *A = nullptr, *state = nullptr, *part = nullptr;
  int *cnt = nullptr, *qh = nullptr, *err = nullptr;
  batch::Desc* D = nullptr;
  int2* items = nullptr;
  const size_t per_state = (size_t)n * C * 3 + (size_t)m * C + (size_t)n * b * 2 + 4 * C + (size_t)C * 2 * b + C * C +
                           4 * b + 64;
  const size_t per_part = (size_t)tmax * ((size_t)n * b + C * C) + (size_t)gmax * ((size_t)n * b + C * C);
  ar.want((void**)&A, (size_t)m * n * 8);
  ar.want((void**)&state, NS * per_state * 8);
  ar.want((void**)&part, NS * per_part * 8);
  ar.want((void**)&cnt, (size_t)NS * (2 + gmax) * 4);
  ar.want((void**)&qh, 64);
  ar.want((void**)&err, 64);
  ar.want((void**)&D, NS * sizeof(batch::Desc));
  ar.want((void**)&items, (size_t)NS * tmax * sizeof(int2));
  RL_TRY(ar.alloc(st));
  int rc = RLOBPCG_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<batch::Desc> hd(NS);
  std::vector<int2> hi;
  float best = 1e30f;
  TileChoice pick = cand[0];
  do {
    if ((rc = fill_random_launch<double>(A, m, n, n, 0x9E3779B97F4A7C15ull, st))) break;
    if ((rc = fill_random_launch<double>(state, (int64_t)NS * per_state / 8, 8, 8, 0xD1B54A32D192ED03ull, st))) break;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = RLOBPCG_ERR_CUDA; break; }
    for (const TileChoice& tc : cand) {
      const int nt = (int)((m + tc.trows - 1) / tc.trows), ng = (nt + batch::GS - 1) / batch::GS;
      hi.clear();
      for (int s = 0; s < NS; ++s) {
        double* q = state + (size_t)s * per_state;
        batch::Desc& d = hd[s];
        d = batch::Desc{};
        d.A = A; d.m = m; d.lda = n; d.n = n; d.b = b;
        d.Tb = q; q += (size_t)n * C;
        d.GTb = q; q += (size_t)n * C;
        d.ATb = q; q += (size_t)m * C;
        d.Rs = q; q += (size_t)n * b;
        d.Res = q; q += (size_t)n * b;
        d.res_norm = q; q += C;
        d.theta = q; q += C;
        d.K = q; q += (size_t)C * 2 * b;
        d.Rfin = q; q += (size_t)C * C;
        d.hist = q; q += 4 * b;
        double* pp = part + (size_t)s * per_part;
        d.Gpart = pp; pp += (size_t)tmax * n * b;
        d.Rpart = pp; pp += (size_t)tmax * C * C;
        d.Ggrp = pp; pp += (size_t)gmax * n * b;
        d.Rgrp = pp;
        d.cnt = cnt + (size_t)s * (2 + gmax);
        d.err = err; d.rr_info = err + 2;
        d.ntiles = nt; d.trows = tc.trows; d.rt = tc.rt; d.ngroups = ng; d.nrb = 1;
        d.iter = 0; d.c = 2 * b; d.nx = 0; d.pending = 0; d.done = 0; d.matvecs = b;
        d.max_iter = 1; d.fixed = 1; d.check_every = 1; d.use_stag = 0;
        d.sigma11 = 1.0; d.tau = 0.0;
        for (int t = 0; t < nt; ++t) hi.push_back(make_int2(s, t));
      }
      const int ab = batch::abuf_need(n, b, tc.rt);
      const size_t smem = batch::tile_smem_bytes(n * b, ab, tc.rt);
      if ((rc = batch::prepare(batch::bcgs2_pre_smem(n, b), smem))) break;
      int per_sm = 1;
      if ((rc = batch::tile_blocks_per_sm(smem, &per_sm))) break;
      const int grid = std::max(1, std::min((int)hi.size(), num_sms() * std::max(1, per_sm)));
      float tot = 0;
      for (int rep = 0; rep < 4 && !rc; ++rep) {
        RL_CUDA(cudaMemcpyAsync(D, hd.data(), NS * sizeof(batch::Desc), cudaMemcpyHostToDevice, st));
        RL_CUDA(cudaMemcpyAsync(items, hi.data(), hi.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
        RL_CUDA(cudaMemsetAsync(cnt, 0, (size_t)NS * (2 + gmax) * 4, st));
        RL_CUDA(cudaMemsetAsync(qh, 0, 64, st));
        RL_CUDA(cudaEventRecord(e0, st));
        rc = batch::tile_launch(false, D, items, (int)hi.size(), qh, grid, n * b, ab, smem, st);
        RL_CUDA(cudaEventRecord(e1, st));
        RL_CUDA(cudaStreamSynchronize(st));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;   // the first launch is a warm-up
      }
      if (rc) break;
      if (tot < best) {
        best = tot;
        pick = tc;
      }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ar.release(st);
  cudaStreamSynchronize(st);
  if (rc) return rc;
  *out = pick;
  return RLOBPCG_OK;
}

int tile_choice(int n, int b, cudaStream_t st, TileChoice* out) {
  const auto key = std::make_pair(n_class(n), b);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_table.find(key);
    if (it != g_tile_table.end()) {
      *out = it->second;
      return RLOBPCG_OK;
    }
  }
  TileChoice tc;
  RL_TRY(tune_class(key.first, b, st, &tc));
  std::lock_guard<std::mutex> lk(g_tile_mu);
  *out = g_tile_table.emplace(key, tc).first->second;   // the first choice made for a class stays
  return RLOBPCG_OK;
}

bool batch_eligible(const rlobpcg_plan_s* p, std::string* why) {
  if (p->dtype != RLOBPCG_F64) { *why = "batched solves are real FP64"; return false; }
  if (p->b > batch::BMAX) { *why = "batched solves need b <= 5"; return false; }
  if (p->n > 512) { *why = "batched solves need n <= 512"; return false; }
  if (p->opts.locking || p->opts.orth_mode != RLOBPCG_ORTH_HOUSEHOLDER || p->opts.residual_refresh_every > 0 ||
      p->opts.precond != RLOBPCG_PRECOND_SKETCH) {
    *why = "batched solves run with the sketch preconditioner, without locking, SVQB or residual refresh";
    return false;
  }
  return true;
}

template <class S>
int batch_setup_one(rlobpcg_plan_s* p, const double* A, int64_t lda, SolveRun& r) {
  return setup_impl<double, S>(p, A, lda, r, p->opts.tau);
}
template <class S>
int batch_finish_one(rlobpcg_plan_s* p, const double* A, int64_t lda, SolveRun& r, double* sigma, double* V, double* U,
                     double* resid, rlobpcg_info* info) {
  return finish_impl<double, S>(p, A, lda, r, sigma, V, U, resid, info);
}

}  // namespace

// -------------------------------------------------------------------------------------------------
// The batch engine: one host thread and one stream that iterate every solve handed to it. Solves
// join and leave between graph replays (continuous batching); a solve's device state of the
// batched iterations is allocated when it joins and freed when it leaves.
// -------------------------------------------------------------------------------------------------
namespace rl {

struct BatchSolve {
  rlobpcg_plan_s* p = nullptr;
  const double* A = nullptr;
  int64_t lda = 0;
  SolveRun r;
  TileChoice tc;
  void* mem = nullptr;       // the solve's batched-iteration buffers (one allocation)
  batch::Desc d{};           // host copy of its descriptor
  std::mutex mu;
  std::condition_variable cv;
  bool finished = false;     // the engine has retired it
  int rc = RLOBPCG_OK;
};

struct BatchEngine {
  int device = 0;
  cudaStream_t st = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<BatchSolve*> incoming;
  bool stop = false;
  std::vector<BatchSolve*> active;
  // device arrays of the current membership
  void* dmem = nullptr;
  size_t dmem_bytes = 0;
  batch::Desc* Dd = nullptr;
  int2 *pre_items = nullptr, *tile_items = nullptr;
  int* qh = nullptr;
  batch::Desc* Dh = nullptr;   // pinned copy the graph writes back after every replay
  size_t Dh_cap = 0;
  int npre = 0, ntile = 0;
  int nwmax = 1, abmax = 1, rtmax = 8;
  size_t pre_smem = 0, tile_smem = 0;
  int pre_grid = 1, tile_grid = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool dirty = true;
  int stable = 0;               // replays since the last membership change
  static constexpr int G = 4;   // iterations per replay
  // telemetry (engine thread writes, readers take mu)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  rlobpcg_engine_stats stats{};
  double active_sum = 0;
};

namespace {

size_t batch_solve_bytes(int64_t m, int64_t n, int b, int trows, int* nt_out, int* ng_out) {
  const int C = 3 * b;
  const int nt = (int)((m + trows - 1) / trows), ng = (nt + batch::GS - 1) / batch::GS;
  if (nt_out) *nt_out = nt;
  if (ng_out) *ng_out = ng;
  auto r = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return r((size_t)n * n * 8) * 2 + r((size_t)n * b * 8) + r((size_t)nt * n * b * 8) + r((size_t)nt * C * C * 8) +
         r((size_t)ng * n * b * 8) + r((size_t)ng * C * C * 8) + r((size_t)C * C * 8) + r((size_t)201 * 2 * b * 8) +
         r((size_t)(2 + ng) * 4);
}

void complete(BatchSolve* s, int rc) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->rc = rc;
  s->finished = true;
  s->cv.notify_all();
}

// device state of a joining solve: its buffers, FP64 copies of R^{-1} (row- and column-major), the
// first history row, and its descriptor
int engine_join(BatchEngine* e, BatchSolve* s) {
  rlobpcg_plan_s* p = s->p;
  const int n = (int)p->n, b = p->b, C = 3 * b;
  int nt = 0, ng = 0;
  const int rows = std::max(p->opts.max_iter, p->opts.fixed_iters) + 1;
  if (rows > 201) {
    set_last_error("batched solves run at most 200 iterations", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  const size_t bytes = batch_solve_bytes(p->m, n, b, s->tc.trows, &nt, &ng);
  if (cudaMallocAsync(&s->mem, bytes, e->st) != cudaSuccess) {
    cudaGetLastError();
    s->mem = nullptr;
    set_last_error("batch: solve workspace", __FILE__, __LINE__);
    return RLOBPCG_ERR_OOM;
  }
  char* q = (char*)s->mem;
  auto take = [&](size_t x) { char* r = q; q += (x + 255) & ~(size_t)255; return r; };
  batch::Desc& d = s->d;
  d = batch::Desc{};
  d.Ru = (double*)take((size_t)n * n * 8);
  d.Rl = (double*)take((size_t)n * n * 8);
  d.Y = (double*)take((size_t)n * b * 8);
  d.Gpart = (double*)take((size_t)nt * n * b * 8);
  d.Rpart = (double*)take((size_t)nt * C * C * 8);
  d.Ggrp = (double*)take((size_t)ng * n * b * 8);
  d.Rgrp = (double*)take((size_t)ng * C * C * 8);
  d.Rfin = (double*)take((size_t)C * C * 8);
  d.hist = (double*)take((size_t)201 * 2 * b * 8);
  d.cnt = (int*)take((size_t)(2 + ng) * 4);
  d.A = s->A; d.m = p->m; d.lda = s->lda; d.n = n; d.b = b;
  d.Tb = (double*)p->Tb; d.ATb = (double*)p->ATb; d.GTb = (double*)p->GTb;
  d.Rs = (double*)p->Rs; d.Res = (double*)p->Res; d.res_norm = p->res_norm; d.theta = p->theta;
  d.K = (double*)p->K; d.err = p->err; d.rr_info = p->info;
  d.ntiles = nt; d.trows = s->tc.trows; d.rt = s->tc.rt; d.ngroups = ng; d.nrb = (n + batch::PR - 1) / batch::PR;
  d.iter = 0; d.c = 2 * b; d.nx = 0; d.pending = 0; d.c_prev = 0; d.done = 0; d.matvecs = b;
  d.fixed = p->opts.fixed_iters;
  d.max_iter = d.fixed > 0 ? d.fixed : p->opts.max_iter;
  d.check_every = std::max(1, p->opts.check_every);
  d.use_stag = p->opts.use_stagnation != 0;
  d.sigma11 = s->r.sigma11;
  d.tau = s->r.tau;
  d.stop_reason = d.fixed > 0 ? RLOBPCG_STOP_FIXED : RLOBPCG_STOP_MAX_ITER;
  const bool f32 = p->opts.sketch_prec == RLOBPCG_SKETCH_F32;
  const int64_t nn = p->n * p->n;
  RL_TRY(f32 ? batch::widen_launch<float>((const float*)p->Rinv_r, nn, (double*)d.Ru, e->st)
             : batch::widen_launch<double>((const double*)p->Rinv_r, nn, (double*)d.Ru, e->st));
  RL_TRY(f32 ? batch::widen_launch<float>((const float*)p->Rinv_c, nn, (double*)d.Rl, e->st)
             : batch::widen_launch<double>((const double*)p->Rinv_c, nn, (double*)d.Rl, e->st));
  // (the host history row lives in the solve's run state until the solve is finished)
  RL_CUDA(cudaMemcpyAsync(d.hist, s->r.hist.r[0].data(), b * sizeof(double), cudaMemcpyHostToDevice, e->st));
  RL_CUDA(cudaMemsetAsync(d.cnt, 0, (size_t)(2 + ng) * 4, e->st));
  return RLOBPCG_OK;
}

// device arrays, work lists and the graph for the current membership (descriptors from the host
// copies, which hold every solve's state after the last replay)
int engine_rebuild(BatchEngine* e) {
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->gexec = nullptr;
  e->graph = nullptr;
  const int count = (int)e->active.size();
  std::vector<int2> hpre, htile;
  e->nwmax = 1; e->abmax = 1; e->rtmax = 8; e->pre_smem = 0;
  for (int i = 0; i < count; ++i) {
    const batch::Desc& d = e->active[i]->d;
    for (int rb = 0; rb < d.nrb; ++rb) hpre.push_back(make_int2(i, rb));
    e->nwmax = std::max(e->nwmax, d.n * d.b);
    e->abmax = std::max(e->abmax, batch::abuf_need(d.n, d.b, d.rt));
    e->rtmax = std::max(e->rtmax, d.rt);
    e->pre_smem = std::max(e->pre_smem, batch::bcgs2_pre_smem(d.n, d.b));
  }
  // tile items: the solves with the most work per iteration first, so that their tails overlap
  // the other solves' tiles
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const batch::Desc &a = e->active[x]->d, &b = e->active[y]->d;
    return (double)a.m * a.n * a.b > (double)b.m * b.n * b.b;
  });
  for (int i : order)
    for (int t = 0; t < e->active[i]->d.ntiles; ++t) htile.push_back(make_int2(i, t));
  e->npre = (int)hpre.size();
  e->ntile = (int)htile.size();
  const size_t need = count * sizeof(batch::Desc) + 256 + hpre.size() * sizeof(int2) + 256 +
                      htile.size() * sizeof(int2) + 256 + (3 * BatchEngine::G + 2) * sizeof(int) + 256;
  if (need > e->dmem_bytes) {
    if (e->dmem) cudaFreeAsync(e->dmem, e->st);
    e->dmem = nullptr;
    e->dmem_bytes = 0;
    if (cudaMallocAsync(&e->dmem, need * 2, e->st) != cudaSuccess) {
      cudaGetLastError();
      return RLOBPCG_ERR_OOM;
    }
    e->dmem_bytes = need * 2;
  }
  if ((size_t)count > e->Dh_cap) {
    if (e->Dh) cudaFreeHost(e->Dh);
    e->Dh = nullptr;
    e->Dh_cap = 0;
    if (cudaMallocHost((void**)&e->Dh, (size_t)count * 2 * sizeof(batch::Desc)) != cudaSuccess) {
      cudaGetLastError();
      return RLOBPCG_ERR_CUDA;
    }
    e->Dh_cap = (size_t)count * 2;
  }
  char* q = (char*)e->dmem;
  auto take = [&](size_t x) { char* r = q; q += (x + 255) & ~(size_t)255; return r; };
  e->Dd = (batch::Desc*)take(count * sizeof(batch::Desc));
  e->pre_items = (int2*)take(hpre.size() * sizeof(int2));
  e->tile_items = (int2*)take(htile.size() * sizeof(int2));
  e->qh = (int*)take((3 * BatchEngine::G + 2) * sizeof(int));
  for (int i = 0; i < count; ++i) e->Dh[i] = e->active[i]->d;
  RL_CUDA(cudaMemcpyAsync(e->Dd, e->Dh, count * sizeof(batch::Desc), cudaMemcpyHostToDevice, e->st));
  RL_CUDA(cudaMemcpyAsync(e->pre_items, hpre.data(), hpre.size() * sizeof(int2), cudaMemcpyHostToDevice, e->st));
  RL_CUDA(cudaMemcpyAsync(e->tile_items, htile.data(), htile.size() * sizeof(int2), cudaMemcpyHostToDevice, e->st));
  e->tile_smem = batch::tile_smem_bytes(e->nwmax, e->abmax, e->rtmax);
  RL_TRY(batch::prepare(e->pre_smem, e->tile_smem));
  int per_sm = 1;
  RL_TRY(batch::tile_blocks_per_sm(e->tile_smem, &per_sm));
  // one CTA per work item (up to 64 waves): CTAs retire all through a launch, so that kernels of
  // other streams (the set-ups of joining solves, at a higher stream priority) start in between
  // instead of waiting for a persistent grid to drain
  const int slots = num_sms() * std::max(1, per_sm);
  e->pre_grid = std::max(1, std::min(e->npre, slots * 64));
  e->tile_grid = std::max(1, std::min(e->ntile, slots * 64));
  RL_CUDA(cudaStreamSynchronize(e->st));   // the item vectors are host locals
  e->dirty = false;
  e->stable = 0;
  return RLOBPCG_OK;
}

// One replay: reset the work queues, (R^{-H} Rs, R^{-1} Y + BCGS2, tiles) x G, then the
// descriptors back to the host. Issued directly on the stream, or captured once as a graph when
// the membership has stayed the same for a replay (and relaunched while it stays so).
int engine_issue(BatchEngine* e) {
  const int G = BatchEngine::G;
  const int count = (int)e->active.size();
  int rc = cudaMemsetAsync(e->qh, 0, (3 * G + 2) * sizeof(int), e->st) == cudaSuccess ? RLOBPCG_OK : RLOBPCG_ERR_CUDA;
  for (int g = 0; g < G && !rc; ++g) {
    rc = batch::pre_launch(0, e->Dd, e->pre_items, e->npre, e->qh + 3 * g, e->pre_grid, e->pre_smem, e->st);
    if (!rc) rc = batch::pre_launch(1, e->Dd, e->pre_items, e->npre, e->qh + 3 * g + 1, e->pre_grid, e->pre_smem, e->st);
    if (!rc)
      rc = batch::tile_launch(false, e->Dd, e->tile_items, e->ntile, e->qh + 3 * g + 2, e->tile_grid, e->nwmax, e->abmax,
                              e->tile_smem, e->st);
  }
  if (!rc && cudaMemcpyAsync(e->Dh, e->Dd, count * sizeof(batch::Desc), cudaMemcpyDeviceToHost, e->st) != cudaSuccess)
    rc = RLOBPCG_ERR_CUDA;
  return rc;
}

int engine_replay(BatchEngine* e) {
  if (e->gexec) return cudaGraphLaunch(e->gexec, e->st) == cudaSuccess ? RLOBPCG_OK : RLOBPCG_ERR_CUDA;
  if (e->stable < 1) {
    ++e->stable;
    return engine_issue(e);
  }
  RL_CUDA(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
  const int crc = engine_issue(e);
  const cudaError_t ce = cudaStreamEndCapture(e->st, &e->graph);
  if (crc || ce != cudaSuccess) {
    cudaGetLastError();
    return crc ? crc : RLOBPCG_ERR_CUDA;
  }
  RL_CUDA(cudaGraphInstantiate(&e->gexec, e->graph, 0));
  return cudaGraphLaunch(e->gexec, e->st) == cudaSuccess ? RLOBPCG_OK : RLOBPCG_ERR_CUDA;
}

// solves that stopped: A V and A X brought up to date, the state handed back, buffers released
int engine_retire(BatchEngine* e, const std::vector<int>& idx) {
  std::vector<int2> items;
  for (int i : idx)
    for (int t = 0; t < e->active[i]->d.ntiles; ++t) items.push_back(make_int2(i, t));
  int2* ditems = nullptr;
  RL_CUDA(cudaMallocAsync((void**)&ditems, items.size() * sizeof(int2), e->st));
  RL_CUDA(cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, e->st));
  RL_CUDA(cudaMemsetAsync(e->qh + 3 * BatchEngine::G, 0, sizeof(int), e->st));
  RL_TRY(batch::tile_launch(true, e->Dd, ditems, (int)items.size(), e->qh + 3 * BatchEngine::G, e->tile_grid, e->nwmax,
                            e->abmax, e->tile_smem, e->st));
  RL_CUDA(cudaFreeAsync(ditems, e->st));
  std::vector<std::vector<double>> hs(idx.size());
  for (size_t q = 0; q < idx.size(); ++q) {
    const batch::Desc& d = e->active[idx[q]]->d;
    hs[q].resize((size_t)(d.iter + 1) * 2 * d.b);
    RL_CUDA(cudaMemcpyAsync(hs[q].data(), d.hist, hs[q].size() * sizeof(double), cudaMemcpyDeviceToHost, e->st));
  }
  RL_CUDA(cudaStreamSynchronize(e->st));
  for (size_t q = 0; q < idx.size(); ++q) {
    BatchSolve* s = e->active[idx[q]];
    const batch::Desc& d = s->d;
    const int b = d.b;
    const std::vector<double>& h = hs[q];
    for (int t = 1; t <= d.iter; ++t) {
      s->r.hist.r.emplace_back(h.begin() + (size_t)t * 2 * b, h.begin() + (size_t)t * 2 * b + b);
      s->r.hist.th.emplace_back(h.begin() + (size_t)t * 2 * b + b, h.begin() + (size_t)(t + 1) * 2 * b);
    }
    s->r.it = d.iter;
    s->r.stop = d.stop_reason;
    s->r.matvecs = d.matvecs;
    s->r.nx = d.nx;
    s->r.theta_s = s->p->theta + (d.iter > 0 ? d.c_prev - b : 0);
    cudaFreeAsync(s->mem, e->st);
    s->mem = nullptr;
  }
  RL_CUDA(cudaStreamSynchronize(e->st));
  return RLOBPCG_OK;
}

void engine_fail_all(BatchEngine* e, int rc) {
  for (BatchSolve* s : e->active) {
    if (s->mem) cudaFreeAsync(s->mem, e->st);
    s->mem = nullptr;
    complete(s, rc);
  }
  e->active.clear();
  e->dirty = true;
}

void engine_main(BatchEngine* e) {
  cudaSetDevice(e->device);
  using clk = std::chrono::steady_clock;
  auto t_host = clk::now();
  auto host_add = [&](clk::time_point a, clk::time_point b) {
    std::lock_guard<std::mutex> lk(e->mu);
    e->stats.host_ms += std::chrono::duration<double, std::milli>(b - a).count();
  };
  for (;;) {
    std::vector<BatchSolve*> joining;
    {
      std::unique_lock<std::mutex> lk(e->mu);
      e->cv.wait(lk, [&] { return e->stop || !e->incoming.empty() || !e->active.empty(); });
      if (e->stop && e->incoming.empty() && e->active.empty()) break;
      joining.assign(e->incoming.begin(), e->incoming.end());
      e->incoming.clear();
    }
    t_host = clk::now();
    for (BatchSolve* s : joining) {
      const int rc = engine_join(e, s);
      if (rc) {
        if (s->mem) cudaFreeAsync(s->mem, e->st);
        s->mem = nullptr;
        complete(s, rc);
      } else {
        e->active.push_back(s);
        e->dirty = true;
      }
    }
    if (e->active.empty()) continue;
    const bool rebuilt = e->dirty;
    int rc = e->dirty ? engine_rebuild(e) : RLOBPCG_OK;
    host_add(t_host, clk::now());
    if (!rc && cudaEventRecord(e->ev0, e->st) != cudaSuccess) rc = RLOBPCG_ERR_CUDA;
    if (!rc) rc = engine_replay(e);
    if (!rc && cudaEventRecord(e->ev1, e->st) != cudaSuccess) rc = RLOBPCG_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(e->st) != cudaSuccess) rc = RLOBPCG_ERR_CUDA;
    t_host = clk::now();
    if (!rc) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e->ev0, e->ev1);
      std::lock_guard<std::mutex> lk(e->mu);
      e->stats.replays += 1;
      e->stats.rebuilds += rebuilt ? 1 : 0;
      e->stats.joins += (int64_t)joining.size();
      e->stats.gpu_ms += ms;
      e->active_sum += (double)e->active.size();
      e->stats.active_mean = e->active_sum / (double)e->stats.replays;
    }
    if (rc) {
      cudaGetLastError();
      engine_fail_all(e, rc);
      continue;
    }
    std::vector<int> done;
    for (size_t i = 0; i < e->active.size(); ++i) {
      e->active[i]->d = e->Dh[i];
      if (e->Dh[i].done) done.push_back((int)i);
    }
    if (done.empty()) {
      host_add(t_host, clk::now());
      continue;
    }
    rc = engine_retire(e, done);
    if (rc) {
      cudaGetLastError();
      engine_fail_all(e, rc);
      continue;
    }
    std::vector<BatchSolve*> keep;
    size_t di = 0;
    for (size_t i = 0; i < e->active.size(); ++i) {
      if (di < done.size() && (size_t)done[di] == i) {
        complete(e->active[i], RLOBPCG_OK);
        ++di;
      } else {
        keep.push_back(e->active[i]);
      }
    }
    e->active.swap(keep);
    e->dirty = true;
    {
      std::lock_guard<std::mutex> lk(e->mu);
      e->stats.retires += (int64_t)done.size();
    }
    host_add(t_host, clk::now());
  }
}

}  // namespace

int batch_engine_create(int device, BatchEngine** out) {
  auto* e = new BatchEngine();
  e->device = device;
  // the lowest stream priority: set-ups and outputs of other solves run first when both wait
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (cudaStreamCreateWithPriority(&e->st, cudaStreamNonBlocking, least) != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return RLOBPCG_ERR_CUDA;
  }
  if (cudaEventCreate(&e->ev0) != cudaSuccess || cudaEventCreate(&e->ev1) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(e->st);
    delete e;
    return RLOBPCG_ERR_CUDA;
  }
  e->th = std::thread(engine_main, e);
  *out = e;
  return RLOBPCG_OK;
}

void batch_engine_stats(BatchEngine* e, rlobpcg_engine_stats* out) {
  std::lock_guard<std::mutex> lk(e->mu);
  *out = e->stats;
}

void batch_engine_destroy(BatchEngine* e) {
  if (!e) return;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->stop = true;
  }
  e->cv.notify_all();
  e->th.join();
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->dmem) cudaFreeAsync(e->dmem, e->st);
  cudaStreamSynchronize(e->st);
  if (e->Dh) cudaFreeHost(e->Dh);
  if (e->ev0) cudaEventDestroy(e->ev0);
  if (e->ev1) cudaEventDestroy(e->ev1);
  cudaStreamDestroy(e->st);
  delete e;
}

bool batch_request_eligible(int64_t n, int k, int dtype, const rlobpcg_opts& o) {
  const int b = o.block > 0 ? o.block : k;
  return dtype == RLOBPCG_F64 && b <= batch::BMAX && n <= 512 && !o.locking && o.orth_mode == RLOBPCG_ORTH_HOUSEHOLDER &&
         o.residual_refresh_every <= 0 && std::max(o.max_iter, o.fixed_iters) <= 200 &&
         o.precond == RLOBPCG_PRECOND_SKETCH;
}

size_t batch_extra_bytes(int64_t m, int64_t n, int b) {
  return batch_solve_bytes(m, n, b, 256, nullptr, nullptr);   // the smallest tile height: the most partials
}

// set-up of one solve on its plan's stream (host-synchronous); A stays valid until finish
int batch_solve_setup(rlobpcg_plan_t p, const double* A, int64_t lda, BatchSolve** out) {
  std::string why;
  if (!batch_eligible(p, &why)) {
    set_last_error(why.c_str(), __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  auto* s = new BatchSolve();
  s->p = p;
  s->A = A;
  s->lda = lda;
  int rc = tile_choice((int)p->n, p->b, p->st, &s->tc);
  if (!rc)
    rc = p->opts.sketch_prec == RLOBPCG_SKETCH_F32 ? batch_setup_one<float>(p, A, lda, s->r)
                                                   : batch_setup_one<double>(p, A, lda, s->r);
  if (rc) {
    delete s;
    return rc;
  }
  *out = s;
  return RLOBPCG_OK;
}

void batch_solve_submit(BatchEngine* e, BatchSolve* s) {
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->incoming.push_back(s);
  }
  e->cv.notify_all();
}

int batch_solve_wait(BatchSolve* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [&] { return s->finished; });
  return s->rc;
}

// outputs of a retired solve on its plan's stream; releases the handle
int batch_solve_finish(BatchSolve* s, double* sigma, void* V, void* U, double* resid, rlobpcg_info* info) {
  rlobpcg_plan_s* p = s->p;
  int rc = s->rc;
  if (!rc)
    rc = p->opts.sketch_prec == RLOBPCG_SKETCH_F32
             ? batch_finish_one<float>(p, s->A, s->lda, s->r, sigma, (double*)V, (double*)U, resid, info)
             : batch_finish_one<double>(p, s->A, s->lda, s->r, sigma, (double*)V, (double*)U, resid, info);
  delete s;
  return rc;
}

}  // namespace rl

namespace {
}  // namespace

extern "C" int rlobpcg_batch_tile(int64_t n, int b, int* trows, int* rt, void* stream) {
  if (n < 1 || n > 512 || b < 1 || b > batch::BMAX) return RLOBPCG_ERR_INVALID_ARG;
  TileChoice tc;
  RL_TRY(tile_choice((int)n, b, (cudaStream_t)stream, &tc));
  if (trows) *trows = tc.trows;
  if (rt) *rt = tc.rt;
  return RLOBPCG_OK;
}

extern "C" int rlobpcg_batch_set_tile(int64_t n, int b, int trows, int rt) {
  if (n < 1 || n > 512 || b < 1 || b > batch::BMAX) return RLOBPCG_ERR_INVALID_ARG;
  size_t s_pre = 0, s_tile = 0;
  RL_TRY(batch::static_smem_bytes(&s_pre, &s_tile));
  const int nc = n_class((int)n);
  bool ok = false;
  for (const TileChoice& c : tile_candidates(nc, b, s_tile)) ok |= (c.trows == trows && c.rt == rt);
  if (!ok) {
    set_last_error("batch: tile shape not among the candidates that fit this class", __FILE__, __LINE__);
    return RLOBPCG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tile_table[std::make_pair(nc, b)] = TileChoice{trows, rt};
  return RLOBPCG_OK;
}


extern "C" int rlobpcg_solve_batch(int count, rlobpcg_plan_t* plans, const void* const* A, const int64_t* lda,
                                   double* const* sigma, void* const* V, void* const* U, double* const* resid,
                                   rlobpcg_info* infos, int* status, void* stream) {
  if (count < 1 || !plans || !A || !lda || !sigma || !V) return RLOBPCG_ERR_INVALID_ARG;
  std::string why;
  for (int i = 0; i < count; ++i) {
    rlobpcg_plan_s* p = plans[i];
    if (!p || !A[i] || !sigma[i] || !V[i] || lda[i] < p->n || !is_device_ptr(A[i])) return RLOBPCG_ERR_INVALID_ARG;
    if (p->async_busy) return async_in_flight(p);
    for (int j = 0; j < i; ++j)
      if (plans[j] == p) return RLOBPCG_ERR_INVALID_ARG;   // one solve per plan
    if (!batch_eligible(p, &why)) {
      set_last_error(why.c_str(), __FILE__, __LINE__);
      return RLOBPCG_ERR_UNSUPPORTED;
    }
  }
  int dev = 0;
  RL_CUDA(cudaGetDevice(&dev));
  // every class's tile shape first (the autotuner times kernels; nothing else runs meanwhile)
  for (int i = 0; i < count; ++i) {
    TileChoice tc;
    RL_TRY(tile_choice((int)plans[i]->n, plans[i]->b, (cudaStream_t)stream, &tc));
  }
  BatchEngine* e = nullptr;
  RL_TRY(batch_engine_create(dev, &e));
  // set-ups on up to 8 host threads; each solve joins the running batch as soon as its set-up ends
  std::vector<BatchSolve*> hs(count, nullptr);
  std::vector<int> rcs(count, RLOBPCG_OK);
  {
    const int nth = std::min(count, 8);
    std::vector<std::thread> th;
    std::atomic<int> next{0};
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&]() {
        cudaSetDevice(dev);
        for (int i = next++; i < count; i = next++) {
          rcs[i] = batch_solve_setup(plans[i], (const double*)A[i], lda[i], &hs[i]);
          if (!rcs[i]) batch_solve_submit(e, hs[i]);
        }
      });
    for (auto& t : th) t.join();
  }
  for (int i = 0; i < count; ++i)
    if (hs[i]) rcs[i] = batch_solve_wait(hs[i]);
  // outputs on each plan's stream
  {
    const int nth = std::min(count, 8);
    std::vector<std::thread> th;
    std::atomic<int> next{0};
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&]() {
        cudaSetDevice(dev);
        for (int i = next++; i < count; i = next++) {
          if (!hs[i]) continue;
          rcs[i] = batch_solve_finish(hs[i], sigma[i], V[i], U ? U[i] : nullptr, resid ? resid[i] : nullptr,
                                      infos ? &infos[i] : nullptr);
          hs[i] = nullptr;
        }
      });
    for (auto& t : th) t.join();
  }
  batch_engine_destroy(e);
  int first = RLOBPCG_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = rcs[i];
    if (rcs[i] < 0 && first >= 0) first = rcs[i];
  }
  return first;
}
