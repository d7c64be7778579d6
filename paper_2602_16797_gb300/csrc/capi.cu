// C ABI entry points for the single steps of the path, status strings and device queries.
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace rl {

int sketch_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int d, int zeta, uint64_t seed,
                    int sketch_prec, void* SA, cudaStream_t st);
size_t factor_workspace_bytes(int64_t d, int64_t n, size_t esz);
template <class S>
int factor_impl(S* SA, int d, int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c, void* work,
                size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err);
size_t refine_workspace_bytes(int64_t d, int64_t n, int dtype);
template <class T>
int factor_refine_impl(T* SA, int d, int n, T* Rout, T* Rout_r, double* sigma, T* Vt, T* Rinv_r, T* Rinv_c,
                       void* work, size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err);
size_t gram_workspace_bytes(int64_t m, int64_t n, int b, int dtype);
int gram_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b, int64_t ldw,
                  void* AW, int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes, int resid_mode,
                  int* err, cudaStream_t st);
size_t tsqr_workspace_bytes(int64_t m, int c, size_t esz);
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
template <class T>
int tsqr_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st);

static thread_local char g_last_error[512] = "";
static thread_local long g_launches = 0;

void note_launch() { ++g_launches; }
long launch_count() { return g_launches; }

void set_last_error(const char* msg, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", msg, base ? base + 1 : file, line);
}
void set_last_error_text(const char* text) { snprintf(g_last_error, sizeof(g_last_error), "%s", text); }
const char* last_error() { return g_last_error; }

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

size_t max_smem_optin() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cached[dev] = v > 0 ? v : 48 * 1024;
  }
  return (size_t)cached[dev];
}

// Scratch error word of the step entry points (bounded device waits report here). One per host
// thread and device: a thread's calls are sequential (each synchronises its stream before it
// returns), so calls from different threads on different streams never share a word. The word
// lives as long as the process.
static int* step_err_word(cudaStream_t st) {
  static thread_local int* w[64] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!w[dev]) {
    if (cudaMalloc(&w[dev], sizeof(int)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  }
  cudaMemsetAsync(w[dev], 0, sizeof(int), st);
  return w[dev];
}

static int finish(cudaStream_t st, int* err) {
  int herr = 0;
  if (err) RL_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RL_CUDA(cudaStreamSynchronize(st));
  return dev_err_status(herr);
}

}  // namespace rl

using namespace rl;

extern "C" const char* rlobpcg_status_string(int s) {
  switch (s) {
    case RLOBPCG_OK: return "ok";
    case RLOBPCG_NOT_CONVERGED: return "not converged (max_iter reached; outputs hold the last iterate)";
    case RLOBPCG_ERR_INVALID_ARG: return "invalid argument";
    case RLOBPCG_ERR_OOM: return "out of device memory";
    case RLOBPCG_ERR_CUDA: return "CUDA runtime error";
    case RLOBPCG_ERR_NONFINITE: return "non-finite value in input or iteration";
    case RLOBPCG_ERR_TIMEOUT: return "bounded device wait ran out";
    case RLOBPCG_ERR_UNSUPPORTED: return "shape not supported by the kernels";
    case RLOBPCG_ERR_CANCELLED: return "request cancelled before it ran";
    default: return "unknown status";
  }
}

extern "C" const char* rlobpcg_last_error(void) { return last_error(); }

extern "C" int rlobpcg_sketch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int d, int zeta,
                              uint64_t seed, int sketch_prec, void* SA, void* stream) {
  if (!A || !SA || m < 1 || n < 1 || lda < n || zeta < 1 || d < zeta || d > (1 << 28) || n > (1 << 28) ||
      (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128) ||
      (sketch_prec != RLOBPCG_SKETCH_F64 && sketch_prec != RLOBPCG_SKETCH_F32 &&
       sketch_prec != RLOBPCG_SKETCH_F32_REFINE))
    return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the refined form keeps the sketch in FP64 (its QR input is rounded to FP32 inside the factor)
  const int sp = sketch_prec == RLOBPCG_SKETCH_F32 ? RLOBPCG_SKETCH_F32 : RLOBPCG_SKETCH_F64;
  int rc = sketch_dispatch(A, m, n, lda, dtype, d, zeta, seed, sp, SA, st);
  if (rc) return rc;
  return finish(st, nullptr);
}

static size_t sketch_elem(int dtype, int prec) {
  return (dtype == RLOBPCG_C128 ? 2 : 1) * (prec == RLOBPCG_SKETCH_F32 ? 4 : 8);
}

static size_t factor_scratch_bytes(int64_t d, int64_t n, int dtype, int sketch_prec) {
  if (sketch_prec == RLOBPCG_SKETCH_F32_REFINE) return refine_workspace_bytes(d, n, dtype);
  return factor_workspace_bytes(d, n, sketch_elem(dtype, sketch_prec));
}

// factorisation scratch plus a column-major copy of R^{-1} (the caller receives the row-major one)
extern "C" size_t rlobpcg_factor_workspace_size(int64_t d, int64_t n, int dtype, int sketch_prec) {
  const size_t esz = sketch_elem(dtype, sketch_prec);
  return factor_scratch_bytes(d, n, dtype, sketch_prec) + (((size_t)n * n * esz + 255) & ~(size_t)255);
}

extern "C" int rlobpcg_factor(void* SA, int64_t d, int64_t n, int dtype, int sketch_prec, void* R, double* sigma,
                              void* Vt, void* Rinv, void* work, size_t work_bytes, void* stream) {
  if (!SA || !sigma || !Vt || !work || n < 1 || d < n || (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128) ||
      (sketch_prec != RLOBPCG_SKETCH_F64 && sketch_prec != RLOBPCG_SKETCH_F32 &&
       sketch_prec != RLOBPCG_SKETCH_F32_REFINE))
    return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (work_bytes < rlobpcg_factor_workspace_size(d, n, dtype, sketch_prec)) return RLOBPCG_ERR_INVALID_ARG;
  const size_t fbytes = factor_scratch_bytes(d, n, dtype, sketch_prec);
  void* Rinv_c = Rinv ? (void*)((unsigned char*)work + fbytes) : nullptr;
  work_bytes = fbytes;
  int* err = step_err_word(st);
  if (!err) return RLOBPCG_ERR_OOM;
  int rc;
  const bool f32 = sketch_prec == RLOBPCG_SKETCH_F32;
  if (sketch_prec == RLOBPCG_SKETCH_F32_REFINE) {
    rc = dtype == RLOBPCG_F64
             ? factor_refine_impl<double>((double*)SA, (int)d, (int)n, (double*)R, nullptr, sigma, (double*)Vt,
                                          (double*)Rinv, (double*)Rinv_c, work, work_bytes, st, nullptr, true, err)
             : factor_refine_impl<cd>((cd*)SA, (int)d, (int)n, (cd*)R, nullptr, sigma, (cd*)Vt, (cd*)Rinv,
                                      (cd*)Rinv_c, work, work_bytes, st, nullptr, true, err);
  } else if (dtype == RLOBPCG_F64) {
    rc = f32 ? factor_impl<float>((float*)SA, (int)d, (int)n, (float*)R, nullptr, sigma, (float*)Vt, (float*)Rinv,
                                  (float*)Rinv_c, work, work_bytes, st, nullptr, true, err)
             : factor_impl<double>((double*)SA, (int)d, (int)n, (double*)R, nullptr, sigma, (double*)Vt, (double*)Rinv,
                                   (double*)Rinv_c, work, work_bytes, st, nullptr, true, err);
  } else {
    rc = f32 ? factor_impl<cf>((cf*)SA, (int)d, (int)n, (cf*)R, nullptr, sigma, (cf*)Vt, (cf*)Rinv, (cf*)Rinv_c, work,
                               work_bytes, st, nullptr, true, err)
             : factor_impl<cd>((cd*)SA, (int)d, (int)n, (cd*)R, nullptr, sigma, (cd*)Vt, (cd*)Rinv, (cd*)Rinv_c, work,
                               work_bytes, st, nullptr, true, err);
  }
  if (rc) return rc;
  return finish(st, err);
}

extern "C" size_t rlobpcg_gram_workspace_size(int64_t m, int64_t n, int b, int dtype) {
  return gram_workspace_bytes(m, n, b, dtype);
}

extern "C" int rlobpcg_gram(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b,
                            int64_t ldw, void* AW, int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes,
                            void* stream) {
  if (!A || !W || !AW || !G || !work || m < 1 || n < 1 || b < 1 || b > 64 || lda < n || ldw < b || ldaw < b ||
      ldg < b || (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128))
    return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = step_err_word(st);
  if (!err) return RLOBPCG_ERR_OOM;
  int rc = gram_dispatch(A, m, n, lda, dtype, W, b, ldw, AW, ldaw, G, ldg, work, work_bytes, 0, err, st);
  if (rc) return rc;
  return finish(st, err);
}

extern "C" size_t rlobpcg_gram_split_prepare_size(int64_t m, int64_t n) { return split_prep_bytes(m, n); }

extern "C" int rlobpcg_gram_split_prepare(const double* A, int64_t m, int64_t n, int64_t lda, void* prep,
                                          size_t prep_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int* err = step_err_word(st);
  if (!err) return RLOBPCG_ERR_OOM;
  const int rc = split_prepare(A, m, n, lda, prep, prep_bytes, err, st);
  if (rc) return rc;
  return finish(st, err);
}

extern "C" size_t rlobpcg_gram_split_workspace_size(int64_t m, int64_t n, int b) { return split_work_bytes(m, n, b); }

extern "C" int rlobpcg_gram_split(const void* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw,
                                  double* AW, int64_t ldaw, double* G, int64_t ldg, void* work, size_t work_bytes,
                                  void* stream) {
  if (!W) return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = step_err_word(st);
  if (!err) return RLOBPCG_ERR_OOM;
  const int rc = split_gram(prep, m, n, W, b, ldw, AW, ldaw, G, ldg, work, work_bytes, 0, err, nullptr, st);
  if (rc) return rc;
  return finish(st, err);
}

extern "C" size_t rlobpcg_gram_split_c128_workspace_size(int64_t m, int64_t n, int b) {
  return split_work_bytes_c128(m, n, b);
}

extern "C" int rlobpcg_gram_split_c128(const void* prep, int64_t m, int64_t n, const void* W, int b, int64_t ldw,
                                       void* AW, int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes,
                                       void* stream) {
  if (!W) return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = step_err_word(st);
  if (!err) return RLOBPCG_ERR_OOM;
  const int rc = split_gram_c128(prep, m, n, (const cd*)W, b, ldw, (cd*)AW, ldaw, (cd*)G, ldg, work, work_bytes, 0,
                                 err, nullptr, st);
  if (rc) return rc;
  return finish(st, err);
}

extern "C" size_t rlobpcg_tsqr_workspace_size(int64_t m, int c, int dtype) {
  return tsqr_workspace_bytes(m, c, dtype == RLOBPCG_C128 ? 16 : 8);
}

extern "C" int rlobpcg_tsqr(const void* X, int64_t m, int c, int64_t ldx, int dtype, void* R, void* work,
                            size_t work_bytes, void* stream) {
  if (!X || !R || !work || m < 1 || c < 1 || c > 64 || ldx < c || (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128))
    return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = dtype == RLOBPCG_C128 ? tsqr_impl<cd>((const cd*)X, m, c, ldx, (cd*)R, work, work_bytes, st)
                                 : tsqr_impl<double>((const double*)X, m, c, ldx, (double*)R, work, work_bytes, st);
  if (rc) return rc;
  return finish(st, nullptr);
}
