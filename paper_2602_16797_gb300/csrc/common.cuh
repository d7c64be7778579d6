// Shared device/host helpers of the RLOBPCG GPU library (sm_103a).
//
// Scalar types: double, float, cd (complex128 as two interleaved doubles, the numpy layout) and
// cf (complex64). The LOBPCG state is double or cd; the sketch side (SA, R, its SVD and R^{-1})
// is float/cf in the mixed-precision form and double/cd otherwise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/rlobpcg.h"

namespace rl {

struct cd { double x, y; };
struct cf { float x, y; };

// ------------------------------------------------------------------ scalar traits and arithmetic
template <class T> struct Tr;
template <> struct Tr<double> { using R = double; static constexpr bool cplx = false; };
template <> struct Tr<float>  { using R = float;  static constexpr bool cplx = false; };
template <> struct Tr<cd>     { using R = double; static constexpr bool cplx = true; };
template <> struct Tr<cf>     { using R = float;  static constexpr bool cplx = true; };

// real scalar of the same precision / the complex or real type of precision R
template <class T> using RealOf = typename Tr<T>::R;

__host__ __device__ inline double conj_(double a) { return a; }
__host__ __device__ inline float conj_(float a) { return a; }
__host__ __device__ inline cd conj_(cd a) { return {a.x, -a.y}; }
__host__ __device__ inline cf conj_(cf a) { return {a.x, -a.y}; }

__host__ __device__ inline double re_(double a) { return a; }
__host__ __device__ inline float re_(float a) { return a; }
__host__ __device__ inline double re_(cd a) { return a.x; }
__host__ __device__ inline float re_(cf a) { return a.x; }

__host__ __device__ inline double im_(double) { return 0.0; }
__host__ __device__ inline float im_(float) { return 0.0f; }
__host__ __device__ inline double im_(cd a) { return a.y; }
__host__ __device__ inline float im_(cf a) { return a.y; }

__host__ __device__ inline double abs2_(double a) { return a * a; }
__host__ __device__ inline float abs2_(float a) { return a * a; }
__host__ __device__ inline double abs2_(cd a) { return fma(a.x, a.x, a.y * a.y); }
__host__ __device__ inline float abs2_(cf a) { return fmaf(a.x, a.x, a.y * a.y); }

template <class T> __host__ __device__ inline T zero_();
template <> __host__ __device__ inline double zero_<double>() { return 0.0; }
template <> __host__ __device__ inline float zero_<float>() { return 0.0f; }
template <> __host__ __device__ inline cd zero_<cd>() { return {0.0, 0.0}; }
template <> __host__ __device__ inline cf zero_<cf>() { return {0.0f, 0.0f}; }

template <class T> __host__ __device__ inline T from_real(RealOf<T> r);
template <> __host__ __device__ inline double from_real<double>(double r) { return r; }
template <> __host__ __device__ inline float from_real<float>(float r) { return r; }
template <> __host__ __device__ inline cd from_real<cd>(double r) { return {r, 0.0}; }
template <> __host__ __device__ inline cf from_real<cf>(float r) { return {r, 0.0f}; }

__host__ __device__ inline double add_(double a, double b) { return a + b; }
__host__ __device__ inline float add_(float a, float b) { return a + b; }
__host__ __device__ inline cd add_(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cf add_(cf a, cf b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline double sub_(double a, double b) { return a - b; }
__host__ __device__ inline float sub_(float a, float b) { return a - b; }
__host__ __device__ inline cd sub_(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cf sub_(cf a, cf b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline double neg_(double a) { return -a; }
__host__ __device__ inline float neg_(float a) { return -a; }
__host__ __device__ inline cd neg_(cd a) { return {-a.x, -a.y}; }
__host__ __device__ inline cf neg_(cf a) { return {-a.x, -a.y}; }

__host__ __device__ inline double scale_(double a, double s) { return a * s; }
__host__ __device__ inline float scale_(float a, float s) { return a * s; }
__host__ __device__ inline cd scale_(cd a, double s) { return {a.x * s, a.y * s}; }
__host__ __device__ inline cf scale_(cf a, float s) { return {a.x * s, a.y * s}; }

__host__ __device__ inline double mul_(double a, double b) { return a * b; }
__host__ __device__ inline float mul_(float a, float b) { return a * b; }
__host__ __device__ inline cd mul_(cd a, cd b) { return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)}; }
__host__ __device__ inline cf mul_(cf a, cf b) { return {fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)}; }

// c + a * b
__host__ __device__ inline double mad_(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ inline float mad_(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ inline cd mad_(cd a, cd b, cd c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
__host__ __device__ inline cf mad_(cf a, cf b, cf c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}
// c + conj(a) * b
__host__ __device__ inline double madc_(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ inline float madc_(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ inline cd madc_(cd a, cd b, cd c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__host__ __device__ inline cf madc_(cf a, cf b, cf c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}

// precision conversions (round to nearest)
template <class To, class From> __host__ __device__ inline To cvt_(From a);
template <> __host__ __device__ inline double cvt_<double, double>(double a) { return a; }
template <> __host__ __device__ inline float cvt_<float, double>(double a) { return (float)a; }
template <> __host__ __device__ inline double cvt_<double, float>(float a) { return (double)a; }
template <> __host__ __device__ inline float cvt_<float, float>(float a) { return a; }
template <> __host__ __device__ inline cd cvt_<cd, cd>(cd a) { return a; }
template <> __host__ __device__ inline cf cvt_<cf, cd>(cd a) { return {(float)a.x, (float)a.y}; }
template <> __host__ __device__ inline cd cvt_<cd, cf>(cf a) { return {(double)a.x, (double)a.y}; }
template <> __host__ __device__ inline cf cvt_<cf, cf>(cf a) { return a; }

// phase e^{i arg a} (1 for a == 0); real: sign with sign(0) = 1
__host__ __device__ inline double phase_(double a) { return a < 0 ? -1.0 : 1.0; }
__host__ __device__ inline float phase_(float a) { return a < 0 ? -1.0f : 1.0f; }
__host__ __device__ inline cd phase_(cd a) {
  double r = hypot(a.x, a.y);
  if (r == 0.0) return {1.0, 0.0};
  return {a.x / r, a.y / r};
}
__host__ __device__ inline cf phase_(cf a) {
  float r = hypotf(a.x, a.y);
  if (r == 0.0f) return {1.0f, 0.0f};
  return {a.x / r, a.y / r};
}

__host__ __device__ inline bool finite_(double a) { return isfinite(a); }
__host__ __device__ inline bool finite_(float a) { return isfinite(a); }
__host__ __device__ inline bool finite_(cd a) { return isfinite(a.x) && isfinite(a.y); }
__host__ __device__ inline bool finite_(cf a) { return isfinite(a.x) && isfinite(a.y); }

// ------------------------------------------------------------------ one-sided Jacobi rotation
// For columns x_p, x_q with a = ||x_p||^2, b = ||x_q||^2, g = x_p^H x_q: the rotation
//   x_p' = c x_p - s conj(e) x_q,   x_q' = s e x_p + c x_q       (e = g / |g|)
// makes x_p'^H x_q' = 0 (Hestenes; the real case is Rutishauser's formula). Its tangent, the
// smaller root of t^2 + 2 zeta t - 1 = 0 with zeta = (b - a) / (2|g|), is written without the
// division by |g|:  t = sign(b - a) 2|g| / (|b - a| + sqrt((b - a)^2 + 4|g|^2)),
// and c = 1/sqrt(1 + t^2), s = c t. On GB300 every dependent FP64 instruction costs ~64 cycles
// and a divide or square root ~10 of them, so this form (one sqrt, one divide, one rsqrt; the
// complex case adds one rsqrt for the phase) matters. Returns false -- no rotation -- when the
// pair is already orthogonal (|g|^2 <= tol^2 a b), when a column is at rounding level (its
// squared norm <= tiny2), or when the angle is below eps (a rotation that changes nothing but
// the smaller column's noise).
__device__ inline double rsqrt_r(double x) { return rsqrt(x); }
__device__ inline float rsqrt_r(float x) { return rsqrtf(x); }
__device__ inline double sqrt_r(double x) { return sqrt(x); }
__device__ inline float sqrt_r(float x) { return sqrtf(x); }

template <class R>
__device__ inline bool jacobi_tangent(R a, R b, R g2, R ga, R tol, R tiny2, R eps, R* c, R* s) {
  if (!(g2 > tol * tol * a * b) || a <= tiny2 || b <= tiny2) return false;
  const R d = b - a;
  // With r = sqrt(d^2 + 4 g^2): cos(2 theta) = |d| / r, cos(theta)^2 = (1 + cos(2 theta)) / 2 and
  // sin(theta) = |g| / (r cos(theta)). Two reciprocal square roots and no square root or division
  // on the dependent chain (FP64 latency); tan(theta) = 2|g| / (|d| + r) as in the usual formula.
  const R q = rsqrt_r(d * d + (R)4 * g2);
  const R u = (R)0.5 + (R)0.5 * (fabs(d) * q);
  const R w = rsqrt_r(u);
  const R cc = u * w;
  const R ss = (ga * q) * w;
  if (ss <= eps * cc) return false;
  *c = cc;
  *s = d >= (R)0 ? ss : -ss;
  return true;
}

__device__ inline bool jacobi_rotation(double a, double b, double g, double tol, double tiny2, double eps, double* c,
                                       double* s, double* e) {
  *e = g < 0.0 ? -1.0 : 1.0;
  return jacobi_tangent(a, b, g * g, fabs(g), tol, tiny2, eps, c, s);
}
__device__ inline bool jacobi_rotation(float a, float b, float g, float tol, float tiny2, float eps, float* c,
                                       float* s, float* e) {
  *e = g < 0.0f ? -1.0f : 1.0f;
  return jacobi_tangent(a, b, g * g, fabsf(g), tol, tiny2, eps, c, s);
}
__device__ inline bool jacobi_rotation(double a, double b, cd g, double tol, double tiny2, double eps, double* c,
                                       double* s, cd* e) {
  const double g2 = abs2_(g);
  if (!(g2 > 0.0)) return false;
  const double rg = rsqrt(g2);
  *e = scale_(g, rg);
  return jacobi_tangent(a, b, g2, g2 * rg, tol, tiny2, eps, c, s);
}
__device__ inline bool jacobi_rotation(float a, float b, cf g, float tol, float tiny2, float eps, float* c, float* s,
                                       cf* e) {
  const float g2 = abs2_(g);
  if (!(g2 > 0.0f)) return false;
  const float rg = rsqrtf(g2);
  *e = scale_(g, rg);
  return jacobi_tangent(a, b, g2, g2 * rg, tol, tiny2, eps, c, s);
}

// ------------------------------------------------------------------ warp helpers
__device__ inline double shfl_xor_(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ inline float shfl_xor_(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ inline cd shfl_xor_(cd v, int m) { return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)}; }
__device__ inline cf shfl_xor_(cf v, int m) { return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)}; }
__device__ inline double shfl_(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ inline float shfl_(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ inline cd shfl_(cd v, int l) { return {__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l)}; }
__device__ inline cf shfl_(cf v, int l) { return {__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l)}; }

// butterfly sum over the 32 lanes (every lane gets the total; fixed order, hence deterministic)
template <class T> __device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = add_(v, shfl_xor_(v, o));
  return v;
}

// ------------------------------------------------------------------ SparseStack randomness
// Output number `counter` (0-based) of SplitMix64 seeded with `seed` (Steele, Lea & Flood,
// OOPSLA 2014): state = seed + (counter + 1) * golden gamma, then the variant-13 finaliser.
__host__ __device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// first row of piece j of a SparseStack column with d rows and zeta pieces: floor(j d / zeta)
__host__ __device__ inline int piece_lo(int j, int d, int zeta) {
  return (int)(((int64_t)j * d) / zeta);
}

// ------------------------------------------------------------------ error handling
struct Status {
  int code = RLOBPCG_OK;
};

#define RL_CUDA(call)                                                           \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) { ::rl::set_last_error(cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RLOBPCG_ERR_CUDA; }                                                \
  } while (0)

// every kernel launch is followed by RL_CHECK_LAUNCH(), which also counts it
#define RL_CHECK_LAUNCH() do { ::rl::note_launch(); RL_CUDA(cudaGetLastError()); } while (0)

void note_launch();
long launch_count();

void set_last_error(const char* msg, const char* file, int line);
void set_last_error_text(const char* text);  // verbatim (an error recorded on another thread)
const char* last_error();

// device-side error flags (bounded waits that ran out, non-finite values)
enum : int { DEV_ERR_TIMEOUT = 1, DEV_ERR_NONFINITE = 2, DEV_ERR_BOUNDS = 4 };

// Status of an entry point from the device error word it read back (one mapping for all of them)
inline int dev_err_status(int herr) {
  if (herr & DEV_ERR_TIMEOUT) return RLOBPCG_ERR_TIMEOUT;
  if (herr & DEV_ERR_NONFINITE) return RLOBPCG_ERR_NONFINITE;
  if (herr & DEV_ERR_BOUNDS) return RLOBPCG_ERR_INVALID_ARG;
  return RLOBPCG_OK;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <class T> __host__ __device__ inline T imin(T a, T b) { return a < b ? a : b; }
template <class T> __host__ __device__ inline T imax(T a, T b) { return a > b ? a : b; }

int num_sms();
size_t max_smem_optin();

// Raise a kernel's dynamic shared-memory limit for a launch of `bytes`. The limit belongs to the
// function, not to the launch, and solves on concurrent streams launch the same kernel with
// different sizes; so it is always raised to the device's opt-in maximum (never to this launch's
// size, which another thread's smaller value could undercut between its set and our launch).
template <class F>
int allow_dynamic_smem(F* kernel, size_t bytes) {
  cudaFuncAttributes fa;
  RL_CUDA(cudaFuncGetAttributes(&fa, kernel));
  const size_t opt = max_smem_optin();
  const size_t cap = opt > fa.sharedSizeBytes ? opt - fa.sharedSizeBytes : 0;  // static smem counts too
  if (bytes > cap) {
    set_last_error("kernel needs more shared memory than the device allows per block", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  // above 48 KB of static + dynamic shared memory a launch needs the opt-in limit
  if (bytes + fa.sharedSizeBytes > 48 * 1024)
    RL_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  return RLOBPCG_OK;
}
#define RL_TRY(call) do { const int rc_ = (call); if (rc_ != RLOBPCG_OK) return rc_; } while (0)

}  // namespace rl
