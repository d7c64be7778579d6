// Factorisation of the sketch (the factorisation step of Alg. 2 of arXiv 2602.16797):
//   1. Householder QR  SA = QR  (the QR route that the footnote in Sec. 1 names as the usual one);
//   2. one-sided Jacobi SVD  R = U~ Sigma~ V~^H  (SVD(SA) = SVD(R): same Sigma~ and V~);
//   3. R^{-1}, so that the preconditioner P P^* = V~ Sigma~^{-2} V~^H = (R^H R)^{-1} is applied
//      as two triangular products.
// All three run in the sketch precision S (float/cf in the mixed form, double/cd otherwise).
//
// GB300 mapping: QR and Jacobi are persistent cooperative kernels (one launch each). The QR runs
// as a dataflow: each reflector is published through a flag and every CTA applies it to its own
// columns when it arrives, so only the chain "update column j+1, form reflector j+1" is serial.
// Jacobi uses grid-wide barriers between rounds, one warp per column pair. The matrices stay
// L2-resident (n <= a few thousand). R^{-1} uses one CTA per column.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rl {

namespace {

constexpr int FQ_THREADS = 256;
constexpr int FQ_WARPS = FQ_THREADS / 32;

template <class S> __device__ inline RealOf<S> eps_of();
template <> __device__ inline double eps_of<double>() { return 2.220446049250313e-16; }
template <> __device__ inline float eps_of<float>() { return 1.1920929e-7f; }
template <> __device__ inline double eps_of<cd>() { return 2.220446049250313e-16; }
template <> __device__ inline float eps_of<cf>() { return 1.1920929e-7f; }

__device__ inline double sqrt_(double a) { return sqrt(a); }
__device__ inline float sqrt_(float a) { return sqrtf(a); }
__device__ inline double hypot_(double a, double b) { return hypot(a, b); }
__device__ inline float hypot_(float a, float b) { return hypotf(a, b); }

// 1 / z. The complex forms scale z by a power of two first (exact), so that |z|^2 neither
// underflows nor overflows: the reflector's 1 / (beta (alpha - beta)) is about |x|^-2 for a
// column of norm |x|, and |z|^2 ~ |x|^4 underflows in FP32 already for |x| ~ 1e-10.
__device__ inline double recip_(double a) { return 1.0 / a; }
__device__ inline float recip_(float a) { return 1.0f / a; }
__device__ inline cd recip_(cd a) {
  int e = 0;
  frexp(fmax(fabs(a.x), fabs(a.y)), &e);
  const double x = ldexp(a.x, -e), y = ldexp(a.y, -e);
  const double s = x * x + y * y;
  return {ldexp(x / s, -e), ldexp(-y / s, -e)};
}
__device__ inline cf recip_(cf a) {
  int e = 0;
  frexpf(fmaxf(fabsf(a.x), fabsf(a.y)), &e);
  const float x = ldexpf(a.x, -e), y = ldexpf(a.y, -e);
  const float s = x * x + y * y;
  return {ldexpf(x / s, -e), ldexpf(-y / s, -e)};
}

// ------------------------------------------------------------------------------------------
// Householder QR (LAPACK geqr2 reflector convention: H = I - tau v v^H, v(0) = 1, H^H x = beta e1)
// M: d x n column-major (ld = d), overwritten: R in the upper triangle, v below the diagonal.
// Column c is owned by CTA c % G; the CTA's 8 warps split its rows, so the dependent FP64 chain
// of each dot product or update is d/256 long (a dependent FP64 instruction costs ~64 cycles on
// GB300). One grid barrier per column step.
// ------------------------------------------------------------------------------------------

// Sum of one value per thread over the CTA (FQ_THREADS threads); every thread gets the total.
// Fixed order: butterfly inside each warp, then warp 0 combines the 8 warp sums.
template <class S>
__device__ inline S cta_sum(S v, S* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    S t = lane < FQ_WARPS ? red[lane] : zero_<S>();
#pragma unroll
    for (int o = FQ_WARPS / 2; o > 0; o >>= 1) t = add_(t, shfl_xor_(t, o));
    if (lane == 0) red[FQ_WARPS] = t;
  }
  __syncthreads();
  const S r = red[FQ_WARPS];
  __syncthreads();
  return r;
}

template <class S>
__device__ void cta_reflector(S* col, int j, int d, S* tau, S* red) {
  using R = RealOf<S>;
  R p0 = 0, p1 = 0;
  int r = j + 1 + threadIdx.x;
  for (; r + FQ_THREADS < d; r += 2 * FQ_THREADS) { p0 += abs2_(col[r]); p1 += abs2_(col[r + FQ_THREADS]); }
  if (r < d) p0 += abs2_(col[r]);
  const R xnorm2 = re_(cta_sum(from_real<S>(p0 + p1), red));
  __shared__ S sc_s;
  if (threadIdx.x == 0) {
    const S alpha = col[j];
    S t = zero_<S>(), beta = alpha, sc = zero_<S>();
    if (!(xnorm2 == (R)0 && im_(alpha) == (R)0)) {
      const R bn = sqrt_(abs2_(alpha) + xnorm2);
      const R b = re_(alpha) >= (R)0 ? -bn : bn;
      beta = from_real<S>(b);
      // one divide: rr = 1 / (beta (alpha - beta)); 1/beta = (alpha - beta) rr, 1/(alpha - beta) = beta rr
      const S amb = sub_(alpha, beta);
      const S rr = recip_(scale_(amb, b));
      t = mul_(sub_(beta, alpha), mul_(amb, rr));
      sc = scale_(rr, b);
    }
    tau[j] = t;
    col[j] = beta;
    sc_s = sc;
  }
  __syncthreads();
  const S sc = sc_s;
  for (int q = j + 1 + threadIdx.x; q < d; q += FQ_THREADS) col[q] = mul_(col[q], sc);
  __syncthreads();
}

template <class S>
__global__ void __launch_bounds__(FQ_THREADS) qr_kernel(S* M, int d, int n, S* tau) {
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x;
  __shared__ S red[FQ_WARPS + 1];
  if (blockIdx.x == 0) cta_reflector(M, 0, d, tau, red);
  grid.sync();
  for (int j = 0; j < n; ++j) {
    const S* v = M + (int64_t)j * d;  // v(j) = 1 implicit, v(r) for r > j stored
    const S tj = tau[j];
    int c = blockIdx.x;
    if (c <= j) c += ((j - c) / G + 1) * G;  // first owned column > j
    for (; c < n; c += G) {
      S* col = M + (int64_t)c * d;
      S a0 = zero_<S>(), a1 = zero_<S>();
      int r = j + 1 + threadIdx.x;
      for (; r + FQ_THREADS < d; r += 2 * FQ_THREADS) {
        a0 = madc_(v[r], col[r], a0);
        a1 = madc_(v[r + FQ_THREADS], col[r + FQ_THREADS], a1);
      }
      if (r < d) a0 = madc_(v[r], col[r], a0);
      S part = add_(a0, a1);
      if (threadIdx.x == 0) part = add_(part, col[j]);   // v(j) = 1
      const S s = cta_sum(part, red);
      const S f = mul_(conj_(tj), s);   // apply H^H = I - conj(tau) v v^H
      if (threadIdx.x == 0) col[j] = sub_(col[j], f);
      for (int q = j + 1 + threadIdx.x; q < d; q += FQ_THREADS) col[q] = sub_(col[q], mul_(v[q], f));
      __syncthreads();
      if (c == j + 1) cta_reflector(col, j + 1, d, tau, red);
    }
    grid.sync();
  }
}

// ------------------------------------------------------------------------------------------
// Dataflow Householder QR (the reflectors of qr_kernel, LAPACK geqr2 convention) for
// d <= 32 * NR * 8 rows. Column c is owned by CTA c % G; row r of every column by thread r % NT
// (NT = blockDim.x, a multiple of 32 with NT * NR >= d), slot r / NT of its registers, so a
// thread only rereads rows of its own columns that it wrote itself. Reflector j is published
// through two flags:
//   ready1[j]: u = column j below the diagonal is in memory (unscaled: v = [1; sc_j u]);
//   ready2[j]: tau_j and sc_j = 1 / (alpha - beta) are in memory.
// A reader starts its dot products u^H x on ready1 and needs tau_j, sc_j only after the
// reduction, so forming reflector j (a norm reduction, a square root, a divide) overlaps the
// readers' loads and reductions. The CTA that owns column j+1 updates it first at step j and
// publishes it at once; the strict lower part of M ends up holding u unscaled (only R is used).
// On GB300 an SM retires about one 32-lane FP64 instruction per 16 cycles, so the cross-thread
// sums and the reflector's scalars run in one warp (or one thread), not redundantly in all.
// Waits are bounded: on timeout the CTA sets DEV_ERR_TIMEOUT and returns.
// ------------------------------------------------------------------------------------------
constexpr long kQrSpin = 1L << 22;
constexpr int kQrMaxThreads = 256;
constexpr int kQrBatch = 2;   // non-critical columns updated per reduction

__device__ __forceinline__ double ldcg_s(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_s(const float* p) { return __ldcg(p); }
__device__ __forceinline__ cd ldcg_s(const cd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cf ldcg_s(const cf* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Release store: orders this thread's earlier writes, and through a preceding __syncthreads()
// those of the whole CTA, before the flag.
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ inline bool qr_poll(const unsigned* flag) {
  for (long it = 0; it < kQrSpin; ++it) {
    if (ld_acquire(flag) != 0u) return true;
    if (it > 32) __nanosleep(32);
  }
  return false;
}

// Called by warp 0 only: sums NV blocks of nt partials (block q at part + q * kQrMaxThreads) in
// a fixed order; the lanes of group q = lane / (32 / NV) all return the total of block q.
template <class S, int NV>
__device__ inline S qr_warp_sum(const S* part, int nt, int lane) {
  constexpr int LPV = 32 / NV;
  const int q = lane / LPV, l = lane % LPV, per = nt / LPV;
  const S* p = part + q * kQrMaxThreads + l * per;
  S a0 = zero_<S>(), a1 = zero_<S>();
  int i = 0;
  for (; i + 1 < per; i += 2) { a0 = add_(a0, p[i]); a1 = add_(a1, p[i + 1]); }
  if (i < per) a0 = add_(a0, p[i]);
  S s = add_(a0, a1);
#pragma unroll
  for (int o = LPV / 2; o > 0; o >>= 1) s = add_(s, shfl_xor_(s, o));
  return s;
}

template <class S>
struct QrShared {
  S part[2][kQrBatch][kQrMaxThreads];   // per-thread partial sums, two phases used alternately
  S xj[2][kQrBatch];                    // x(j) of the reduced columns, or alpha
  S f[kQrBatch], fs[kQrBatch];          // f = conj(tau_j) v^H x and f sc_j
  S tj, scj;
  int stop[2];                          // stage-1 / stage-2 wait outcome
};

// Reflector c of the column held in x (every reflector before c applied): the partial norms go
// through phase ph of the shared buffers; thread 0 writes beta, tau_c, sc_c and sets ready2[c].
template <class S, int NR>
__device__ inline void qr_form(const S (&x)[NR], S* col, int d, int c, S* tau, S* scv, unsigned* ready2,
                               QrShared<S>& sh, int& ph) {
  using R = RealOf<S>;
  const int nt = blockDim.x, tid = threadIdx.x;
  R p = 0;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int r = tid + i * nt;
    if (r > c && r < d) p += abs2_(x[i]);
    if (r == c) sh.xj[ph][0] = x[i];
  }
  sh.part[ph][0][tid] = from_real<S>(p);
  __syncthreads();
  if (tid < 32) {
    const R xnorm2 = re_(qr_warp_sum<S, 1>(sh.part[ph][0], nt, tid));
    if (tid == 0) {
      const S alpha = sh.xj[ph][0];
      S t = zero_<S>(), beta = alpha, sc = zero_<S>();
      if (!(xnorm2 == (R)0 && im_(alpha) == (R)0)) {
        const R bn = sqrt_(abs2_(alpha) + xnorm2);
        const R b = re_(alpha) >= (R)0 ? -bn : bn;
        beta = from_real<S>(b);
        const S amb = sub_(alpha, beta);
        const S rr = recip_(scale_(amb, b));   // 1 / (beta (alpha - beta))
        t = mul_(sub_(beta, alpha), mul_(amb, rr));
        sc = scale_(rr, b);
      }
      col[c] = beta;
      tau[c] = t;
      scv[c] = sc;
      st_release(ready2 + c, 1u);
    }
  }
  ph ^= 1;
}

template <class S, int NR>
__global__ void __launch_bounds__(kQrMaxThreads) qr_flow_kernel(S* M, int d, int n, S* tau, S* scv,
                                                               unsigned* ready, int* err) {
  __shared__ QrShared<S> sh;
  unsigned* ready1 = ready;
  unsigned* ready2 = ready + n;
  const int G = gridDim.x, b0 = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  if (b0 >= n) return;
  const int lastc = b0 + ((n - 1 - b0) / G) * G;
  int ph = 0;
  S u[NR];
  if (b0 == 0) {   // reflector 0: the sketch itself is in memory, so ready1[0] holds at launch
    S x[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int r = tid + i * nt;
      x[i] = r < d ? M[r] : zero_<S>();
    }
    if (tid == 0) st_release(ready1, 1u);
    qr_form<S, NR>(x, M, d, 0, tau, scv, ready2, sh, ph);
  }
  for (int j = 0; j < lastc; ++j) {
    if (tid == 0) {
      const bool ok = qr_poll(ready1 + j);
      sh.stop[0] = ok ? 0 : 1;
      if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
    }
    __syncthreads();
    if (sh.stop[0]) return;
    const S* uj = M + (int64_t)j * d;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int r = tid + i * nt;
      u[i] = (r > j && r < d) ? ldcg_s(uj + r) : zero_<S>();
    }
    bool have_tau = false;
    int c = b0 > j ? b0 : b0 + ((j - b0) / G + 1) * G;   // first owned column > j
    while (c < n) {
      // the next pivot column j+1 alone (it is then published at once), else up to kQrBatch
      const int kb = (c == j + 1) ? 1 : min(kQrBatch, (n - 1 - c) / G + 1);
      S x[kQrBatch][NR];
#pragma unroll
      for (int k = 0; k < kQrBatch; ++k) {
        S a0 = zero_<S>(), a1 = zero_<S>();
        if (k < kb) {
          const S* col = M + (int64_t)(c + k * G) * d;
#pragma unroll
          for (int i = 0; i < NR; ++i) {
            const int r = tid + i * nt;
            x[k][i] = (r >= j && r < d) ? col[r] : zero_<S>();
            if (i & 1) a1 = madc_(u[i], x[k][i], a1);   // conj(u) x
            else a0 = madc_(u[i], x[k][i], a0);
            if (r == j) sh.xj[ph][k] = x[k][i];
          }
        }
        sh.part[ph][k][tid] = add_(a0, a1);
      }
      __syncthreads();
      if (tid < 32) {
        const S s = kb == 1 ? qr_warp_sum<S, 1>(sh.part[ph][0], nt, tid) : qr_warp_sum<S, 2>(sh.part[ph][0], nt, tid);
        if (!have_tau && tid == 0) {
          const bool ok = qr_poll(ready2 + j);
          sh.stop[1] = ok ? 0 : 1;
          if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
          sh.tj = ldcg_s(tau + j);
          sh.scj = ldcg_s(scv + j);
        }
        __syncwarp();
        const int lpv = kb == 1 ? 32 : 16;
        if (tid % lpv == 0) {
          // H_j^H x = x - f v,  f = conj(tau_j) (x(j) + conj(sc_j) u^H x(j+1:)),  v = [1; sc_j u]
          const int q = tid / lpv;
          const S tj = sh.tj, scj = sh.scj;
          const S f = mul_(conj_(tj), add_(sh.xj[ph][q], mul_(conj_(scj), s)));
          sh.f[q] = f;
          sh.fs[q] = mul_(f, scj);
        }
      }
      __syncthreads();
      if (sh.stop[1]) return;
      have_tau = true;
#pragma unroll
      for (int k = 0; k < kQrBatch; ++k) {
        if (k < kb) {
          S* col = M + (int64_t)(c + k * G) * d;
          const S f = sh.f[k], fs = sh.fs[k];
#pragma unroll
          for (int i = 0; i < NR; ++i) {
            const int r = tid + i * nt;
            if (r > j && r < d) {
              x[k][i] = sub_(x[k][i], mul_(fs, u[i]));
              col[r] = x[k][i];
            } else if (r == j) {
              x[k][i] = sub_(x[k][i], f);
              col[r] = x[k][i];
            }
          }
        }
      }
      ph ^= 1;
      if (c == j + 1) {
        __syncthreads();   // every thread's rows of u_{j+1} are stored
        if (tid == 0) st_release(ready1 + c, 1u);
        qr_form<S, NR>(x[0], M + (int64_t)c * d, d, c, tau, scv, ready2, sh, ph);
      }
      c += kb * G;
    }
  }
}

// copy the upper triangle of M (d x n col-major) into R (n x n col-major), zero below
template <class S>
__global__ void extract_r_kernel(const S* M, int d, int n, S* R) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int c = (int)(idx / n), r = (int)(idx % n);
  R[idx] = (r <= c) ? M[(int64_t)c * d + r] : zero_<S>();
}

// R row-major from R column-major (n x n)
template <class S>
__global__ void transpose_kernel(const S* Rc, int n, S* Rr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int r = (int)(idx / n), c = (int)(idx % n);
  Rr[idx] = Rc[(int64_t)c * n + r];
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi SVD (Hestenes; rotation formulas of Demmel & Veselic, SIMAX 1992) on the
// columns of X (n x n col-major), accumulating V (n x n col-major, starts as I). Round-robin
// ordering: in round r of a sweep the N = n + (n odd) slots pair up as (slot 0 fixed, others
// rotated), every pair meeting once per sweep; one warp per pair, a grid barrier per round.
// A sweep without any rotation ends the iteration (or max_sweeps).
// ------------------------------------------------------------------------------------------
__device__ inline int rr_slot(int k, int r, int N) { return k == 0 ? 0 : ((k - 1 + r) % (N - 1)) + 1; }

template <class S>
__device__ void jacobi_pair(S* X, S* V, int n, int p, int q, RealOf<S> tol, RealOf<S> tiny2, int lane,
                            int* changed) {
  using R = RealOf<S>;
  S* xp = X + (int64_t)p * n;
  S* xq = X + (int64_t)q * n;
  R a = 0, b = 0;
  S g = zero_<S>();
  for (int r = lane; r < n; r += 32) {
    const S u = xp[r], w = xq[r];
    a += abs2_(u);
    b += abs2_(w);
    g = madc_(u, w, g);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  // columns at rounding level (||x|| <= n eps max_j ||x_j||) are not rotated: their directions
  // are arbitrary inside the noise subspace, and rotating them would never converge; neither
  // are pairs whose rotation angle is below eps (see jacobi_rotation)
  R c, s;
  S e;
  if (!jacobi_rotation(a, b, g, tol, tiny2, eps_of<S>(), &c, &s, &e)) return;
  const S se = scale_(e, s);                     // s e
  const S sec = conj_(se);                       // s conj(e)
  for (int r = lane; r < n; r += 32) {
    const S u = xp[r], w = xq[r];
    xp[r] = sub_(scale_(u, c), mul_(sec, w));
    xq[r] = add_(mul_(se, u), scale_(w, c));
  }
  S* vp = V + (int64_t)p * n;
  S* vq = V + (int64_t)q * n;
  for (int r = lane; r < n; r += 32) {
    const S u = vp[r], w = vq[r];
    vp[r] = sub_(scale_(u, c), mul_(sec, w));
    vq[r] = add_(mul_(se, u), scale_(w, c));
  }
  if (lane == 0) *changed = 1;
}

template <class S>
__global__ void __launch_bounds__(FQ_THREADS) jacobi_kernel(S* X, S* V, int n, int max_sweeps,
                                                            int* flags, int* sweeps_out, const double* nrm0) {
  cg::grid_group grid = cg::this_grid();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * FQ_WARPS + warp;
  const int NW = gridDim.x * FQ_WARPS;
  const int N = n + (n & 1);
  using R = RealOf<S>;
  // a pair counts as orthogonal when |x_p^H x_q| <= n eps ||x_p|| ||x_q||: the computed cosine
  // carries about n u of rounding noise, so a tighter test would never be met and every sweep
  // would rotate noise
  const R tol = (R)n * eps_of<S>();
  // rounding-level threshold from the initial column norms (computed before the launch)
  double mx = 0;
  for (int j = 0; j < n; ++j) mx = fmax(mx, nrm0[j]);
  const R tiny = (R)(mx * (double)n * (double)eps_of<S>());
  const R tiny2 = tiny * tiny;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[(sweep + 1) % 3] = 0;
    int* changed = flags + (sweep % 3);
    for (int r = 0; r < N - 1; ++r) {
      for (int i = gw; i < N / 2; i += NW) {
        int p = rr_slot(i, r, N), q = rr_slot(N - 1 - i, r, N);
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= n) continue;  // dummy slot of an odd n
        jacobi_pair(X, V, n, p, q, tol, tiny2, lane, changed);
      }
      grid.sync();
    }
    const bool done = (*(volatile int*)changed) == 0;
    if (done) { ++sweep; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep;
}

template <class S>
__global__ void set_identity_kernel(S* V, int n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int c = (int)(idx / n), r = (int)(idx % n);
  V[idx] = (r == c) ? from_real<S>((RealOf<S>)1) : zero_<S>();
}

// column norms of X (one warp per column): sigma_j = ||x_j||
template <class S>
__global__ void colnorm_kernel(const S* X, int n, double* nrm) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const S* x = X + (int64_t)warp * n;
  RealOf<S> a = 0;
  for (int r = lane; r < n; r += 32) a += abs2_(x[r]);
  a = warp_sum(a);
  if (lane == 0) nrm[warp] = (double)sqrt_(a);
}

// sort descending (stable in column index) and permute V's columns accordingly
template <class S>
__global__ void sort_svd_kernel(const double* nrm, const S* V, int n, double* sigma, S* Vt) {
  const int j = blockIdx.x;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double sj = nrm[j];
  int local = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = nrm[i];
    local += (si > sj) || (si == sj && i < j);
  }
  atomicAdd(&cnt, local);
  __syncthreads();
  const int rank = cnt;
  if (threadIdx.x == 0) sigma[rank] = sj;
  for (int r = threadIdx.x; r < n; r += blockDim.x) Vt[(int64_t)rank * n + r] = V[(int64_t)j * n + r];
}

// ------------------------------------------------------------------------------------------
// Triangular inverse X = R^{-1} (R upper, n x n col-major): one CTA per column j of X,
// backward column sweep x(l) = acc(l) / R(l,l); acc(0:l) -= R(0:l, l) x(l).
// An exactly zero pivot is replaced by eps * max|R(i,i)| (R from a rank-deficient sketch).
// Writes X both row-major (Xr) and column-major (Xc).
// ------------------------------------------------------------------------------------------
template <class S>
__global__ void trinv_kernel(const S* Rm, int n, S* Xr, S* Xc) {
  using Rl = RealOf<S>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* acc = reinterpret_cast<S*>(smem_raw);   // n entries, then n pivot reciprocals
  S* rdiag = acc + n;
  __shared__ Rl red[32];
  const int j = blockIdx.x;
  // max |R_ii| (parallel), the floor for zero pivots, and the pivot reciprocals 1/R_ll, l <= j,
  // all before the dependent back substitution
  Rl mx = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, sqrt_(abs2_(Rm[(int64_t)i * n + i])));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) acc[i] = (i == j) ? from_real<S>((Rl)1) : zero_<S>();
  __syncthreads();
  mx = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  const Rl floor_ = eps_of<S>() * mx;
  for (int l = threadIdx.x; l <= j; l += blockDim.x) {
    S piv = Rm[(int64_t)l * n + l];
    if (abs2_(piv) == (Rl)0) piv = from_real<S>(floor_ > (Rl)0 ? floor_ : (Rl)1);
    rdiag[l] = recip_(piv);
  }
  __syncthreads();
  for (int l = j; l >= 0; --l) {
    if (threadIdx.x == 0) acc[l] = mul_(acc[l], rdiag[l]);
    __syncthreads();
    const S xl = acc[l];
    const S* col = Rm + (int64_t)l * n;
    for (int i = threadIdx.x; i < l; i += blockDim.x) acc[i] = sub_(acc[i], mul_(col[i], xl));
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const S v = (i <= j) ? acc[i] : zero_<S>();
    Xc[(int64_t)j * n + i] = v;
    Xr[(int64_t)i * n + j] = v;
  }
}

template <class K>
int coop_grid(K kernel, int threads, size_t smem, int* grid) {
  int per_sm = 0;
  RL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  if (per_sm < 1) return RLOBPCG_ERR_UNSUPPORTED;
  *grid = num_sms();   // one CTA per SM: measured faster than two (cheaper grid barriers)
  return RLOBPCG_OK;
}

}  // namespace

// workspace: tau (n), sc (n), X copy (n*n), V (n*n), norms (n doubles), flags (4 ints),
// reflector ready flags (2n)
size_t factor_workspace_bytes(int64_t d, int64_t n, size_t esz) {
  (void)d;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  add(n * esz);
  add(n * esz);
  add(n * n * esz);
  add(n * n * esz);
  add(n * sizeof(double));
  add(4 * sizeof(int));
  add(2 * n * sizeof(unsigned));
  return b;
}

template <class S, int NR>
int qr_flow_launch(S* SA, int d, int n, S* tau, S* scv, unsigned* ready, int* err, cudaStream_t st) {
  const int nt = 32 * ((d + 32 * NR - 1) / (32 * NR));   // NT * NR >= d, fewer than 32 * NR idle rows
  int per_sm = 0;
  RL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_flow_kernel<S, NR>, nt, 0));
  if (per_sm < 1) return RLOBPCG_ERR_UNSUPPORTED;
  // two CTAs per SM measured faster than one (a CTA's backlog of non-pivot columns no longer
  // delays its next pivot) and than more (the SM's FP64 pipe is shared)
  const int G = (int)min((int64_t)min(per_sm, 2) * num_sms(), (int64_t)n);
  RL_CUDA(cudaMemsetAsync(ready, 0, (size_t)2 * n * sizeof(unsigned), st));
  void* args[] = {(void*)&SA, (void*)&d, (void*)&n, (void*)&tau, (void*)&scv, (void*)&ready, (void*)&err};
  RL_CUDA(cudaLaunchCooperativeKernel((void*)qr_flow_kernel<S, NR>, dim3(G), dim3(nt), args, 0, st));
  note_launch();
  return RLOBPCG_OK;
}

namespace {
// Pointers of the factor workspace (layout of factor_workspace_bytes)
template <class S>
struct FactorWs {
  S *tau, *scv, *X, *V;
  double* nrm;
  int* flags;
  unsigned* ready;
  FactorWs(void* work, int n) {
    unsigned char* p = (unsigned char*)work;
    auto take = [&](size_t x) { void* r = p; p += (x + 255) & ~(size_t)255; return r; };
    tau = (S*)take((size_t)n * sizeof(S));
    scv = (S*)take((size_t)n * sizeof(S));
    X = (S*)take((size_t)n * n * sizeof(S));
    V = (S*)take((size_t)n * n * sizeof(S));
    nrm = (double*)take((size_t)n * sizeof(double));
    flags = (int*)take(4 * sizeof(int));
    ready = (unsigned*)take((size_t)2 * n * sizeof(unsigned));
  }
};
}  // namespace

// Householder QR of SA (d x n col-major, overwritten); R (n x n col-major, zero below the
// diagonal) is left in the workspace's X (factor_r_of). err: device word that receives
// DEV_ERR_TIMEOUT if a bounded wait of the QR runs out.
template <class S>
int factor_qr(S* SA, int d, int n, void* work, size_t work_bytes, cudaStream_t st, int* err) {
  if (work_bytes < factor_workspace_bytes(d, n, sizeof(S)) || !err) return RLOBPCG_ERR_INVALID_ARG;
  FactorWs<S> w(work, n);
  // the dataflow kernel holds each thread's rows of a column in registers (d <= 4096); taller
  // sketches take the kernel with one grid barrier per column
  int G = 0, rc = 0;
  if (d <= 8 * kQrMaxThreads) {
    RL_TRY((qr_flow_launch<S, 8>(SA, d, n, w.tau, w.scv, w.ready, err, st)));
  } else if (d <= 16 * kQrMaxThreads) {
    RL_TRY((qr_flow_launch<S, 16>(SA, d, n, w.tau, w.scv, w.ready, err, st)));
  } else {
    rc = coop_grid(qr_kernel<S>, FQ_THREADS, 0, &G);
    if (rc) return rc;
    G = min(G, max(1, n));
    void* args[] = {(void*)&SA, (void*)&d, (void*)&n, (void*)&w.tau};
    RL_CUDA(cudaLaunchCooperativeKernel((void*)qr_kernel<S>, dim3(G), dim3(FQ_THREADS), args, 0, st));
    note_launch();
  }
  const int64_t nn = (int64_t)n * n;
  const int eb = 256, eg = (int)((nn + eb - 1) / eb);
  extract_r_kernel<S><<<eg, eb, 0, st>>>(SA, d, n, w.X);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

// X = R^{-1} for an upper-triangular R (n x n col-major), row- and column-major outputs.
template <class S>
int trinv_launch(const S* R, int n, S* Xr, S* Xc, cudaStream_t st) {
  const size_t sm = (size_t)2 * n * sizeof(S);
  RL_TRY(allow_dynamic_smem(trinv_kernel<S>, sm));
  trinv_kernel<S><<<n, 256, sm, st>>>(R, n, Xr, Xc);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

// Where factor_qr leaves R, and where factor_post reads it (the workspace's X).
template <class S>
S* factor_r_of(void* work, int n) { return FactorWs<S>(work, n).X; }

// From R in the workspace's X (n x n col-major, consumed): copies of R (col- and row-major),
// R^{-1} (row- and col-major), and the one-sided Jacobi SVD of R (sigma descending, V~).
template <class S>
int factor_post(int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c, void* work, cudaStream_t st,
                int* sweeps_host, bool do_svd) {
  FactorWs<S> w(work, n);
  S* X = w.X;
  const int64_t nn = (int64_t)n * n;
  const int eb = 256, eg = (int)((nn + eb - 1) / eb);
  if (Rout) RL_CUDA(cudaMemcpyAsync(Rout, X, nn * sizeof(S), cudaMemcpyDeviceToDevice, st));
  if (Rout_r) {
    transpose_kernel<S><<<eg, eb, 0, st>>>(X, n, Rout_r);
    RL_CHECK_LAUNCH();
  }
  // R^{-1} (before Jacobi overwrites X)
  if (Rinv_r && Rinv_c) {
    size_t sm = (size_t)2 * n * sizeof(S);
    RL_TRY(allow_dynamic_smem(trinv_kernel<S>, sm));
    trinv_kernel<S><<<n, 256, sm, st>>>(X, n, Rinv_r, Rinv_c);
    RL_CHECK_LAUNCH();
  }
  if (!do_svd) {
    if (sweeps_host) *sweeps_host = 0;
    return RLOBPCG_OK;
  }
  // Jacobi SVD of R
  set_identity_kernel<S><<<eg, eb, 0, st>>>(w.V, n);
  RL_CHECK_LAUNCH();
  RL_CUDA(cudaMemsetAsync(w.flags, 0, 4 * sizeof(int), st));
  int G = 0;
  const int rc = coop_grid(jacobi_kernel<S>, FQ_THREADS, 0, &G);
  if (rc) return rc;
  G = min(G, max(1, (n / 2 + FQ_WARPS - 1) / FQ_WARPS));
  int max_sweeps = 40;
  int* sweeps_dev = w.flags + 3;
  colnorm_kernel<S><<<(n * 32 + 255) / 256, 256, 0, st>>>(X, n, w.nrm);
  RL_CHECK_LAUNCH();
  {
    const double* nrm0 = w.nrm;
    S* V = w.V;
    int* flags = w.flags;
    void* args[] = {(void*)&X, (void*)&V, (void*)&n, (void*)&max_sweeps, (void*)&flags, (void*)&sweeps_dev,
                    (void*)&nrm0};
    RL_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_kernel<S>, dim3(G), dim3(FQ_THREADS), args, 0, st));
    note_launch();
  }
  colnorm_kernel<S><<<(n * 32 + 255) / 256, 256, 0, st>>>(X, n, w.nrm);
  RL_CHECK_LAUNCH();
  sort_svd_kernel<S><<<n, 256, 0, st>>>(w.nrm, w.V, n, sigma, Vt);
  RL_CHECK_LAUNCH();
  if (sweeps_host) RL_CUDA(cudaMemcpyAsync(sweeps_host, sweeps_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  return RLOBPCG_OK;
}

// The factorisation step of Alg. 2: QR of SA, then R, R^{-1} and (optionally) the SVD of R.
template <class S>
int factor_impl(S* SA, int d, int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c,
                void* work, size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err) {
  RL_TRY(factor_qr<S>(SA, d, n, work, work_bytes, st, err));
  return factor_post<S>(n, Rout, Rout_r, sigma, Vt, Rinv_r, Rinv_c, work, st, sweeps_host, do_svd);
}

template int factor_impl<double>(double*, int, int, double*, double*, double*, double*, double*, double*, void*, size_t, cudaStream_t, int*, bool, int*);
template int factor_impl<float>(float*, int, int, float*, float*, double*, float*, float*, float*, void*, size_t, cudaStream_t, int*, bool, int*);
template int factor_impl<cd>(cd*, int, int, cd*, cd*, double*, cd*, cd*, cd*, void*, size_t, cudaStream_t, int*, bool, int*);
template int factor_impl<cf>(cf*, int, int, cf*, cf*, double*, cf*, cf*, cf*, void*, size_t, cudaStream_t, int*, bool, int*);
template int factor_qr<float>(float*, int, int, void*, size_t, cudaStream_t, int*);
template int factor_qr<cf>(cf*, int, int, void*, size_t, cudaStream_t, int*);
template int trinv_launch<double>(const double*, int, double*, double*, cudaStream_t);
template int trinv_launch<cd>(const cd*, int, cd*, cd*, cudaStream_t);
template float* factor_r_of<float>(void*, int);
template cf* factor_r_of<cf>(void*, int);
template double* factor_r_of<double>(void*, int);
template cd* factor_r_of<cd>(void*, int);
template int factor_post<double>(int, double*, double*, double*, double*, double*, double*, void*, cudaStream_t, int*, bool);
template int factor_post<cd>(int, cd*, cd*, double*, cd*, cd*, cd*, void*, cudaStream_t, int*, bool);

}  // namespace rl
