// Factorisation of the sketch (Alg. 2, second and third lines of arXiv 2602.16797):
//   1. Householder QR  SA = QR  (the QR route that the footnote in Sec. 1 names as the usual one);
//   2. one-sided Jacobi SVD  R = U~ Sigma~ V~^H  (SVD(SA) = SVD(R): same Sigma~ and V~);
//   3. R^{-1}, so that the preconditioner P P^* = V~ Sigma~^{-2} V~^H = (R^H R)^{-1} is applied
//      as two triangular products.
// All three run in the sketch precision S (float/cf in the mixed form, double/cd otherwise).
//
// GB300 mapping: QR and Jacobi are persistent cooperative kernels (one launch each, grid-wide
// barriers between the dependent steps) with one warp per column (QR) or per column pair
// (Jacobi); the matrices stay L2-resident (n <= a few thousand). R^{-1} uses one CTA per column.
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

// 1 / z
__device__ inline double recip_(double a) { return 1.0 / a; }
__device__ inline float recip_(float a) { return 1.0f / a; }
__device__ inline cd recip_(cd a) { double s = a.x * a.x + a.y * a.y; return {a.x / s, -a.y / s}; }
__device__ inline cf recip_(cf a) { float s = a.x * a.x + a.y * a.y; return {a.x / s, -a.y / s}; }

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

// workspace: tau (n), X copy (n*n), V (n*n), norms (n doubles), flags (4 ints)
size_t factor_workspace_bytes(int64_t d, int64_t n, size_t esz) {
  (void)d;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
  add(n * esz);
  add(n * n * esz);
  add(n * n * esz);
  add(n * sizeof(double));
  add(4 * sizeof(int));
  return b;
}

// Rout (col-major) and Rout_r (row-major) are optional copies of R; with do_svd == false the
// Jacobi SVD (sigma, Vt) is skipped.
template <class S>
int factor_impl(S* SA, int d, int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c,
                void* work, size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd) {
  if (work_bytes < factor_workspace_bytes(d, n, sizeof(S))) return RLOBPCG_ERR_INVALID_ARG;
  unsigned char* p = (unsigned char*)work;
  auto take = [&](size_t x) { void* r = p; p += (x + 255) & ~(size_t)255; return r; };
  S* tau = (S*)take((size_t)n * sizeof(S));
  S* X = (S*)take((size_t)n * n * sizeof(S));
  S* V = (S*)take((size_t)n * n * sizeof(S));
  double* nrm = (double*)take((size_t)n * sizeof(double));
  int* flags = (int*)take(4 * sizeof(int));

  // 1. Householder QR
  int G = 0;
  int rc = coop_grid(qr_kernel<S>, FQ_THREADS, 0, &G);
  if (rc) return rc;
  G = min(G, max(1, n));
  {
    void* args[] = {(void*)&SA, (void*)&d, (void*)&n, (void*)&tau};
    RL_CUDA(cudaLaunchCooperativeKernel((void*)qr_kernel<S>, dim3(G), dim3(FQ_THREADS), args, 0, st));
    note_launch();
  }
  const int64_t nn = (int64_t)n * n;
  const int eb = 256, eg = (int)((nn + eb - 1) / eb);
  extract_r_kernel<S><<<eg, eb, 0, st>>>(SA, d, n, X);
  RL_CHECK_LAUNCH();
  if (Rout) RL_CUDA(cudaMemcpyAsync(Rout, X, nn * sizeof(S), cudaMemcpyDeviceToDevice, st));
  if (Rout_r) {
    transpose_kernel<S><<<eg, eb, 0, st>>>(X, n, Rout_r);
    RL_CHECK_LAUNCH();
  }

  // 3. R^{-1} (before Jacobi overwrites X)
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
  // 2. Jacobi SVD of R
  set_identity_kernel<S><<<eg, eb, 0, st>>>(V, n);
  RL_CHECK_LAUNCH();
  RL_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  rc = coop_grid(jacobi_kernel<S>, FQ_THREADS, 0, &G);
  if (rc) return rc;
  G = min(G, max(1, (n / 2 + FQ_WARPS - 1) / FQ_WARPS));
  int max_sweeps = 40;
  int* sweeps_dev = flags + 3;
  colnorm_kernel<S><<<(n * 32 + 255) / 256, 256, 0, st>>>(X, n, nrm);
  RL_CHECK_LAUNCH();
  {
    const double* nrm0 = nrm;
    void* args[] = {(void*)&X, (void*)&V, (void*)&n, (void*)&max_sweeps, (void*)&flags, (void*)&sweeps_dev,
                    (void*)&nrm0};
    RL_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_kernel<S>, dim3(G), dim3(FQ_THREADS), args, 0, st));
    note_launch();
  }
  colnorm_kernel<S><<<(n * 32 + 255) / 256, 256, 0, st>>>(X, n, nrm);
  RL_CHECK_LAUNCH();
  sort_svd_kernel<S><<<n, 256, 0, st>>>(nrm, V, n, sigma, Vt);
  RL_CHECK_LAUNCH();
  if (sweeps_host) RL_CUDA(cudaMemcpyAsync(sweeps_host, sweeps_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  return RLOBPCG_OK;
}

template int factor_impl<double>(double*, int, int, double*, double*, double*, double*, double*, double*, void*, size_t, cudaStream_t, int*, bool);
template int factor_impl<float>(float*, int, int, float*, float*, double*, float*, float*, float*, void*, size_t, cudaStream_t, int*, bool);
template int factor_impl<cd>(cd*, int, int, cd*, cd*, double*, cd*, cd*, cd*, void*, size_t, cudaStream_t, int*, bool);
template int factor_impl<cf>(cf*, int, int, cf*, cf*, double*, cf*, cf*, cf*, void*, size_t, cudaStream_t, int*, bool);

}  // namespace rl
