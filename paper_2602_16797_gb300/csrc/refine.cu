// The FP32 factor of the sketch, corrected once in FP64 (sketch precision
// RLOBPCG_SKETCH_F32_REFINE).
//
// The preconditioner of Alg. 2 (arXiv 2602.16797) is P = V~ Sigma~^{-1}, P P^* = (R^H R)^{-1} for
// a QR factor R of the sketch SA (footnote of Sec. 1). The paper's point that P only has to be
// well conditioned (Fact 2, Sec. 3.1) invites a single-precision factor, but an FP32 QR perturbs
// SA by about u_32 ||SA||: when kappa(A) >> 1 / u_32 the FP32 factor R_32 cannot see the bottom
// singular directions, kappa(SA R_32^{-1}) grows to about u_32 kappa(SA), and the LOBPCG
// iteration slows. One Cholesky-QR step in FP64 removes that error (a preconditioned Cholesky QR):
//     Y   = SA M,  M = R_32^{-1}        (SA in FP64: the sketch keeps its FP64 information)
//     H   = Y^H Y + s I,  s = n u max_i H_ii      (kappa(Y) ~ u_32 kappa(SA), so H is far
//                                                  from singular in FP64; the shift covers an
//                                                  exactly rank-deficient SA)
//     R_c = chol(H)  (H = R_c^H R_c, upper),   R = R_c R_32.
// Then SA R^{-1} = Y R_c^{-1} is orthonormal to O(u kappa(Y)^2), i.e. R is an FP64-quality QR
// factor of SA, and everything downstream (R^{-1}, the SVD of R, the start block) is the plain
// form's. FP64 work: d n^2 (Y) + d n^2 (upper half of H) + n^3 / 3 flops.
#include "common.cuh"

namespace rl {

size_t factor_workspace_bytes(int64_t d, int64_t n, size_t esz);
template <class S>
int factor_qr(S* SA, int d, int n, void* work, size_t work_bytes, cudaStream_t st, int* err);
template <class S>
S* factor_r_of(void* work, int n);
template <class S>
int factor_post(int n, S* Rout, S* Rout_r, double* sigma, S* Vt, S* Rinv_r, S* Rinv_c, void* work, cudaStream_t st,
                int* sweeps_host, bool do_svd);
template <class S>
int trinv_launch(const S* R, int n, S* Xr, S* Xc, cudaStream_t st);

namespace {

template <class T> struct Low;   // the FP32 type of an FP64 working type
template <> struct Low<double> { using type = float; };
template <> struct Low<cd> { using type = cf; };

template <class O, class I>
__global__ void convert_kernel(const I* __restrict__ x, O* __restrict__ y, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cvt_<O, I>(x[i]);
}

// ---------------------------------------------------------------------------------------------
// C = alpha op(A) B + beta C, all column-major; op(A) = A (M x K, lda) or A^H (A is K x M, lda).
// 64 x 64 tiles, 256 threads, 4 x 4 outputs per thread (rows tx + 16 r, columns ty + 16 c), K
// slices through shared memory. Triangular operands shrink the K range of a tile: a_upper (op(A)
// upper triangular: k >= i), b_upper (B upper triangular: k <= j). c_upper: only the upper
// triangle of C (i <= j) is computed and written.
// ---------------------------------------------------------------------------------------------
constexpr int GT = 64;
template <class T> constexpr int gbk() { return sizeof(T) == 8 ? 16 : 8; }

template <class T, bool CONJ_A>
__global__ void __launch_bounds__(256) gemm_kernel(const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                                                   int64_t ldb, T* __restrict__ C, int64_t ldc, int M, int N, int K,
                                                   int a_upper, int b_upper, int c_upper, double alpha, int beta) {
  constexpr int BK = gbk<T>();
  __shared__ T As[BK][GT + 1];
  __shared__ T Bs[BK][GT + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (c_upper && i0 > j0 + GT - 1) return;
  const int klo = a_upper ? i0 : 0;
  const int khi = b_upper ? imin(K, j0 + GT) : K;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = zero_<T>();
  for (int k0 = klo; k0 < khi; k0 += BK) {
    for (int e = tid; e < GT * BK; e += 256) {
      int ii, kk;
      if (CONJ_A) { kk = e % BK; ii = e / BK; } else { ii = e % GT; kk = e / GT; }
      const int i = i0 + ii, k = k0 + kk;
      T v = zero_<T>();
      if (i < M && k < khi) v = CONJ_A ? conj_(A[(int64_t)i * lda + k]) : A[(int64_t)k * lda + i];
      As[kk][ii] = v;
    }
    for (int e = tid; e < GT * BK; e += 256) {
      const int kk = e % BK, jj = e / BK;
      const int j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < N && k < khi) ? B[(int64_t)j * ldb + k] : zero_<T>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = mad_(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
      if (i < M && j < N && (!c_upper || i <= j)) {
        T v = scale_(acc[r][c], (RealOf<T>)alpha);
        if (beta) v = add_(v, C[(int64_t)j * ldc + i]);
        C[(int64_t)j * ldc + i] = v;
      }
    }
}

template <class T, bool CONJ_A>
int gemm_launch(const T* A, int64_t lda, const T* B, int64_t ldb, T* C, int64_t ldc, int M, int N, int K, int a_upper,
                int b_upper, int c_upper, double alpha, int beta, cudaStream_t st) {
  if (M <= 0 || N <= 0) return RLOBPCG_OK;
  const dim3 grid((unsigned)((M + GT - 1) / GT), (unsigned)((N + GT - 1) / GT));
  gemm_kernel<T, CONJ_A><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, a_upper, b_upper, c_upper, alpha, beta);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

// ---------------------------------------------------------------------------------------------
// Shifted Cholesky H = R^H R (R upper), in place on the upper triangle of H (n x n col-major),
// blocked right-looking with 64-column panels: the diagonal block (one CTA), the panel row
// R[k:k+nb, k+nb:] = R_kk^{-H} H[k:k+nb, k+nb:] (a CTA per four columns), the trailing update
// H[k+nb:, k+nb:] -= R[k:k+nb, k+nb:]^H R[k:k+nb, k+nb:] (upper triangle, the tiled GEMM).
// ---------------------------------------------------------------------------------------------
template <class T> constexpr int cbk() { return sizeof(T) == 8 ? 64 : 32; }   // panel width (static smem)

// s = n u max_i Re H_ii (written to *shift) and H_ii += s
template <class T>
__global__ void shift_kernel(T* H, int n, double* shift) {
  __shared__ double red[32];
  double mx = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, re_(H[(int64_t)i * n + i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  const double s = (double)n * ldexp(1.0, -53) * mx;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) H[(int64_t)i * n + i] = add_(H[(int64_t)i * n + i], from_real<T>(s));
  if (threadIdx.x == 0) *shift = s;
}

// Unblocked Cholesky of the nb x nb diagonal block at (k, k). A pivot that is not positive after
// the shift (rounding in an exactly singular H) is replaced by the shift itself and counted.
template <class T>
__global__ void __launch_bounds__(256) chol_diag_kernel(T* H, int n, int k, int nb, const double* shift, int* clamped) {
  constexpr int CB = cbk<T>();
  __shared__ T Bk[CB][CB + 1];   // Bk[col][row]
  __shared__ double piv_s;
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    Bk[c][r] = r <= c ? H[(int64_t)(k + c) * n + k + r] : zero_<T>();
  }
  __syncthreads();
  const double s = *shift > 0 ? *shift : 1.0;
  for (int l = 0; l < nb; ++l) {
    if (tid == 0) {
      double p = re_(Bk[l][l]);
      if (!(p > 0)) {
        p = s;
        atomicAdd(clamped, 1);
      }
      piv_s = sqrt(p);
      Bk[l][l] = from_real<T>(piv_s);
    }
    __syncthreads();
    const double inv = 1.0 / piv_s;
    for (int j = l + 1 + tid; j < nb; j += blockDim.x) Bk[j][l] = scale_(Bk[j][l], inv);   // row l of R
    __syncthreads();
    // trailing: B[i][j] -= conj(R[l][i]) R[l][j], l < i <= j
    for (int e = tid; e < (nb - l - 1) * (nb - l - 1); e += blockDim.x) {
      const int i = l + 1 + e / (nb - l - 1), j = l + 1 + e % (nb - l - 1);
      if (i <= j) Bk[j][i] = sub_(Bk[j][i], mul_(conj_(Bk[i][l]), Bk[j][l]));
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, r = e % nb;
    H[(int64_t)(k + c) * n + k + r] = r <= c ? Bk[c][r] : zero_<T>();
  }
}

// Panel row: for each column j >= k + nb, x = H[k:k+nb, j] solved from R_kk^H x = h (forward
// substitution; R_kk^H is lower triangular with entries conj(R_kk[p][l])). 256 threads =
// 256 / CB columns x CB rows.
template <class T>
__global__ void __launch_bounds__(256) chol_panel_kernel(T* H, int n, int k, int nb) {
  constexpr int CB = cbk<T>(), NQ = 256 / CB;
  __shared__ T Rk[CB][CB + 1];   // Rk[col][row] of the factored diagonal block
  __shared__ T X[NQ][CB];
  const int tid = threadIdx.x, q = tid % NQ, r = tid / NQ;
  const int j = k + nb + blockIdx.x * NQ + q;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int c = e / nb, rr = e % nb;
    Rk[c][rr] = H[(int64_t)(k + c) * n + k + rr];
  }
  if (r < nb) X[q][r] = j < n ? H[(int64_t)j * n + k + r] : zero_<T>();
  __syncthreads();
  for (int l = 0; l < nb; ++l) {
    if (r == l) X[q][l] = scale_(X[q][l], 1.0 / re_(Rk[l][l]));
    __syncthreads();
    if (r > l && r < nb) X[q][r] = sub_(X[q][r], mul_(conj_(Rk[r][l]), X[q][l]));
    __syncthreads();
  }
  if (r < nb && j < n) H[(int64_t)j * n + k + r] = X[q][r];
}

template <class T>
__global__ void zero_lower_kernel(T* R, int n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int c = (int)(idx / n), r = (int)(idx % n);
  if (r > c) R[idx] = zero_<T>();
}

template <class T>
int chol_upper(T* H, int n, double* shift, int* clamped, cudaStream_t st) {
  shift_kernel<T><<<1, 1024, 0, st>>>(H, n, shift);
  RL_CHECK_LAUNCH();
  constexpr int CB = cbk<T>(), NQ = 256 / CB;
  for (int k = 0; k < n; k += CB) {
    const int nb = imin(CB, n - k);
    chol_diag_kernel<T><<<1, 256, 0, st>>>(H, n, k, nb, shift, clamped);
    RL_CHECK_LAUNCH();
    const int rest = n - k - nb;
    if (rest <= 0) break;
    chol_panel_kernel<T><<<(rest + NQ - 1) / NQ, 256, 0, st>>>(H, n, k, nb);
    RL_CHECK_LAUNCH();
    T* P = H + (int64_t)(k + nb) * n + k;   // R[k:k+nb, k+nb:], nb x rest, ld n
    T* Ct = H + (int64_t)(k + nb) * n + k + nb;
    RL_TRY((gemm_launch<T, true>(P, n, P, n, Ct, n, rest, rest, nb, 0, 0, 1, -1.0, 1, st)));
  }
  const int64_t nn = (int64_t)n * n;
  zero_lower_kernel<T><<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(H, n);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class T>
struct RefineWs {
  using Tf = typename Low<T>::type;
  void* f64;        // factor workspace of T (R ends in its X for factor_post)
  void* f32;        // factor workspace of Tf (the FP32 QR)
  Tf* SA32;         // d x n
  T *R32, *M, *Mr, *Y, *H;
  double* shift;
  int* clamped;
  size_t total;
  RefineWs(void* base, int64_t d, int64_t n) {
    unsigned char* p = (unsigned char*)base;
    size_t off = 0;
    auto take = [&](size_t x) { void* r = p ? (void*)(p + off) : nullptr; off += a256(x); return r; };
    f64 = take(factor_workspace_bytes(d, n, sizeof(T)));
    f32 = take(factor_workspace_bytes(d, n, sizeof(Tf)));
    SA32 = (Tf*)take((size_t)d * n * sizeof(Tf));
    R32 = (T*)take((size_t)n * n * sizeof(T));
    M = (T*)take((size_t)n * n * sizeof(T));
    Mr = (T*)take((size_t)n * n * sizeof(T));
    Y = (T*)take((size_t)d * n * sizeof(T));
    H = (T*)take((size_t)n * n * sizeof(T));
    shift = (double*)take(sizeof(double));
    clamped = (int*)take(sizeof(int));
    total = off;
  }
};

}  // namespace

size_t refine_workspace_bytes(int64_t d, int64_t n, int dtype) {
  return dtype == RLOBPCG_C128 ? RefineWs<cd>(nullptr, d, n).total : RefineWs<double>(nullptr, d, n).total;
}

// SA: d x n col-major FP64 (or complex128) sketch, consumed. Outputs as factor_impl (all FP64).
template <class T>
int factor_refine_impl(T* SA, int d, int n, T* Rout, T* Rout_r, double* sigma, T* Vt, T* Rinv_r, T* Rinv_c,
                       void* work, size_t work_bytes, cudaStream_t st, int* sweeps_host, bool do_svd, int* err) {
  using Tf = typename Low<T>::type;
  RefineWs<T> w(work, d, n);
  if (work_bytes < w.total || !err) return RLOBPCG_ERR_INVALID_ARG;
  const int64_t dn = (int64_t)d * n, nn = (int64_t)n * n;
  const unsigned cg = (unsigned)imin<int64_t>((dn + 255) / 256, 65535);
  RL_CUDA(cudaMemsetAsync(w.clamped, 0, sizeof(int), st));
  // FP32 QR of the rounded sketch
  convert_kernel<Tf, T><<<cg, 256, 0, st>>>(SA, w.SA32, dn);
  RL_CHECK_LAUNCH();
  RL_TRY(factor_qr<Tf>(w.SA32, d, n, w.f32, factor_workspace_bytes(d, n, sizeof(Tf)), st, err));
  const Tf* R32f = factor_r_of<Tf>(w.f32, n);
  convert_kernel<T, Tf><<<(unsigned)imin<int64_t>((nn + 255) / 256, 65535), 256, 0, st>>>(R32f, w.R32, nn);
  RL_CHECK_LAUNCH();
  // M = R_32^{-1} in FP64, Y = SA M, H = Y^H Y (upper), R_c = chol(H + s I)
  RL_TRY(trinv_launch<T>(w.R32, n, w.Mr, w.M, st));
  RL_TRY((gemm_launch<T, false>(SA, d, w.M, n, w.Y, d, d, n, n, 0, 1, 0, 1.0, 0, st)));
  RL_TRY((gemm_launch<T, true>(w.Y, d, w.Y, d, w.H, n, n, n, d, 0, 0, 1, 1.0, 0, st)));
  RL_TRY(chol_upper<T>(w.H, n, w.shift, w.clamped, st));
  // R = R_c R_32 into the FP64 factor workspace, then the plain form's post-processing
  T* X = factor_r_of<T>(w.f64, n);
  RL_TRY((gemm_launch<T, false>(w.H, n, w.R32, n, X, n, n, n, n, 1, 1, 0, 1.0, 0, st)));
  return factor_post<T>(n, Rout, Rout_r, sigma, Vt, Rinv_r, Rinv_c, w.f64, st, sweeps_host, do_svd);
}

template int factor_refine_impl<double>(double*, int, int, double*, double*, double*, double*, double*, double*, void*,
                                        size_t, cudaStream_t, int*, bool, int*);
template int factor_refine_impl<cd>(cd*, int, int, cd*, cd*, double*, cd*, cd*, cd*, void*, size_t, cudaStream_t, int*,
                                    bool, int*);

}  // namespace rl
