// The per-iteration kernels around the Gram pass (Alg. 2 of arXiv 2602.16797):
//   * TSQR: R factor of A_T = [A_V A_W A_X] (m x c) -- Rayleigh-Ritz needs SVD(A_T), and
//     SVD(A_T) = SVD(R_T) on the right, without ever forming A_T^H A_T (which would square the
//     condition number and wipe out sigma ~ 1e-10 ||A||).
//   * rr_small: one-sided Jacobi SVD of R_T (c x c), Theta descending, and the coefficient block
//     K = [C_s | C(:, 1:c-b) Q] with Q = Orth(C(1:b, 1:c-b)^H) (the x-trick of Sec. 2.1).
//   * update: [V X] <- T K, [A_V A_X] <- A_T K, [G_V G_X] <- G_T K in place, row by row.
//   * residual: R = G_V - V Theta_s^2, its column norms, and R / ||R(:,j)|| in the sketch
//     precision for the preconditioner.
//   * precondition: W = R^{-1} (R^{-H} R~) (= P P^* R~ with P = V~ Sigma~^{-1}).
//   * bcgs2_orth: W <- W - [V X]([V X]^H W) twice, then Orth(W) (thin Householder Q with
//     diag(R) real non-negative).
// State layout: T, A_T and G_T are row-major with leading dimension 3b and column blocks
// [V | W | X] (X absent, i.e. c = 2b, in iteration 0).
#include <cooperative_groups.h>
#include <type_traits>

#include "batch.cuh"
#include "common.cuh"
#include "split.cuh"

namespace rl {

namespace {

__device__ inline double sqrt_(double a) { return sqrt(a); }
__device__ inline float sqrt_(float a) { return sqrtf(a); }
__device__ inline double hypot_(double a, double b) { return hypot(a, b); }
__device__ inline double recip_(double a) { return 1.0 / a; }
__device__ inline cd recip_(cd a) { double s = a.x * a.x + a.y * a.y; return {a.x / s, -a.y / s}; }
__device__ inline float recip_(float a) { return 1.0f / a; }
__device__ inline cf recip_(cf a) { float s = a.x * a.x + a.y * a.y; return {a.x / s, -a.y / s}; }

// Householder scalars (LAPACK larfg convention) from alpha = x(0) and ||x(1:)||^2:
// beta = -sign(Re alpha) ||x||, tau = (beta - alpha)/beta, v = [1; x(1:) / (alpha - beta)].
// tau = 0 (H = I) when x(1:) = 0 and alpha is real.
// One divide instead of two: with r = 1 / (beta (alpha - beta)), 1/beta = (alpha - beta) r and
// 1/(alpha - beta) = beta r (FP64 divides are ~10 dependent FMAs on GB300).
template <class T>
__device__ inline void householder_scalars(T alpha, double xnorm2, T* tau, T* beta, T* inv_ab) {
  if (xnorm2 == 0.0 && im_(alpha) == 0.0) {
    *tau = zero_<T>(); *beta = alpha; *inv_ab = zero_<T>();
    return;
  }
  const double bn = sqrt(abs2_(alpha) + xnorm2);
  const double bb = re_(alpha) >= 0.0 ? -bn : bn;
  *beta = from_real<T>(bb);
  const T amb = sub_(alpha, *beta);
  const T r = recip_(scale_(amb, bb));
  *tau = mul_(sub_(*beta, alpha), mul_(amb, r));
  *inv_ab = scale_(r, bb);
}

// ------------------------------------------------------------------------------------------
// TSQR level: CTA i reduces rows [i*rpc, min((i+1)*rpc, rows)) of X (row-major, ldx, c cols)
// to a c x c upper-triangular R by Householder steps on [R_running; next chunk of CH rows].
// Q is never formed. For column j the a = c - j active columns (cc = j .. c-1) each get L lanes,
// L the largest power of two with a L <= 256 (at most 32): as the active columns shrink, the lanes
// per column grow, so the threads issuing FP64 instructions stay contiguous and nearly all lanes
// of an issuing warp do useful work (an FP64 warp instruction costs its sub-partition the same
// issue slot whatever the number of active lanes). Thread (q, p) = (tid / L, tid % L) takes
// column cc = j + q and rows r = j+1+p, j+1+p+L, ...; the L lanes of a column are contiguous,
// so its sums are shuffle trees. Per column j:
//   d_cc = sum_{r > j} conj(S[r][j]) S[r][cc]   (cc = j gives ||x(1:)||^2)
//   reflector scalars from alpha = S[j][j] and d_j (one thread), then for cc > j
//   s = S[j][cc] + conj(1/(alpha - beta)) d_cc,  f = conj(tau) s,
//   S[j][cc] -= f,  S[r][cc] -= S[r][j] (f / (alpha - beta))  for r > j.
// Rows of the running R below the diagonal of column j are zero and are skipped.
// ------------------------------------------------------------------------------------------
__device__ inline int lanes_for(int a) {
  int L = 32;
  while (L > 1 && a * L > 256) L >>= 1;
  return L;
}

template <class T>
__global__ void __launch_bounds__(256) tsqr_level_kernel(const T* __restrict__ X, int64_t rows, int c, int64_t ldx,
                                                          int64_t rpc, int CH, int RP, T* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const int tid = threadIdx.x;
  T* S = reinterpret_cast<T*>(smem_raw);       // (c + CH) x c row-major
  __shared__ T s_d[64], s_fv[64];              // per active column: its sum d, then f / (alpha - beta)
  (void)RP;

  const int64_t r_begin = (int64_t)blockIdx.x * rpc;
  const int64_t r_end = imin<int64_t>(rows, r_begin + rpc);
  for (int i = tid; i < c * c; i += NT) S[i] = zero_<T>();
  for (int64_t r0 = r_begin; r0 < r_end || r0 == r_begin; r0 += CH) {
    const int nr = (int)imax<int64_t>(0, imin<int64_t>(CH, r_end - r0));
    // keep the upper triangle of the running R, load the next chunk below it
    for (int i = tid; i < c * c; i += NT) {
      const int r = i / c, q = i % c;
      if (q < r) S[i] = zero_<T>();
    }
    for (int i = tid; i < CH * c; i += NT) {
      const int r = i / c, q = i % c;
      S[(size_t)(c + r) * c + q] = (r < nr) ? X[(r0 + r) * ldx + q] : zero_<T>();
    }
    __syncthreads();
    const int SRu = c + imax(nr, 1);            // rows that can be nonzero
    for (int j = 0; j < c; ++j) {
      const int a = c - j, L = lanes_for(a);
      const int q = tid / L, p = tid % L;
      const int cc = j + q;
      const bool on = q < a;
      // rows of column j that can be nonzero: row j of R (the pivot), then the chunk (rows c..)
      const int rs = c;                         // first chunk row (R rows j+1..c-1 are zero in column j)
      T d = zero_<T>();
      if (on) {
        // two accumulators: the FP64 pipe, not the dependency chain, bounds this loop
        T a0 = zero_<T>(), a1 = zero_<T>();
        int r = rs + p;
        for (; r + L < SRu; r += 2 * L) {
          a0 = madc_(S[(size_t)r * c + j], S[(size_t)r * c + cc], a0);
          a1 = madc_(S[(size_t)(r + L) * c + j], S[(size_t)(r + L) * c + cc], a1);
        }
        if (r < SRu) a0 = madc_(S[(size_t)r * c + j], S[(size_t)r * c + cc], a0);
        d = add_(a0, a1);
      }
      for (int o = L >> 1; o > 0; o >>= 1) d = add_(d, shfl_xor_(d, o));
      if (on && p == 0) s_d[q] = d;
      __syncthreads();
      // Warp 0 forms the reflector (lane 0) and then f and f / (alpha - beta) of every active
      // column, a lane per column: done by the column groups themselves, these few FP64
      // instructions would be issued by every warp at one active lane in L.
      if (tid < 32) {
        T tau = zero_<T>(), beta = zero_<T>(), inv_ab = zero_<T>();
        if (tid == 0) householder_scalars(S[(size_t)j * c + j], re_(s_d[0]), &tau, &beta, &inv_ab);
        tau = shfl_(tau, 0);
        inv_ab = shfl_(inv_ab, 0);
        for (int l = 1 + tid; l < a; l += 32) {
          T* rj = S + (size_t)j * c + j + l;
          const T f = mul_(conj_(tau), add_(*rj, mul_(conj_(inv_ab), s_d[l])));
          s_fv[l] = mul_(inv_ab, f);             // v_r = S[r][j] / (alpha - beta) folded into f
          *rj = sub_(*rj, f);
        }
        if (tid == 0) S[(size_t)j * c + j] = beta;
      }
      __syncthreads();
      if (on && q > 0) {
        const T fv = s_fv[q];
        for (int r = rs + p; r < SRu; r += L)
          S[(size_t)r * c + cc] = sub_(S[(size_t)r * c + cc], mul_(S[(size_t)r * c + j], fv));
      }
      __syncthreads();
    }
    if (r_end <= r_begin) break;
  }
  T* out = Rout + (size_t)blockIdx.x * c * c;
  for (int i = tid; i < c * c; i += NT) {
    const int r = i / c, q = i % c;
    out[i] = (q >= r) ? S[i] : zero_<T>();
  }
}

// Upper levels of the TSQR tree: merge F stacked c x c upper-triangular R factors into one.
// Block 0 is the running R; the reflector of column j touches row j of block 0 and rows 0..j of
// blocks 1..F-1 only (every other entry of the column is zero and stays zero), so both the FP64
// work and the rows per thread of column j shrink with j (half the work of a dense stack).
// Thread (column cc, row phase p) as in tsqr_level_kernel; the reflector is applied with its
// 1/(alpha - beta) scaling folded into the update, and Q is never formed.
template <class T>
__global__ void __launch_bounds__(256) tsqr_merge_kernel(const T* __restrict__ Rin, int nblk, int c, int F, int RP,
                                                         T* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);   // F c rows x c, row-major
  __shared__ T sh_tau, sh_inv, sh_beta;
  const int tid = threadIdx.x, NT = blockDim.x, cc = tid / RP, p = tid % RP;
  const int b0 = blockIdx.x * F;
  const int nb = imin(F, nblk - b0);
  for (int i = tid; i < nb * c * c; i += NT) S[i] = Rin[(size_t)b0 * c * c + i];
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    const int jr = j + 1;
    const int act = (nb - 1) * jr;   // rows of blocks 1.. that can be nonzero in column j
    T d = zero_<T>();
    // active row t = (block 1 + t / jr, local row t % jr), walked incrementally (no divides)
    if (cc < c && cc >= j) {
      T a0 = zero_<T>(), a1 = zero_<T>();
      int f = 1 + p / jr, lr = p % jr;
      const int df = RP / jr, dl = RP % jr;
      for (int t = p; t < act; t += 2 * RP) {
        const int r0 = f * c + lr;
        a0 = madc_(S[(size_t)r0 * c + j], S[(size_t)r0 * c + cc], a0);
        f += df;
        lr += dl;
        if (lr >= jr) { lr -= jr; ++f; }
        if (t + RP < act) {
          const int r1 = f * c + lr;
          a1 = madc_(S[(size_t)r1 * c + j], S[(size_t)r1 * c + cc], a1);
        }
        f += df;
        lr += dl;
        if (lr >= jr) { lr -= jr; ++f; }
      }
      d = add_(a0, a1);
    }
    for (int o = RP >> 1; o > 0; o >>= 1) d = add_(d, shfl_xor_(d, o));
    if (cc == j && p == 0) {
      T tau, beta, inv_ab;
      householder_scalars(S[(size_t)j * c + j], re_(d), &tau, &beta, &inv_ab);
      sh_tau = tau; sh_inv = inv_ab; sh_beta = beta;
    }
    __syncthreads();
    if (cc < c && cc > j) {
      const T inv_ab = sh_inv;
      const T f = mul_(conj_(sh_tau), add_(S[(size_t)j * c + cc], mul_(conj_(inv_ab), d)));
      const T fv = mul_(inv_ab, f);
      if (p == 0) S[(size_t)j * c + cc] = sub_(S[(size_t)j * c + cc], f);
      int fb = 1 + p / jr, lr = p % jr;
      const int df = RP / jr, dl = RP % jr;
      for (int t = p; t < act; t += RP) {
        const int r = fb * c + lr;
        S[(size_t)r * c + cc] = sub_(S[(size_t)r * c + cc], mul_(S[(size_t)r * c + j], fv));
        fb += df;
        lr += dl;
        if (lr >= jr) { lr -= jr; ++fb; }
      }
    }
    if (cc == j && p == 0) S[(size_t)j * c + j] = sh_beta;
    __syncthreads();
  }
  T* out = Rout + (size_t)blockIdx.x * c * c;
  for (int i = tid; i < c * c; i += NT) {
    const int r = i / c, q = i % c;
    out[i] = (q >= r) ? S[i] : zero_<T>();
  }
}

// scale rows of a c x c R so that diag(R) is real and non-negative
template <class T>
__global__ void r_phase_fix_kernel(T* R, int c) {
  const int r = blockIdx.x;
  const T ph = conj_(phase_(R[(size_t)r * c + r]));
  for (int q = threadIdx.x; q < c; q += blockDim.x) R[(size_t)r * c + q] = mul_(ph, R[(size_t)r * c + q]);
}

// ------------------------------------------------------------------------------------------
// rr_small: one CTA. X = R_T (c x c) column-major in smem, V = I; one-sided Jacobi, one warp
// per pair (round-robin), __syncthreads per round. Then Theta (descending, stable), C, and
// K = [C_s | C(:,1:c-b) Q] with Q = Orth(C(1:b,1:c-b)^H).
// Outputs: theta (c, descending), K (c x 2b row-major), sweeps.
// ------------------------------------------------------------------------------------------
__device__ inline int rr_slot(int k, int r, int N) { return k == 0 ? 0 : ((k - 1 + r) % (N - 1)) + 1; }

// One-sided Jacobi on c <= 16 real columns (X, V column-major c x c in shared memory) with two
// disjoint pairs per warp (a half-warp each, lane = row): on GB300 every FP64 warp instruction
// costs its sub-partition ~64 cycles whatever the number of active lanes, so packing two pairs per
// instruction halves the FP64 time of a round. A half-warp forms its pair's three sums with a
// 4-level butterfly. The rotation test is the FP64 one of jacobi_tangent; the angle comes from an
// FP32 evaluation of tan(theta) = sign(d) 2|g| / (|d| + sqrt(d^2 + 4 g^2)) on d = b - a and g
// taken in FP64 and scaled by a power of two, and (c, s) = (1, t) / sqrt(1 + t^2) in FP64, which
// is orthogonal to FP64 rounding for any t; an FP32-accurate angle leaves ~1e-7 of the pair's
// cosine, which the next sweep removes. A pair that needs no rotation uses (c, s) = (1, 0), so
// both halves execute the same instructions. Returns the number of sweeps.
__device__ int jacobi_pairs16(double* X, double* V, int c, int N, double tol, double tiny2, const uint8_t* sched,
                              int max_sweeps) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int half = lane >> 4, row = lane & 15;
  const double tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int p0 = 2 * warp; p0 < N / 2; p0 += 2 * nw) {   // warp-uniform
        const int pi = p0 + half;
        const int code = pi < N / 2 ? sched[r * 8 + pi] : 0xFF;
        const int pp = code & 15, qq = code >> 4;
        const bool valid = code != 0xFF;
        const bool live = valid && row < c;
        const double xp = live ? X[pp * c + row] : 0.0, xq = live ? X[qq * c + row] : 0.0;
        double a = xp * xp, bb = xq * xq, g = xp * xq;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        bool rot = valid && (g * g > tol2 * a * bb) && a > tiny2 && bb > tiny2;
        double cs = 1.0, se = 0.0;
        {
          const double mx = rot ? fmax(a, bb) : 1.0;
          const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023;
          const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
          const float df = (float)((bb - a) * sc), gf = fabsf((float)(g * sc));
          const float tf = copysignf(2.0f * gf, df) / (fabsf(df) + sqrtf(df * df + 4.0f * gf * gf));
          rot = rot && fabsf(tf) > 2.220446049250313e-16f;
          const double t = rot ? (double)tf : 0.0;
          cs = rsqrt(fma(t, t, 1.0));
          const double sn = cs * t;
          se = g < 0.0 ? -sn : sn;
        }
        if (live) {
          const double vp = V[pp * c + row], vq = V[qq * c + row];
          X[pp * c + row] = cs * xp - se * xq;
          X[qq * c + row] = se * xp + cs * xq;
          V[pp * c + row] = cs * vp - se * vq;
          V[qq * c + row] = se * vp + cs * vq;
        }
        rotated |= rot;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// Would a sweep still rotate any column pair of X (c x c, column-major)? The same two tests as
// the sweep -- the cosine test and a rotation angle above eps (a pair whose angle is below eps is
// never rotated) -- in one pass over all pairs instead of a whole confirming sweep.
__device__ bool jacobi_pending(const double* X, int c, double tol, double tiny2) {
  const double tol2 = tol * tol;
  int bad = 0;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j <= i) continue;
    double a = 0, bb = 0, g = 0;
    for (int r = 0; r < c; ++r) {
      const double x = X[i * c + r], y = X[j * c + r];
      a = fma(x, x, a);
      bb = fma(y, y, bb);
      g = fma(x, y, g);
    }
    if ((g * g > tol2 * a * bb) && a > tiny2 && bb > tiny2) {
      const double d = bb - a;
      const double t = 2.0 * fabs(g) / (fabs(d) + sqrt(d * d + 4.0 * g * g));
      bad |= t > 2.220446049250313e-16;
    }
  }
  return __syncthreads_or(bad) != 0;
}

// The same sweeps in FP32 (on GB300 the FP32 pipe issues ~64x the FP64 rate): used on a scaled
// FP32 copy of R_T to find a V that nearly diagonalises it (cosines ~ c u_32).
__device__ int jacobi_pairs16_f32(float* X, float* V, int c, int N, float tol, float tiny2, const uint8_t* sched) {
  // same layout as the FP64 sweeps: two pairs per warp, a half-warp per pair, lane = row
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int half = lane >> 4, row = lane & 15;
  const float tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < 12; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int p0 = 2 * warp; p0 < N / 2; p0 += 2 * nw) {   // warp-uniform
        const int pi = p0 + half;
        const int code = pi < N / 2 ? sched[r * 8 + pi] : 0xFF;
        const int pp = code & 15, qq = code >> 4;
        const bool valid = code != 0xFF;
        const bool live = valid && row < c;
        const float xp = live ? X[pp * c + row] : 0.f, xq = live ? X[qq * c + row] : 0.f;
        float a = xp * xp, bb = xq * xq, g = xp * xq;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        const float d = bb - a, ga = fabsf(g);
        const float tf = copysignf(2.0f * ga, d) / (fabsf(d) + sqrtf(d * d + 4.0f * ga * ga));
        const bool rot = valid && (g * g > tol2 * a * bb) && a > tiny2 && bb > tiny2 && fabsf(tf) > 1.0e-12f;
        const float t = rot ? tf : 0.0f;
        const float cs = rsqrtf(fmaf(t, t, 1.0f));
        const float sn = cs * t;
        const float se = g < 0.0f ? -sn : sn;
        if (live && rot) {
          const float vp = V[pp * c + row], vq = V[qq * c + row];
          X[pp * c + row] = cs * xp - se * xq;
          X[qq * c + row] = se * xp + cs * xq;
          V[pp * c + row] = cs * vp - se * vq;
          V[qq * c + row] = se * vp + cs * vq;
        }
        rotated |= rot;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// Out = In * M for c x c column-major matrices in shared memory (all threads; result in Out).
__device__ void small_matmul(const double* In, const double* M, double* Out, int c) {
  for (int o = threadIdx.x; o < c * c; o += blockDim.x) {
    const int j = o / c, r = o % c;
    double s0 = 0, s1 = 0;
    int i = 0;
    for (; i + 1 < c; i += 2) {
      s0 = fma(In[i * c + r], M[j * c + i], s0);
      s1 = fma(In[(i + 1) * c + r], M[j * c + i + 1], s1);
    }
    if (i < c) s0 = fma(In[i * c + r], M[j * c + i], s0);
    Out[o] = s0 + s1;
  }
}

// Preconditioned one-sided Jacobi for real c <= 16 (X = R_T, V = I on entry, column-major):
//   1. FP32 sweeps on X scaled by a power of two -> Vf with X Vf nearly column-orthogonal;
//   2. V = Vf made orthonormal in FP64 by two Newton-Schulz steps V <- V (3 I - V^T V) / 2
//      (orthogonality error ~1e-6 -> ~1e-12 -> rounding level);
//   3. X <- X V in FP64 and FP64 sweeps from there (usually one with rotations, one to confirm).
// The FP64 stage runs to the same convergence test as the plain FP64 sweeps, on X V with V
// orthonormal to rounding; the FP32 stage only changes where it starts (and saves FP64 sweeps).
__device__ int jacobi_mixed16(double* X, double* V, int c, int N, double tol, double tiny2, double mx0, float* Xf,
                              float* Vf, double* Ms, double* Ws) {
  const int tid = threadIdx.x, NT = blockDim.x;
  // power-of-two scale so that the largest column norm is about 1 in FP32
  const int ex = (int)((__double_as_longlong(fmax(mx0, 1e-300)) >> 52) & 0x7ff) - 1023;
  const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
  for (int i = tid; i < c * c; i += NT) {
    Xf[i] = (float)(X[i] * sc);
    Vf[i] = (i / c == i % c) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const float tol32 = (float)imax(c, 4) * 1.1920929e-7f;
  const float tiny32 = (float)(tiny2 * sc * sc);
  // round-robin schedule: pair i of round r is (slot(i), slot(N - 1 - i)), ordered, 0xFF if a
  // member is the padding column c (odd c)
  __shared__ uint8_t sched[15 * 8];
  for (int e = tid; e < (N - 1) * 8; e += NT) {
    const int r = e / 8, i = e % 8;
    uint8_t code = 0xFF;
    if (i < N / 2) {
      int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
      if (pp > qq) { const int t = pp; pp = qq; qq = t; }
      if (qq < c) code = (uint8_t)(pp | (qq << 4));
    }
    sched[e] = code;
  }
  __syncthreads();
  jacobi_pairs16_f32(Xf, Vf, c, N, tol32, tiny32, sched);
  for (int i = tid; i < c * c; i += NT) V[i] = (double)Vf[i];
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    // Ms = (3 I - V^T V) / 2
    for (int o = tid; o < c * c; o += NT) {
      const int i = o / c, j = o % c;
      double s0 = 0, s1 = 0;
      int k = 0;
      for (; k + 1 < c; k += 2) {
        s0 = fma(V[i * c + k], V[j * c + k], s0);
        s1 = fma(V[i * c + k + 1], V[j * c + k + 1], s1);
      }
      if (k < c) s0 = fma(V[i * c + k], V[j * c + k], s0);
      Ms[o] = (i == j ? 1.5 : 0.0) - 0.5 * (s0 + s1);
    }
    __syncthreads();
    small_matmul(V, Ms, Ws, c);
    __syncthreads();
    for (int i = tid; i < c * c; i += NT) V[i] = Ws[i];
    __syncthreads();
  }
  small_matmul(X, V, Ws, c);
  __syncthreads();
  for (int i = tid; i < c * c; i += NT) X[i] = Ws[i];
  __syncthreads();
  // FP64 sweeps while they rotate; after two, a single check of all pairs replaces the sweep
  // that would only confirm convergence
  int sweeps = 0;
  for (int round = 0; round < 30; ++round) {
    const int s2 = jacobi_pairs16(X, V, c, N, tol, tiny2, sched, 2);
    sweeps += s2;
    if (s2 < 2 || !jacobi_pending(X, c, tol, tiny2)) break;
  }
  return sweeps;
}

// ---- complex c <= 16: the preconditioned scheme of jacobi_mixed16 -------------------------
// Column pair (p, q) with a = ||x_p||^2, b = ||x_q||^2, g = x_p^H x_q: the phase e = g / |g|
// turns it into the real problem of jacobi_pairs16 on (|g|, a, b), and the rotation
//     x_p <- c x_p - conj(s e) x_q,   x_q <- s e x_p + c x_q      (c = 1 / sqrt(1 + t^2), s = c t)
// is unitary to FP64 rounding for any t; V takes the same rotation. FP64 sums, FP32 angle (as in
// jacobi_pairs16), two pairs per warp (a half-warp each, lane = row).
__device__ int jacobi_pairs16_c(cd* X, cd* V, int c, int N, double tol, double tiny2, const uint8_t* sched,
                                int max_sweeps) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int half = lane >> 4, row = lane & 15;
  const double tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int p0 = 2 * warp; p0 < N / 2; p0 += 2 * nw) {   // warp-uniform
        const int pi = p0 + half;
        const int code = pi < N / 2 ? sched[r * 8 + pi] : 0xFF;
        const int pp = code & 15, qq = code >> 4;
        const bool valid = code != 0xFF;
        const bool live = valid && row < c;
        const cd xp = live ? X[pp * c + row] : zero_<cd>(), xq = live ? X[qq * c + row] : zero_<cd>();
        double a = abs2_(xp), bb = abs2_(xq);
        cd g = madc_(xp, xq, zero_<cd>());
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g = add_(g, shfl_xor_(g, o));
        }
        const double g2 = abs2_(g);
        bool rot = valid && (g2 > tol2 * a * bb) && a > tiny2 && bb > tiny2;
        double cs = 1.0, sn = 0.0;
        cd e = from_real<cd>(1.0);
        {
          const double mx = rot ? fmax(a, bb) : 1.0;
          const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023;
          const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
          const float df = (float)((bb - a) * sc), gf = sqrtf((float)(g2 * sc * sc));
          const float tf = copysignf(2.0f * gf, df) / (fabsf(df) + sqrtf(df * df + 4.0f * gf * gf));
          rot = rot && fabsf(tf) > 2.220446049250313e-16f;
          const double t = rot ? (double)tf : 0.0;
          cs = rsqrt(fma(t, t, 1.0));
          sn = cs * t;
          if (rot) e = scale_(g, rsqrt(g2));
        }
        const cd se = scale_(e, sn), sec = conj_(se);
        if (live) {
          const cd vp = V[pp * c + row], vq = V[qq * c + row];
          X[pp * c + row] = sub_(scale_(xp, cs), mul_(sec, xq));
          X[qq * c + row] = add_(mul_(se, xp), scale_(xq, cs));
          V[pp * c + row] = sub_(scale_(vp, cs), mul_(sec, vq));
          V[qq * c + row] = add_(mul_(se, vp), scale_(vq, cs));
        }
        rotated |= rot;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// jacobi_pending for complex columns
__device__ bool jacobi_pending_c(const cd* X, int c, double tol, double tiny2) {
  const double tol2 = tol * tol;
  int bad = 0;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j <= i) continue;
    double a = 0, bb = 0;
    cd g = zero_<cd>();
    for (int r = 0; r < c; ++r) {
      const cd x = X[i * c + r], y = X[j * c + r];
      a += abs2_(x);
      bb += abs2_(y);
      g = madc_(x, y, g);
    }
    const double g2 = abs2_(g);
    if ((g2 > tol2 * a * bb) && a > tiny2 && bb > tiny2) {
      const double d = bb - a;
      const double t = 2.0 * sqrt(g2) / (fabs(d) + sqrt(d * d + 4.0 * g2));
      bad |= t > 2.220446049250313e-16;
    }
  }
  return __syncthreads_or(bad) != 0;
}

// FP32 sweeps for complex c <= 16 (same layout and rule as jacobi_pairs16_f32)
__device__ int jacobi_pairs16_f32_c(cf* X, cf* V, int c, int N, float tol, float tiny2, const uint8_t* sched) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int half = lane >> 4, row = lane & 15;
  const float tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < 12; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int p0 = 2 * warp; p0 < N / 2; p0 += 2 * nw) {   // warp-uniform
        const int pi = p0 + half;
        const int code = pi < N / 2 ? sched[r * 8 + pi] : 0xFF;
        const int pp = code & 15, qq = code >> 4;
        const bool valid = code != 0xFF;
        const bool live = valid && row < c;
        const cf zf = {0.f, 0.f};
        const cf xp = live ? X[pp * c + row] : zf, xq = live ? X[qq * c + row] : zf;
        float a = abs2_(xp), bb = abs2_(xq);
        cf g = madc_(xp, xq, zf);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g = add_(g, shfl_xor_(g, o));
        }
        const float g2 = abs2_(g), ga = sqrtf(g2);
        const float d = bb - a;
        const float tf = copysignf(2.0f * ga, d) / (fabsf(d) + sqrtf(d * d + 4.0f * g2));
        const bool rot = valid && (g2 > tol2 * a * bb) && a > tiny2 && bb > tiny2 && fabsf(tf) > 1.0e-12f;
        const float t = rot ? tf : 0.0f;
        const float cs = rsqrtf(fmaf(t, t, 1.0f));
        const float sn = cs * t;
        const cf e = rot ? scale_(g, 1.0f / ga) : cf{1.0f, 0.0f};
        const cf se = scale_(e, sn), sec = conj_(se);
        if (live && rot) {
          const cf vp = V[pp * c + row], vq = V[qq * c + row];
          X[pp * c + row] = sub_(scale_(xp, cs), mul_(sec, xq));
          X[qq * c + row] = add_(mul_(se, xp), scale_(xq, cs));
          V[pp * c + row] = sub_(scale_(vp, cs), mul_(sec, vq));
          V[qq * c + row] = add_(mul_(se, vp), scale_(vq, cs));
        }
        rotated |= rot;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// Out = In * M for complex c x c column-major matrices in shared memory (all threads)
__device__ void small_matmul_c(const cd* In, const cd* M, cd* Out, int c) {
  for (int o = threadIdx.x; o < c * c; o += blockDim.x) {
    const int j = o / c, r = o % c;
    cd s0 = zero_<cd>(), s1 = zero_<cd>();
    int i = 0;
    for (; i + 1 < c; i += 2) {
      s0 = mad_(In[i * c + r], M[j * c + i], s0);
      s1 = mad_(In[(i + 1) * c + r], M[j * c + i + 1], s1);
    }
    if (i < c) s0 = mad_(In[i * c + r], M[j * c + i], s0);
    Out[o] = add_(s0, s1);
  }
}

// jacobi_mixed16 for complex c <= 16: FP32 sweeps on the scaled complex64 copy, V made unitary
// in FP64 by two Newton-Schulz steps V <- V (3 I - V^H V) / 2, X <- X V, FP64 sweeps from there.
__device__ int jacobi_mixed16_c(cd* X, cd* V, int c, int N, double tol, double tiny2, double mx0, cf* Xf, cf* Vf,
                                cd* Ms, cd* Ws) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ex = (int)((__double_as_longlong(fmax(mx0, 1e-300)) >> 52) & 0x7ff) - 1023;
  const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
  for (int i = tid; i < c * c; i += NT) {
    Xf[i] = cvt_<cf, cd>(scale_(X[i], sc));
    Vf[i] = (i / c == i % c) ? cf{1.0f, 0.0f} : cf{0.0f, 0.0f};
  }
  __syncthreads();
  const float tol32 = (float)imax(c, 4) * 1.1920929e-7f;
  const float tiny32 = (float)(tiny2 * sc * sc);
  __shared__ uint8_t sched[15 * 8];
  for (int e = tid; e < (N - 1) * 8; e += NT) {
    const int r = e / 8, i = e % 8;
    uint8_t code = 0xFF;
    if (i < N / 2) {
      int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
      if (pp > qq) { const int t = pp; pp = qq; qq = t; }
      if (qq < c) code = (uint8_t)(pp | (qq << 4));
    }
    sched[e] = code;
  }
  __syncthreads();
  jacobi_pairs16_f32_c(Xf, Vf, c, N, tol32, tiny32, sched);
  for (int i = tid; i < c * c; i += NT) V[i] = cvt_<cd, cf>(Vf[i]);
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    // Ms = (3 I - V^H V) / 2
    for (int o = tid; o < c * c; o += NT) {
      const int i = o / c, j = o % c;
      cd s0 = zero_<cd>(), s1 = zero_<cd>();
      int k = 0;
      for (; k + 1 < c; k += 2) {
        s0 = madc_(V[j * c + k], V[i * c + k], s0);
        s1 = madc_(V[j * c + k + 1], V[i * c + k + 1], s1);
      }
      if (k < c) s0 = madc_(V[j * c + k], V[i * c + k], s0);
      const cd s = add_(s0, s1);   // (V^H V)(j, i), stored at column i, row j
      Ms[o] = cd{(i == j ? 1.5 : 0.0) - 0.5 * s.x, -0.5 * s.y};
    }
    __syncthreads();
    small_matmul_c(V, Ms, Ws, c);
    __syncthreads();
    for (int i = tid; i < c * c; i += NT) V[i] = Ws[i];
    __syncthreads();
  }
  small_matmul_c(X, V, Ws, c);
  __syncthreads();
  for (int i = tid; i < c * c; i += NT) X[i] = Ws[i];
  __syncthreads();
  int sweeps = 0;
  for (int round = 0; round < 30; ++round) {
    const int s2 = jacobi_pairs16_c(X, V, c, N, tol, tiny2, sched, 2);
    sweeps += s2;
    if (s2 < 2 || !jacobi_pending_c(X, c, tol, tiny2)) break;
  }
  return sweeps;
}

// ---- real c in (16, 32]: the same preconditioned scheme with one pair per warp -------------
// Round-robin schedule for N <= 32 slots: pair i of round r is coded pp | qq << 8 (pp < qq), or
// 0xFFFF when a member is the padding column c (odd c).
__device__ void rr_schedule32(uint16_t* sched, int c, int N) {
  for (int e = threadIdx.x; e < (N - 1) * 16; e += blockDim.x) {
    const int r = e / 16, i = e % 16;
    uint16_t code = 0xFFFF;
    if (i < N / 2) {
      int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
      if (pp > qq) { const int t = pp; pp = qq; qq = t; }
      if (qq < c) code = (uint16_t)(pp | (qq << 8));
    }
    sched[e] = code;
  }
}

// FP32 sweeps for c <= 32: a warp per pair, lane = row, the three sums by a 5-level butterfly
// (FP32 work runs on the fast pipe). Same rotation rule as jacobi_pairs16_f32.
__device__ int jacobi_sweeps32_f32(float* X, float* V, int c, int N, float tol, float tiny2, const uint16_t* sched) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const float tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < 15; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pi = warp; pi < N / 2; pi += nw) {   // warp-uniform
        const int code = sched[r * 16 + pi];
        const bool valid = code != 0xFFFF;
        const int pp = code & 0xFF, qq = code >> 8;
        const bool live = valid && lane < c;
        const float xp = live ? X[pp * c + lane] : 0.f, xq = live ? X[qq * c + lane] : 0.f;
        float a = xp * xp, bb = xq * xq, g = xp * xq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        const float d = bb - a, ga = fabsf(g);
        const float tf = copysignf(2.0f * ga, d) / (fabsf(d) + sqrtf(d * d + 4.0f * ga * ga));
        const bool rot = valid && (g * g > tol2 * a * bb) && a > tiny2 && bb > tiny2 && fabsf(tf) > 1.0e-12f;
        const float t = rot ? tf : 0.0f;
        const float cs = rsqrtf(fmaf(t, t, 1.0f));
        const float sn = cs * t;
        const float se = g < 0.0f ? -sn : sn;
        if (live && rot) {
          const float vp = V[pp * c + lane], vq = V[qq * c + lane];
          X[pp * c + lane] = cs * xp - se * xq;
          X[qq * c + lane] = se * xp + cs * xq;
          V[pp * c + lane] = cs * vp - se * vq;
          V[qq * c + lane] = se * vp + cs * vq;
        }
        rotated |= rot;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// FP64 sweeps for c <= 32, in three phases per round so that few FP64 warp instructions are
// issued (each costs an SM sub-partition ~64 cycles however many lanes are active):
//   1. the 3 sums of each of the <= 16 pairs, 8 lanes per sum (4 rows each, 3 butterfly levels);
//   2. the rotations, one lane of warp 0 per pair (same rule as jacobi_pairs16);
//   3. a warp per pair applies its rotation to X and V, lane = row.
// Needs blockDim.x >= 384. dots: 48 doubles, rot: 32 doubles, rflag: 16 ints (shared).
__device__ int jacobi_sweeps32_f64(double* X, double* V, int c, int N, double tol, double tiny2,
                                   const uint16_t* sched, int max_sweeps, double* dots, double* rotp, int* rflag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const double tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < N - 1; ++r) {
      const uint16_t* sr = sched + r * 16;
      if (tid < 384) {
        const int t = tid >> 3, sub = tid & 7, pi = t / 3, kind = t % 3;
        const int code = pi < N / 2 ? sr[pi] : 0xFFFF;
        double sum = 0.0;
        if (code != 0xFFFF) {
          const int pp = code & 0xFF, qq = code >> 8;
          const double* u = X + (kind == 1 ? qq : pp) * c;
          const double* v = X + (kind == 0 ? pp : qq) * c;
          for (int row = sub; row < c; row += 8) sum = fma(u[row], v[row], sum);
        }
        sum += __shfl_xor_sync(0xffffffffu, sum, 4);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if (sub == 0) dots[t] = sum;
      }
      __syncthreads();
      if (tid < 16) {
        const int pi = tid;
        const int code = pi < N / 2 ? sr[pi] : 0xFFFF;
        const double a = dots[3 * pi], bb = dots[3 * pi + 1], g = dots[3 * pi + 2];
        bool rot = code != 0xFFFF && (g * g > tol2 * a * bb) && a > tiny2 && bb > tiny2;
        double cs = 1.0, se = 0.0;
        if (rot) {
          const double mx = fmax(a, bb);
          const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023;
          const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
          const float df = (float)((bb - a) * sc), gf = fabsf((float)(g * sc));
          const float tf = copysignf(2.0f * gf, df) / (fabsf(df) + sqrtf(df * df + 4.0f * gf * gf));
          rot = fabsf(tf) > 2.220446049250313e-16f;
          const double t = rot ? (double)tf : 0.0;
          cs = rsqrt(fma(t, t, 1.0));
          const double sn = cs * t;
          se = g < 0.0 ? -sn : sn;
        }
        rotp[2 * pi] = cs;
        rotp[2 * pi + 1] = se;
        rflag[pi] = rot;
        rotated |= rot;
      }
      __syncthreads();
      for (int pi = warp; pi < N / 2; pi += nw) {   // warp-uniform
        if (!rflag[pi] || lane >= c) continue;
        const int code = sr[pi];
        const int pp = code & 0xFF, qq = code >> 8;
        const double cs = rotp[2 * pi], se = rotp[2 * pi + 1];
        const double xp = X[pp * c + lane], xq = X[qq * c + lane];
        const double vp = V[pp * c + lane], vq = V[qq * c + lane];
        X[pp * c + lane] = cs * xp - se * xq;
        X[qq * c + lane] = se * xp + cs * xq;
        V[pp * c + lane] = cs * vp - se * vq;
        V[qq * c + lane] = se * vp + cs * vq;
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) { ++sweep; break; }
  }
  return sweep;
}

// Preconditioned one-sided Jacobi for real 16 < c <= 32, as jacobi_mixed16: FP32 sweeps on a
// power-of-two scaled copy, V made orthonormal in FP64 by two Newton-Schulz steps, X <- X V, and
// FP64 sweeps from there to the n eps test (confirmed by one pass over all pairs).
__device__ int jacobi_mixed32(double* X, double* V, int c, int N, double tol, double tiny2, double mx0, float* Xf,
                              float* Vf, double* Ms, double* Ws, uint16_t* sched, double* dots, double* rotp,
                              int* rflag) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ex = (int)((__double_as_longlong(fmax(mx0, 1e-300)) >> 52) & 0x7ff) - 1023;
  const double sc = __longlong_as_double((long long)(1023 - imax(-1022, imin(1022, ex))) << 52);
  for (int i = tid; i < c * c; i += NT) {
    Xf[i] = (float)(X[i] * sc);
    Vf[i] = (i / c == i % c) ? 1.0f : 0.0f;
  }
  rr_schedule32(sched, c, N);
  __syncthreads();
  const float tol32 = (float)imax(c, 4) * 1.1920929e-7f;
  const float tiny32 = (float)(tiny2 * sc * sc);
  jacobi_sweeps32_f32(Xf, Vf, c, N, tol32, tiny32, sched);
  for (int i = tid; i < c * c; i += NT) V[i] = (double)Vf[i];
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    for (int o = tid; o < c * c; o += NT) {
      const int i = o / c, j = o % c;
      double s0 = 0, s1 = 0;
      int k = 0;
      for (; k + 1 < c; k += 2) {
        s0 = fma(V[i * c + k], V[j * c + k], s0);
        s1 = fma(V[i * c + k + 1], V[j * c + k + 1], s1);
      }
      if (k < c) s0 = fma(V[i * c + k], V[j * c + k], s0);
      Ms[o] = (i == j ? 1.5 : 0.0) - 0.5 * (s0 + s1);
    }
    __syncthreads();
    small_matmul(V, Ms, Ws, c);
    __syncthreads();
    for (int i = tid; i < c * c; i += NT) V[i] = Ws[i];
    __syncthreads();
  }
  small_matmul(X, V, Ws, c);
  __syncthreads();
  for (int i = tid; i < c * c; i += NT) X[i] = Ws[i];
  __syncthreads();
  int sweeps = 0;
  for (int round = 0; round < 30; ++round) {
    const int s2 = jacobi_sweeps32_f64(X, V, c, N, tol, tiny2, sched, 2, dots, rotp, rflag);
    sweeps += s2;
    if (s2 < 2 || !jacobi_pending(X, c, tol, tiny2)) break;
  }
  return sweeps;
}

// One CTA (any multiple of 32 threads); smem_raw: rr_small_smem(c, b) bytes of dynamic shared memory.
template <class T, int CMAX = 32>   // CMAX: the largest c the FP32-preconditioned Jacobi path serves
__device__ void rr_small_cta(unsigned char* smem_raw, const T* __restrict__ Rt, int c, int b, double* theta_out,
                             T* K_out, int* info) {
  T* X = reinterpret_cast<T*>(smem_raw);        // c x c col-major
  T* V = X + c * c;                             // c x c col-major
  T* C = V + c * c;                             // c x c col-major (sorted)
  T* Qm = C + c * c;                            // (c-b) x b col-major
  double* nrm = reinterpret_cast<double*>(Qm + c * b);
  int* rank = reinterpret_cast<int*>(nrm + c);
  __shared__ int changed;
  __shared__ T tau_s[64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;

  for (int i = tid; i < c * c; i += blockDim.x) {
    const int col = i / c, row = i % c;
    X[i] = Rt[(size_t)row * c + col];
    V[i] = (row == col) ? from_real<T>(1.0) : zero_<T>();
  }
  __syncthreads();
  const int N = c + (c & 1);
  // orthogonality test |x_p^H x_q| <= c eps ||x_p|| ||x_q|| (the cosine carries ~c u of noise)
  const double tol = (double)imax(c, 4) * 2.220446049250313e-16;
  // columns at rounding level (<= c eps max_j ||x_j||) are not rotated (rank-deficient R_T, e.g.
  // A_V at noise level for an exact nullspace): they would never converge
  for (int j = warp; j < c; j += nwarp) {
    double a = 0;
    for (int rr = lane; rr < c; rr += 32) a += abs2_(X[j * c + rr]);
    a = warp_sum(a);
    if (lane == 0) nrm[j] = sqrt(a);
  }
  __syncthreads();
  double mx0 = 0;
  for (int j = 0; j < c; ++j) mx0 = fmax(mx0, nrm[j]);
  const double tiny = mx0 * (double)imax(c, 4) * 2.220446049250313e-16;
  const double tiny2 = tiny * tiny;
  int sweep = 0;
  bool fast = false;
  if constexpr (std::is_same<T, double>::value) {
    if (c <= CMAX) {
      __shared__ float Xf[CMAX * CMAX], Vf[CMAX * CMAX];
      __shared__ double Ms[CMAX * CMAX], Ws2[CMAX * CMAX];
      if (c <= 16) {
        sweep = jacobi_mixed16(X, V, c, N, tol, tiny2, mx0, Xf, Vf, Ms, Ws2);
      } else if constexpr (CMAX > 16) {
        __shared__ uint16_t sched32[31 * 16];
        __shared__ double dots[48], rotp[32];
        __shared__ int rflag[16];
        sweep = jacobi_mixed32(X, V, c, N, tol, tiny2, mx0, Xf, Vf, Ms, Ws2, sched32, dots, rotp, rflag);
      }
      fast = true;
    }
  } else {
    if (c <= 16) {
      __shared__ cf Xc[16 * 16], Vc[16 * 16];
      __shared__ cd Mc[16 * 16], Wc[16 * 16];
      sweep = jacobi_mixed16_c(X, V, c, N, tol, tiny2, mx0, Xc, Vc, Mc, Wc);
      fast = true;
    }
  }
  for (; !fast && sweep < 60; ++sweep) {
    if (tid == 0) changed = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int i = warp; i < N / 2; i += nwarp) {
        int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
        if (pp > qq) { int t = pp; pp = qq; qq = t; }
        if (qq >= c) continue;
        T* xp = X + pp * c;
        T* xq = X + qq * c;
        double a = 0, bb = 0;
        T g = zero_<T>();
        for (int rr = lane; rr < c; rr += 32) {
          a += abs2_(xp[rr]); bb += abs2_(xq[rr]); g = madc_(xp[rr], xq[rr], g);
        }
        a = warp_sum(a); bb = warp_sum(bb); g = warp_sum(g);
        double cs, sn;
        T e;
        if (!jacobi_rotation(a, bb, g, tol, tiny2, 2.220446049250313e-16, &cs, &sn, &e)) continue;
        const T se = scale_(e, sn), sec = conj_(se);
        for (int rr = lane; rr < c; rr += 32) {
          const T u = xp[rr], w = xq[rr];
          xp[rr] = sub_(scale_(u, cs), mul_(sec, w));
          xq[rr] = add_(mul_(se, u), scale_(w, cs));
          const T vu = V[pp * c + rr], vw = V[qq * c + rr];
          V[pp * c + rr] = sub_(scale_(vu, cs), mul_(sec, vw));
          V[qq * c + rr] = add_(mul_(se, vu), scale_(vw, cs));
        }
        if (lane == 0) changed = 1;
      }
      __syncthreads();
    }
    const int ch = changed;
    __syncthreads();
    if (!ch) { ++sweep; break; }
  }
  // singular values = column norms (a thread per column: no reductions on the dependent chain);
  // sort descending, ties by index
  for (int j = tid; j < c; j += blockDim.x) {
    double a0 = 0, a1 = 0;
    int rr = 0;
    for (; rr + 1 < c; rr += 2) {
      a0 += abs2_(X[j * c + rr]);
      a1 += abs2_(X[j * c + rr + 1]);
    }
    if (rr < c) a0 += abs2_(X[j * c + rr]);
    nrm[j] = sqrt(a0 + a1);
  }
  __syncthreads();
  for (int j = tid; j < c; j += blockDim.x) {
    int rk = 0;
    for (int i = 0; i < c; ++i) rk += (nrm[i] > nrm[j]) || (nrm[i] == nrm[j] && i < j);
    rank[j] = rk;
  }
  __syncthreads();
  for (int i = tid; i < c * c; i += blockDim.x) {
    const int j = i / c, row = i % c;
    C[rank[j] * c + row] = V[j * c + row];
  }
  for (int j = tid; j < c; j += blockDim.x) theta_out[rank[j]] = nrm[j];
  __syncthreads();

  // Q = Orth(M), M = C(0:b, 0:p)^H  (p x b, p = c - b >= b); Householder by warp 0 serially.
  // The initial Rayleigh-Ritz (c == b) has no momentum block: K = [C | 0].
  const int pdim = c - b;
  const bool with_x = pdim >= b;
  for (int i = tid; i < pdim * b; i += blockDim.x) {
    const int col = i / pdim, row = i % pdim;     // M(row, col) = conj(C(col, row))
    Qm[col * pdim + row] = conj_(C[row * c + col]);
  }
  __syncthreads();
  // (warp 0 forms each reflector; the columns it updates are spread over the warps)
  for (int j = 0; with_x && j < b; ++j) {
    T* x = Qm + j * pdim;
    if (warp == 0) {
      double part = 0;
      for (int r = j + 1 + lane; r < pdim; r += 32) part += abs2_(x[r]);
      const double xn2 = warp_sum(part);
      T tau, beta, inv_ab;
      householder_scalars(x[j], xn2, &tau, &beta, &inv_ab);
      for (int r = j + 1 + lane; r < pdim; r += 32) x[r] = mul_(x[r], inv_ab);
      __syncwarp();
      if (lane == 0) { x[j] = beta; tau_s[j] = tau; }
    }
    __syncthreads();
    const T tau = tau_s[j];
    for (int q = j + 1 + warp; q < b; q += nwarp) {
      T* y = Qm + q * pdim;
      T s = zero_<T>();
      for (int r = j + 1 + lane; r < pdim; r += 32) s = madc_(x[r], y[r], s);
      s = warp_sum(s);
      s = add_(s, y[j]);
      const T f = mul_(conj_(tau), s);
      __syncwarp();
      if (lane == 0) y[j] = sub_(y[j], f);
      for (int r = j + 1 + lane; r < pdim; r += 32) y[r] = sub_(y[r], mul_(x[r], f));
    }
    __syncthreads();
  }
  T* E = reinterpret_cast<T*>(rank + c + 4);  // p x b col-major scratch
  E = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(E) + 15) & ~(uintptr_t)15);
  for (int i = tid; i < pdim * b; i += blockDim.x) {
    const int col = i / pdim, row = i % pdim;
    E[i] = (row == col) ? from_real<T>(1.0) : zero_<T>();
  }
  __syncthreads();
  // form Q explicitly: E = I(:, 0:b); E <- H_j E for j = b-1 .. 0 (H_j = I - tau_j v_j v_j^H)
  for (int j = b - 1; with_x && j >= 0; --j) {
    const T* v = Qm + j * pdim;
    const T tau = tau_s[j];
    for (int q = j + warp; q < b; q += nwarp) {
      T* y = E + q * pdim;
      T s = zero_<T>();
      for (int r = j + 1 + lane; r < pdim; r += 32) s = madc_(v[r], y[r], s);
      s = warp_sum(s);
      s = add_(s, y[j]);
      const T f = mul_(tau, s);
      __syncwarp();
      if (lane == 0) y[j] = sub_(y[j], f);
      for (int r = j + 1 + lane; r < pdim; r += 32) y[r] = sub_(y[r], mul_(v[r], f));
    }
    __syncthreads();
  }
  // make diag(R) real non-negative: Q(:, j) *= phase(R(j, j))
  if (with_x)
    for (int e = tid; e < pdim * b; e += blockDim.x) {
      const int j = e / pdim;
      E[e] = mul_(E[e], phase_(Qm[j * pdim + j]));
    }
  __syncthreads();
  // K = [C(:, p:c) | C(:, 0:p) E]  (c x 2b row-major)
  for (int i = tid; i < c * 2 * b; i += blockDim.x) {
    const int row = i / (2 * b), col = i % (2 * b);
    T v;
    if (col < b) {
      v = C[(pdim + col) * c + row];
    } else if (!with_x) {
      v = zero_<T>();
    } else {
      const int q = col - b;
      v = zero_<T>();
      for (int l = 0; l < pdim; ++l) v = mad_(C[l * c + row], E[q * pdim + l], v);
    }
    K_out[i] = v;
  }
  if (tid == 0 && info) { info[0] += sweep; info[1] += 1; }   // totals over the solve
}

template <class T>
__global__ void __launch_bounds__(1024) rr_small_kernel(const T* __restrict__ Rt, int c, int b, double* theta_out,
                                                         T* K_out, int* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rr_small_cta<T>(smem_raw, Rt, c, b, theta_out, K_out, info);
}

template <class T>
inline size_t rr_small_smem(int c, int b) {
  const int pdim = c - b;
  return (size_t)3 * c * c * sizeof(T) + (size_t)c * b * sizeof(T) + c * sizeof(double) + (c + 4) * sizeof(int) + 16 +
         (size_t)pdim * b * sizeof(T);
}

// ------------------------------------------------------------------------------------------
// update: rows of buf (row-major, ld): x = buf[row, 0:c]; buf[row, 0:b] = x K(:, 0:b),
// buf[row, 2b:3b] = x K(:, b:2b). Three buffers (T, A_T, G_T) in one launch.
// ------------------------------------------------------------------------------------------
template <class T>
struct UpdSeg { T* buf; int64_t rows; int64_t ld; int blocks; };

template <class T>
__global__ void __launch_bounds__(256) update_kernel(UpdSeg<T> s0, UpdSeg<T> s1, UpdSeg<T> s2, int c, int b,
                                                     const T* __restrict__ K) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TRW = 64;
  T* Ks = reinterpret_cast<T*>(smem_raw);       // c x 2b
  T* tile = Ks + c * 2 * b;                     // TRW x c
  int blk = blockIdx.x;
  UpdSeg<T> s = s0;
  if (blk >= s0.blocks) { blk -= s0.blocks; s = s1; if (blk >= s1.blocks) { blk -= s1.blocks; s = s2; } }
  for (int i = threadIdx.x; i < c * 2 * b; i += blockDim.x) Ks[i] = K[i];
  const int64_t r0 = (int64_t)blk * TRW;
  const int nr = (int)imin<int64_t>(TRW, s.rows - r0);
  for (int i = threadIdx.x; i < nr * c; i += blockDim.x) tile[i] = s.buf[(r0 + i / c) * s.ld + (i % c)];
  __syncthreads();
  for (int i = threadIdx.x; i < nr * 2 * b; i += blockDim.x) {
    const int r = i / (2 * b), o = i % (2 * b);
    T v = zero_<T>();
    for (int l = 0; l < c; ++l) v = mad_(tile[r * c + l], Ks[l * 2 * b + o], v);
    const int col = o < b ? o : (o + b);        // V -> [0,b), X -> [2b,3b)
    s.buf[(r0 + r) * s.ld + col] = v;
  }
}

// ------------------------------------------------------------------------------------------
// residual: Res = G_V - V diag(theta_s^2); norms; Rs = Res / ||Res(:,j)|| (the preconditioner
// input, unit columns). One CTA, one warp per column.
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(1024) residual_kernel(const T* __restrict__ Tbuf, const T* __restrict__ Gbuf,
                                                         int n, int b, int64_t ld, const double* theta_s,
                                                         T* Res, double* res_norm, T* Rs, int* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int j = warp; j < b; j += nwarp) {
    const double th2 = theta_s[j] * theta_s[j];
    double a = 0;
    for (int k = lane; k < n; k += 32) {
      const T r = sub_(Gbuf[(int64_t)k * ld + j], scale_(Tbuf[(int64_t)k * ld + j], th2));
      Res[(int64_t)k * b + j] = r;
      a += abs2_(r);
    }
    a = warp_sum(a);
    const double nr = sqrt(a);
    if (lane == 0) {
      res_norm[j] = nr;
      if (!isfinite(nr)) atomicOr(err, DEV_ERR_NONFINITE);
    }
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int k = lane; k < n; k += 32) Rs[(int64_t)k * b + j] = scale_(Res[(int64_t)k * b + j], inv);
  }
}

// ------------------------------------------------------------------------------------------
// trimul: Y = L X with L an n x n matrix (row-major, only the triangle l in [lo(k), hi(k)] used)
// STORED in precision S (the sketch side: FP32 in the mixed form), X and Y (n x b, row-major) in
// the working precision T. Every entry of L is widened to T on load and all arithmetic is in T:
// the factor may be rounded to FP32, its application may not (with kappa(R) >> 1/u_32 an FP32
// product would lose exactly the directions of the smallest singular values). One warp per row.
// ------------------------------------------------------------------------------------------
template <class S, class T>
__global__ void trimul_kernel(const S* __restrict__ L, int n, const T* __restrict__ X, int64_t ldx, int b,
                              T* __restrict__ Y, int64_t ldy, int lower, int conj_l) {
  const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const int lo = lower ? 0 : k, hi = lower ? k : n - 1;
  const S* Lk = L + (int64_t)k * n;
  for (int c0 = 0; c0 < b; c0 += 8) {
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = zero_<T>();
    // four steps of a lane's walk per trip: their loads are issued together (the latency of
    // L2 loads, not the FP64 work, bounds this kernel); each lane still adds its terms in
    // ascending l, so the sums are the same as one step at a time
    int l = lo + lane;
    for (; l + 96 <= hi; l += 128) {
      T lk[4], xv[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        lk[u] = cvt_<T, S>(conj_l ? conj_(Lk[l + 32 * u]) : Lk[l + 32 * u]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          xv[u][q] = (c0 + q < b) ? X[(int64_t)(l + 32 * u) * ldx + c0 + q] : zero_<T>();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + q < b) acc[q] = mad_(lk[u], xv[u][q], acc[q]);
    }
    for (; l <= hi; l += 32) {
      const T lk = cvt_<T, S>(conj_l ? conj_(Lk[l]) : Lk[l]);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (c0 + q < b) acc[q] = mad_(lk, X[(int64_t)l * ldx + c0 + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (c0 + q < b) {
        const T s = warp_sum(acc[q]);
        if (lane == 0) Y[(int64_t)k * ldy + c0 + q] = s;
      }
    }
  }
}

// Warp-cooperative sum_{k = k0 + lane, step 32} conj(x[k*ldx]) y[k*ldy] for k < n with four
// independent accumulators per lane (dependent FP64 FMAs cost ~64 cycles each on GB300), then a
// butterfly over the warp. Every lane returns the total.
template <class T>
__device__ inline T warp_dotc(const T* x, int64_t ldx, const T* y, int64_t ldy, int k0, int n) {
  T a0 = zero_<T>(), a1 = zero_<T>(), a2 = zero_<T>(), a3 = zero_<T>();
  const int lane = threadIdx.x & 31;
  int k = k0 + lane;
  for (; k + 96 < n; k += 128) {
    a0 = madc_(x[(int64_t)k * ldx], y[(int64_t)k * ldy], a0);
    a1 = madc_(x[(int64_t)(k + 32) * ldx], y[(int64_t)(k + 32) * ldy], a1);
    a2 = madc_(x[(int64_t)(k + 64) * ldx], y[(int64_t)(k + 64) * ldy], a2);
    a3 = madc_(x[(int64_t)(k + 96) * ldx], y[(int64_t)(k + 96) * ldy], a3);
  }
  for (; k < n; k += 32) a0 = madc_(x[(int64_t)k * ldx], y[(int64_t)k * ldy], a0);
  return warp_sum(add_(add_(a0, a1), add_(a2, a3)));
}

// ------------------------------------------------------------------------------------------
// bcgs2_orth (one CTA): W (n x b at column offset wo of T, ld) is made orthogonal to the
// columns listed in [0, b) (V) and, when nx > 0, [2b, 3b) (X), twice (BCGS2), then replaced by
// Orth(W). E is an n x b scratch (row-major).
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(1024) bcgs2_orth_kernel(T* Tb, int n, int b, int64_t ld, int wo, int nx,
                                                           T* E, int passes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);     // q x b, q = b + nx
  T* tauv = P + 2 * b * b;                   // b
  T* sv = tauv + b;                          // b (s values)
  T* dg = sv + b;                            // b diag(R)
  __shared__ T sh_inv;
  __shared__ double sh_x2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5, NT = blockDim.x;
  const int q = b + nx;
  auto bcol = [&](int j) { return j < b ? j : (2 * b + (j - b)); };  // basis column -> T column
  for (int pass = 0; pass < passes && q > 0; ++pass) {
    for (int o = warp; o < q * b; o += nwarp) {
      const int j = o / b, cw = o % b;
      const T s = warp_dotc(Tb + bcol(j), ld, Tb + wo + cw, ld, 0, n);
      if (lane == 0) P[o] = s;
    }
    __syncthreads();
    for (int i = tid; i < n * b; i += NT) {
      const int k = i / b, cw = i % b;
      T w = Tb[(int64_t)k * ld + wo + cw];
      for (int j = 0; j < q; ++j) w = sub_(w, mul_(Tb[(int64_t)k * ld + bcol(j)], P[j * b + cw]));
      Tb[(int64_t)k * ld + wo + cw] = w;
    }
    __syncthreads();
  }
  // Householder QR of W (n x b) in place; v stored below the diagonal.
  for (int j = 0; j < b; ++j) {
    // d_cc = sum_{k > j} conj(W[k][j]) W[k][cc], cc >= j
    for (int cc = j + warp; cc < b; cc += nwarp) {
      const T s = warp_dotc(Tb + wo + j, ld, Tb + wo + cc, ld, j + 1, n);
      if (lane == 0) sv[cc] = s;
    }
    __syncthreads();
    if (tid == 0) {
      T tau, beta, inv_ab;
      const T alpha = Tb[(int64_t)j * ld + wo + j];
      householder_scalars(alpha, re_(sv[j]), &tau, &beta, &inv_ab);
      tauv[j] = tau; dg[j] = beta; sh_inv = inv_ab; sh_x2 = re_(sv[j]);
      for (int cc = j + 1; cc < b; ++cc)
        sv[cc] = add_(Tb[(int64_t)j * ld + wo + cc], mul_(conj_(inv_ab), sv[cc]));
    }
    __syncthreads();
    const T tau = tauv[j], inv_ab = sh_inv;
    for (int i = tid; i < (n - j) * b; i += NT) {
      const int k = j + i / b, cc = i % b;
      if (cc <= j) continue;
      const T f = mul_(conj_(tau), sv[cc]);
      const T vk = (k == j) ? from_real<T>(1.0) : mul_(Tb[(int64_t)k * ld + wo + j], inv_ab);
      Tb[(int64_t)k * ld + wo + cc] = sub_(Tb[(int64_t)k * ld + wo + cc], mul_(vk, f));
    }
    __syncthreads();
    for (int k = j + 1 + tid; k < n; k += NT) Tb[(int64_t)k * ld + wo + j] = mul_(Tb[(int64_t)k * ld + wo + j], inv_ab);
    if (tid == 0) Tb[(int64_t)j * ld + wo + j] = dg[j];
    __syncthreads();
  }
  // Q = H_0 ... H_{b-1} I(:, 0:b) into E, phases of diag(R) folded in, copied back to W
  for (int i = tid; i < n * b; i += NT) {
    const int k = i / b, cc = i % b;
    E[i] = (k == cc) ? from_real<T>(1.0) : zero_<T>();
  }
  __syncthreads();
  for (int j = b - 1; j >= 0; --j) {
    for (int cc = j + warp; cc < b; cc += nwarp) {
      const T s = E[(int64_t)j * b + cc];
      const T part = warp_dotc(Tb + wo + j, ld, E + cc, b, j + 1, n);
      if (lane == 0) sv[cc] = mul_(tauv[j], add_(s, part));
    }
    __syncthreads();
    for (int i = tid; i < (n - j) * b; i += NT) {
      const int k = j + i / b, cc = i % b;
      if (cc < j) continue;
      const T vk = (k == j) ? from_real<T>(1.0) : Tb[(int64_t)k * ld + wo + j];
      E[(int64_t)k * b + cc] = sub_(E[(int64_t)k * b + cc], mul_(vk, sv[cc]));
    }
    __syncthreads();
  }
  for (int i = tid; i < n * b; i += NT) {
    const int k = i / b, cc = i % b;
    Tb[(int64_t)k * ld + wo + cc] = mul_(E[i], phase_(dg[cc]));
  }
}

// BCGS2 + Orth with the rows of [V X] and W staged in shared memory (one CTA of 256 threads,
// used whenever n (q + b) elements fit; the kernel above is the fallback). Shared-memory operands
// avoid the L2 latency of every dependent step; the FP64 work (2 passes x 2 n q b FMAs, then
// 2 n b^2 for Householder and Q) runs at the single SM's DFMA rate. With wd.Wsl set (real FP64),
// the final W is also written as bf16 digits for the split Gram pass (see split.cuh).
// ------------------------------------------------------------------------------------------
// SVQB (Stathopoulos & Wu, SISC 2002), the alternative to Orth that Sec. 2.1 names: with
// S = W^H W and D = diag(S)^{-1/2}, the eigendecomposition D S D = Z Theta Z^H, eigenvalues below
// eps max(Theta) raised to it, and W <- W D Z Theta^{-1/2}. The b x b eigenproblem runs as a
// cyclic two-sided Jacobi with the round-robin parallel ordering: per round, the rotations of the
// disjoint pairs (one thread each), then U^H on their rows and U on their columns (and on Z), with
// U = diag(1, e^{-i phi}) J on (p, q), phi the phase of M_pq and J the real rotation of
// Golub & Van Loan's symmetric Schur step. One CTA; M, Z column-major b x b in shared memory.
// ------------------------------------------------------------------------------------------

// S (col-major b x b) = W^H W over rows [0, rows) of W (row-major rows x b); a warp per entry
// of the upper triangle, the lower one mirrored.
template <class T>
__device__ void cta_gram(const T* Ws, int rows, int b, T* S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = blockDim.x >> 5;
  for (int e = warp; e < b * b; e += NW) {
    const int i = e / b, j = e % b;
    if (j < i) continue;
    T a0 = zero_<T>(), a1 = zero_<T>();
    int r = lane;
    for (; r + 32 < rows; r += 64) {
      a0 = madc_(Ws[(size_t)r * b + i], Ws[(size_t)r * b + j], a0);
      a1 = madc_(Ws[(size_t)(r + 32) * b + i], Ws[(size_t)(r + 32) * b + j], a1);
    }
    if (r < rows) a0 = madc_(Ws[(size_t)r * b + i], Ws[(size_t)r * b + j], a0);
    const T v = warp_sum(add_(a0, a1));
    if (lane == 0) {
      S[(size_t)j * b + i] = v;          // (i, j) = sum conj(w_i) w_j
      S[(size_t)i * b + j] = conj_(v);
    }
  }
  __syncthreads();
}

template <class T>
__device__ inline T phase_of_(T g, double ag) { return scale_(g, 1.0 / ag); }

// Hermitian b x b M (b <= 32) -> diagonal; Z accumulates the rotations (starts as I). rot: 2
// doubles per pair, ph: phases, rf: flags (16 pairs). Returns the sweeps taken.
template <class T>
__device__ int herm_jacobi(T* M, T* Z, int b, double* rot, T* ph, int* rf, int* any) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int N = b + (b & 1);
  const double tol = (double)imax(b, 4) * 2.220446049250313e-16;
  for (int e = tid; e < b * b; e += NT) Z[e] = (e / b == e % b) ? from_real<T>(1.0) : zero_<T>();
  __syncthreads();
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (tid == 0) *any = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      if (tid < N / 2) {
        int pp = rr_slot(tid, r, N), qq = rr_slot(N - 1 - tid, r, N);
        if (pp > qq) { const int t = pp; pp = qq; qq = t; }
        int f = 0;
        if (qq < b) {
          const double a = re_(M[(size_t)pp * b + pp]), d = re_(M[(size_t)qq * b + qq]);
          const T g = M[(size_t)qq * b + pp];   // row pp, column qq
          const double ag = sqrt(abs2_(g));
          if (ag > tol * sqrt(fabs(a * d)) && ag > 0.0) {
            const double tau = (d - a) / (2.0 * ag);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t);
            rot[2 * tid] = c;
            rot[2 * tid + 1] = t * c;
            ph[tid] = phase_of_(g, ag);
            f = 1;
            *any = 1;
          }
        }
        rf[tid] = f;
      }
      __syncthreads();
      // rows p, q <- U^H rows: p: c row_p - s e row_q, q: s row_p + c e row_q
      for (int e = tid; e < (N / 2) * b; e += NT) {
        const int i = e / b, col = e % b;
        if (!rf[i]) continue;
        int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
        if (pp > qq) { const int t = pp; pp = qq; qq = t; }
        const double c = rot[2 * i], sn = rot[2 * i + 1];
        const T ep = ph[i];
        const T mp = M[(size_t)col * b + pp], mq = M[(size_t)col * b + qq];
        M[(size_t)col * b + pp] = sub_(scale_(mp, c), scale_(mul_(ep, mq), sn));
        M[(size_t)col * b + qq] = add_(scale_(mp, sn), scale_(mul_(ep, mq), c));
      }
      __syncthreads();
      // columns p, q of M and Z <- U: p: c col_p - s conj(e) col_q, q: s col_p + c conj(e) col_q
      for (int e = tid; e < (N / 2) * b * 2; e += NT) {
        const int which = e / ((N / 2) * b), e2 = e % ((N / 2) * b);
        const int i = e2 / b, row = e2 % b;
        if (!rf[i]) continue;
        int pp = rr_slot(i, r, N), qq = rr_slot(N - 1 - i, r, N);
        if (pp > qq) { const int t = pp; pp = qq; qq = t; }
        T* A = which ? Z : M;
        const double c = rot[2 * i], sn = rot[2 * i + 1];
        const T ec = conj_(ph[i]);
        const T ap = A[(size_t)pp * b + row], aq = A[(size_t)qq * b + row];
        A[(size_t)pp * b + row] = sub_(scale_(ap, c), scale_(mul_(ec, aq), sn));
        A[(size_t)qq * b + row] = add_(scale_(ap, sn), scale_(mul_(ec, aq), c));
      }
      __syncthreads();
      if (tid < N / 2 && rf[tid]) {
        int pp = rr_slot(tid, r, N), qq = rr_slot(N - 1 - tid, r, N);
        if (pp > qq) { const int t = pp; pp = qq; qq = t; }
        M[(size_t)qq * b + pp] = zero_<T>();
        M[(size_t)pp * b + qq] = zero_<T>();
      }
      __syncthreads();
    }
    if (!*any) { ++sweep; break; }
    __syncthreads();
  }
  return sweep;
}

// W (rows x b, row-major) -> out (rows x b): W D Z Theta^{-1/2} from S = W^H W (already summed,
// col-major in S; consumed). M, Z: b x b scratch; dsc, th: b doubles; rot, ph, rf, any: the
// Jacobi scratch. Every thread of the CTA takes part.
template <class T>
__device__ void cta_svqb(const T* Ws, int rows, int b, T* S, T* Z, double* dsc, double* th, T* out, double* rot,
                         T* ph, int* rf, int* any) {
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int j = tid; j < b; j += NT) {
    const double s = re_(S[(size_t)j * b + j]);
    dsc[j] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += NT) {
    const int col = e / b, row = e % b;
    S[e] = scale_(S[e], dsc[row] * dsc[col]);
  }
  __syncthreads();
  herm_jacobi<T>(S, Z, b, rot, ph, rf, any);
  if (tid == 0) {
    double top = 0.0;
    for (int j = 0; j < b; ++j) top = fmax(top, re_(S[(size_t)j * b + j]));
    for (int j = 0; j < b; ++j) {
      const double t = top > 0.0 ? fmax(re_(S[(size_t)j * b + j]), 2.220446049250313e-16 * top) : 1.0;
      th[j] = 1.0 / sqrt(t);
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * b; e += NT) {
    const int k = e / b, j = e % b;
    T v = zero_<T>();
    for (int i = 0; i < b; ++i) v = mad_(scale_(Ws[(size_t)k * b + i], dsc[i]), Z[(size_t)j * b + i], v);
    out[e] = scale_(v, th[j]);
  }
  __syncthreads();
}

// One CTA of exactly 256 threads; smem_raw: bcgs2_smem_bytes(n, b, nx + nl) bytes.
template <class T>
__device__ void bcgs2_orth_cta(unsigned char* smem_raw, T* __restrict__ Tb, int n, int b, int64_t ld, int wo, int nx,
                               int passes, split::WDigits wd, int* err, int svqb, const T* __restrict__ Dl, int nl,
                               int64_t ldl) {
  constexpr int NT = 256, NW = NT / 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = b + nx + nl;   // V, X, and the deflated (locked) columns Dl
  const int QB = q * b;
  T* Bs = reinterpret_cast<T*>(smem_raw);   // n x q: V then X (row-major); later E = Q (n x b)
  T* Ws = Bs + (size_t)n * q;               // n x b
  T* Pp = Ws + (size_t)n * b;               // up to 4 x q x b partial projections
  T* P = Pp + 4 * (size_t)QB;               // q x b
  T* tauv = P + QB;
  T* dg = tauv + b;
  T* sv = dg + b;
  double* red = reinterpret_cast<double*>(sv + b);   // NW x 16 column maxima
  __shared__ T sh_inv;
  __shared__ int Fs[32];   // digit-block width of the split Gram pass, <= 32
  auto pcol = [&](int64_t k, int j) {   // column j of the projection set [V X Dl] in row k
    return j < b ? Tb[k * ld + j] : j < b + nx ? Tb[k * ld + 2 * b + (j - b)] : Dl[k * ldl + (j - b - nx)];
  };
  for (int e = tid; e < n * b; e += NT) {
    const int k = e / b, cw = e % b;
    Ws[e] = Tb[(int64_t)k * ld + wo + cw];
  }
  if (passes > 0)
    for (int e = tid; e < n * q; e += NT) {
      const int k = e / q, j = e % q;
      Bs[e] = pcol(k, j);
    }
  __syncthreads();
  const int G = QB >= NT ? 1 : imin(4, NT / QB);
  for (int pass = 0; pass < passes; ++pass) {
    // P = [V X]^H W, rows split into G groups per output
    for (int t = tid; t < G * QB; t += NT) {
      const int o = t % QB, g = t / QB;
      const int j = o / b, cw = o % b;
      const int r0 = (int)((int64_t)g * n / G), r1 = (int)((int64_t)(g + 1) * n / G);
      T a0 = zero_<T>(), a1 = zero_<T>(), a2 = zero_<T>(), a3 = zero_<T>();
      int r = r0;
      for (; r + 3 < r1; r += 4) {
        a0 = madc_(Bs[(size_t)r * q + j], Ws[(size_t)r * b + cw], a0);
        a1 = madc_(Bs[(size_t)(r + 1) * q + j], Ws[(size_t)(r + 1) * b + cw], a1);
        a2 = madc_(Bs[(size_t)(r + 2) * q + j], Ws[(size_t)(r + 2) * b + cw], a2);
        a3 = madc_(Bs[(size_t)(r + 3) * q + j], Ws[(size_t)(r + 3) * b + cw], a3);
      }
      for (; r < r1; ++r) a0 = madc_(Bs[(size_t)r * q + j], Ws[(size_t)r * b + cw], a0);
      Pp[(size_t)g * QB + o] = add_(add_(a0, a1), add_(a2, a3));
    }
    __syncthreads();
    for (int o = tid; o < QB; o += NT) {
      T sum = Pp[o];
      for (int g = 1; g < G; ++g) sum = add_(sum, Pp[(size_t)g * QB + o]);
      P[o] = sum;
    }
    __syncthreads();
    // W -= [V X] P
    for (int e = tid; e < n * b; e += NT) {
      const int k = e / b, cw = e % b;
      T w = Ws[e];
      for (int j = 0; j < q; ++j) w = sub_(w, mul_(Bs[(size_t)k * q + j], P[j * b + cw]));
      Ws[e] = w;
    }
    __syncthreads();
  }
  T* E = Bs;
  if (svqb) {
    // SVQB in place of Orth: S = W^H W, then W D Z Theta^{-1/2} into E (Pp holds S and Z)
    __shared__ double sq_rot[32];
    __shared__ T sq_ph[16];
    __shared__ int sq_rf[16], sq_any;
    cta_gram<T>(Ws, n, b, Pp);
    cta_svqb<T>(Ws, n, b, Pp, Pp + (size_t)b * b, reinterpret_cast<double*>(tauv), reinterpret_cast<double*>(sv), E,
                sq_rot, sq_ph, sq_rf, &sq_any);
    for (int j = tid; j < b; j += NT) dg[j] = from_real<T>(1.0);
    __syncthreads();
  } else {
  // Householder QR of W (n x b) in place; v (scaled by 1/(alpha - beta)) stored below the diagonal
  for (int j = 0; j < b; ++j) {
    for (int cc = j + warp; cc < b; cc += NW) {
      T a0 = zero_<T>(), a1 = zero_<T>();
      int k = j + 1 + lane;
      for (; k + 32 < n; k += 64) {
        a0 = madc_(Ws[(size_t)k * b + j], Ws[(size_t)k * b + cc], a0);
        a1 = madc_(Ws[(size_t)(k + 32) * b + j], Ws[(size_t)(k + 32) * b + cc], a1);
      }
      if (k < n) a0 = madc_(Ws[(size_t)k * b + j], Ws[(size_t)k * b + cc], a0);
      const T s = warp_sum(add_(a0, a1));
      if (lane == 0) sv[cc] = s;
    }
    __syncthreads();
    if (tid == 0) {
      T tau, beta, inv_ab;
      householder_scalars(Ws[(size_t)j * b + j], re_(sv[j]), &tau, &beta, &inv_ab);
      tauv[j] = tau;
      dg[j] = beta;
      sh_inv = inv_ab;
      for (int cc = j + 1; cc < b; ++cc) sv[cc] = add_(Ws[(size_t)j * b + cc], mul_(conj_(inv_ab), sv[cc]));
    }
    __syncthreads();
    const T tau = tauv[j], inv_ab = sh_inv;
    for (int e = tid; e < (n - j) * b; e += NT) {
      const int k = j + e / b, cc = e % b;
      if (cc <= j) continue;
      const T f = mul_(conj_(tau), sv[cc]);
      const T vk = (k == j) ? from_real<T>(1.0) : mul_(Ws[(size_t)k * b + j], inv_ab);
      Ws[(size_t)k * b + cc] = sub_(Ws[(size_t)k * b + cc], mul_(vk, f));
    }
    __syncthreads();
    for (int k = j + 1 + tid; k < n; k += NT) Ws[(size_t)k * b + j] = mul_(Ws[(size_t)k * b + j], inv_ab);
    if (tid == 0) Ws[(size_t)j * b + j] = dg[j];
    __syncthreads();
  }
  // Q = H_0 ... H_{b-1} I(:, 0:b) into E (the space of [V X]), phases of diag(R) folded in
  for (int e = tid; e < n * b; e += NT) {
    const int k = e / b, cc = e % b;
    E[e] = (k == cc) ? from_real<T>(1.0) : zero_<T>();
  }
  __syncthreads();
  for (int j = b - 1; j >= 0; --j) {
    for (int cc = j + warp; cc < b; cc += NW) {
      T a0 = zero_<T>(), a1 = zero_<T>();
      int k = j + 1 + lane;
      for (; k + 32 < n; k += 64) {
        a0 = madc_(Ws[(size_t)k * b + j], E[(size_t)k * b + cc], a0);
        a1 = madc_(Ws[(size_t)(k + 32) * b + j], E[(size_t)(k + 32) * b + cc], a1);
      }
      if (k < n) a0 = madc_(Ws[(size_t)k * b + j], E[(size_t)k * b + cc], a0);
      const T s = warp_sum(add_(a0, a1));
      if (lane == 0) sv[cc] = mul_(tauv[j], add_(E[(size_t)j * b + cc], s));
    }
    __syncthreads();
    for (int e = tid; e < (n - j) * b; e += NT) {
      const int k = j + e / b, cc = e % b;
      if (cc < j) continue;
      const T vk = (k == j) ? from_real<T>(1.0) : Ws[(size_t)k * b + j];
      E[(size_t)k * b + cc] = sub_(E[(size_t)k * b + cc], mul_(vk, sv[cc]));
    }
    __syncthreads();
  }
  }  // Householder
  for (int e = tid; e < n * b; e += NT) {
    const int k = e / b, cc = e % b;
    const T v = mul_(E[e], phase_(dg[cc]));
    E[e] = v;
    Tb[(int64_t)k * ld + wo + cc] = v;
  }
  if (wd.Wsl == nullptr) return;
  // digits of the final W (real FP64 only): column exponents, then digit tiles
  __syncthreads();
  const int BP = wd.BP, N = split::SL * BP;
  bool bad = false;
  for (int cc = warp; cc < BP; cc += NW) {
    double mx = 0;
    if (cc < b)
      for (int k = lane; k < n; k += 32) {
        const double a = fabs(re_(E[(size_t)k * b + cc]));
        bad |= !(a <= 1.7976931348623157e308);
        mx = fmax(mx, a);
      }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      Fs[cc] = split::group_exp(mx);
      wd.F[cc] = Fs[cc];
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(err, DEV_ERR_NONFINITE);
  const int64_t total = wd.NKB * split::TK * BP;
  for (int64_t e = tid; e < total; e += NT) {
    const int j = (int)(e % BP);
    const int64_t k = e / BP;
    const double x = (k < n && j < b) ? re_(E[(size_t)k * b + j]) : 0.0;
    int d[split::SL];
    split::split8(x, Fs[j], d);
    uint16_t* out = wd.Wsl + (size_t)(k / split::TK) * (N * split::TK);
    const int kk = (int)(k % split::TK);
#pragma unroll
    for (int qd = 0; qd < split::SL; ++qd) out[split::core_off(qd * BP + j, kk, N)] = split::bf16_of(d[qd]);
  }
  (void)red;
}

template <class T>
__global__ void __launch_bounds__(256) bcgs2_orth_smem_kernel(T* __restrict__ Tb, int n, int b, int64_t ld, int wo,
                                                              int nx, int passes, split::WDigits wd, int* err,
                                                              int svqb, const T* __restrict__ Dl, int nl,
                                                              int64_t ldl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bcgs2_orth_cta<T>(smem_raw, Tb, n, b, ld, wo, nx, passes, wd, err, svqb, Dl, nl, ldl);
}

// dynamic shared memory of bcgs2_orth_cta for q = b + (columns projected out besides V)
template <class T>
inline size_t bcgs2_smem_bytes(int n, int b, int extra) {
  const int q = b + extra;
  return ((size_t)n * (q + b) + 5 * (size_t)q * b + 3 * b) * sizeof(T) + 16 * 8 * sizeof(double) + 64;
}

// L2-coherent load (data written by other CTAs of a cooperative grid)
__device__ __forceinline__ double ldcg_(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cd ldcg_(const cd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Householder QR of a rows x b block (row-major, ld b) in shared memory by one CTA: on return the
// upper triangle holds R (diag = beta), the strict lower part the reflector vectors scaled by
// 1/(alpha - beta) (v_j = 1 implicit) and tau[j] their scalars; H_j = I - tau_j v_j v_j^H and the
// block equals H_0 ... H_{b-1} [R; 0]. dgo[j] = beta_j.
template <class T>
__device__ void cta_householder(T* Wm, int rows, int b, T* tau, T* dgo, T* sv, T* sh_inv) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NT = blockDim.x, NW = NT >> 5;
  for (int j = 0; j < b; ++j) {
    for (int cc = j + warp; cc < b; cc += NW) {
      T a0 = zero_<T>(), a1 = zero_<T>();
      int k = j + 1 + lane;
      for (; k + 32 < rows; k += 64) {
        a0 = madc_(Wm[(size_t)k * b + j], Wm[(size_t)k * b + cc], a0);
        a1 = madc_(Wm[(size_t)(k + 32) * b + j], Wm[(size_t)(k + 32) * b + cc], a1);
      }
      if (k < rows) a0 = madc_(Wm[(size_t)k * b + j], Wm[(size_t)k * b + cc], a0);
      const T sum = warp_sum(add_(a0, a1));
      if (lane == 0) sv[cc] = sum;
    }
    __syncthreads();
    if (tid == 0) {
      T t, beta, inv_ab;
      householder_scalars(Wm[(size_t)j * b + j], re_(sv[j]), &t, &beta, &inv_ab);
      tau[j] = t;
      dgo[j] = beta;
      *sh_inv = inv_ab;
      for (int cc = j + 1; cc < b; ++cc) sv[cc] = add_(Wm[(size_t)j * b + cc], mul_(conj_(inv_ab), sv[cc]));
    }
    __syncthreads();
    const T tj = tau[j], inv_ab = *sh_inv;
    for (int e = tid; e < (rows - j) * b; e += NT) {
      const int k = j + e / b, cc = e % b;
      if (cc <= j) continue;
      const T f = mul_(conj_(tj), sv[cc]);
      const T vk = (k == j) ? from_real<T>(1.0) : mul_(Wm[(size_t)k * b + j], inv_ab);
      Wm[(size_t)k * b + cc] = sub_(Wm[(size_t)k * b + cc], mul_(vk, f));
    }
    __syncthreads();
    for (int k = j + 1 + tid; k < rows; k += NT) Wm[(size_t)k * b + j] = mul_(Wm[(size_t)k * b + j], inv_ab);
    if (tid == 0) Wm[(size_t)j * b + j] = dgo[j];
    __syncthreads();
  }
}

// E (rows x b) <- H_0 ... H_{b-1} E with the reflectors stored by cta_householder in Vm (rows x b).
// from_identity: E = [I; 0] on entry, so H_j only touches columns >= j.
template <class T>
__device__ void cta_apply_q(const T* Vm, const T* tau, int rows, int b, T* E, T* sv, bool from_identity) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NT = blockDim.x, NW = NT >> 5;
  for (int j = b - 1; j >= 0; --j) {
    const int c0 = from_identity ? j : 0;
    for (int cc = c0 + warp; cc < b; cc += NW) {
      T a0 = zero_<T>(), a1 = zero_<T>();
      int k = j + 1 + lane;
      for (; k + 32 < rows; k += 64) {
        a0 = madc_(Vm[(size_t)k * b + j], E[(size_t)k * b + cc], a0);
        a1 = madc_(Vm[(size_t)(k + 32) * b + j], E[(size_t)(k + 32) * b + cc], a1);
      }
      if (k < rows) a0 = madc_(Vm[(size_t)k * b + j], E[(size_t)k * b + cc], a0);
      const T sum = warp_sum(add_(a0, a1));
      if (lane == 0) sv[cc] = mul_(tau[j], add_(E[(size_t)j * b + cc], sum));
    }
    __syncthreads();
    for (int e = tid; e < (rows - j) * b; e += NT) {
      const int k = j + e / b, cc = e % b;
      if (cc < c0) continue;
      const T vk = (k == j) ? from_real<T>(1.0) : Vm[(size_t)k * b + j];
      E[(size_t)k * b + cc] = sub_(E[(size_t)k * b + cc], mul_(vk, sv[cc]));
    }
    __syncthreads();
  }
}

// BCGS2 + Orth over G cooperating CTAs, CTA g owning rows [g n / G, (g+1) n / G). The projections
// [V X]^H W are summed from per-CTA partials in CTA order after a grid barrier (two alternating
// global buffers, one barrier per pass). Orth(W) is a one-level TSQR: each CTA reduces its rows
// to R_g by Householder steps, every CTA then factors the same stack [R_0; ...; R_{G-1}] (same
// arithmetic, so all hold the same R and stack Q_s) and applies its local reflectors to its
// b x b block of Q_s. Q = blockdiag(Q_g) Q_s is the thin Householder Q of W (diag(R) made real
// non-negative as in the single-CTA kernel). With wd.Wsl set, the column maxima go through one
// more barrier and every CTA writes the bf16 digits of its rows.
template <class T>
__global__ void __launch_bounds__(256) bcgs2_orth_coop_kernel(T* __restrict__ Tb, int n, int b, int64_t ld, int wo,
                                                              int nx, int passes, T* __restrict__ gs,
                                                              split::WDigits wd, int* err, int svqb,
                                                              const T* __restrict__ Dl, int nl, int64_t ldl) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NT = blockDim.x, NW = NT >> 5;
  const int G = gridDim.x, g = blockIdx.x;
  const int q = b + nx + nl, QB = q * b, SB = G * b;   // projection set [V X Dl]
  const int r0 = (int)((int64_t)g * n / G), r1 = (int)((int64_t)(g + 1) * n / G), rows = r1 - r0;
  const int rmax = (n + G - 1) / G;
  T* Bs = reinterpret_cast<T*>(smem_raw);   // rmax x q (V, X); later this CTA's rows of Q
  T* Ws = Bs + (size_t)rmax * imax(q, b);   // rmax x b
  T* P = Ws + (size_t)rmax * b;             // q x b
  T* S = P + QB;                            // SB x b: the stack of R factors, then its reflectors
  T* E = S + (size_t)SB * b;                // SB x b: Q_s
  T* tl = E + (size_t)SB * b;               // local taus
  T* ts = tl + b;                           // stack taus
  T* sv = ts + b;
  T* dl = sv + b;                           // local betas (unused after the stack)
  T* dg = dl + b;                           // stack betas = diag(R)
  __shared__ T sh_inv;
  __shared__ int Fs[32];   // digit-block width of the split Gram pass, <= 32
  T* gP0 = gs;
  T* gP1 = gP0 + (size_t)G * QB;
  T* gR = gP1 + (size_t)G * QB;
  double* gmx = reinterpret_cast<double*>(gR + (size_t)G * b * b);
  auto pcol = [&](int64_t k, int j) {   // column j of the projection set [V X Dl] in row k
    return j < b ? Tb[k * ld + j] : j < b + nx ? Tb[k * ld + 2 * b + (j - b)] : Dl[k * ldl + (j - b - nx)];
  };

  for (int e = tid; e < rows * b; e += NT) {
    const int k = e / b, cw = e % b;
    Ws[e] = Tb[(int64_t)(r0 + k) * ld + wo + cw];
  }
  if (passes > 0)
    for (int e = tid; e < rows * q; e += NT) {
      const int k = e / q, j = e % q;
      Bs[e] = pcol((int64_t)(r0 + k), j);
    }
  __syncthreads();
  for (int pass = 0; pass < passes; ++pass) {
    T* gP = (pass & 1) ? gP1 : gP0;
    for (int o = tid; o < QB; o += NT) {
      const int j = o / b, cw = o % b;
      T a0 = zero_<T>(), a1 = zero_<T>();
      int k = 0;
      for (; k + 1 < rows; k += 2) {
        a0 = madc_(Bs[(size_t)k * q + j], Ws[(size_t)k * b + cw], a0);
        a1 = madc_(Bs[(size_t)(k + 1) * q + j], Ws[(size_t)(k + 1) * b + cw], a1);
      }
      if (k < rows) a0 = madc_(Bs[(size_t)k * q + j], Ws[(size_t)k * b + cw], a0);
      gP[(size_t)g * QB + o] = add_(a0, a1);
    }
    grid.sync();
    for (int o = tid; o < QB; o += NT) {
      T sum = ldcg_(gP + o);
      for (int h = 1; h < G; ++h) sum = add_(sum, ldcg_(gP + (size_t)h * QB + o));
      P[o] = sum;
    }
    __syncthreads();
    for (int e = tid; e < rows * b; e += NT) {
      const int k = e / b, cw = e % b;
      T w = Ws[e];
      for (int j = 0; j < q; ++j) w = sub_(w, mul_(Bs[(size_t)k * q + j], P[j * b + cw]));
      Ws[e] = w;
    }
    __syncthreads();
  }
  T* QL = Bs;
  if (svqb) {
    // SVQB in place of Orth: every CTA sums the same per-CTA Gram partials in CTA order, solves
    // the same b x b eigenproblem and scales its own rows
    __shared__ double sq_rot[32];
    __shared__ T sq_ph[16];
    __shared__ int sq_rf[16], sq_any;
    cta_gram<T>(Ws, rows, b, S);
    for (int e = tid; e < b * b; e += NT) gR[(size_t)g * b * b + e] = S[e];
    grid.sync();
    for (int e = tid; e < b * b; e += NT) {
      T sum = ldcg_(gR + e);
      for (int h = 1; h < G; ++h) sum = add_(sum, ldcg_(gR + (size_t)h * b * b + e));
      S[e] = sum;
    }
    __syncthreads();
    cta_svqb<T>(Ws, rows, b, S, E, reinterpret_cast<double*>(tl), reinterpret_cast<double*>(ts), QL, sq_rot, sq_ph,
                sq_rf, &sq_any);
    for (int j = tid; j < b; j += NT) dg[j] = from_real<T>(1.0);
    __syncthreads();
  } else {
  // local R_g
  cta_householder<T>(Ws, rows, b, tl, dl, sv, &sh_inv);
  for (int e = tid; e < b * b; e += NT) {
    const int r = e / b, cc = e % b;
    gR[(size_t)g * b * b + e] = (cc >= r) ? Ws[e] : zero_<T>();
  }
  grid.sync();
  for (int e = tid; e < SB * b; e += NT) S[e] = ldcg_(gR + e);
  __syncthreads();
  cta_householder<T>(S, SB, b, ts, dg, sv, &sh_inv);
  for (int e = tid; e < SB * b; e += NT) {
    const int k = e / b, cc = e % b;
    E[e] = (k == cc) ? from_real<T>(1.0) : zero_<T>();
  }
  __syncthreads();
  cta_apply_q<T>(S, ts, SB, b, E, sv, true);
  // this CTA's rows of Q: H_local [Q_s block g; 0]
  for (int e = tid; e < rows * b; e += NT) {
    const int k = e / b, cc = e % b;
    QL[e] = (k < b) ? E[(size_t)(g * b + k) * b + cc] : zero_<T>();
  }
  __syncthreads();
  cta_apply_q<T>(Ws, tl, rows, b, QL, sv, false);
  }  // Householder
  for (int e = tid; e < rows * b; e += NT) {
    const int k = e / b, cc = e % b;
    const T v = mul_(QL[e], phase_(dg[cc]));
    QL[e] = v;
    Tb[(int64_t)(r0 + k) * ld + wo + cc] = v;
  }
  if (wd.Wsl == nullptr) return;
  const int BP = wd.BP, N = split::SL * BP;
  __syncthreads();
  bool bad = false;
  for (int cc = warp; cc < BP; cc += NW) {
    double mx = 0;
    if (cc < b)
      for (int k = lane; k < rows; k += 32) {
        const double a = fabs(re_(QL[(size_t)k * b + cc]));
        bad |= !(a <= 1.7976931348623157e308);
        mx = fmax(mx, a);
      }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) gmx[(size_t)g * 32 + cc] = mx;
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(err, DEV_ERR_NONFINITE);
  grid.sync();
  if (tid < BP) {
    double mx = 0;
    for (int h = 0; h < G; ++h) mx = fmax(mx, __ldcg(gmx + (size_t)h * 32 + tid));
    Fs[tid] = split::group_exp(mx);
    if (g == 0) wd.F[tid] = Fs[tid];
  }
  __syncthreads();
  const int64_t k_end = (g == G - 1) ? wd.NKB * split::TK : r1;   // the last CTA writes the padding rows
  const int64_t total = (k_end - r0) * BP;
  for (int64_t e = tid; e < total; e += NT) {
    const int j = (int)(e % BP);
    const int64_t k = r0 + e / BP;
    const double x = (k < n && j < b) ? re_(QL[(size_t)(k - r0) * b + j]) : 0.0;
    int d[split::SL];
    split::split8(x, Fs[j], d);
    uint16_t* out = wd.Wsl + (size_t)(k / split::TK) * (N * split::TK);
    const int kk = (int)(k % split::TK);
#pragma unroll
    for (int qd = 0; qd < split::SL; ++qd) out[split::core_off(qd * BP + j, kk, N)] = split::bf16_of(d[qd]);
  }
}

// V0 = Vt(:, n-b:n) (sketch precision, col-major n x n) -> T columns [0, b) in double/complex128
template <class S, class T>
__global__ void take_start_kernel(const S* Vt, int n, int b, T* Tb, int64_t ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * b) return;
  const int k = (int)(i / b), j = (int)(i % b);
  Tb[(int64_t)k * ld + j] = cvt_<T, S>(Vt[(int64_t)(n - b + j) * n + k]);
}

// copy columns [src, src+w) of a row-major buffer to [dst, dst+w) (used to move V0 into the
// W slot for the first Gram pass and back), or out to a compact row-major array.
template <class T>
__global__ void copy_cols_kernel(const T* src, int64_t lds, int so, T* dst, int64_t ldd, int dof, int64_t rows, int w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * w) return;
  const int64_t r = i / w;
  const int c = (int)(i % w);
  dst[r * ldd + dof + c] = src[r * lds + so + c];
}

// outputs: ascending order (reverse of the descending Theta_s block), first k of b
// Per row of buf (row-major, ld): columns dst[t] <- old columns src[t], t < cnt (all reads of a row
// before its writes, so the map may move columns in place). Compacts the active block when
// columns are locked and orders the final columns.
struct ColMap { int cnt; int src[64]; int dst[64]; };

template <class T>
__global__ void gather_cols_kernel(T* buf, int64_t rows, int64_t ld, ColMap map) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  T v[64];
  for (int t = 0; t < map.cnt; ++t) v[t] = buf[r * ld + map.src[t]];
  for (int t = 0; t < map.cnt; ++t) buf[r * ld + map.dst[t]] = v[t];
}

template <class T>
__global__ void outputs_kernel(const T* Tb, const T* ATb, int64_t n, int64_t m, int b, int k, int64_t ld,
                               const double* theta_s, const double* res_norm, double* sigma, T* Vout, T* Uout,
                               double* resid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (n + (Uout ? m : 0)) * k;
  if (i < k) {
    sigma[i] = theta_s[b - 1 - i];
    if (resid) resid[i] = res_norm[b - 1 - i];
  }
  if (i >= tot) return;
  const int64_t r = i / k;
  const int j = (int)(i % k);
  const int src = b - 1 - j;
  if (r < n) {
    Vout[r * k + j] = Tb[r * ld + src];
  } else {
    const int64_t rr = r - n;
    const double s = theta_s[src];
    Uout[rr * k + j] = scale_(ATb[rr * ld + src], 1.0 / s);
  }
}

// Z (rows x q, row-major, ld) with entries uniform in [-1, 1) (real and imaginary parts) from
// SplitMix64 output number 2 (r q + j) (+1 for the imaginary part) of the stream `seed`.
__device__ inline double uniform_pm1(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; }
__device__ inline void fill_value(double* z, uint64_t seed, uint64_t c) { *z = uniform_pm1(splitmix64_at(seed, 2 * c)); }
__device__ inline void fill_value(cd* z, uint64_t seed, uint64_t c) {
  z->x = uniform_pm1(splitmix64_at(seed, 2 * c));
  z->y = uniform_pm1(splitmix64_at(seed, 2 * c + 1));
}
template <class T>
__global__ void fill_random_kernel(T* Z, int64_t rows, int q, int64_t ld, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * q) return;
  fill_value(&Z[(i / q) * ld + (i % q)], seed, (uint64_t)i);
}

// Out (rows x b, ldo) = In (rows x q, ldi) K (q x b, ldk); one thread per output element
template <class T>
__global__ void small_gemm_kernel(const T* __restrict__ In, int64_t ldi, int q, const T* __restrict__ K, int ldk, int b,
                                  T* __restrict__ Out, int64_t ldo, int64_t rows) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * b) return;
  const int64_t r = i / b;
  const int j = (int)(i % b);
  T acc = zero_<T>();
  for (int l = 0; l < q; ++l) acc = mad_(In[r * ldi + l], K[(int64_t)l * ldk + j], acc);
  Out[r * ldo + j] = acc;
}

template <class T>
__global__ void nonfinite_scan_kernel(const T* A, int64_t m, int n, int64_t lda, int* err) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !finite_(A[(i / n) * lda + (i % n)]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, DEV_ERR_NONFINITE);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
// the most rows of one chunk: [R; chunk] in ~100 KB of shared memory (2 CTAs per SM)
static int tsqr_chunk(int c, size_t esz) { return imax(32, (int)(100 * 1024 / ((size_t)c * esz)) - c); }

static int pow2_at_least(int x) { int p = 1; while (p < x) p <<= 1; return p; }

static int tsqr_rp(int c) { return imin(32, 256 / pow2_at_least(c)); }

static size_t tsqr_level_smem(int c, int CH, size_t esz) { return (size_t)(c + CH) * c * esz; }

// Level 1: two CTAs per SM, each with at least 256 rows: the level is bound by FP64 issue (about
// m c^2 FMAs), so all SMs' FP64 pipes take part, while short blocks keep few R factors to merge.
static int64_t tsqr_level1_ctas(int64_t m, int c, size_t esz) {
  (void)c;
  (void)esz;
  return imin<int64_t>(2 * (int64_t)num_sms(), imax<int64_t>(1, (m + 255) / 256));
}

static constexpr int kTsqrFan = 20;   // R factors merged per CTA in the upper levels

size_t tsqr_workspace_bytes(int64_t m, int c, size_t esz) {
  const int64_t g1 = tsqr_level1_ctas(m, c, esz);
  // level buffers ping-pong
  return 2 * (((size_t)g1 * c * c * esz + 255) & ~(size_t)255);
}

static int tsqr_fan(int c, size_t esz) {
  return (int)imax<int64_t>(2, imin<int64_t>(kTsqrFan, (int64_t)(max_smem_optin() * 9 / 10) / ((int64_t)c * c * esz)));
}

// CTAs of the first merge level (0 when the level kernel leaves a single R)
int tsqr_merge1_ctas(int64_t m, int c, size_t esz) {
  const int64_t g1 = tsqr_level1_ctas(m, c, esz);
  const int64_t rpc = (m + g1 - 1) / g1;
  const int64_t grid = (m + rpc - 1) / rpc;
  if (grid <= 1) return 0;
  const int fan = tsqr_fan(c, esz);
  return (int)((grid + fan - 1) / fan);
}

// The level kernel on st; with mst, the merges (and the copy of R) on mst after lvl_done, so that
// they can run beside other work of st.
template <class T>
int tsqr_split_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st,
                    cudaStream_t mst, cudaEvent_t lvl_done);

template <class T>
int tsqr_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st) {
  return tsqr_split_impl<T>(X, m, c, ldx, R, work, work_bytes, st, nullptr, nullptr);
}

template <class T>
int tsqr_split_impl(const T* X, int64_t m, int c, int64_t ldx, T* R, void* work, size_t work_bytes, cudaStream_t st,
                    cudaStream_t mst, cudaEvent_t lvl_done) {
  if (c < 1 || c > 64) return RLOBPCG_ERR_INVALID_ARG;
  const size_t esz = sizeof(T);
  if (work_bytes < tsqr_workspace_bytes(m, c, esz)) return RLOBPCG_ERR_INVALID_ARG;
  const int RP = tsqr_rp(c);
  const int64_t g1 = tsqr_level1_ctas(m, c, esz);
  const size_t half = (((size_t)g1 * c * c * esz + 255) & ~(size_t)255);
  T* buf[2] = {(T*)work, (T*)((unsigned char*)work + half)};
  int64_t rpc = (m + g1 - 1) / g1;
  int64_t grid = (m + rpc - 1) / rpc;
  if (grid < 1) grid = 1;
  // a CTA's rows in equal chunks of at most tsqr_chunk rows (each chunk costs a fixed serial
  // part per column, so no short remainder chunk)
  const int64_t nch = (rpc + tsqr_chunk(c, esz) - 1) / tsqr_chunk(c, esz);
  const int CH = (int)imax<int64_t>(1, (rpc + nch - 1) / nch);
  const size_t smem = tsqr_level_smem(c, CH, esz);
  RL_TRY(allow_dynamic_smem(tsqr_level_kernel<T>, smem));
  tsqr_level_kernel<T><<<(int)grid, 256, smem, st>>>(X, m, c, ldx, rpc, CH, RP, buf[0]);
  RL_CHECK_LAUNCH();
  if (mst) {
    RL_CUDA(cudaEventRecord(lvl_done, st));
    RL_CUDA(cudaStreamWaitEvent(mst, lvl_done, 0));
    st = mst;
  }
  int cur = 0;
  // fixed-order tree of triangular merges, up to kTsqrFan factors per CTA (balanced)
  const int fan = tsqr_fan(c, esz);
  while (grid > 1) {
    const int64_t g2 = (grid + fan - 1) / fan;
    const int F = (int)((grid + g2 - 1) / g2);
    const size_t msmem = (size_t)F * c * c * esz;
    RL_TRY(allow_dynamic_smem(tsqr_merge_kernel<T>, msmem));
    tsqr_merge_kernel<T><<<(int)g2, 256, msmem, st>>>(buf[cur], (int)grid, c, F, RP, buf[cur ^ 1]);
    RL_CHECK_LAUNCH();
    cur ^= 1;
    grid = g2;
  }
  RL_CUDA(cudaMemcpyAsync(R, buf[cur], (size_t)c * c * esz, cudaMemcpyDeviceToDevice, st));
  r_phase_fix_kernel<T><<<c, 64, 0, st>>>(R, c);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int tsqr_impl<double>(const double*, int64_t, int, int64_t, double*, void*, size_t, cudaStream_t);
template int tsqr_impl<cd>(const cd*, int64_t, int, int64_t, cd*, void*, size_t, cudaStream_t);
template int tsqr_split_impl<double>(const double*, int64_t, int, int64_t, double*, void*, size_t, cudaStream_t,
                                     cudaStream_t, cudaEvent_t);
template int tsqr_split_impl<cd>(const cd*, int64_t, int, int64_t, cd*, void*, size_t, cudaStream_t, cudaStream_t,
                                 cudaEvent_t);

template <class T>
int rr_small_launch(const T* Rt, int c, int b, double* theta, T* K, size_t k_cap, int* info, cudaStream_t st) {
  if ((size_t)c * 2 * b > k_cap || c > 64 || b > c) {
    set_last_error("rr_small: coefficient block larger than its buffer", __FILE__, __LINE__);
    return RLOBPCG_ERR_INVALID_ARG;
  }
  const size_t smem = rr_small_smem<T>(c, b);
  RL_TRY(allow_dynamic_smem(rr_small_kernel<T>, smem));
  int threads = min(1024, max(64, ((c + 1) / 2) * 32));
  if (c <= 16) threads = 128;   // two Jacobi pairs per warp (real and complex)
  else if (std::is_same<T, double>::value && c <= 32) threads = 512;   // a warp per pair, 16 pairs
  rr_small_kernel<T><<<1, threads, smem, st>>>(Rt, c, b, theta, K, info);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int rr_small_launch<double>(const double*, int, int, double*, double*, size_t, int*, cudaStream_t);
template int rr_small_launch<cd>(const cd*, int, int, double*, cd*, size_t, int*, cudaStream_t);

template <class T>
int update_launch(T* Tb, int64_t n, T* ATb, int64_t m, T* GTb, int64_t ld, int c, int b, const T* K, cudaStream_t st) {
  constexpr int TRW = 64;
  UpdSeg<T> s0{Tb, n, ld, ceil_div(n, TRW)}, s1{ATb, m, ld, ceil_div(m, TRW)}, s2{GTb, n, ld, ceil_div(n, TRW)};
  const size_t smem = ((size_t)c * 2 * b + (size_t)TRW * c) * sizeof(T);
  RL_TRY(allow_dynamic_smem(update_kernel<T>, smem));
  const int blocks = s0.blocks + s1.blocks + s2.blocks;
  update_kernel<T><<<blocks, 256, smem, st>>>(s0, s1, s2, c, b, K);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int update_launch<double>(double*, int64_t, double*, int64_t, double*, int64_t, int, int, const double*, cudaStream_t);
template int update_launch<cd>(cd*, int64_t, cd*, int64_t, cd*, int64_t, int, int, const cd*, cudaStream_t);

template <class T>
int residual_launch(const T* Tb, const T* Gb, int n, int b, int64_t ld, const double* theta_s, T* Res, double* res_norm,
                    T* Rs, int* err, cudaStream_t st) {
  residual_kernel<T><<<1, min(1024, b * 32), 0, st>>>(Tb, Gb, n, b, ld, theta_s, Res, res_norm, Rs, err);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int residual_launch<double>(const double*, const double*, int, int, int64_t, const double*, double*, double*, double*, int*, cudaStream_t);
template int residual_launch<cd>(const cd*, const cd*, int, int, int64_t, const double*, cd*, double*, cd*, int*, cudaStream_t);

// W = Rinv (Rinv^H Rs): Rinv stored in precision S, applied in precision T; Y (n x b, T) scratch;
// W written into T columns [wo, wo+b)
template <class T, class S>
int precond_launch(const S* Rinv_r, const S* Rinv_c, int n, int b, const T* Rs, T* Y, T* Tb, int64_t ld, int wo,
                   cudaStream_t st) {
  const int blocks = (n * 32 + 127) / 128;   // a warp per row, four per CTA (rows over more SMs)
  // Y(k) = sum_{l <= k} conj(Rinv(l, k)) Rs(l): row k of Rinv^H = conj(column k of Rinv)
  trimul_kernel<S, T><<<blocks, 128, 0, st>>>(Rinv_c, n, Rs, b, b, Y, b, 1, 1);
  RL_CHECK_LAUNCH();
  // W(k) = sum_{l >= k} Rinv(k, l) Y(l)
  trimul_kernel<S, T><<<blocks, 128, 0, st>>>(Rinv_r, n, Y, b, b, Tb + wo, ld, 0, 0);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int precond_launch<double, double>(const double*, const double*, int, int, const double*, double*, double*, int64_t, int, cudaStream_t);
template int precond_launch<double, float>(const float*, const float*, int, int, const double*, double*, double*, int64_t, int, cudaStream_t);
template int precond_launch<cd, cd>(const cd*, const cd*, int, int, const cd*, cd*, cd*, int64_t, int, cudaStream_t);
template int precond_launch<cd, cf>(const cf*, const cf*, int, int, const cd*, cd*, cd*, int64_t, int, cudaStream_t);

template <class T>
int fill_random_launch(T* Z, int64_t rows, int q, int64_t ld, uint64_t seed, cudaStream_t st) {
  fill_random_kernel<T><<<ceil_div(rows * q, 256), 256, 0, st>>>(Z, rows, q, ld, seed);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int fill_random_launch<double>(double*, int64_t, int, int64_t, uint64_t, cudaStream_t);
template int fill_random_launch<cd>(cd*, int64_t, int, int64_t, uint64_t, cudaStream_t);

template <class T>
int small_gemm_launch(const T* In, int64_t ldi, int q, const T* K, int ldk, int b, T* Out, int64_t ldo, int64_t rows,
                      cudaStream_t st) {
  small_gemm_kernel<T><<<ceil_div(rows * b, 256), 256, 0, st>>>(In, ldi, q, K, ldk, b, Out, ldo, rows);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int small_gemm_launch<double>(const double*, int64_t, int, const double*, int, int, double*, int64_t, int64_t, cudaStream_t);
template int small_gemm_launch<cd>(const cd*, int64_t, int, const cd*, int, int, cd*, int64_t, int64_t, cudaStream_t);

// Y (n x q) = L X with L stored in precision S (row-major; lower: rows use l <= k, else l >= k)
template <class T, class S>
int trimul_launch(const S* L, int n, const T* X, int64_t ldx, int q, T* Y, int64_t ldy, int lower, int conj_l,
                  cudaStream_t st) {
  trimul_kernel<S, T><<<(n * 32 + 255) / 256, 256, 0, st>>>(L, n, X, ldx, q, Y, ldy, lower, conj_l);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int trimul_launch<double, double>(const double*, int, const double*, int64_t, int, double*, int64_t, int, int, cudaStream_t);
template int trimul_launch<double, float>(const float*, int, const double*, int64_t, int, double*, int64_t, int, int, cudaStream_t);
template int trimul_launch<cd, cd>(const cd*, int, const cd*, int64_t, int, cd*, int64_t, int, int, cudaStream_t);
template int trimul_launch<cd, cf>(const cf*, int, const cd*, int64_t, int, cd*, int64_t, int, int, cudaStream_t);

size_t bcgs2_coop_bytes(int64_t n, int qmax, int b, size_t esz);

template <class T>
int bcgs2_orth_launch(T* Tb, int n, int b, int64_t ld, int wo, int nx, T* E, int passes, cudaStream_t st,
                      const split::WDigits* wd, int* err, bool* digits_done, void* coop, size_t coop_bytes,
                      int svqb, const T* Dl, int nl, int64_t ldl) {
  if (digits_done) *digits_done = false;
  if (svqb && b > 32) {
    set_last_error("SVQB orthonormalisation takes blocks of at most 32 columns", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  if (nl > 0 && passes == 0) return RLOBPCG_ERR_INVALID_ARG;
  if (nl <= 0) { nl = 0; Dl = Tb; ldl = ld; }
  const int q = b + nx + nl;
  {
    // cooperative version over G CTAs when n is large enough for the grid barriers to pay (every
    // CTA keeps at least max(32, b) rows; below n = 256 the one-CTA kernel is faster)
    const int G = imin(16, n / imax(32, b));
    if (n >= 256 && G >= 2 && coop && coop_bytes >= bcgs2_coop_bytes(n, b + imax(nx, 0) + nl, b, sizeof(T))) {
      const int rmax = (n + G - 1) / G, SB = G * b;
      const size_t smem = ((size_t)rmax * (imax(q, b) + b) + (size_t)q * b + 2 * (size_t)SB * b + 6 * b) * sizeof(T);
      if (smem <= max_smem_optin() - 2048) {
        split::WDigits w{};
        if (wd && wd->Wsl && sizeof(T) == sizeof(double) && b <= wd->BP) w = *wd;
        RL_TRY(allow_dynamic_smem(bcgs2_orth_coop_kernel<T>, smem));
        T* gsp = (T*)coop;
        void* args[] = {&Tb, &n, &b, &ld, &wo, &nx, &passes, &gsp, &w, &err, &svqb, &Dl, &nl, &ldl};
        RL_CUDA(cudaLaunchCooperativeKernel((void*)bcgs2_orth_coop_kernel<T>, dim3(G), dim3(256), args, smem, st));
        note_launch();
        if (digits_done) *digits_done = w.Wsl != nullptr;
        return RLOBPCG_OK;
      }
    }
  }
  const size_t smem_s = bcgs2_smem_bytes<T>(n, b, nx + nl);
  if (smem_s <= max_smem_optin() - 1024) {
    split::WDigits w{};
    if (wd && wd->Wsl && sizeof(T) == sizeof(double) && b <= wd->BP) w = *wd;
    RL_TRY(allow_dynamic_smem(bcgs2_orth_smem_kernel<T>, smem_s));
    bcgs2_orth_smem_kernel<T><<<1, 256, smem_s, st>>>(Tb, n, b, ld, wo, nx, passes, w, err, svqb, Dl, nl, ldl);
    RL_CHECK_LAUNCH();
    if (digits_done) *digits_done = w.Wsl != nullptr;
    return RLOBPCG_OK;
  }
  if (svqb || nl > 0) {
    set_last_error("SVQB orthonormalisation and locking: n too large for the shared-memory and cooperative kernels",
                   __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  const size_t smem = ((size_t)2 * b * b + 3 * b) * sizeof(T);
  bcgs2_orth_kernel<T><<<1, 1024, smem, st>>>(Tb, n, b, ld, wo, nx, E, passes);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int bcgs2_orth_launch<double>(double*, int, int, int64_t, int, int, double*, int, cudaStream_t,
                                       const split::WDigits*, int*, bool*, void*, size_t, int, const double*, int,
                                       int64_t);
template int bcgs2_orth_launch<cd>(cd*, int, int, int64_t, int, int, cd*, int, cudaStream_t, const split::WDigits*,
                                   int*, bool*, void*, size_t, int, const cd*, int, int64_t);

// global scratch of the cooperative BCGS2 + Orth kernel for up to qmax basis columns and b columns
size_t bcgs2_coop_bytes(int64_t n, int qmax, int b, size_t esz) {
  const int64_t G = 16;
  (void)n;
  return ((size_t)2 * G * qmax * b + (size_t)G * b * b) * esz + (size_t)G * 32 * sizeof(double) + 256;
}

template <class S, class T>
int take_start_launch(const S* Vt, int n, int b, T* Tb, int64_t ld, cudaStream_t st) {
  take_start_kernel<S, T><<<ceil_div((int64_t)n * b, 256), 256, 0, st>>>(Vt, n, b, Tb, ld);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int take_start_launch<double, double>(const double*, int, int, double*, int64_t, cudaStream_t);
template int take_start_launch<float, double>(const float*, int, int, double*, int64_t, cudaStream_t);
template int take_start_launch<cd, cd>(const cd*, int, int, cd*, int64_t, cudaStream_t);
template int take_start_launch<cf, cd>(const cf*, int, int, cd*, int64_t, cudaStream_t);

template <class T>
int copy_cols_launch(const T* src, int64_t lds, int so, T* dst, int64_t ldd, int dof, int64_t rows, int w, cudaStream_t st) {
  if (rows * w == 0) return RLOBPCG_OK;
  copy_cols_kernel<T><<<ceil_div(rows * w, 256), 256, 0, st>>>(src, lds, so, dst, ldd, dof, rows, w);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int copy_cols_launch<double>(const double*, int64_t, int, double*, int64_t, int, int64_t, int, cudaStream_t);
template int copy_cols_launch<cd>(const cd*, int64_t, int, cd*, int64_t, int, int64_t, int, cudaStream_t);

template <class T>
int outputs_launch(const T* Tb, const T* ATb, int64_t n, int64_t m, int b, int k, int64_t ld, const double* theta_s,
                   const double* res_norm, double* sigma, T* Vout, T* Uout, double* resid, cudaStream_t st) {
  const int64_t tot = imax<int64_t>((n + (Uout ? m : 0)) * k, k);
  outputs_kernel<T><<<ceil_div(tot, 256), 256, 0, st>>>(Tb, ATb, n, m, b, k, ld, theta_s, res_norm, sigma, Vout, Uout, resid);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int outputs_launch<double>(const double*, const double*, int64_t, int64_t, int, int, int64_t, const double*, const double*, double*, double*, double*, double*, cudaStream_t);
template int outputs_launch<cd>(const cd*, const cd*, int64_t, int64_t, int, int, int64_t, const double*, const double*, double*, cd*, cd*, double*, cudaStream_t);

template <class T>
int nonfinite_scan_launch(const T* A, int64_t m, int n, int64_t lda, int* err, cudaStream_t st) {
  nonfinite_scan_kernel<T><<<num_sms() * 4, 256, 0, st>>>(A, m, n, lda, err);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int nonfinite_scan_launch<double>(const double*, int64_t, int, int64_t, int*, cudaStream_t);
template int nonfinite_scan_launch<cd>(const cd*, int64_t, int, int64_t, int*, cudaStream_t);

}  // namespace rl

namespace rl {
template <class T>
int gather_cols_launch(T* buf, int64_t rows, int64_t ld, const int* src, const int* dst, int cnt, cudaStream_t st) {
  if (cnt <= 0) return RLOBPCG_OK;
  if (cnt > 64) return RLOBPCG_ERR_INVALID_ARG;
  ColMap map{};
  map.cnt = cnt;
  for (int t = 0; t < cnt; ++t) { map.src[t] = src[t]; map.dst[t] = dst[t]; }
  gather_cols_kernel<T><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(buf, rows, ld, map);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int gather_cols_launch<double>(double*, int64_t, int64_t, const int*, const int*, int, cudaStream_t);
template int gather_cols_launch<cd>(cd*, int64_t, int64_t, const int*, const int*, int, cudaStream_t);

// ---- the preconditioner variants of Sec. 1.1 ------------------------------------------------
// Squared column norms of A (m x n row-major): block g sums rows [g rb, (g+1) rb) of every column
// (thread per column, rows in order), then one thread per column adds the blocks in order.
constexpr int kColnormParts = 256;
int colnorm_parts(int64_t m) { return (int)imin<int64_t>(kColnormParts, imax<int64_t>(1, (m + 1023) / 1024)); }

template <class T>
__global__ void colnorm_part_kernel(const T* __restrict__ A, int64_t m, int n, int64_t lda, int64_t rb,
                                    double* __restrict__ part) {
  const int64_t g = blockIdx.y;
  const int j = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= n) return;
  const int64_t r0 = g * rb, r1 = imin<int64_t>(m, r0 + rb);
  double s0 = 0, s1 = 0;
  int64_t r = r0;
  for (; r + 1 < r1; r += 2) {
    s0 += abs2_(A[r * lda + j]);
    s1 += abs2_(A[(r + 1) * lda + j]);
  }
  if (r < r1) s0 += abs2_(A[r * lda + j]);
  part[g * n + j] = s0 + s1;
}

__global__ void colnorm_sum_kernel(const double* __restrict__ part, int G, int n, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0;
  for (int g = 0; g < G; ++g) s += part[(int64_t)g * n + j];
  out[j] = s;
}

template <class T>
int colnorm2_launch(const T* A, int64_t m, int n, int64_t lda, double* part, double* out, cudaStream_t st) {
  const int G = colnorm_parts(m);
  const int64_t rb = (m + G - 1) / G;
  colnorm_part_kernel<T><<<dim3((unsigned)((n + 127) / 128), (unsigned)G), 128, 0, st>>>(A, m, n, lda, rb, part);
  RL_CHECK_LAUNCH();
  colnorm_sum_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, G, n, out);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int colnorm2_launch<double>(const double*, int64_t, int, int64_t, double*, double*, cudaStream_t);
template int colnorm2_launch<cd>(const cd*, int64_t, int, int64_t, double*, double*, cudaStream_t);

// W(k, :) = Rs(k, :) / d2(k) (diagonal preconditioner, d2 = squared column norms of A), or
// W = Rs when d2 is null (no preconditioner); W into columns [wo, wo + b) of Tb (ld)
template <class T>
__global__ void scale_rows_kernel(const T* __restrict__ Rs, int n, int b, const double* __restrict__ d2, T* Tb,
                                  int64_t ld, int wo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * b) return;
  const int64_t k = e / b;
  const int j = (int)(e % b);
  const T r = Rs[e];
  Tb[k * ld + wo + j] = d2 ? scale_(r, 1.0 / d2[k]) : r;
}

template <class T>
int scale_rows_launch(const T* Rs, int n, int b, const double* d2, T* Tb, int64_t ld, int wo, cudaStream_t st) {
  const int64_t tot = (int64_t)n * b;
  scale_rows_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Rs, n, b, d2, Tb, ld, wo);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int scale_rows_launch<double>(const double*, int, int, const double*, double*, int64_t, int, cudaStream_t);
template int scale_rows_launch<cd>(const cd*, int, int, const double*, cd*, int64_t, int, cudaStream_t);

// batched iterations of many small solves (they reuse the one-CTA bodies above)
#include "batch_kernels.cuh"
}  // namespace rl
