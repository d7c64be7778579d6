// Batched LOBPCG iterations for many small solves (real FP64), included at the end of small.cu so
// that the one-CTA bodies it reuses (bcgs2_orth_cta, rr_small_cta, cta_householder) are in the
// same translation unit.
//
// One iteration of Alg. 2 for every solve of the batch is two persistent kernels, each pulling
// work items from a device queue (an atomic counter over a fixed item list):
//
//   pre_kernel   the preconditioner W = P P^* Rs = R^{-1} (R^{-H} Rs) in two launches of row
//                blocks (32 rows per item): phase 0 forms Y = R^{-H} Rs, phase 1 W = R^{-1} Y, and
//                the CTA that finishes a solve's last block of phase 1 runs BCGS2 + Orth of W
//                against [V X] for that solve (Alg. 2). The two triangular factors are kept
//                separate on purpose: the rounding error of R^{-1} (R^{-H} Rs) lies mostly along
//                the smallest singular directions of R (which BCGS2 then removes with V), while an
//                explicit (R^H R)^{-1} would spread an error of u ||(R^H R)^{-1}|| over every
//                direction and swamp the components of W that correct V.
//   tile_kernel  items (solve, tile of trows rows of A): applies the previous iteration's
//                coefficients to the tile's rows of A_T (A V and A X of Rayleigh-Ritz, deferred
//                from the last iteration), forms A W for the tile and its share of A^H (A W), and
//                reduces its rows of A_T = [A V  A W  A X] to a c x c triangular factor. The last
//                tile of each group of 16 sums the group's G partials and merges its factors; the
//                last group of a solve runs the rest of the iteration for that solve in the same
//                launch: Rayleigh-Ritz on the merged R (SVD of A_T, Sec. 2.1), the update of V, X
//                and G = A^H A T, the residual A^H A_V - V Theta^2 and its norms, the history and
//                the stopping rule of Sec. 2.1.
//
// Nothing waits on another CTA: a dependency is met by the CTA that completes it (a fenced atomic
// counter), so there are no spin waits. Every sum runs in an order fixed by the solve's own shape
// and tile height (tiles in order, groups in order, a fixed butterfly per row), so a solve gives
// the same bits alone and in any batch. A solve that has stopped skips its items.
namespace batch {

// ---- device helpers ---------------------------------------------------------------------------

__device__ inline int pop_item(int* qhead, int* s_item) {
  if (threadIdx.x == 0) *s_item = atomicAdd(qhead, 1);
  __syncthreads();
  const int it = *s_item;
  __syncthreads();
  return it;
}

// Called by every thread after the CTA's writes that the counter publishes: returns true in the
// CTA that brings cnt to `total` (then the other CTAs' writes are visible to it).
__device__ inline bool arrive_last(int* cnt, int total, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = (atomicAdd(cnt, 1) == total - 1);
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Running triangular factor: Wm (row-major, (c + QRC) x c in shared memory) holds R_acc in its
// first c rows; fold(rows) factors [R_acc; the next `rows` rows already staged below it] and
// leaves the new R_acc (upper triangle, strict lower part zeroed) in the first c rows.
__device__ inline void fold_staged(double* Wm, int c, int rows, double* tau, double* dg, double* sv, double* sh_inv) {
  cta_householder<double>(Wm, c + rows, c, tau, dg, sv, sh_inv);
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    if (j < i) Wm[e] = 0.0;
  }
  __syncthreads();
}

__device__ inline void zero_smem(double* p, int cnt) {
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) p[e] = 0.0;
  __syncthreads();
}

// rows [r0, r0 + rows) of buf (ld 3b): x = buf[r, 0:c]; buf[r, 0:b] = x K(:, 0:b),
// buf[r, 2b:3b] = x K(:, b:2b)  (the Rayleigh-Ritz recombination of V and X, Alg. 2)
__device__ inline void apply_coeffs(double* buf, int64_t r0, int64_t rows, int b, int c, const double* Kg,
                                    double* stage) {
  const int C = 3 * b, b2 = 2 * b;
  double* Ks = stage;                 // c x 2b
  double* xs = stage + C * b2;        // UR x c
  for (int e = threadIdx.x; e < c * b2; e += blockDim.x) Ks[e] = Kg[e];
  for (int64_t q0 = 0; q0 < rows; q0 += UR) {
    const int nr = (int)min((int64_t)UR, rows - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * c; e += blockDim.x) xs[e] = buf[(r0 + q0 + e / c) * C + (e % c)];
    __syncthreads();
    for (int e = threadIdx.x; e < nr * b2; e += blockDim.x) {
      const int r = e / b2, o = e % b2;
      double v = 0.0;
      for (int l = 0; l < c; ++l) v = fma(xs[r * c + l], Ks[l * b2 + o], v);
      buf[(r0 + q0 + r) * C + (o < b ? o : o + b)] = v;
    }
  }
  __syncthreads();
}

// ---- inner products, specialised on the block size (a DFMA predicated off still takes an FP64
// issue slot, so no instruction is issued for a column that does not exist) ----------------------

#define RL_BATCH_DISPATCH_B(b, call) \
  switch (b) {                       \
    case 1: call(1); break;          \
    case 2: call(2); break;          \
    case 3: call(3); break;          \
    case 4: call(4); break;          \
    default: call(5); break;         \
  }

// rows [k0, k1) of Out = L In for a triangular L (row-major, FP64): lower (l <= k) or upper
// (l >= k); In, Out n x B row-major with leading dimensions ldi, ldo (a warp per row)
template <int B>
__device__ inline void tri_rows(const double* L, int n, bool lower, const double* In, int64_t ldi, double* Out,
                                int64_t ldo, int k0, int k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = k0 + warp; k < k1; k += NT / 32) {
    double acc[B];
#pragma unroll
    for (int j = 0; j < B; ++j) acc[j] = 0.0;
    const double* Lk = L + (size_t)k * n;
    const int lo = lower ? 0 : k, hi = lower ? k + 1 : n;
    for (int l = lo + lane; l < hi; l += 32) {
      const double lkl = Lk[l];
      const double* xl = In + (size_t)l * ldi;
#pragma unroll
      for (int j = 0; j < B; ++j) acc[j] = fma(lkl, xl[j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const double v = warp_sum(acc[j]);
      if (lane == 0) Out[(int64_t)k * ldo + j] = v;
    }
  }
}

// phase 1: a warp per row r of the stage: lane l sums A[r, k] W[k, j] over k = l (mod 32), then a
// butterfly over the warp (a fixed order); lane 0 writes Y[r, :] (shared) and A W (global)
template <int B>
__device__ inline void gram_phase1(const double* cur, int nr, int n, const double* Wt, double* Ys, double* aw,
                                   int64_t ldaw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < nr; r += NT / 32) {
    double y[B];
#pragma unroll
    for (int j = 0; j < B; ++j) y[j] = 0.0;
    const double* ar = cur + (size_t)r * n;
    for (int k = lane; k < n; k += 32) {
      const double a = ar[k];
#pragma unroll
      for (int j = 0; j < B; ++j) y[j] = fma(a, Wt[(size_t)j * n + k], y[j]);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const double v = warp_sum(y[j]);
      if (lane == 0) {
        Ys[r * B + j] = v;
        aw[(int64_t)r * ldaw + j] = v;
      }
    }
  }
}

// phase 2: Gacc[k, :] += A[r, k] Y[r, :] over the rows in order
template <int B>
__device__ inline void gram_phase2(const double* cur, int nr, int n, const double* Ys, double* Gacc) {
  for (int k = threadIdx.x; k < n; k += NT) {
    double g[B];
#pragma unroll
    for (int j = 0; j < B; ++j) g[j] = Gacc[(size_t)k * B + j];
    for (int r = 0; r < nr; ++r) {
      const double a = cur[(size_t)r * n + k];
#pragma unroll
      for (int j = 0; j < B; ++j) g[j] = fma(a, Ys[r * B + j], g[j]);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) Gacc[(size_t)k * B + j] = g[j];
  }
}

// ---- precondition + BCGS2 ------------------------------------------------------------------------

template <int PHASE>
__global__ void __launch_bounds__(NT) pre_kernel(Desc* D, const int2* __restrict__ items, int nitems, int* qhead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  __shared__ int s_item, s_flag;
  const int tid = threadIdx.x;
  for (;;) {
    const int it = pop_item(qhead, &s_item);
    if (it >= nitems) break;
    const int2 item = items[it];
    if (tid == 0) sd = D[item.x];
    __syncthreads();
    if (!sd.done) {
      const int n = sd.n, b = sd.b;
      const int64_t C = 3 * b;
      const int k0 = item.y * PR, k1 = min(n, k0 + PR);
      if (PHASE == 0) {
#define RL_PRE(B) tri_rows<B>(sd.Rl, n, true, sd.Rs, B, sd.Y, B, k0, k1)
        RL_BATCH_DISPATCH_B(b, RL_PRE)
#undef RL_PRE
      } else {
#define RL_PRE(B) tri_rows<B>(sd.Ru, n, false, sd.Y, B, sd.Tb + B, C, k0, k1)
        RL_BATCH_DISPATCH_B(b, RL_PRE)
#undef RL_PRE
        if (arrive_last(sd.cnt, sd.nrb, &s_flag)) {
          if (tid == 0) sd.cnt[0] = 0;
          split::WDigits wd{};
          bcgs2_orth_cta<double>(smem_raw, sd.Tb, n, b, C, b, sd.nx, 2, wd, sd.err, 0, sd.Tb, 0, C);
        }
      }
    }
    __syncthreads();
  }
}

// ---- stopping rule of Sec. 2.1 (the host rule, on the device) ------------------------------------

__device__ inline bool stop_check(const double* hist, int b, int i, double sigma11, double tau, bool stag) {
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  auto rv = [&](int t, int j) { return t >= 0 ? hist[(size_t)t * 2 * b + j] : inf; };
  auto tv = [&](int t, int j) { return t >= 0 ? (t == 0 ? inf : hist[(size_t)t * 2 * b + b + j]) : inf; };
  double mx = 0;
  for (int j = 0; j < b; ++j) mx = fmax(mx, rv(i + 1, j));
  const double thr = sigma11 * sigma11 * tau;
  if (!(mx <= thr)) return false;
  if (!stag) return true;
  for (int j = 0; j < b; ++j) {
    if (!(__dmul_rn(1.1, rv(i + 1, j)) >= rv(i - 4, j))) return false;
    const double lhs = __ddiv_rn(__dmul_rn(1.1, __dsub_rn(tv(i - 4, j), tv(i + 1, j))), tv(i + 1, j));
    const double rhs = __ddiv_rn(__dsub_rn(tv(i - 9, j), tv(i - 4, j)), tv(i - 4, j));
    if (!(lhs >= rhs)) return false;
  }
  return true;
}

// ---- the rest of an iteration for one solve (one CTA) ------------------------------------------

__device__ void tail(Desc& sd, Desc* Dg, double* sm, double* qtau, double* qdg, double* qsv, double* qinv) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NW = blockDim.x >> 5;
  const int n = sd.n, b = sd.b, c = sd.c, C = 3 * b;
  // G_W = sum of the group sums, in group order
  for (int e = tid; e < n * b; e += blockDim.x) {
    double s = __ldcg(sd.Ggrp + e);
    for (int g = 1; g < sd.ngroups; ++g) s += __ldcg(sd.Ggrp + (size_t)g * n * b + e);
    sd.GTb[(int64_t)(e / b) * C + b + (e % b)] = s;
  }
  // R of A_T: fold the group factors in group order
  zero_smem(sm, c * c);
  for (int g0 = 0; g0 < sd.ngroups; g0 += QRC / c) {
    const int ng = min(QRC / c, sd.ngroups - g0);
    for (int e = tid; e < ng * c * c; e += blockDim.x) {
      const int gi = e / (c * c), rr = (e / c) % c, cc = e % c;
      sm[(size_t)(c + gi * c + rr) * c + cc] = __ldcg(sd.Rgrp + (size_t)(g0 + gi) * C * C + rr * C + cc);
    }
    __syncthreads();
    fold_staged(sm, c, ng * c, qtau, qdg, qsv, qinv);
  }
  for (int e = tid; e < c * c; e += blockDim.x) sd.Rfin[e] = sm[e];
  __syncthreads();
  // Rayleigh-Ritz: [~, Theta, C] = SVD(A_T) through R (Alg. 2)
  rr_small_cta<double, 16>(reinterpret_cast<unsigned char*>(sm), sd.Rfin, c, b, sd.theta, sd.K, sd.rr_info);
  __syncthreads();
  // V, X and their G columns (the A_T columns follow in the next launch's tiles)
  apply_coeffs(sd.Tb, 0, n, b, c, sd.K, sm);
  apply_coeffs(sd.GTb, 0, n, b, c, sd.K, sm);
  // residual R = A^H A_V - V Theta^2, its column norms, and the unit columns for P
  const double* theta_s = sd.theta + (c - b);
  for (int j = warp; j < b; j += NW) {
    const double th2 = theta_s[j] * theta_s[j];
    double a = 0;
    for (int k = lane; k < n; k += 32) {
      const double r = sd.GTb[(int64_t)k * C + j] - sd.Tb[(int64_t)k * C + j] * th2;
      sd.Res[(int64_t)k * b + j] = r;
      a += r * r;
    }
    a = warp_sum(a);
    const double nr = sqrt(a);
    if (lane == 0) {
      sd.res_norm[j] = nr;
      sd.hist[(size_t)(sd.iter + 1) * 2 * b + j] = nr;
      sd.hist[(size_t)(sd.iter + 1) * 2 * b + b + j] = theta_s[j];
      if (!isfinite(nr)) atomicOr(sd.err, DEV_ERR_NONFINITE);
    }
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int k = lane; k < n; k += 32) sd.Rs[(int64_t)k * b + j] = sd.Res[(int64_t)k * b + j] * inv;
  }
  __syncthreads();
  if (tid == 0) {
    const int i = sd.iter;
    int done = 0, reason = sd.fixed > 0 ? RLOBPCG_STOP_FIXED : RLOBPCG_STOP_MAX_ITER;
    if (sd.fixed <= 0 && i % sd.check_every == 0 &&
        stop_check(sd.hist, b, i, sd.sigma11, sd.tau, sd.use_stag != 0)) {
      done = 1;
      reason = RLOBPCG_STOP_CONVERGED;
    }
    if (!done && i + 1 >= sd.max_iter) done = 1;
    Desc* dg = Dg;
    dg->iter = i + 1;
    dg->matvecs = sd.matvecs + b;
    dg->c_prev = c;
    dg->pending = 1;
    dg->nx = b;
    dg->c = 3 * b;
    dg->done = done;
    dg->stop_reason = reason;
    sd.cnt[1] = 0;
  }
}

// ---- Gram tile + local factor + reductions + tail ----------------------------------------------

template <int FLUSH>
__global__ void __launch_bounds__(NT, 2) tile_kernel(Desc* D, const int2* __restrict__ items, int nitems, int* qhead,
                                                     int nw, int abuf_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Desc sd;
  __shared__ int s_item, s_flag;
  __shared__ double qtau[3 * BMAX], qdg[3 * BMAX], qsv[3 * BMAX], qinv;
  double* Wt = reinterpret_cast<double*>(smem_raw);        // b x n (transposed W); nw >= n b over the batch
  double* Gacc = Wt + nw;                                   // n x b
  double* Abuf = Gacc + nw;                                 // staging (A rows, A_T rows, tail scratch)
  double* Ps = Abuf + abuf_elems;                           // phase-1 partials
  const int tid = threadIdx.x;
  for (;;) {
    const int it = pop_item(qhead, &s_item);
    if (it >= nitems) break;
    const int2 item = items[it];
    if (tid == 0) sd = D[item.x];
    __syncthreads();
    const bool skip = FLUSH ? (sd.pending == 0) : (sd.done != 0);
    if (!skip) {
      const int n = sd.n, b = sd.b, C = 3 * b;
      const int64_t r0 = (int64_t)item.y * sd.trows;
      const int rows = (int)min((int64_t)sd.trows, sd.m - r0);
      // (a) A V, A X of the last Rayleigh-Ritz step for these rows
      if (sd.pending) apply_coeffs(sd.ATb, r0, rows, b, sd.c_prev, sd.K, Abuf);
      if (!FLUSH) {
        const int rt = sd.rt, c = sd.c;
        // (b) A W and A^H (A W): W^T and the accumulator in shared memory
        for (int e = tid; e < n * b; e += NT) {
          const int k = e / b, j = e % b;
          Wt[(size_t)j * n + k] = sd.Tb[(int64_t)k * C + b + j];
          Gacc[e] = 0.0;
        }
        double* Ys = Ps;
        auto issue = [&](int q, double* dst) {   // cp.async of rows [q, q + rt) of the tile
          const int nr = min(rt, rows - q);
          const double* src = sd.A + (r0 + q) * sd.lda;
          for (int e = tid; e < nr * n; e += NT) {
            const int r = e / n, k = e % n;
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + e);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + (int64_t)r * sd.lda + k)
                         : "memory");
          }
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        // two stages of rt rows: the next stage loads while this one computes
        const int nsub = (rows + rt - 1) / rt;
        issue(0, Abuf);
        for (int q = 0; q < nsub; ++q) {
          double* cur = Abuf + (size_t)(q & 1) * rt * n;
          if (q + 1 < nsub) {
            issue((q + 1) * rt, Abuf + (size_t)((q + 1) & 1) * rt * n);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
          } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
          }
          __syncthreads();
          const int nr = min(rt, rows - q * rt);
          double* aw = sd.ATb + (r0 + q * rt) * C + b;
          // phase 1: Y = A W for the stage's rows (also the A W columns of A_T)
#define RL_P1(B) gram_phase1<B>(cur, nr, n, Wt, Ys, aw, C)
          RL_BATCH_DISPATCH_B(b, RL_P1)
#undef RL_P1
          __syncthreads();
          // phase 2: Gacc[k, :] += A[r, k] Y[r, :] over the rows in order
#define RL_P2(B) gram_phase2<B>(cur, nr, n, Ys, Gacc)
          RL_BATCH_DISPATCH_B(b, RL_P2)
#undef RL_P2
          __syncthreads();
        }
        double* gp = sd.Gpart + (size_t)item.y * n * b;
        for (int e = tid; e < n * b; e += NT) gp[e] = Gacc[e];
        // (c) triangular factor of the tile's rows of A_T = [A V  A W  A X] (width c)
        zero_smem(Abuf, c * c);
        for (int q0 = 0; q0 < rows; q0 += QRC) {
          const int nr = min(QRC, rows - q0);
          for (int e = tid; e < nr * c; e += NT) Abuf[(size_t)c * c + e] = sd.ATb[(r0 + q0 + e / c) * C + (e % c)];
          __syncthreads();
          fold_staged(Abuf, c, nr, qtau, qdg, qsv, &qinv);
        }
        double* rp = sd.Rpart + (size_t)item.y * C * C;
        for (int e = tid; e < c * c; e += NT) rp[(e / c) * C + (e % c)] = Abuf[e];
        // (d) group reduction, then the solve's tail
        const int g = item.y / GS, t0 = g * GS, t1 = min(sd.ntiles, t0 + GS);
        if (arrive_last(sd.cnt + 2 + g, t1 - t0, &s_flag)) {
          if (tid == 0) sd.cnt[2 + g] = 0;
          double* gg = sd.Ggrp + (size_t)g * n * b;
          for (int e = tid; e < n * b; e += NT) {
            double s = __ldcg(sd.Gpart + (size_t)t0 * n * b + e);
            for (int t = t0 + 1; t < t1; ++t) s += __ldcg(sd.Gpart + (size_t)t * n * b + e);
            gg[e] = s;
          }
          zero_smem(Abuf, c * c);
          for (int ta = t0; ta < t1; ta += QRC / c) {
            const int nt = min(QRC / c, t1 - ta);
            for (int e = tid; e < nt * c * c; e += NT) {
              const int ti = e / (c * c), rr = (e / c) % c, cc = e % c;
              Abuf[(size_t)(c + ti * c + rr) * c + cc] = __ldcg(sd.Rpart + (size_t)(ta + ti) * C * C + rr * C + cc);
            }
            __syncthreads();
            fold_staged(Abuf, c, nt * c, qtau, qdg, qsv, &qinv);
          }
          double* rg = sd.Rgrp + (size_t)g * C * C;
          for (int e = tid; e < c * c; e += NT) rg[(e / c) * C + (e % c)] = Abuf[e];
          if (arrive_last(sd.cnt + 1, sd.ngroups, &s_flag)) tail(sd, D + item.x, Abuf, qtau, qdg, qsv, &qinv);
        }
      }
    }
    __syncthreads();
  }
}

// number of solves not yet stopped (one CTA)
__global__ void active_kernel(const Desc* D, int count, int* out) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int a = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) a += D[i].done ? 0 : 1;
  atomicAdd(&s, a);
  __syncthreads();
  if (threadIdx.x == 0) *out = s;
}

// FP64 copy of a factor stored in the sketch precision
template <class S>
__global__ void widen_kernel(const S* __restrict__ in, int64_t cnt, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (double)in[i];
}

}  // namespace batch

// ---- launchers (host) --------------------------------------------------------------------------

namespace batch {

// staging the tile kernel needs for one solve: two A sub-tiles, the A_T fold, the coefficient
// update and the tail's Rayleigh-Ritz scratch
int abuf_need(int n, int b, int rt) {
  const int C = 3 * b;
  size_t need = (size_t)2 * rt * n;
  need = std::max(need, (size_t)(C + QRC) * C);
  need = std::max(need, (size_t)C * 2 * b + (size_t)UR * C);
  need = std::max(need, (rr_small_smem<double>(C, b) + 7) / 8 + 2);   // 3b <= 15
  return (int)need;
}

size_t bcgs2_pre_smem(int n, int b) { return bcgs2_smem_bytes<double>(n, b, b); }

int prepare(size_t pre_smem, size_t tile_smem) {
  RL_TRY(allow_dynamic_smem(pre_kernel<0>, pre_smem));
  RL_TRY(allow_dynamic_smem(pre_kernel<1>, pre_smem));
  RL_TRY(allow_dynamic_smem(tile_kernel<0>, tile_smem));
  RL_TRY(allow_dynamic_smem(tile_kernel<1>, tile_smem));
  return RLOBPCG_OK;
}

int tile_blocks_per_sm(size_t tile_smem, int* out) {
  RL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, tile_kernel<0>, NT, tile_smem));
  return RLOBPCG_OK;
}

int pre_launch(int phase, Desc* D, const int2* items, int nitems, int* qhead, int grid, size_t smem, cudaStream_t st) {
  if (phase == 0)
    pre_kernel<0><<<grid, NT, 0, st>>>(D, items, nitems, qhead);
  else
    pre_kernel<1><<<grid, NT, smem, st>>>(D, items, nitems, qhead);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

int tile_launch(bool flush, Desc* D, const int2* items, int nitems, int* qhead, int grid, int nw, int abuf,
                size_t smem, cudaStream_t st) {
  if (flush)
    tile_kernel<1><<<grid, NT, smem, st>>>(D, items, nitems, qhead, nw, abuf);
  else
    tile_kernel<0><<<grid, NT, smem, st>>>(D, items, nitems, qhead, nw, abuf);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

int active_launch(const Desc* D, int count, int* out, cudaStream_t st) {
  active_kernel<<<1, 256, 0, st>>>(D, count, out);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

template <class S>
int widen_launch(const S* in, int64_t cnt, double* out, cudaStream_t st) {
  widen_kernel<S><<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(in, cnt, out);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}
template int widen_launch<double>(const double*, int64_t, double*, cudaStream_t);
template int widen_launch<float>(const float*, int64_t, double*, cudaStream_t);

int static_smem_bytes(size_t* pre, size_t* tile) {
  cudaFuncAttributes a;
  RL_CUDA(cudaFuncGetAttributes(&a, pre_kernel<1>));
  *pre = a.sharedSizeBytes;
  RL_CUDA(cudaFuncGetAttributes(&a, tile_kernel<0>));
  *tile = a.sharedSizeBytes;
  return RLOBPCG_OK;
}

}  // namespace batch
