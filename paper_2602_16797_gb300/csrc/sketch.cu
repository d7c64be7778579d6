// Sketch SA = S A with the SparseStack embedding (Sec. 2.2 of arXiv 2602.16797).
//
// Design (GB300): S is never stored. A CTA owns (a block of w columns of A) x (one piece j of
// the SparseStack columns) x (a sub-range of that piece's destination rows); its accumulator
// block of SA lives in shared memory. The CTA streams the rows of its column block through a
// cp.async ring; for each row i it derives the destination row and sign of piece j from
// SplitMix64 (one hash per row, computed once per CTA). Warp kk owns column kk and its lanes own
// 32 consecutive rows: lanes that hit the same destination are grouped with match_any and their
// values are added by the group's first lane in ascending row order. Every SA entry therefore
// sums its sources in ascending source row -- the same order as a sequential reference -- and
// only then is scaled by zeta^{-1/2}: the result is reproducible bit for bit.
// The 8 piece-CTAs of a column block read the same A rows at nearly the same time, so A comes
// from HBM once and from L2 the other zeta-1 times.
#include "common.cuh"

namespace rl {

namespace {

constexpr int SK_TR = 64;      // rows per staged tile
constexpr int SK_STAGES = 4;   // cp.async ring depth

__device__ inline void cp_async_elem(void* smem, const void* gmem, int bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  }
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <class TA, class TS>
__global__ void __launch_bounds__(1024) sketch_kernel(const TA* __restrict__ A, int64_t m, int n,
                                                      int64_t lda, int d, int zeta, uint64_t seed,
                                                      int w, int sub, RealOf<TS> scale,
                                                      TS* __restrict__ SA) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.x * w;
  const int wcols = min(w, n - k0);
  const int j = blockIdx.y;
  const int plo = piece_lo(j, d, zeta);
  const int plen = piece_lo(j + 1, d, zeta) - plo;
  const int slo = blockIdx.z * sub;
  const int shi = min(slo + sub, plen);
  if (slo >= shi) return;  // whole CTA: this piece has no rows in this sub-range
  const int slen = shi - slo;

  TS* acc = reinterpret_cast<TS*>(smem_raw);                         // [sub][w]
  size_t off = ((size_t)sub * w * sizeof(TS) + 15) & ~(size_t)15;
  TA* tiles = reinterpret_cast<TA*>(smem_raw + off);                 // [STAGES][TR][w+1]
  off += (size_t)SK_STAGES * SK_TR * (w + 1) * sizeof(TA);
  int* codes = reinterpret_cast<int*>(smem_raw + off);               // [STAGES][TR]

  for (int idx = threadIdx.x; idx < slen * w; idx += blockDim.x) acc[idx] = zero_<TS>();

  const int64_t ntiles = (m + SK_TR - 1) / SK_TR;
  const int rows_per_warp = SK_TR / nwarps;

  auto issue = [&](int64_t t) {
    int s = (int)(t % SK_STAGES);
    TA* tile = tiles + (size_t)s * SK_TR * (w + 1);
    for (int rr = 0; rr < rows_per_warp; ++rr) {
      int r = warp * rows_per_warp + rr;
      int64_t i = t * SK_TR + r;
      if (i < m && lane < wcols) cp_async_elem(&tile[r * (w + 1) + lane], &A[i * lda + k0 + lane], (int)sizeof(TA));
    }
    if (warp == 0) {
      for (int r = lane; r < SK_TR; r += 32) {
        int64_t i = t * SK_TR + r;
        int code = -1;
        if (i < m) {
          uint64_t h = splitmix64_at(seed, (uint64_t)i * (uint64_t)zeta + (uint64_t)j);
          int pos = (int)(((h >> 32) * (uint64_t)plen) >> 32);
          if (pos >= slo && pos < shi) code = ((pos - slo) << 1) | (int)(h & 1ull);
        }
        codes[s * SK_TR + r] = code;
      }
    }
  };

  for (int64_t t = 0; t < SK_STAGES - 1; ++t) {
    if (t < ntiles) issue(t);
    cp_async_commit();
  }
  for (int64_t t = 0; t < ntiles; ++t) {
    if (t + SK_STAGES - 1 < ntiles) issue(t + SK_STAGES - 1);
    cp_async_commit();
    cp_async_wait<SK_STAGES - 1>();
    __syncthreads();
    const int s = (int)(t % SK_STAGES);
    const TA* tile = tiles + (size_t)s * SK_TR * (w + 1);
    const int* cd_ = codes + s * SK_TR;
    if (warp < wcols) {
      const int kk = warp;
#pragma unroll
      for (int h = 0; h < SK_TR / 32; ++h) {
        const int code = cd_[h * 32 + lane];
        const int key = code < 0 ? -1 : (code >> 1);
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(grp) - 1) {
          TS a = acc[key * w + kk];
          unsigned mm = grp;
          while (mm) {
            const int q = __ffs(mm) - 1;
            mm &= mm - 1;
            const TS v = cvt_<TS, TA>(tile[(h * 32 + q) * (w + 1) + kk]);
            a = (cd_[h * 32 + q] & 1) ? sub_(a, v) : add_(a, v);
          }
          acc[key * w + kk] = a;
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  // write out, scaled once by zeta^{-1/2}; SA is column-major (d rows)
  for (int idx = threadIdx.x; idx < slen * wcols; idx += blockDim.x) {
    const int kk = idx / slen, p = idx % slen;
    SA[(int64_t)(k0 + kk) * d + plo + slo + p] = scale_(acc[p * w + kk], scale);
  }
}

template <class TA, class TS>
int launch_sketch(const TA* A, int64_t m, int n, int64_t lda, int d, int zeta, uint64_t seed,
                  TS* SA, cudaStream_t st) {
  const size_t budget = 150 * 1024;
  const int maxlen = (d + zeta - 1) / zeta + 1;
  int w = sizeof(TA) == 16 ? 16 : 32;
  w = min(w, n);
  int sub = maxlen;
  while (w > 8 && (size_t)sub * w * sizeof(TS) > budget) w >>= 1;
  int nsub = 1;
  while ((size_t)sub * w * sizeof(TS) > budget) { ++nsub; sub = (maxlen + nsub - 1) / nsub; }
  // at least 2 warps per CTA so that the 64-row tile load divides evenly
  int nwarps = max(w, 2);
  while (SK_TR % nwarps) ++nwarps;
  size_t smem = (((size_t)sub * w * sizeof(TS) + 15) & ~(size_t)15) +
                (size_t)SK_STAGES * SK_TR * (w + 1) * sizeof(TA) + (size_t)SK_STAGES * SK_TR * sizeof(int);
  if (smem > max_smem_optin()) return RLOBPCG_ERR_UNSUPPORTED;
  RL_CUDA(cudaFuncSetAttribute(sketch_kernel<TA, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((n + w - 1) / w, zeta, nsub);
  using R = RealOf<TS>;
  const R scale = (R)(1.0 / sqrt((double)zeta));
  sketch_kernel<TA, TS><<<grid, nwarps * 32, smem, st>>>(A, m, n, lda, d, zeta, seed, w, sub, scale, SA);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

}  // namespace

int sketch_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, int d, int zeta,
                    uint64_t seed, int sketch_prec, void* SA, cudaStream_t st) {
  if (dtype == RLOBPCG_F64) {
    if (sketch_prec == RLOBPCG_SKETCH_F32)
      return launch_sketch<double, float>((const double*)A, m, (int)n, lda, d, zeta, seed, (float*)SA, st);
    return launch_sketch<double, double>((const double*)A, m, (int)n, lda, d, zeta, seed, (double*)SA, st);
  }
  if (sketch_prec == RLOBPCG_SKETCH_F32)
    return launch_sketch<cd, cf>((const cd*)A, m, (int)n, lda, d, zeta, seed, (cf*)SA, st);
  return launch_sketch<cd, cd>((const cd*)A, m, (int)n, lda, d, zeta, seed, (cd*)SA, st);
}

}  // namespace rl
