// Sketch SA = S A with the SparseStack embedding (Sec. 2.2 of arXiv 2602.16797).
//
// Design (GB300): S is never stored. A CTA owns a block of R destination rows of one piece j
// and a block of up to 256 columns; its slice of SA accumulates in shared memory. The CTA scans
// all m source rows in chunks: each warp hashes 256 consecutive rows (SplitMix64, integer work
// only) and keeps, in ascending row order, those whose piece-j destination falls in its block.
// Then every thread (one column each) walks the kept rows in ascending order and adds +-A[i, k]
// into its column of the accumulator, loading whole rows of A with coalesced reads. Each SA entry
// therefore sums its sources in ascending source row -- the order of a sequential reference --
// and is scaled by zeta^{-1/2} once at the end: the result is reproducible bit for bit. Every row
// of A is read zeta times in total (once per piece), which costs less than the zeta m n adds.
#include "common.cuh"

namespace rl {

namespace {

constexpr int SK_NT = 256;           // threads per CTA (one column each in the add phase)
constexpr int SK_WARPS = SK_NT / 32;
constexpr int SK_GROUPS = 8;         // 32-row groups hashed per warp per chunk
constexpr int SK_CHUNK = SK_WARPS * SK_GROUPS * 32;   // rows per chunk (2048)

// x with its sign flipped when s = 1, by an integer XOR on the sign bit(s): acc + flip(v, 1) is
// exactly acc - v, and the FP64 pipe (the sketch's bound) sees one add instead of an add and a
// subtract with a select
__device__ __forceinline__ double flip_(double x, int s) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)s << 63));
}
__device__ __forceinline__ float flip_(float x, int s) { return __int_as_float(__float_as_int(x) ^ (s << 31)); }
__device__ __forceinline__ cd flip_(cd x, int s) { return {flip_(x.x, s), flip_(x.y, s)}; }
__device__ __forceinline__ cf flip_(cf x, int s) { return {flip_(x.x, s), flip_(x.y, s)}; }

template <class TA, class TS>
__global__ void __launch_bounds__(SK_NT) sketch_kernel(const TA* __restrict__ A, int64_t m, int n, int64_t lda,
                                                       int d, int zeta, uint64_t seed, int R, int bpp,
                                                       RealOf<TS> scale, TS* __restrict__ SA) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j = blockIdx.x / bpp;                 // piece
  const int sblk = blockIdx.x % bpp;              // destination block inside the piece
  const int plo = piece_lo(j, d, zeta);
  const int plen = piece_lo(j + 1, d, zeta) - plo;
  const int dlo = sblk * R;
  const int dhi = imin(dlo + R, plen);
  if (dlo >= dhi) return;                         // whole CTA: empty block
  const int k0 = blockIdx.y * SK_NT;
  const int kk = k0 + tid;
  const bool has_col = kk < n;

  TS* acc = reinterpret_cast<TS*>(smem_raw);                       // [R][SK_NT]
  int* lst = reinterpret_cast<int*>(smem_raw + (size_t)R * SK_NT * sizeof(TS));  // [WARPS][GROUPS*32]
  int* code = lst + SK_WARPS * SK_GROUPS * 32;                     // matching (dest - dlo) << 1 | sign
  __shared__ int cnt[SK_WARPS];
  for (int r = 0; r < dhi - dlo; ++r) acc[r * SK_NT + tid] = zero_<TS>();

  for (int64_t c0 = 0; c0 < m; c0 += SK_CHUNK) {
    // phase 1: warp w hashes rows c0 + w*256 + [0, 256) and keeps its matches in row order
    int mine = 0;
    const int64_t wbase = c0 + (int64_t)warp * SK_GROUPS * 32;
    for (int g = 0; g < SK_GROUPS; ++g) {
      const int64_t i = wbase + g * 32 + lane;
      bool hit = false;
      int cd = 0;
      if (i < m) {
        const uint64_t h = splitmix64_at(seed, (uint64_t)i * (uint64_t)zeta + (uint64_t)j);
        const int pos = (int)(((h >> 32) * (uint64_t)plen) >> 32);
        hit = pos >= dlo && pos < dhi;
        cd = ((pos - dlo) << 1) | (int)(h & 1ull);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int slot = mine + __popc(bal & ((1u << lane) - 1u));
        lst[warp * SK_GROUPS * 32 + slot] = (int)(i - c0);
        code[warp * SK_GROUPS * 32 + slot] = cd;
      }
      mine += __popc(bal);
    }
    if (lane == 0) cnt[warp] = mine;
    __syncthreads();
    // phase 2: each thread adds its column of the kept rows, warps' lists in order = row order
    if (has_col) {
      for (int w = 0; w < SK_WARPS; ++w) {
        const int nw = cnt[w];
        const int* L = lst + w * SK_GROUPS * 32;
        const int* C = code + w * SK_GROUPS * 32;
        int e = 0;
        for (; e + 3 < nw; e += 4) {   // four loads in flight, adds in order
          const TA v0 = A[(c0 + L[e]) * lda + kk];
          const TA v1 = A[(c0 + L[e + 1]) * lda + kk];
          const TA v2 = A[(c0 + L[e + 2]) * lda + kk];
          const TA v3 = A[(c0 + L[e + 3]) * lda + kk];
          int q = C[e];
          acc[(q >> 1) * SK_NT + tid] = add_(acc[(q >> 1) * SK_NT + tid], flip_(cvt_<TS, TA>(v0), q & 1));
          q = C[e + 1];
          acc[(q >> 1) * SK_NT + tid] = add_(acc[(q >> 1) * SK_NT + tid], flip_(cvt_<TS, TA>(v1), q & 1));
          q = C[e + 2];
          acc[(q >> 1) * SK_NT + tid] = add_(acc[(q >> 1) * SK_NT + tid], flip_(cvt_<TS, TA>(v2), q & 1));
          q = C[e + 3];
          acc[(q >> 1) * SK_NT + tid] = add_(acc[(q >> 1) * SK_NT + tid], flip_(cvt_<TS, TA>(v3), q & 1));
        }
        for (; e < nw; ++e) {
          const TA v = A[(c0 + L[e]) * lda + kk];
          const int q = C[e];
          acc[(q >> 1) * SK_NT + tid] = add_(acc[(q >> 1) * SK_NT + tid], flip_(cvt_<TS, TA>(v), q & 1));
        }
      }
    }
    __syncthreads();
  }
  // write out, scaled once by zeta^{-1/2}; SA is column-major (d rows)
  if (has_col)
    for (int r = 0; r < dhi - dlo; ++r) SA[(int64_t)kk * d + plo + dlo + r] = scale_(acc[r * SK_NT + tid], scale);
}

template <class TA, class TS>
int launch_sketch(const TA* A, int64_t m, int n, int64_t lda, int d, int zeta, uint64_t seed, TS* SA,
                  cudaStream_t st) {
  const int maxlen = (d + zeta - 1) / zeta + 1;
  const int cblocks = (n + SK_NT - 1) / SK_NT;
  // destination rows per CTA: at most 32 (smem), fewer while that keeps ~2 CTAs per SM busy
  int R = 32;
  while (R > 4 && (int64_t)((maxlen + R - 1) / R) * zeta * cblocks < 2 * num_sms()) R >>= 1;
  R = imin(R, maxlen);
  const int bpp = (maxlen + R - 1) / R;
  const size_t smem = (size_t)R * SK_NT * sizeof(TS) + (size_t)2 * SK_WARPS * SK_GROUPS * 32 * sizeof(int);
  if (smem > max_smem_optin()) return RLOBPCG_ERR_UNSUPPORTED;
  RL_TRY(allow_dynamic_smem(sketch_kernel<TA, TS>, smem));
  dim3 grid(bpp * zeta, cblocks);
  using Rl = RealOf<TS>;
  const Rl scale = (Rl)(1.0 / sqrt((double)zeta));
  sketch_kernel<TA, TS><<<grid, SK_NT, smem, st>>>(A, m, n, lda, d, zeta, seed, R, bpp, scale, SA);
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
