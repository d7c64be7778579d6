// Split-bf16 Gram pass on the 5th-generation tensor cores: the products of the Gram pass of
// Alg. 2 (arXiv 2602.16797; per iteration only the new block W is multiplied by A), real FP64,
//     AW = A W      (m x b)   and   G = A^T AW   (n x b),
// computed as an error-free split of every FP64 operand into bf16 digits (the Ozaki scheme:
// Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012; on tensor cores: Mukunoki,
// Ozaki, Ogita, Imamura, "DGEMM using Tensor Cores, and Its Accurate and Reproducible Versions",
// ISC 2020).
//
// Split. A group of FP64 values (a row of A for the first product, a column of A within a
// 128-row chunk for the second, a column of W, a column of AW within a 128-row chunk) shares one
// exponent E with max |x| < 2^E. Each x becomes V = rint(x 2^(55-E)) (|V| <= 2^55) and V is
// written in balanced base 128, most significant digit first:
//     x ~= 2^(E+1) sum_{p=0}^{7} d_p 2^(-7(p+1)),   d_p integers in [-64, 64],
// with |error| <= 2^(E-56). A digit is exact in bf16 and a digit product (|.| <= 2^12) is exact.
//
// Products. For a digit pair (p, q) the tensor core forms sum_k a_p[k] b_q[k] in f32. Pairs of
// the same level l = p + q share one accumulator: the MMA for A-digit p writes its output
// columns (B-digits q, BP columns each) at TMEM column offset BP * p, so pair (p, q) lands on
// columns BP * l + j. Only levels l <= 8 are kept: a level-9 term is at most 2^12 2^(-7 * 11)
// = 2^-65 of 2^(E+F+2) and the six of them (with everything above) stay below 2^-60 of the
// leading term, far under the 2^-55 of the digit truncation itself. The MMA of A-digit p
// therefore spans only the B-digits q <= 8 - p (N = BP min(8, 9 - p), rounded up to the MMA's
// granularity of 16: the rounding adds a few level >= 9 products in columns that are never
// read), 43 of the 64 pairs. A level holds at most 8 pairs, so with at most 512 terms per
// accumulation |L_l| <= 8 * 512 * 2^12 = 2^24 and the f32 accumulator is exact (integers).
// The result is then
//     2^(E+F-12) sum_{l=0}^{8} 2^(-7 l) L_l,
// evaluated as: levels 8..5 by Horner's rule in f32 (their weight is below 2^-35 of level 0,
// so f32 rounding there stays below 2^-59 of the leading term), levels 4..0 exactly as one int64
// (sum L_l 2^(7 (4 - l)) < 2^53), the two joined and scaled in FP64. The error
// is that of the digit truncation, about 2^-55 of the group maxima per term, which is the size
// of an FP64 dot product's own rounding. Tensor cores do the O(m n b) work; FP64 does O((m+n) b).
// BP, the block width of the digits of W and A W, is 8, 12, 16 or 24 (b <= 24): levels 0..8
// of BP columns take 128 TMEM columns for BP <= 12 (two accumulator buffers and two A stages fit
// in TMEM) and 256 above.
//
// Layouts. A is split once per solve and kept as one BYTE per digit, u_p = d_p + 64 in [0, 127]
// (8 bytes per element, as many as the FP64 value itself); the kernel expands them to bf16 on
// chip: a byte permute puts 0x43 above each byte, giving the bf16 128 + u_p, and one bf16x2 add
// of -192 leaves d_p, exactly (two digits per two instructions). Digits in [-64, 63] need
// |rint(x 2^(55-E))| below 0.992 * 2^55, so an A group takes E with max |x| * 65/64 < 2^E. A
// digit tile is 128 x 16 elements: 256 units of (M index i, K half h), each 64 bytes [p][8 k]
// stored as four 16-byte chunks at 4096 c + 16 u (unit u = 128 h + i), so that a warp of
// converter threads reads 512 consecutive bytes per chunk and writes 32 consecutive 16-byte rows of
// the no-swizzle K-major core-matrix order of tc.cuh (row i of K half h sits at byte
// 2048 h + 16 i of each 4 KB bf16 digit tile). A_rt[r][kb] -- row tile r (128 rows), column
// block kb (16 columns) -- for the first product; A_ct[ct][rc][kb] -- column tile ct (128
// columns) as the M side, row chunk rc (128 rows = 8 blocks of 16) as the K side -- for the
// second. W and AW are split once per pass, straight into bf16 digit tiles.
//
// Kernel shape: one CTA per SM, 448 threads. Warp 0 streams the A digit bytes and the B digits
// of each stage (two k-blocks when A goes through TMEM, else one) into a ring of five or six staging
// slots with bulk copies; warps 6-13 expand each stage's bytes into the eight bf16 digit tiles -- in TMEM beside
// the accumulators for BP <= 12 (the MMAs then read A without shared-memory traffic), else in
// shared memory; warp 1 owns TMEM and issues the MMAs from one thread, B read in the staging
// slot; warps 2-5 read the accumulators (two TMEM buffers, so reading one unit overlaps the MMAs
// of the next), zero them, and do the FP64 recombination. The last CTA of each column tile of
// the second product sums the per-CTA partials in a fixed order. Every wait is bounded and
// reports DEV_ERR_TIMEOUT.
#include "common.cuh"
#include "split.cuh"
#include "tc.cuh"

namespace rl {

namespace {

using split::SL;
using split::TK;
using split::core_off;
using split::group_exp;
using split::split8;
using split::bf16_of;
using split::SPLIT_RESID;
using split::SPLIT_W_READY;
constexpr int TM = 128;                // MMA M: rows (first product) or columns (second) per tile
constexpr int KC_KB = 32;              // k-blocks per exact accumulation: 32 x 16 = 512 terms
constexpr int CH_KB = TM / TK;         // k-blocks per 128-row chunk of the second product
constexpr int NLEV = 9;                // digit-pair levels kept (l = p + q <= 8)
// TMEM columns of one accumulator buffer, and whether the A digits go through TMEM (BP <= 12:
// two stages of two k-blocks fit beside the two buffers) or shared memory
template <int BP> constexpr uint32_t accw() { return NLEV * BP <= 128 ? 128u : 256u; }
template <int BP> constexpr bool ta_of() { return accw<BP>() == 128u; }
// B rows (digits x BP) the MMA of A-digit p reads: the digits q <= 8 - p, rounded up to 16
__host__ __device__ constexpr int np_of(int BP, int p) {
  return ((((9 - p) < 8 ? (9 - p) : 8) * BP + 15) / 16) * 16;
}
// every MMA's output columns [BP p, BP p + np_of(BP, p)) lie inside one accumulator buffer, and
// its B rows inside the 8 BP rows of the B tile
template <int BP>
constexpr bool mma_cols_fit() {
  for (int p = 0; p < SL; ++p)
    if (BP * p + np_of(BP, p) > (int)accw<BP>() || np_of(BP, p) > SL * BP || np_of(BP, p) < 16) return false;
  return true;
}
// bf16 digit stages (MMA operands): in TMEM two stages of two k-blocks; in shared memory three
// stages of one k-block
template <bool TA> constexpr int nst() { return TA ? 2 : 3; }
template <bool TA> constexpr int kps() { return TA ? 2 : 1; }   // k-blocks per stage
// staging slots (bulk copies in flight), each the A digit bytes of a stage and its B digits: the
// bf16 A stages take 32 KB of shared memory each when the MMAs read A from there, none when A
// goes through TMEM; as many slots as fit in 227 KB, at most six
constexpr size_t kSmemMax = 227 * 1024;
template <int BP> constexpr size_t slot_bytes() { return (size_t)kps<ta_of<BP>()>() * (TM * TK * SL + SL * BP * TK * 2); }
template <int BP> constexpr size_t fixed_smem() {
  return (size_t)nst<ta_of<BP>()>() * (ta_of<BP>() ? 0 : SL * TM * TK * 2) + 512 + 2 * 4 * BP * sizeof(double);
}
template <int BP> constexpr int nsb() {
  return (int)((kSmemMax - fixed_smem<BP>()) / slot_bytes<BP>() < 6 ? (kSmemMax - fixed_smem<BP>()) / slot_bytes<BP>() : 6);
}
template <int BP> constexpr size_t pass_smem() { return fixed_smem<BP>() + (size_t)nsb<BP>() * slot_bytes<BP>(); }
constexpr int SLICE_BYTES = TM * TK * 2;   // one bf16 digit tile
constexpr int TILE_U8 = TM * TK * SL;      // the byte digits of one 128 x 16 tile (all 8 digits)
constexpr int NCW = 8;                     // converter warps (one 64-byte unit per thread per stage)
constexpr int NTH = 192 + 32 * NCW;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Dims {
  int64_t R1, NKB, CT, NC;
};
Dims dims_of(int64_t m, int64_t n) { return {cdiv(m, TM), cdiv(n, TK), cdiv(n, TM), cdiv(n, TM) * TM}; }

struct PrepLayout {
  size_t art, act, erow, ecol, cnt, total;
};
PrepLayout prep_layout(int64_t m, int64_t n) {
  const Dims d = dims_of(m, n);
  PrepLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
  L.art = take((size_t)d.R1 * d.NKB * TILE_U8);
  L.act = take((size_t)d.CT * d.R1 * CH_KB * TILE_U8);
  L.erow = take((size_t)d.R1 * TM * sizeof(int));
  L.ecol = take((size_t)d.R1 * d.NC * sizeof(int));
  L.cnt = take((size_t)d.CT * sizeof(int));   // finished-CTA counters of the second product
  L.total = off;
  return L;
}

struct WorkLayout {
  int BP, NR;
  size_t wsl, f, ysl, h, part, total;
};
WorkLayout work_layout(int64_t m, int64_t n, int b) {
  const Dims d = dims_of(m, n);
  WorkLayout L;
  L.BP = b <= 8 ? 8 : b <= 12 ? 12 : b <= 16 ? 16 : 24;
  const int N = SL * L.BP;
  L.NR = (int)std::max<int64_t>(1, std::min<int64_t>(d.R1, num_sms() / std::max<int64_t>(1, d.CT)));
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
  L.wsl = take((size_t)d.NKB * N * TK * 2);
  L.f = take(64 * sizeof(int));
  L.ysl = take((size_t)d.R1 * CH_KB * N * TK * 2);
  L.h = take((size_t)d.R1 * L.BP * sizeof(int));
  L.part = take((size_t)L.NR * d.NC * L.BP * sizeof(double));
  L.total = off;
  return L;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---- one-time split of A ---------------------------------------------------------------------------
// Exponent of a group of A: max |x| * 65/64 < 2^E (see the byte form above).
__device__ __forceinline__ int group_exp_a(double amax) { return group_exp(amax * 1.015625); }

// Byte digits of 8 values sharing exponent E: w[2p + kk/4] holds u_p of value kk in byte kk%4,
// u_p the base-128 digits of V + OFF, V = rint(x 2^(55-E)), OFF = 64 sum_p 128^p, so that
// V = sum_p (u_p - 64) 128^(7-p) with every u_p in [0, 127].
__device__ __forceinline__ void digit_bytes(const double (&x)[8], int E, uint32_t (&w)[16]) {
  constexpr unsigned long long OFF = (64ull * ((1ull << 56) - 1)) / 127;
#pragma unroll
  for (int q = 0; q < 16; ++q) w[q] = 0;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const unsigned long long Y = (unsigned long long)split::scaled_int(x[kk], E) + OFF;
    const uint32_t lo = (uint32_t)Y, hi = (uint32_t)(Y >> 32);
    // digit p holds bits [7 (7 - p), 7 (7 - p) + 7) of Y
    const uint32_t d[SL] = {(hi >> 17) & 127u, (hi >> 10) & 127u, (hi >> 3) & 127u, __funnelshift_r(lo, hi, 28) & 127u,
                            (lo >> 21) & 127u, (lo >> 14) & 127u, (lo >> 7) & 127u, lo & 127u};
#pragma unroll
    for (int p = 0; p < SL; ++p) w[2 * p + (kk >> 2)] |= d[p] << (8 * (kk & 3));
  }
}

__device__ __forceinline__ void store_unit(unsigned char* tile, int t, const uint32_t (&w)[16]) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<uint4*>(tile + c * 4096 + t * 16) = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
}

// One CTA per 128-row chunk rc: the row exponents of its rows and the column exponents of the
// chunk (the groups of the two products), from one read of A; maxima are taken on the bit
// patterns of |x| (ordered like the values), which also flags NaN and infinity.
__global__ void __launch_bounds__(256) exp_scan_kernel(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                       int64_t NC, int* __restrict__ erow, int* __restrict__ ecol,
                                                       int* err) {
  constexpr unsigned long long ABS = 0x7fffffffffffffffull, INF = 0x7ff0000000000000ull;
  __shared__ unsigned long long cmax[8][512];
  __shared__ unsigned long long rmax[TM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t rc = blockIdx.x, i0 = rc * TM;
  const int nrow = (int)min((int64_t)TM, m - i0);
  bool bad = false;
  for (int r = threadIdx.x; r < TM; r += 256) rmax[r] = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < NC; c0 += 512) {
    unsigned long long cm[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) cm[q] = 0;
    for (int r = warp; r < nrow; r += 8) {
      const double* row = A + (i0 + r) * lda;
      unsigned long long rm = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int64_t c = c0 + q * 32 + lane;
        if (c < n) {
          const unsigned long long key = (unsigned long long)__double_as_longlong(row[c]) & ABS;
          rm = max(rm, key);
          cm[q] = max(cm[q], key);
        }
      }
      const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(rm >> 32));
      const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(rm >> 32) == hi ? (unsigned)rm : 0u);
      if (lane == 0) rmax[r] = max(rmax[r], ((unsigned long long)hi << 32) | lo);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) cmax[warp][q * 32 + lane] = cm[q];
    __syncthreads();
    for (int c = threadIdx.x; c < 512; c += 256) {
      unsigned long long v = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) v = max(v, cmax[w][c]);
      if (c0 + c < NC) {
        bad |= v >= INF;
        ecol[rc * NC + c0 + c] = group_exp_a(__longlong_as_double((long long)v));
      }
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < TM; r += 256) {
    const unsigned long long v = rmax[r];
    bad |= v >= INF;
    erow[i0 + r] = group_exp_a(__longlong_as_double((long long)v));
  }
  if (bad && err) atomicOr(err, DEV_ERR_NONFINITE);
}

// one CTA per 128 x 16 tile (r, kb); thread t writes unit t (row t % 128, K half t / 128)
__global__ void __launch_bounds__(256) rt_digits_kernel(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                        const int* __restrict__ erow, int64_t NKB,
                                                        unsigned char* __restrict__ Art) {
  const int64_t r = blockIdx.x, kb = blockIdx.y;
  const int t = threadIdx.x, row = t & 127, h = t >> 7;
  const int64_t i = r * TM + row, k0 = kb * TK + h * 8;
  double x[8];
  int E = 0;
  if (i < m) E = erow[i];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) x[kk] = (i < m && k0 + kk < n) ? A[i * lda + k0 + kk] : 0.0;
  uint32_t w[16];
  digit_bytes(x, E, w);
  store_unit(Art + (size_t)(r * NKB + kb) * TILE_U8, t, w);
}

// one CTA per tile (ct, rc, kb): rows rc * 128 + kb * 16 + [0, 16) of columns ct * 128 + [0, 128),
// staged through shared memory so that the loads are coalesced; thread t writes unit t
// (column t % 128 as the M index, K half t / 128)
__global__ void __launch_bounds__(256) ct_digits_kernel(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                        const int* __restrict__ ecol, int64_t NC, int64_t R1,
                                                        unsigned char* __restrict__ Act) {
  __shared__ double tile[TK][TM + 1];
  const int64_t rc = blockIdx.x / CH_KB;
  const int kb = (int)(blockIdx.x % CH_KB);
  const int64_t ct = blockIdx.y;
  const int64_t i0 = rc * TM + kb * TK, c0 = ct * TM;
  for (int e = threadIdx.x; e < TK * TM; e += 256) {
    const int rr = e >> 7, cc = e & 127;
    const int64_t i = i0 + rr, c = c0 + cc;
    tile[rr][cc] = (i < m && c < n) ? A[i * lda + c] : 0.0;
  }
  __syncthreads();
  const int t = threadIdx.x, cc = t & 127, h = t >> 7;
  double x[8];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) x[kk] = tile[h * 8 + kk][cc];
  uint32_t w[16];
  digit_bytes(x, ecol[rc * NC + c0 + cc], w);
  store_unit(Act + (size_t)(((ct * R1 + rc) * CH_KB + kb)) * TILE_U8, t, w);
}

// Expands one 64-byte unit (8 digits of 8 values) into the bf16 digit tiles of a stage: digit p
// goes to the 16-byte row at dst + p * SLICE_BYTES.
__device__ __forceinline__ uint32_t bf16x2_minus192(uint32_t v) {
  uint32_t r;
  asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0xC340C340u));
  return r;
}
template <class Put>
__device__ __forceinline__ void expand_unit_to(const uint4 (&b)[4], Put put) {
  const uint32_t w[16] = {b[0].x, b[0].y, b[0].z, b[0].w, b[1].x, b[1].y, b[1].z, b[1].w,
                          b[2].x, b[2].y, b[2].z, b[2].w, b[3].x, b[3].y, b[3].z, b[3].w};
  constexpr uint32_t HI = 0x43434343u;   // bf16 0x43uu = 128 + uu for uu < 128
#pragma unroll
  for (int p = 0; p < SL; ++p)
    put(p, bf16x2_minus192(__byte_perm(w[2 * p], HI, 0x4140)), bf16x2_minus192(__byte_perm(w[2 * p], HI, 0x4342)),
        bf16x2_minus192(__byte_perm(w[2 * p + 1], HI, 0x4140)), bf16x2_minus192(__byte_perm(w[2 * p + 1], HI, 0x4342)));
}
__device__ __forceinline__ void expand_unit(const uint4 (&b)[4], unsigned char* dst) {
  expand_unit_to(b, [&](int p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    *reinterpret_cast<uint4*>(dst + p * SLICE_BYTES) = make_uint4(x, y, z, w);
  });
}

// ---- per-pass split of W (one CTA) ---------------------------------------------------------------
template <int BP>
__global__ void __launch_bounds__(512) w_digits_kernel(const double* __restrict__ W, int n, int b, int64_t ldw,
                                                       int64_t NKB, uint16_t* __restrict__ Wsl, int* __restrict__ F,
                                                       int* err) {
  constexpr int N = SL * BP;
  __shared__ double red[16][BP];
  __shared__ int Fs[BP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double mx[BP];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < BP; ++j) mx[j] = 0;
  for (int k = threadIdx.x; k < n; k += 512)
#pragma unroll
    for (int j = 0; j < BP; ++j)
      if (j < b) {
        const double a = fabs(W[(int64_t)k * ldw + j]);
        bad |= !(a <= 1.7976931348623157e308);
        mx[j] = fmax(mx[j], a);
      }
#pragma unroll
  for (int j = 0; j < BP; ++j) {
    const double v = warp_max(mx[j]);
    if (lane == 0) red[warp][j] = v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, DEV_ERR_NONFINITE);
  if (threadIdx.x < BP) {
    double v = 0;
    for (int w = 0; w < 16; ++w) v = fmax(v, red[w][threadIdx.x]);
    Fs[threadIdx.x] = group_exp(v);
    F[threadIdx.x] = Fs[threadIdx.x];
  }
  __syncthreads();
  const int64_t total = NKB * TK * BP;
  for (int64_t e = threadIdx.x; e < total; e += 512) {
    const int j = (int)(e % BP);
    const int64_t k = e / BP;
    const double x = (k < n && j < b) ? W[k * ldw + j] : 0.0;
    int d[SL];
    split8(x, Fs[j], d);
    uint16_t* out = Wsl + (size_t)(k / TK) * (N * TK);
    const int kk = (int)(k % TK);
#pragma unroll
    for (int q = 0; q < SL; ++q) out[core_off(q * BP + j, kk, N)] = bf16_of(d[q]);
  }
}

// Digits of one 128-row chunk of Y = AW (B operand of the second product): the chunk's column
// maxima set H_j, then row `row` writes its digits. `bar` synchronises the 128 threads of the chunk.
template <int BP, class Bar>
__device__ __forceinline__ void emit_y_digits(const double (&y)[BP], int b, int row, int lane, int quarter,
                                              double* red, int64_t rc, uint16_t* __restrict__ Ysl,
                                              int* __restrict__ H, Bar bar) {
  constexpr int N = SL * BP;
  // group maxima on the bit patterns of |y| (integer instructions; red holds the bits)
  unsigned long long* redb = reinterpret_cast<unsigned long long*>(red);
#pragma unroll
  for (int j = 0; j < BP; ++j) {
    const unsigned long long v = split::warp_max_abs_bits(j < b ? y[j] : 0.0);
    if (lane == 0) redb[quarter * BP + j] = v;
  }
  bar();
  int Hj[BP];
#pragma unroll
  for (int j = 0; j < BP; ++j)
    Hj[j] = group_exp(__longlong_as_double(
        (long long)max(max(redb[j], redb[BP + j]), max(redb[2 * BP + j], redb[3 * BP + j]))));
  if (row == 0)
#pragma unroll
    for (int j = 0; j < BP; ++j) H[rc * BP + j] = j < b ? Hj[j] : 0;
  uint16_t* out = Ysl + (size_t)(rc * CH_KB + (row >> 4)) * (N * TK);
  const int kk = row & 15;
#pragma unroll
  for (int j = 0; j < BP; ++j) {
    int d[SL];
    split8(j < b ? y[j] : 0.0, Hj[j], d);
#pragma unroll
    for (int q = 0; q < SL; ++q) out[core_off(q * BP + j, kk, N)] = bf16_of(d[q]);
  }
}

// Y given (the residual refresh: G = A^T A_V for a stored A_V): one CTA of 128 threads per chunk
template <int BP>
__global__ void __launch_bounds__(128) y_digits_kernel(const double* __restrict__ Y, int64_t m, int b, int64_t ldy,
                                                       uint16_t* __restrict__ Ysl, int* __restrict__ H, int* err) {
  __shared__ double red[4 * BP];
  const int64_t rc = blockIdx.x;
  const int row = threadIdx.x;
  const int64_t i = rc * TM + row;
  double y[BP];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < BP; ++j) {
    y[j] = (i < m && j < b) ? Y[i * ldy + j] : 0.0;
    bad |= !(fabs(y[j]) <= 1.7976931348623157e308);
  }
  if (bad) atomicOr(err, DEV_ERR_NONFINITE);
  emit_y_digits<BP>(y, b, row, row & 31, row >> 5, red, rc, Ysl, H, [] { __syncthreads(); });
}

// ---- the tensor-core pass ---------------------------------------------------------------------
struct PassArgs {
  const unsigned char* Aop;   // byte digits A_rt (first product) or A_ct (second)
  const uint16_t* Bop;   // W digits or AW digits
  const int* eA;         // row exponents of A, or column exponents per chunk
  const int* eB;         // W column exponents, or AW column exponents per chunk
  int64_t m, R1, NKB, CT, NC;
  int b, NR;
  double* AW;            // first product: output (m x b, ldaw)
  int64_t ldaw;
  uint16_t* Ysl;         // first product: digits of AW for the second product (or null)
  int* H;
  double* part;          // second product: partials [NR][NC][BP]
  double* G;             // second product: output (n x b, ldg), summed by the last CTA per column tile
  int64_t ldg, n;
  int* cnt;              // per column tile: CTAs finished (zero between launches)
  int* err;
};

// Bounded wait by the four epilogue warps; the outcome is made uniform over all 128 threads, so
// that they either all go on (and meet every later named barrier) or all stop.
__device__ __forceinline__ bool epi_wait(uint64_t* bar, uint32_t parity) {
  return tc::named_bar_and<2>(128, tc::mbar_wait(bar, parity));
}

template <int BP>
__device__ __forceinline__ void ld_level8(uint32_t taddr, uint32_t (&r)[BP], int h) {
  tc::tmem_ld8(taddr, r[h], r[h + 1], r[h + 2], r[h + 3], r[h + 4], r[h + 5], r[h + 6], r[h + 7]);
}

// Reads one accumulator buffer (levels 0..8 of BP columns) eight columns at a time, hands
// s_j = 2^28 sum_l 2^(-7 l) L_l[j] of every column j < b to put(j, s_j), then zeroes the buffer
// for reuse and releases it. Levels 4..0 are integers below 2^24 held exactly in f32, so
// S = sum_{l<=4} L_l 2^(7 (4 - l)) is an exact int64 below 2^53 and converts to FP64 exactly;
// levels 8..5 by Horner's rule in f32: three FP64-pipe instructions per column (the FP64 pipe is
// the scarce one in the epilogue).
template <int BP, class Put>
__device__ __forceinline__ void drain_levels(uint32_t ta, uint64_t* release, int b, Put put) {
  constexpr int BR = (BP + 7) / 8 * 8;
#pragma unroll
  for (int h = 0; h < BR; h += 8) {
    // levels 8..5 (Horner in f32), then levels 0..4 (exact int64): two waits, a smaller peak
    uint32_t r[5][8];
    float t[8];
#pragma unroll
    for (int l = 0; l < 4; ++l)
      tc::tmem_ld8(ta + BP * (8 - l) + h, r[l][0], r[l][1], r[l][2], r[l][3], r[l][4], r[l][5], r[l][6], r[l][7]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      t[jj] = __uint_as_float(r[0][jj]);
#pragma unroll
      for (int l = 1; l < 4; ++l) t[jj] = fmaf(t[jj], 0x1p-7f, __uint_as_float(r[l][jj]));
    }
#pragma unroll
    for (int l = 0; l < 5; ++l)
      tc::tmem_ld8(ta + BP * l + h, r[l][0], r[l][1], r[l][2], r[l][3], r[l][4], r[l][5], r[l][6], r[l][7]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = h + jj;
      if (j < BP && j < b) {
        long long S = __float2int_rn(__uint_as_float(r[0][jj]));
#pragma unroll
        for (int l = 1; l <= 4; ++l) S = S * 128 + __float2int_rn(__uint_as_float(r[l][jj]));
        put(j, fma((double)t[jj], 0x1p-7, __ll2double_rn(S)));
      }
    }
  }
  // the buffer is free again once it is zero
  constexpr uint32_t ACCW = accw<BP>();
#pragma unroll
  for (uint32_t c = 0; c < ACCW; c += 8) tc::tmem_st8_zero(ta + c);
  tc::tmem_st_wait();
  tc::fence_before_sync();
  tc::mbar_arrive(release);
}

// MODE 0: AW = A W (+ digits of AW). MODE 1: partial G = A^T AW over each CTA's row chunks.
template <int BP, int MODE>
__global__ void __launch_bounds__(NTH, 1) split_pass_kernel(PassArgs g) {
  constexpr int N = SL * BP;
  constexpr uint32_t ACCW = accw<BP>();
  constexpr uint32_t BBYTES = N * TK * 2;
  static_assert(BP % 4 == 0 && mma_cols_fit<BP>(), "digit block width outside the TMEM layout");
  static_assert(nsb<BP>() >= 4 && pass_smem<BP>() <= kSmemMax, "staging ring does not fit in shared memory");
  // BP <= 12: the A digits of a stage go to TMEM (8 columns per digit, after the two accumulator
  // buffers), so shared memory holds only B and the MMAs read A without shared-memory traffic
  constexpr bool TA = ta_of<BP>();
  // A stage covers KPS k-blocks (a unit of KC_KB or CH_KB k-blocks -- both even -- never splits
  // a stage; the last stage of a unit may hold one k-block)
  constexpr int KPS = kps<TA>();
  constexpr uint32_t STG = TA ? 0 : SL * SLICE_BYTES;      // bf16 A stage in shared memory
  constexpr uint32_t SLOT = KPS * (TILE_U8 + BBYTES);      // staging slot: KPS A byte tiles, KPS B tiles
  constexpr int NSB = nsb<BP>();
  constexpr int NST = nst<TA>();
  constexpr uint32_t TCOLS = TA ? 512 : 2 * ACCW;
  constexpr uint32_t ACOL0 = 2 * ACCW;   // TMEM column of the A digits of stage 0 (TA)
  constexpr uint32_t ASTW = 64 * KPS;    // TMEM columns of one A stage (TA)
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* bring = sm + NST * STG;   // staging slots, SLOT bytes each
  uint64_t* full = reinterpret_cast<uint64_t*>(bring + NSB * SLOT);
  uint64_t* empty = full + NST;
  uint64_t* bfull = empty + NST;
  uint64_t* bempty = bfull + NSB;
  uint64_t* accf = bempty + NSB;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  double* red = reinterpret_cast<double*>(bring + NSB * SLOT + 512);   // [2][4][BP]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      tc::mbar_init(full + s, NCW);       // the converter warps
      tc::mbar_init(empty + s, 1);        // the MMAs of the stage
    }
    for (int s = 0; s < NSB; ++s) {
      tc::mbar_init(bfull + s, 1);        // the copies (with their bytes)
      tc::mbar_init(bempty + s, NCW + 1); // the converter warps and the MMAs (which read B there)
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(accf + a, 1);
      tc::mbar_init(acce + a, 128);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tslot, TCOLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  // work of this CTA: MODE 0 -- row tiles r = blockIdx.x (+ gridDim.x ...), each ceil(NKB / 32)
  // units of up to 32 k-blocks; MODE 1 -- column tile ct and row chunks [rc0, rc1), one unit each
  const int64_t ct = MODE == 1 ? blockIdx.x % g.CT : 0;
  const int64_t rng = MODE == 1 ? blockIdx.x / g.CT : 0;
  const int64_t rc0 = MODE == 1 ? rng * g.R1 / g.NR : 0;
  const int64_t rc1 = MODE == 1 ? (rng + 1) * g.R1 / g.NR : 0;
  const int64_t NKC = cdiv(g.NKB, KC_KB);

  if (warp == 0) {
    // the A digit bytes and the B digits of every stage, NSB stages ahead of the converters
    if (lane == 0) {
      uint32_t u = 0;
      bool ok = true;
      // the nk tiles of a stage are consecutive in both digit layouts
      auto load = [&](const unsigned char* srcA, const uint16_t* srcB, int nk) {
        const int s = (int)(u % NSB);
        if (!tc::mbar_wait(bempty + s, ((u / NSB) & 1) ^ 1)) return false;
        unsigned char* slot = bring + (size_t)s * SLOT;
        tc::mbar_expect_tx(bfull + s, (uint32_t)nk * (TILE_U8 + BBYTES));
        tc::bulk_g2s(slot, srcA, (uint32_t)nk * TILE_U8, bfull + s);
        tc::bulk_g2s(slot + KPS * TILE_U8, srcB, (uint32_t)nk * BBYTES, bfull + s);
        ++u;
        return true;
      };
      if (MODE == 0) {
        for (int64_t r = blockIdx.x; ok && r < g.R1; r += gridDim.x)
          for (int64_t kb = 0; ok && kb < g.NKB; kb += KPS)
            ok = load(g.Aop + (size_t)(r * g.NKB + kb) * TILE_U8, g.Bop + (size_t)kb * (N * TK),
                      (int)std::min<int64_t>(KPS, g.NKB - kb));
      } else {
        for (int64_t rc = rc0; ok && rc < rc1; ++rc)
          for (int kb = 0; ok && kb < CH_KB; kb += KPS)
            ok = load(g.Aop + (size_t)((ct * g.R1 + rc) * CH_KB + kb) * TILE_U8,
                      g.Bop + (size_t)(rc * CH_KB + kb) * (N * TK), KPS);
      }
      if (!ok) atomicOr(g.err, DEV_ERR_TIMEOUT);
      // copies into the last NSB slots have landed before the CTA may finish
      for (uint32_t w = u > (uint32_t)NSB ? u - NSB : 0; w < u; ++w) tc::mbar_wait(bfull + (w % NSB), (w / NSB) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t u = 0, v = 0;
      bool ok = true;
      auto unit = [&](int nkb) {
        const int a = (int)(v & 1);
        if (!tc::mbar_wait(acce + a, (v >> 1) & 1)) return false;
        tc::fence_after_sync();
        const uint32_t dbase = tmem + (uint32_t)a * ACCW;
        for (int kb = 0; kb < nkb; kb += KPS) {
          const int s = (int)(u % NST), ds = (int)(u % NSB);
          if (!tc::mbar_wait(full + s, (u / NST) & 1)) return false;
          tc::fence_after_sync();
          unsigned char* stg = sm + (size_t)s * STG;
          const int nk = nkb - kb < KPS ? nkb - kb : KPS;
          for (int q = 0; q < nk; ++q) {
            const uint64_t bdesc =
                tc::smem_desc(bring + (size_t)ds * SLOT + KPS * TILE_U8 + q * BBYTES, (N / 8) * 128, 128);
#pragma unroll
            for (int p = 0; p < SL; ++p) {
              // A-digit p against the B-digits of levels p + q <= 8 only
              const uint32_t idesc = tc::idesc_bf16_f32(TM, np_of(BP, p));
              if (TA)
                tc::mma_bf16_ta(dbase + (uint32_t)(BP * p), tmem + ACOL0 + (uint32_t)(ASTW * s + 64 * q + 8 * p), bdesc,
                                idesc, 1u);
              else
                tc::mma_bf16(dbase + (uint32_t)(BP * p), tc::smem_desc(stg + p * SLICE_BYTES, 2048, 128), bdesc, idesc,
                             1u);
            }
          }
          tc::mma_commit(empty + s);
          tc::mma_commit(bempty + ds);
          ++u;
        }
        tc::mma_commit(accf + a);
        ++v;
        return true;
      };
      if (MODE == 0) {
        for (int64_t r = blockIdx.x; ok && r < g.R1; r += gridDim.x)
          for (int64_t kc = 0; ok && kc < NKC; ++kc) ok = unit((int)std::min<int64_t>(KC_KB, g.NKB - kc * KC_KB));
      } else {
        for (int64_t rc = rc0; ok && rc < rc1; ++rc) ok = unit(CH_KB);
      }
      if (!ok) atomicOr(g.err, DEV_ERR_TIMEOUT);
      // every MMA issued here has finished before TMEM is released
      tc::mma_commit(done);
      tc::mbar_wait(done, 0);
    }
  } else if (warp < 6) {
    const int quarter = warp & 3;                 // TMEM lanes 32 * quarter .. + 31
    const int row = 32 * quarter + lane;          // MODE 0: row of the tile; MODE 1: column
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
    for (uint32_t c = 0; c < 2 * ACCW; c += 8) tc::tmem_st8_zero(tq + c);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::mbar_arrive(acce + 0);
    tc::mbar_arrive(acce + 1);
    uint32_t v = 0;
    bool ok = true;
    if (MODE == 0) {
      int Fj[BP];
#pragma unroll
      for (int j = 0; j < BP; ++j) Fj[j] = g.eB[j];
      int t = 0;
      for (int64_t r = blockIdx.x; ok && r < g.R1; r += gridDim.x, ++t) {
        const int64_t i = r * TM + row;
        const int Ei = g.eA[i];
        double y[BP];
#pragma unroll
        for (int j = 0; j < BP; ++j) y[j] = 0;
        for (int64_t kc = 0; kc < NKC; ++kc) {
          const int a = (int)(v & 1);
          ok = epi_wait(accf + a, (v >> 1) & 1);
          if (!ok) break;
          tc::fence_after_sync();
          drain_levels<BP>(tq + (uint32_t)a * ACCW, acce + a, g.b,
                           [&](int j, double sj) { y[j] += split::mul_pow2(sj, Ei + Fj[j] - 40); });
          ++v;
        }
        if (!ok) break;
        if (i < g.m)
#pragma unroll
          for (int j = 0; j < BP; ++j)
            if (j < g.b) g.AW[i * g.ldaw + j] = y[j];
        if (g.Ysl)
          emit_y_digits<BP>(y, g.b, row, lane, quarter, red + (t & 1) * 4 * BP, r, g.Ysl, g.H,
                            [] { tc::named_bar<1>(128); });
      }
    } else {
      const int64_t c = ct * TM + row;
      double acc[BP];
#pragma unroll
      for (int j = 0; j < BP; ++j) acc[j] = 0;
      for (int64_t rc = rc0; ok && rc < rc1; ++rc) {
        const int a = (int)(v & 1);
        ok = epi_wait(accf + a, (v >> 1) & 1);
        if (!ok) break;
        tc::fence_after_sync();
        const int Ec = g.eA[rc * g.NC + c];
        const int* eBr = g.eB + rc * BP;
        drain_levels<BP>(tq + (uint32_t)a * ACCW, acce + a, g.b,
                         [&](int j, double sj) { acc[j] += split::mul_pow2(sj, Ec + eBr[j] - 40); });
        ++v;
      }
      double* out = g.part + (size_t)(rng * g.NC + c) * BP;
#pragma unroll
      for (int j = 0; j < BP; ++j) out[j] = (ok && j < g.b) ? acc[j] : 0.0;
      // the last CTA of this column tile to finish sums the NR partials in range order
      // (deterministic); the counter is left at zero for the next launch
      __shared__ int s_last;
      __threadfence();
      tc::named_bar<1>(128);
      if (row == 0) s_last = atomicAdd(g.cnt + ct, 1) == g.NR - 1;
      tc::named_bar<1>(128);
      if (s_last) {
        __threadfence();
        if (c < g.n) {
          // 4 interleaved accumulators per column keep several L2 loads in flight; the
          // combination order is fixed
          double sum[4][BP];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < BP; ++j) sum[u][j] = 0;
          int r = 0;
          for (; r + 3 < g.NR; r += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const double* pr = g.part + (size_t)((r + u) * g.NC + c) * BP;
#pragma unroll
              for (int j = 0; j < BP; ++j)
                if (j < g.b) sum[u][j] += __ldcg(pr + j);
            }
          for (; r < g.NR; ++r) {
            const double* pr = g.part + (size_t)(r * g.NC + c) * BP;
#pragma unroll
            for (int j = 0; j < BP; ++j)
              if (j < g.b) sum[0][j] += __ldcg(pr + j);
          }
#pragma unroll
          for (int j = 0; j < BP; ++j)
            if (j < g.b) g.G[c * g.ldg + j] = (sum[0][j] + sum[1][j]) + (sum[2][j] + sum[3][j]);
        }
        if (row == 0) g.cnt[ct] = 0;
      }
    }
    if (!ok) atomicOr(g.err, DEV_ERR_TIMEOUT);
  } else {
    // converter warps: thread ci expands unit ci (M index ci % 128, K half ci / 128) of each of
    // the stage's nk A tiles from the staging slot into the bf16 digit tiles; warp w covers rows
    // 32 (w % 4) .. + 31 (its TMEM lane quarter) of K half (w - 6) / 4
    const int quarter = warp & 3, h = (warp - 6) >> 2, row = 32 * quarter + lane;
    const int ci = 128 * h + row;
    const uint32_t soff = (uint32_t)(h * 2048 + row * 16);
    const uint32_t tq = tmem + ((uint32_t)(32 * quarter) << 16) + ACOL0 + 4 * h;
    uint32_t u = 0;
    auto stage = [&](int nk) {
      const int ds = (int)(u % NSB), s = (int)(u % NST);
      if (!__all_sync(0xffffffffu, tc::mbar_wait(bfull + ds, (u / NSB) & 1))) return false;
      uint4 b[KPS][4];
      const unsigned char* sp = bring + (size_t)ds * SLOT + (size_t)ci * 16;
#pragma unroll
      for (int q = 0; q < KPS; ++q)
        if (q < nk)
#pragma unroll
          for (int c = 0; c < 4; ++c) b[q][c] = *reinterpret_cast<const uint4*>(sp + q * TILE_U8 + c * 4096);
      if (!__all_sync(0xffffffffu, tc::mbar_wait(empty + s, ((u / NST) & 1) ^ 1))) return false;
      // the staging slot is free once every lane's bytes are in registers (the expansion consumed
      // them); the tensor core reads the digits just written through TMEM or the async proxy
      if (TA) {
#pragma unroll
        for (int q = 0; q < KPS; ++q)
          if (q < nk)
            expand_unit_to(b[q], [&](int p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
              tc::tmem_st4(tq + (uint32_t)(ASTW * s + 64 * q + 8 * p), x, y, z, w);
            });
        tc::tmem_st_wait();
        tc::fence_before_sync();
      } else {
        expand_unit(b[0], sm + (size_t)s * STG + soff);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      }
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(bempty + ds);
        tc::mbar_arrive(full + s);
      }
      ++u;
      return true;
    };
    bool ok = true;
    if (MODE == 0) {
      for (int64_t r = blockIdx.x; ok && r < g.R1; r += gridDim.x)
        for (int64_t kb = 0; ok && kb < g.NKB; kb += KPS) ok = stage((int)std::min<int64_t>(KPS, g.NKB - kb));
    } else {
      for (int64_t rc = rc0; ok && rc < rc1; ++rc)
        for (int kb = 0; ok && kb < CH_KB; kb += KPS) ok = stage(KPS);
    }
    if (!ok && lane == 0) atomicOr(g.err, DEV_ERR_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TCOLS);
  }
}

template <int BP, int MODE>
int launch_pass(const PassArgs& a, int grid, cudaStream_t st) {
  const size_t smem = pass_smem<BP>();
  RL_TRY(allow_dynamic_smem(split_pass_kernel<BP, MODE>, smem));
  split_pass_kernel<BP, MODE><<<grid, NTH, smem, st>>>(a);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

template <int BP>
int split_gram_bp(const unsigned char* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw, double* AW,
                  int64_t ldaw, double* G, int64_t ldg, unsigned char* work, int flags, int* err,
                  cudaEvent_t mid, cudaStream_t st) {
  const bool resid_mode = (flags & SPLIT_RESID) != 0;
  const bool first = (flags & split::SPLIT_SECOND_ONLY) == 0, second = (flags & split::SPLIT_FIRST_ONLY) == 0;
  const Dims d = dims_of(m, n);
  const PrepLayout P = prep_layout(m, n);
  const WorkLayout L = work_layout(m, n, b);
  uint16_t* Ysl = (uint16_t*)(work + L.ysl);
  int* H = (int*)(work + L.h);
  if (!first) {
    // the second product alone
  } else if (!resid_mode) {
    if (!(flags & SPLIT_W_READY)) {
      w_digits_kernel<BP><<<1, 512, 0, st>>>(W, (int)n, b, ldw, d.NKB, (uint16_t*)(work + L.wsl), (int*)(work + L.f),
                                            err);
      RL_CHECK_LAUNCH();
    }
    PassArgs a{};
    a.Aop = prep + P.art;
    a.Bop = (const uint16_t*)(work + L.wsl);
    a.eA = (const int*)(prep + P.erow);
    a.eB = (const int*)(work + L.f);
    a.m = m; a.R1 = d.R1; a.NKB = d.NKB; a.CT = d.CT; a.NC = d.NC;
    a.b = b; a.NR = L.NR;
    a.AW = AW; a.ldaw = ldaw; a.Ysl = Ysl; a.H = H; a.err = err;
    RL_TRY((launch_pass<BP, 0>(a, (int)std::min<int64_t>(d.R1, num_sms()), st)));
  } else {
    y_digits_kernel<BP><<<(unsigned)d.R1, 128, 0, st>>>(AW, m, b, ldaw, Ysl, H, err);
    RL_CHECK_LAUNCH();
  }
  if (mid) RL_CUDA(cudaEventRecord(mid, st));
  if (!second) return RLOBPCG_OK;
  // row ranges per column tile: fewer when SMs are to be left free for another stream (the
  // partials of the ranges are summed in range order either way)
  const int reserve = (flags >> 16) & 0xff;
  const int NR = (int)std::max<int64_t>(
      1, std::min<int64_t>(L.NR, (num_sms() - reserve) / std::max<int64_t>(1, d.CT)));
  PassArgs a{};
  a.Aop = prep + P.act;
  a.Bop = Ysl;
  a.eA = (const int*)(prep + P.ecol);
  a.eB = H;
  a.m = m; a.R1 = d.R1; a.NKB = d.NKB; a.CT = d.CT; a.NC = d.NC;
  a.b = b; a.NR = NR;
  a.part = (double*)(work + L.part);
  a.G = G;
  a.ldg = ldg;
  a.n = n;
  a.cnt = (int*)(prep + P.cnt);
  a.err = err;
  RL_TRY((launch_pass<BP, 1>(a, (int)(d.CT * NR), st)));
  return RLOBPCG_OK;
}

}  // namespace

size_t split_prep_bytes(int64_t m, int64_t n) { return (m < 1 || n < 1) ? 0 : prep_layout(m, n).total; }

size_t split_work_bytes(int64_t m, int64_t n, int b) {
  return (m < 1 || n < 1 || b < 1 || b > 24) ? 0 : work_layout(m, n, b).total;
}

int split_prepare(const double* A, int64_t m, int64_t n, int64_t lda, void* prep, size_t prep_bytes, int* err,
                  cudaStream_t st) {
  if (!A || !prep || m < 1 || n < 1 || lda < n) return RLOBPCG_ERR_INVALID_ARG;
  const PrepLayout P = prep_layout(m, n);
  if (prep_bytes < P.total) return RLOBPCG_ERR_INVALID_ARG;
  const Dims d = dims_of(m, n);
  if (d.NKB > 65535 || d.R1 * CH_KB > 2147483647LL) return RLOBPCG_ERR_UNSUPPORTED;
  unsigned char* base = (unsigned char*)prep;
  int* erow = (int*)(base + P.erow);
  int* ecol = (int*)(base + P.ecol);
  RL_CUDA(cudaMemsetAsync(base + P.cnt, 0, (size_t)d.CT * sizeof(int), st));
  exp_scan_kernel<<<(unsigned)d.R1, 256, 0, st>>>(A, m, (int)n, lda, d.NC, erow, ecol, err);
  RL_CHECK_LAUNCH();
  rt_digits_kernel<<<dim3((unsigned)d.R1, (unsigned)d.NKB), 256, 0, st>>>(A, m, (int)n, lda, erow, d.NKB,
                                                                         base + P.art);
  RL_CHECK_LAUNCH();
  ct_digits_kernel<<<dim3((unsigned)(d.R1 * CH_KB), (unsigned)d.CT), 256, 0, st>>>(A, m, (int)n, lda, ecol, d.NC, d.R1,
                                                                                  base + P.act);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

split::WDigits split_w_digits(void* work, int64_t m, int64_t n, int b) {
  const WorkLayout L = work_layout(m, n, b);
  split::WDigits w;
  w.Wsl = (uint16_t*)((unsigned char*)work + L.wsl);
  w.F = (int*)((unsigned char*)work + L.f);
  w.NKB = dims_of(m, n).NKB;
  w.BP = L.BP;
  return w;
}

int split_gram(const void* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw, double* AW, int64_t ldaw,
               double* G, int64_t ldg, void* work, size_t work_bytes, int flags, int* err, cudaEvent_t mid,
               cudaStream_t st) {
  const bool resid_mode = (flags & SPLIT_RESID) != 0;
  if (!prep || !AW || !G || !work || m < 1 || n < 1 || b < 1 || b > 24 || ldaw < b || ldg < b ||
      (!resid_mode && (!W || ldw < b)))
    return RLOBPCG_ERR_INVALID_ARG;
  if (work_bytes < split_work_bytes(m, n, b)) return RLOBPCG_ERR_INVALID_ARG;
  const unsigned char* pp = (const unsigned char*)prep;
  unsigned char* wk = (unsigned char*)work;
  if (b <= 8) return split_gram_bp<8>(pp, m, n, W, b, ldw, AW, ldaw, G, ldg, wk, flags, err, mid, st);
  if (b <= 12) return split_gram_bp<12>(pp, m, n, W, b, ldw, AW, ldaw, G, ldg, wk, flags, err, mid, st);
  if (b <= 16) return split_gram_bp<16>(pp, m, n, W, b, ldw, AW, ldaw, G, ldg, wk, flags, err, mid, st);
  return split_gram_bp<24>(pp, m, n, W, b, ldw, AW, ldaw, G, ldg, wk, flags, err, mid, st);
}

}  // namespace rl
