// Digit split of FP64 values for the tensor-core Gram pass (the Ozaki scheme of gram_tc.cu):
// a group of values with max |x| < 2^E is written as rint(x 2^(55-E)) in balanced base 128,
//     x ~= 2^(E+1) sum_{p=0}^{7} d_p 2^(-7(p+1)),   d_p integers in [-64, 64],
// each digit exact in bf16. Shared by gram_tc.cu (A, A W) and small.cu (W, at the end of the
// BCGS2 + Orth kernel that produces it).
#pragma once
#include <cstdint>

namespace rl {
namespace split {

constexpr int SL = 8;   // digits per FP64 value
constexpr int TK = 16;  // K depth of one MMA / one digit tile

__device__ __forceinline__ int group_exp(double amax) {
  int e = 0;
  frexp(amax, &e);   // amax = f 2^e with f in [0.5, 1), so every |x| <= amax is < 2^e
  return amax > 0 ? e : 0;
}

// x 2^k: one exact multiply by a power of two built from its bits (FP64 instructions are the
// scarce resource on GB300); scalbn only for k outside the normal exponent range
__device__ __forceinline__ double mul_pow2(double x, int k) {
  return (k >= -1022 && k <= 1023) ? x * __longlong_as_double((long long)(k + 1023) << 52) : scalbn(x, k);
}

// rint(x 2^(55-E)) (ties away from zero) for |x| < 2^E, from the bits of x with integer
// instructions only (the FP64 pipe is the scarce one on GB300)
__device__ __forceinline__ long long scaled_int(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  unsigned long long M = bits & 0xfffffffffffffull;
  int eb = 1;                     // x = M 2^(eb - 1075); subnormals keep eb = 1
  if (e) {
    M |= 1ull << 52;
    eb = e;
  }
  const int sh = eb - 1020 - E;   // x 2^(55-E) = M 2^sh, sh <= 2 since |x| < 2^E
  unsigned long long X = 0;
  if (sh >= 0) {
    X = M << sh;
  } else if (sh > -64) {
    const int r = -sh;
    X = (M + (1ull << (r - 1))) >> r;   // M + 2^62 < 2^63: no overflow
  }
  return (bits >> 63) ? -(long long)X : (long long)X;
}

// largest |x| of a warp's values, on the bit patterns (ordered like the values for |x|)
__device__ __forceinline__ unsigned long long warp_max_abs_bits(double x) {
  const unsigned long long k = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(k >> 32));
  const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(k >> 32) == hi ? (unsigned)k : 0u);
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ void split8(double x, int E, int (&d)[SL]) {
  long long V = scaled_int(x, E);
#pragma unroll
  for (int p = SL - 1; p > 0; --p) {
    const int r = (int)(V & 127);
    const int dd = r - ((r & 64) << 1);   // balanced remainder in [-64, 63]
    d[p] = dd;
    V = (V - dd) >> 7;                    // exact: V - dd is a multiple of 128
  }
  d[0] = (int)V;                          // |V| <= 64 here since |V| <= 2^55 at the start
}

__device__ __forceinline__ uint16_t bf16_of(int v) { return (uint16_t)(__float_as_uint((float)v) >> 16); }

// element (row, kk) of an R-row x 16 digit tile in tcgen05's no-swizzle K-major core-matrix order
__device__ __forceinline__ int core_off(int row, int kk, int R) {
  return (kk >> 3) * (R * 8) + (row >> 3) * 64 + (row & 7) * 8 + (kk & 7);
}

// Where the digits of W (n x b) go: Wsl[kb][N x 16 tile], N = 8 x BP, row q * BP + j of the tile
// holding digit q of W[kb * 16 + kk][j]; F[j] the exponent of column j. NKB = ceil(n / 16).
struct WDigits {
  uint16_t* Wsl = nullptr;
  int* F = nullptr;
  int64_t NKB = 0;
  int BP = 0;
};

// flags of split_gram
constexpr int SPLIT_RESID = 1;    // G = A^T Y for the given Y = AW (no first product)
constexpr int SPLIT_W_READY = 2;  // the digits of W are already in the work buffer
constexpr int SPLIT_FIRST_ONLY = 4;    // only the first product (A W and its digits)
constexpr int SPLIT_SECOND_ONLY = 8;   // only the second product, from the digits of A W in the work buffer
// SMs the second product leaves free for other streams (bits 16..23 of the flags)
constexpr int split_reserve_flag(int sms) { return (sms & 0xff) << 16; }

}  // namespace split
}  // namespace rl
