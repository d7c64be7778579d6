// Split-bf16 Gram pass for complex128 A: the products of the Gram pass of Alg. 2 (arXiv
// 2602.16797),
//     AW = A W      (m x b)   and   G = A^H AW   (n x b),
// carried out by the real tensor-core pass of gram_tc.cu on a real view of the operands.
//
// A complex m x n matrix stored row-major (lda complex elements per row) is, read as doubles, the
// real m x 2n row-major matrix B with leading dimension 2 lda: B(i, 2j) = Re A(i, j) and
// B(i, 2j + 1) = Im A(i, j). So the split of A is the real split of B, and
//   * A W: each complex w = W(j, c) becomes the real 2 x 2 block  [ Re w   Im w ]
//                                                                 [ -Im w  Re w ]
//     at rows 2j, 2j+1 and columns 2c, 2c+1 of W' (2n x 2b). Then
//         (B W')(i, 2c)     = sum_j Re A Re w - Im A Im w = Re (A W)(i, c),
//         (B W')(i, 2c + 1) = sum_j Re A Im w + Im A Re w = Im (A W)(i, c),
//     i.e. B W' is A W itself in its interleaved storage (real leading dimension 2 ldaw).
//   * A^H AW: with Y = B W' (the real view of Z = A W), G' = B^T Y (2n x 2b) holds the four real
//     products of Re/Im A with Re/Im Z, and
//         Re G(j, c) = G'(2j, 2c) + G'(2j + 1, 2c + 1)   (Re A Re Z + Im A Im Z),
//         Im G(j, c) = G'(2j, 2c + 1) - G'(2j + 1, 2c)   (Re A Im Z - Im A Re Z).
// Every real product keeps the split's error bound (about 2^-55 of the product of the group
// maxima per term); the recombination adds one FP64 rounding per entry of G. The block width of
// the real pass is 2b, so b <= 12.
#include "common.cuh"
#include "split.cuh"

namespace rl {

size_t split_work_bytes(int64_t m, int64_t n, int b);
int split_gram(const void* prep, int64_t m, int64_t n, const double* W, int b, int64_t ldw, double* AW, int64_t ldaw,
               double* G, int64_t ldg, void* work, size_t work_bytes, int flags, int* err, cudaEvent_t mid,
               cudaStream_t st);

namespace {

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct CLayout {
  size_t wr, gr, real, total;
};

CLayout clayout(int64_t m, int64_t n, int b) {
  CLayout L;
  const size_t blk = al256((size_t)(2 * n) * (size_t)(2 * b) * sizeof(double));
  L.wr = 0;
  L.gr = blk;
  L.real = 2 * blk;
  L.total = L.real + split_work_bytes(m, 2 * n, 2 * b);
  return L;
}

// W (n x b complex, ldw) -> W' (2n x 2b real, leading dimension 2b): one thread per entry of W
__global__ void __launch_bounds__(256) cplx_w_kernel(const cd* __restrict__ W, int n, int b, int64_t ldw,
                                                     double* __restrict__ Wr) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * b) return;
  const int64_t j = t / b;
  const int c = (int)(t - j * b);
  const cd w = W[j * ldw + c];
  double* r0 = Wr + (2 * j) * (2 * b) + 2 * c;
  double* r1 = r0 + 2 * b;
  r0[0] = w.x;
  r0[1] = w.y;
  r1[0] = -w.y;
  r1[1] = w.x;
}

// G' (2n x 2b real, leading dimension 2b) -> G (n x b complex, ldg)
__global__ void __launch_bounds__(256) cplx_g_kernel(const double* __restrict__ Gr, int n, int b, cd* __restrict__ G,
                                                     int64_t ldg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * b) return;
  const int64_t j = t / b;
  const int c = (int)(t - j * b);
  const double* r0 = Gr + (2 * j) * (2 * b) + 2 * c;
  const double* r1 = r0 + 2 * b;
  G[j * ldg + c] = cd{r0[0] + r1[1], r0[1] - r1[0]};
}

unsigned blocks_of(int64_t count) { return (unsigned)((count + 255) / 256); }

}  // namespace

size_t split_work_bytes_c128(int64_t m, int64_t n, int b) {
  return (m < 1 || n < 1 || b < 1 || 2 * b > 24) ? 0 : clayout(m, n, b).total;
}

// prep: the real split of B (split_prepare of A read as doubles, m x 2n, leading dimension 2 lda).
// flags: split::SPLIT_RESID (G = A^H AW for the AW given), SPLIT_FIRST_ONLY / SPLIT_SECOND_ONLY and
// the reserved SMs of the real pass; W digits are always formed here.
int split_gram_c128(const void* prep, int64_t m, int64_t n, const cd* W, int b, int64_t ldw, cd* AW, int64_t ldaw,
                    cd* G, int64_t ldg, void* work, size_t work_bytes, int flags, int* err, cudaEvent_t mid,
                    cudaStream_t st) {
  const bool resid_mode = (flags & split::SPLIT_RESID) != 0;
  const bool first = (flags & split::SPLIT_SECOND_ONLY) == 0, second = (flags & split::SPLIT_FIRST_ONLY) == 0;
  if (!prep || !AW || !G || !work || m < 1 || n < 1 || b < 1 || 2 * b > 24 || ldaw < b || ldg < b ||
      (!resid_mode && (!W || ldw < b)))
    return RLOBPCG_ERR_INVALID_ARG;
  if (n > (int64_t)1 << 30 || (int64_t)n * b > ((int64_t)1 << 31) - 256) return RLOBPCG_ERR_UNSUPPORTED;
  const CLayout L = clayout(m, n, b);
  if (work_bytes < L.total) return RLOBPCG_ERR_INVALID_ARG;
  unsigned char* wk = (unsigned char*)work;
  double* Wr = (double*)(wk + L.wr);
  double* Gr = (double*)(wk + L.gr);
  if (!resid_mode && first) {
    cplx_w_kernel<<<blocks_of(n * b), 256, 0, st>>>(W, (int)n, b, ldw, Wr);
    RL_CHECK_LAUNCH();
  }
  const int pass_flags =
      flags & (split::SPLIT_RESID | split::SPLIT_FIRST_ONLY | split::SPLIT_SECOND_ONLY | split::split_reserve_flag(255));
  RL_TRY(split_gram(prep, m, 2 * n, Wr, 2 * b, 2 * b, (double*)AW, 2 * ldaw, Gr, 2 * b, wk + L.real,
                    work_bytes - L.real, pass_flags, err, mid, st));
  if (second) {
    cplx_g_kernel<<<blocks_of(n * b), 256, 0, st>>>(Gr, (int)n, b, G, ldg);
    RL_CHECK_LAUNCH();
  }
  return RLOBPCG_OK;
}

}  // namespace rl
