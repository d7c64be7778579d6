// Batched iterations of many small solves: the per-solve descriptor shared by the kernels
// (batch_kernels.cuh, in small.cu's translation unit) and the host engine (solver.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rl {
namespace batch {

constexpr int NT = 256;         // threads of every batched kernel
constexpr int GS = 16;          // tiles per group of the two-level reduction
constexpr int PR = 32;          // rows of W per precondition item
constexpr int QRC = 128;        // rows folded into the running R per Householder step
constexpr int UR = 64;          // rows per staging step of the coefficient update
constexpr int BMAX = 5;         // block size limit of the batched path (3b <= 15: the 16-column Jacobi)

struct Desc {
  const double* A;
  int64_t m, lda;
  int n, b;
  double* Tb;        // n x 3b row-major: [V W X]
  double* ATb;       // m x 3b: [A V  A W  A X]
  double* GTb;       // n x 3b: A^H A of the same columns
  const double* Ru;  // n x n row-major R^{-1} (upper triangle), FP64
  const double* Rl;  // n x n row-major R^{-H} (lower triangle), FP64
  double* Y;         // n x b, R^{-H} Rs
  double* Rs;        // n x b, residual columns scaled to unit norm (the preconditioner input)
  double* Res;       // n x b
  double* res_norm;  // b
  double* theta;     // c singular values of A_T (descending); the b smallest are the estimates
  double* K;         // c x 2b coefficients of the last Rayleigh-Ritz step (row-major)
  double* Gpart;     // ntiles x n x b
  double* Rpart;     // ntiles x 3b x 3b
  double* Ggrp;      // ngroups x n x b
  double* Rgrp;      // ngroups x 3b x 3b
  double* Rfin;      // 3b x 3b
  double* hist;      // rows t = 0 .. max_iter: [residual norms (b) | estimates (b)]
  int* cnt;          // [0] precondition blocks done, [1] groups done, [2 + g] tiles of group g done
  int* err;
  int* rr_info;
  int ntiles, trows, rt, ngroups, nrb;
  int iter, c, nx, pending, c_prev, done, stop_reason, matvecs;
  int max_iter, fixed, check_every, use_stag;
  double sigma11, tau;
};


// dynamic shared memory of the tile kernel: W^T and the G accumulator (nw doubles each, nw >= n b
// for every solve of the launch), the staging area (two stages of A rows, or the factor and tail
// scratch), and the stage's row products Y
inline size_t tile_smem_bytes(int nw, int abuf_elems, int rtmax) {
  return ((size_t)2 * nw + (size_t)abuf_elems + (size_t)rtmax * BMAX) * sizeof(double);
}

int abuf_need(int n, int b, int rt);
size_t bcgs2_pre_smem(int n, int b);
int prepare(size_t pre_smem, size_t tile_smem);
int tile_blocks_per_sm(size_t tile_smem, int* out);
int pre_launch(int phase, Desc* D, const int2* items, int nitems, int* qhead, int grid, size_t smem, cudaStream_t st);
int tile_launch(bool flush, Desc* D, const int2* items, int nitems, int* qhead, int grid, int nw, int abuf,
                size_t smem, cudaStream_t st);
int active_launch(const Desc* D, int count, int* out, cudaStream_t st);
template <class S>
int widen_launch(const S* in, int64_t cnt, double* out, cudaStream_t st);
int static_smem_bytes(size_t* pre, size_t* tile);

}  // namespace batch
}  // namespace rl
