// Fused Gram pass: the one product with A per LOBPCG iteration (Alg. 2 of arXiv 2602.16797 keeps
// A V and A X from earlier products and multiplies only the new block W), extended so that the
// same read of A also gives A^H (A W):
//     AW = A W            (m x b)     -- the new columns of A_T
//     G  = A^H AW         (n x b)     -- keeps G_T = A^H A T current, so the residual
//                                        A^H A_V - V Theta^2 needs no second pass over A.
// Mode RESID instead computes G = A^H Y for a given Y (the paper's direct residual A^H A_V).
//
// GB300 design: FP64 FMA throughput (not HBM) bounds this kernel: 4 m n b flop against 8 m n
// bytes, far above the FP64 ridge. So the kernel spends FP64 instructions on the 2 m n b FMAs
// only. One persistent CTA per SM owns a contiguous slab of rows (split-m). Row tiles (RT full
// rows) arrive in shared memory by TMA bulk copies (cp.async.bulk + mbarrier, double-buffered,
// no multicast). Phase 1: thread (r, s) forms partial dot products of row r with W over the
// columns k = s (mod g); the g partials are summed in a fixed order (no shuffle tree, g-1 adds
// per output). Phase 2: thread k accumulates G[k, :] += conj(A[r, k]) Y[r, :] over the tile
// into a shared-memory accumulator. Each CTA writes its n x b partial; a second kernel sums the
// partials in CTA order. Every result is deterministic.
#include <mutex>

#include "common.cuh"

namespace rl {

namespace {

constexpr int GR_NT = 256;

__device__ inline unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline void tma_bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Bounded wait on an mbarrier phase. Returns false when the bound ran out (the caller records
// an error and carries on, so that every thread still meets every barrier).
__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (int it = 0; it < (1 << 24); ++it) {
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

template <class T> __device__ inline T ldg_(const T* p) { return __ldg(p); }
template <> __device__ inline cd ldg_<cd>(const cd* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

enum { MODE_FUSED = 0, MODE_RESID = 1 };

// Phase 1 for N columns c0 .. c0+N-1 (N exact: no DFMA is issued for a column that does not
// exist; predicated-off FMAs would still occupy FP64 issue slots).
template <class T, int N>
__device__ __forceinline__ void phase1_chunk(const T* arow, int n, int g, int ps, const T* __restrict__ W,
                                             int64_t ldw, int c0, T* Ps, size_t pbase, int b) {
  T y[N];
#pragma unroll
  for (int cc = 0; cc < N; ++cc) y[cc] = zero_<T>();
  for (int k = ps; k < n; k += g) {
    const T a = arow[k];
    const T* wk = W + (int64_t)k * ldw + c0;
#pragma unroll
    for (int cc = 0; cc < N; ++cc) y[cc] = mad_(a, ldg_(wk + cc), y[cc]);
  }
#pragma unroll
  for (int cc = 0; cc < N; ++cc) Ps[(pbase + c0 + cc) * g + ps] = y[cc];
  (void)b;
}

// Phase 2 for N columns: G[k, c0 .. c0+N-1] += sum_r conj(A[r, k]) Y[r, c0 ..]
template <class T, int N>
__device__ __forceinline__ void phase2_chunk(const T* tile, int n, int k, int rows, const T* Ys, int b, int c0,
                                             T* Gacc) {
  T gk[N];
#pragma unroll
  for (int cc = 0; cc < N; ++cc) gk[cc] = Gacc[(size_t)k * b + c0 + cc];
  for (int r = 0; r < rows; ++r) {
    const T a = tile[(size_t)r * n + k];
    const T* yr = Ys + (size_t)r * b + c0;
#pragma unroll
    for (int cc = 0; cc < N; ++cc) gk[cc] = madc_(a, yr[cc], gk[cc]);
  }
#pragma unroll
  for (int cc = 0; cc < N; ++cc) Gacc[(size_t)k * b + c0 + cc] = gk[cc];
}

// CB: width of the full column chunks; CR = b mod CB, the width of the last chunk (both exact).
template <class T, int CB, int CR>
__global__ void __launch_bounds__(GR_NT, 1)
gram_kernel(const T* __restrict__ A, int64_t m, int n, int64_t lda, const T* __restrict__ W, int b,
            int64_t ldw, T* __restrict__ AW, int64_t ldaw, T* __restrict__ part, int64_t rows_per_cta,
            int RT, int use_tma, int mode, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int g = GR_NT / RT;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  size_t off = 128;
  T* tiles = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)2 * RT * n * sizeof(T);
  T* Gacc = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)n * b * sizeof(T);
  T* Ps = reinterpret_cast<T*>(smem_raw + off);
  off += (size_t)GR_NT * b * sizeof(T);
  T* Ys = reinterpret_cast<T*>(smem_raw + off);

  const int64_t row_begin = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t row_end = min(m, row_begin + rows_per_cta);
  const int ntile = row_end > row_begin ? (int)((row_end - row_begin + RT - 1) / RT) : 0;
  const int bfull = b - CR;  // columns covered by full chunks

  for (int i = tid; i < n * b; i += GR_NT) Gacc[i] = zero_<T>();
  if (tid == 0 && use_tma) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](int t) {  // thread 0 only
    const int64_t r0 = row_begin + (int64_t)t * RT;
    const int rows = (int)min((int64_t)RT, row_end - r0);
    const int buf = t & 1;
    T* dst = tiles + (size_t)buf * RT * n;
    const unsigned rbytes = (unsigned)(n * sizeof(T));
    mbar_expect_tx(&mbar[buf], rbytes * rows);
    for (int r = 0; r < rows; ++r) tma_bulk_g2s(dst + (size_t)r * n, A + (r0 + r) * lda, rbytes, &mbar[buf]);
  };
  if (use_tma && tid == 0) {
    if (ntile > 0) issue(0);
    if (ntile > 1) issue(1);
  }

  bool ok = true;
  const int pr = tid / g, ps = tid % g;  // phase-1 role: row pr, column phase ps
  for (int t = 0; t < ntile; ++t) {
    const int buf = t & 1;
    const int64_t r0 = row_begin + (int64_t)t * RT;
    const int rows = (int)min((int64_t)RT, row_end - r0);
    T* tile = tiles + (size_t)buf * RT * n;
    if (use_tma) {
      ok = mbar_wait(&mbar[buf], (unsigned)((t >> 1) & 1)) && ok;
    } else {
      for (int64_t i = tid; i < (int64_t)rows * n; i += GR_NT) tile[i] = A[(r0 + i / n) * lda + i % n];
      __syncthreads();
    }

    if (mode == MODE_FUSED) {
      // ---- phase 1: partial dot products of row pr with W over columns k = ps (mod g)
      if (pr < rows) {
        const T* arow = tile + (size_t)pr * n;
        const size_t pbase = (size_t)pr * b;
        for (int c0 = 0; c0 < bfull; c0 += CB) phase1_chunk<T, CB>(arow, n, g, ps, W, ldw, c0, Ps, pbase, b);
        if constexpr (CR > 0) phase1_chunk<T, CR>(arow, n, g, ps, W, ldw, bfull, Ps, pbase, b);
      }
      __syncthreads();
      // fixed-order sum of the g partials of each (row, column)
      for (int i = tid; i < rows * b; i += GR_NT) {
        const T* p = Ps + (size_t)i * g;
        T s = p[0];
        for (int q = 1; q < g; ++q) s = add_(s, p[q]);
        Ys[i] = s;
        AW[(r0 + i / b) * ldaw + (i % b)] = s;
      }
    } else {
      for (int i = tid; i < rows * b; i += GR_NT) Ys[i] = AW[(r0 + i / b) * ldaw + (i % b)];
    }
    __syncthreads();

    // ---- phase 2: G[k, :] += conj(A[r, k]) Y[r, :]
    for (int k = tid; k < n; k += GR_NT) {
      for (int c0 = 0; c0 < bfull; c0 += CB) phase2_chunk<T, CB>(tile, n, k, rows, Ys, b, c0, Gacc);
      if constexpr (CR > 0) phase2_chunk<T, CR>(tile, n, k, rows, Ys, b, bfull, Gacc);
    }
    __syncthreads();
    if (use_tma && tid == 0 && t + 2 < ntile) {
      fence_proxy_async();
      issue(t + 2);
    }
  }
  if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);

  T* mypart = part + (size_t)blockIdx.x * n * b;
  for (int i = tid; i < n * b; i += GR_NT) mypart[i] = Gacc[i];
}

// G[k, c] = sum over CTAs (in CTA order) of the partials
template <class T>
__global__ void gram_reduce_kernel(const T* __restrict__ part, int nparts, int n, int b, T* G, int64_t ldg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * b) return;
  T s = part[i];
  for (int p = 1; p < nparts; ++p) s = add_(s, part[(int64_t)p * n * b + i]);
  G[(i / b) * ldg + (i % b)] = s;
}

struct GramPlan {
  int grid = 0, RT = 0;
  int64_t rows_per_cta = 0;
  size_t smem = 0;
};

template <class T>
size_t gram_smem(int n, int b, int RT) {
  return 128 + (size_t)2 * RT * n * sizeof(T) + (size_t)n * b * sizeof(T) + (size_t)GR_NT * b * sizeof(T) +
         (size_t)RT * b * sizeof(T);
}

template <class T>
int gram_plan(int64_t m, int n, int b, GramPlan* gp) {
  const size_t cap = max_smem_optin();
  int RT = 256;
  while (RT > 1 && gram_smem<T>(n, b, RT) > cap) RT >>= 1;
  if (gram_smem<T>(n, b, RT) > cap) return RLOBPCG_ERR_UNSUPPORTED;
  // do not make tiles taller than the rows a CTA gets
  const int sms = num_sms();
  while (RT > 1 && (int64_t)RT * sms > m) RT >>= 1;
  gp->RT = RT;
  gp->smem = gram_smem<T>(n, b, RT);
  const int64_t tiles = (m + RT - 1) / RT;
  gp->grid = (int)imax<int64_t>(1, imin<int64_t>(sms, tiles));
  const int64_t tiles_per = (tiles + gp->grid - 1) / gp->grid;
  gp->rows_per_cta = tiles_per * RT;
  gp->grid = (int)imax<int64_t>(1, (m + gp->rows_per_cta - 1) / gp->rows_per_cta);
  return RLOBPCG_OK;
}

template <class T, int CB, int CR>
int launch_gram_cr(const GramPlan& gp, const T* A, int64_t m, int n, int64_t lda, const T* W, int b, int64_t ldw,
                   T* AW, int64_t ldaw, T* part, int use_tma, int mode, int* err, cudaStream_t st) {
  RL_TRY(allow_dynamic_smem(gram_kernel<T, CB, CR>, gp.smem));
  gram_kernel<T, CB, CR><<<gp.grid, GR_NT, gp.smem, st>>>(A, m, n, lda, W, b, ldw, AW, ldaw, part, gp.rows_per_cta,
                                                         gp.RT, use_tma, mode, err);
  RL_CHECK_LAUNCH();
  return RLOBPCG_OK;
}

// choose the instantiation whose remainder chunk is exactly b mod CB
template <class T>
int launch_gram_kernel(const GramPlan& gp, const T* A, int64_t m, int n, int64_t lda, const T* W, int b, int64_t ldw,
                       T* AW, int64_t ldaw, T* part, int use_tma, int mode, int* err, cudaStream_t st) {
  if constexpr (sizeof(T) == 16) {
    switch (b % 4) {
      case 0: return launch_gram_cr<T, 4, 0>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 1: return launch_gram_cr<T, 4, 1>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 2: return launch_gram_cr<T, 4, 2>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      default: return launch_gram_cr<T, 4, 3>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
    }
  } else {
    switch (b % 8) {
      case 0: return launch_gram_cr<T, 8, 0>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 1: return launch_gram_cr<T, 8, 1>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 2: return launch_gram_cr<T, 8, 2>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 3: return launch_gram_cr<T, 8, 3>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 4: return launch_gram_cr<T, 8, 4>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 5: return launch_gram_cr<T, 8, 5>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      case 6: return launch_gram_cr<T, 8, 6>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
      default: return launch_gram_cr<T, 8, 7>(gp, A, m, n, lda, W, b, ldw, AW, ldaw, part, use_tma, mode, err, st);
    }
  }
}

#define RL_TRY_GRAM(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

// Largest column group bc <= b whose accumulators fit on chip; the pass over A is repeated per
// group (FP64 arithmetic, not the extra reads of A, bounds the kernel).
template <class T>
int gram_group(int64_t m, int n, int b, GramPlan* gp) {
  for (int bc = b; bc >= 1; --bc)
    if (gram_plan<T>(m, n, bc, gp) == RLOBPCG_OK) return bc;
  return 0;
}

template <class T>
int gram_impl(const T* A, int64_t m, int n, int64_t lda, const T* W, int b, int64_t ldw, T* AW, int64_t ldaw,
              T* G, int64_t ldg, void* work, size_t work_bytes, int mode, int* err, cudaStream_t st) {
  GramPlan gp;
  const int bc = gram_group<T>(m, n, b, &gp);
  if (bc < 1) return RLOBPCG_ERR_UNSUPPORTED;
  const size_t need = (size_t)gp.grid * n * bc * sizeof(T);
  if (work_bytes < need) return RLOBPCG_ERR_INVALID_ARG;
  T* part = (T*)work;
  const int use_tma = ((uintptr_t)A % 16 == 0) && ((lda * (int64_t)sizeof(T)) % 16 == 0) &&
                      (((int64_t)n * (int64_t)sizeof(T)) % 16 == 0);
  for (int c0 = 0; c0 < b; c0 += bc) {
    const int bw = imin(bc, b - c0);
    GramPlan gq = gp;
    if (bw != bc) gram_plan<T>(m, n, bw, &gq);
    RL_TRY_GRAM(launch_gram_kernel<T>(gq, A, m, n, lda, W ? W + c0 : nullptr, bw, ldw, AW + c0, ldaw, part, use_tma,
                                      mode, err, st));
    const int64_t nb = (int64_t)n * bw;
    gram_reduce_kernel<T><<<(int)((nb + 255) / 256), 256, 0, st>>>(part, gq.grid, n, bw, G + c0, ldg);
    RL_CHECK_LAUNCH();
  }
  return RLOBPCG_OK;
}

}  // namespace

size_t gram_workspace_bytes(int64_t m, int64_t n, int b, int dtype) {
  GramPlan gp;
  const int bc = dtype == RLOBPCG_C128 ? gram_group<cd>(m, (int)n, b, &gp) : gram_group<double>(m, (int)n, b, &gp);
  if (bc < 1) return 0;
  return (size_t)gp.grid * n * bc * (dtype == RLOBPCG_C128 ? 16 : 8);
}

int gram_dispatch(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b, int64_t ldw,
                  void* AW, int64_t ldaw, void* G, int64_t ldg, void* work, size_t work_bytes, int resid_mode,
                  int* err, cudaStream_t st) {
  const int mode = resid_mode ? MODE_RESID : MODE_FUSED;
  if (dtype == RLOBPCG_C128)
    return gram_impl<cd>((const cd*)A, m, (int)n, lda, (const cd*)W, b, ldw, (cd*)AW, ldaw, (cd*)G, ldg, work,
                         work_bytes, mode, err, st);
  return gram_impl<double>((const double*)A, m, (int)n, lda, (const double*)W, b, ldw, (double*)AW, ldaw,
                           (double*)G, ldg, work, work_bytes, mode, err, st);
}

// kernel-level launch parameters, for the benchmark's roofline report
int gram_launch_info(int64_t m, int64_t n, int b, int dtype, int* grid, int* rt, size_t* smem, int* group) {
  GramPlan gp;
  const int bc = dtype == RLOBPCG_C128 ? gram_group<cd>(m, (int)n, b, &gp) : gram_group<double>(m, (int)n, b, &gp);
  if (bc < 1) return RLOBPCG_ERR_UNSUPPORTED;
  *grid = gp.grid; *rt = gp.RT; *smem = gp.smem; *group = bc;
  return RLOBPCG_OK;
}


// ------------------------------------------------------------------------------------------------
// Allocation-free entry point of the fused Gram pass.
//
// Some callers cannot let a library allocate device memory: a serving process that budgets all
// of HBM up front and admits work only into memory it already owns, or a real-time loop that
// must not call cudaMalloc/cudaFree because they synchronise the whole device and stall every
// other stream's work. rlobpcg_gram_noalloc serves them: its scratch (the per-SM partial
// sums and the device error word) is a file-scope device array of fixed size, so the call makes
// no allocation at all. The array lives as long as the library is loaded, on every GPU that uses
// it, and all calls share it.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocPartBytes = (size_t)16 << 20;  // room for the split-m partials: 16 MiB
constexpr size_t kNoallocHeadBytes = 256;                // the error word, padded to 256 bytes

static __device__ __align__(256) unsigned char g_gram_noalloc_scratch[kNoallocHeadBytes + kNoallocPartBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_base[64] = {};

// Device address of the static scratch on the current device, looked up once per device.
int noalloc_scratch(void** out) {
  int dev = 0;
  RL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RLOBPCG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_gram_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address", __FILE__, __LINE__);
      return RLOBPCG_ERR_CUDA;
    }
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return RLOBPCG_OK;
}

}  // namespace

}  // namespace rl

extern "C" int rlobpcg_gram_noalloc(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* W, int b,
                                    int64_t ldw, void* AW, int64_t ldaw, void* G, int64_t ldg, void* stream) {
  using namespace rl;
  if (!A || !W || !AW || !G || m < 1 || n < 1 || b < 1 || b > 64 || lda < n || ldw < b || ldaw < b || ldg < b ||
      (dtype != RLOBPCG_F64 && dtype != RLOBPCG_C128))
    return RLOBPCG_ERR_INVALID_ARG;
  const size_t need = gram_workspace_bytes(m, n, b, dtype);
  if (need == 0) {
    set_last_error("rlobpcg_gram_noalloc: n * b too large for on-chip accumulation", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  if (need > kNoallocPartBytes) {
    set_last_error("rlobpcg_gram_noalloc: this m, n, b needs more split-m scratch than its fixed 16 MiB "
                   "buffer holds; use rlobpcg_gram with caller-provided workspace", __FILE__, __LINE__);
    return RLOBPCG_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = (int*)base;
  void* part = (unsigned char*)base + kNoallocHeadBytes;
  // the partials are fully overwritten by every call; only the error word must start at zero
  RL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  rc = gram_dispatch(A, m, n, lda, dtype, W, b, ldw, AW, ldaw, G, ldg, part, kNoallocPartBytes, 0, err, st);
  if (rc) return rc;
  int herr = 0;
  RL_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RL_CUDA(cudaStreamSynchronize(st));
  return dev_err_status(herr);
}
