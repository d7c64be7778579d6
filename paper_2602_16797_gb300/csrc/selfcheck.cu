// Health check of the bounded-wait path: a kernel whose wait cannot complete.
//
// Every device-side wait of the library (mbarrier phases in the tensor-core Gram kernels, the
// reflector flags of the dataflow QR) spins a bounded number of times and, when the bound runs
// out, records DEV_ERR_TIMEOUT in the launch's error word, releases what it holds and returns, so
// that a lost arrival turns into RLOBPCG_ERR_TIMEOUT on the host instead of a hung GPU.
// rlobpcg_check_bounded_wait exercises that path on purpose: the kernel below holds TMEM (as the
// Gram kernels do) and waits, with a caller-given bound, on an mbarrier that nothing arrives at
// (kind 0) or on a global flag that nothing sets (kind 1); nothing else is in flight.
#include "common.cuh"
#include "tc.cuh"

namespace rl {
namespace {

__global__ void __launch_bounds__(64) bounded_wait_kernel(int kind, int spins, const unsigned* flag, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);   // expects one arrival that never comes
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  bool ok = true;
  if (threadIdx.x == 32) {
    if (kind == 0) {
      ok = tc::mbar_wait_bounded(&bar, 0, spins);
    } else {
      ok = false;
      for (int it = 0; it < spins; ++it)
        if (*(volatile const unsigned*)flag != 0u) { ok = true; break; }
    }
    if (!ok) atomicOr(err, DEV_ERR_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(*(volatile uint32_t*)&tslot, 32);
  }
}

}  // namespace
}  // namespace rl

using namespace rl;

extern "C" int rlobpcg_check_bounded_wait(int kind, int spins, void* stream) {
  if ((kind != 0 && kind != 1) || spins < 1 || spins > (1 << 24)) return RLOBPCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* word = nullptr;   // [0] error word, [1] the flag nothing sets
  RL_CUDA(cudaMallocAsync((void**)&word, 2 * sizeof(int), st));
  RL_CUDA(cudaMemsetAsync(word, 0, 2 * sizeof(int), st));
  bounded_wait_kernel<<<1, 64, 0, st>>>(kind, spins, (const unsigned*)(word + 1), word);
  note_launch();
  const cudaError_t le = cudaGetLastError();
  int herr = 0;
  if (le == cudaSuccess) RL_CUDA(cudaMemcpyAsync(&herr, word, sizeof(int), cudaMemcpyDeviceToHost, st));
  RL_CUDA(cudaFreeAsync(word, st));
  RL_CUDA(cudaStreamSynchronize(st));
  if (le != cudaSuccess) {
    set_last_error(cudaGetErrorString(le), __FILE__, __LINE__);
    return RLOBPCG_ERR_CUDA;
  }
  if (herr & DEV_ERR_TIMEOUT) set_last_error("bounded device wait ran out (as intended by the check)", __FILE__, __LINE__);
  return dev_err_status(herr);
}
