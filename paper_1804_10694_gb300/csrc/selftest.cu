// Self-test of the pipeline's bounded waits: one CTA initialises an mbarrier
// that expects one arrival and waits on it with the same bounded wait the
// gemm kernels use; nothing ever arrives, so the wait must give up after its
// limit, record kErrTimeout in the device error word and return.  The kernel
// neither faults nor hangs: it ends after the limit (2 s).
#include <cuda_runtime.h>

#include "ptx.cuh"
#include "runtime.h"

namespace gb {
namespace {

__global__ void wait_timeout_kernel(int* err, int* finished) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, err);   // no arrival ever comes
  __syncthreads();
  if (threadIdx.x == 0) *finished = ok ? 2 : 1;
}

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" gemm_status gemm_selftest_wait_timeout(void) {
  clear_error();
  int* err = nullptr;
  gemm_status st = device_err_word(&err);
  if (st != GEMM_OK) return st;
  int* finished = nullptr;
  cudaError_t e = cudaMalloc(&finished, sizeof(int));
  if (e != cudaSuccess) return fail(GEMM_ERR_ALLOC, "selftest flag");
  cudaMemset(finished, 0, sizeof(int));
  wait_timeout_kernel<<<1, 32>>>(err, finished);
  e = cudaDeviceSynchronize();
  int f = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&f, finished, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(finished);
  if (e != cudaSuccess) return cuda_fail(e, "selftest kernel");
  if (f != 1) return fail(GEMM_ERR_CUDA, "bounded wait did not report a timeout (flag %d)", f);
  // the kernel returned and the context is usable: report what the error word holds
  return gemm_device_error();
}
