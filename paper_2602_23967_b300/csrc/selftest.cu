// selftest.cu — makes the solver's bounded device waits run out, on purpose and
// harmlessly, so that tests can check that a wait which never completes ends
// in an error status the host reads, with the context still usable.
//
// Two waits of the solve kernel are exercised with its own code:
//   * the group barrier inside group_reduce() (device_common.cuh), for a group
//     of two CTAs where CTA 1 returns at once and never arrives;
//   * spin_geq() on a flag that nothing sets (the form of a queue wait).
// Both stop after timeout_ns of device time.  No trap, fault or unbounded loop.
#include <cuda_runtime.h>

#include <string>

#include "device_common.cuh"
#include "host_problem.h"

namespace pdhcg {

int cuda_fail(cudaError_t e, const char* where);

template <int BS>
__global__ void __launch_bounds__(BS) bounded_wait_kernel(unsigned long long* bar, double* part, int32_t* err,
                                                          int32_t* err2, const unsigned long long* flag,
                                                          uint64_t timeout_ns, unsigned long long* out) {
  __shared__ double sm_warp[2 * (BS / 32) * kSlots];
  __shared__ double sm_tot[2 * kSlots];
  __shared__ int sm_flag;
  if (blockIdx.x == 1) return;  // the other member of the group never arrives
  Group<BS> g;
  g.nblk = 2;
  g.rank = 0;
  g.bar32 = reinterpret_cast<unsigned*>(bar);
  g.part = part;
  g.sm_warp = sm_warp;
  g.sm_tot = sm_tot;
  g.sm_flag = &sm_flag;
  g.err = err;
  g.timeout_ns = timeout_ns;
  g.failed = false;
  g.epoch = 0;
  if (threadIdx.x == 0) sm_flag = 0;
  __syncthreads();
  const uint64_t t0 = globaltimer_ns();
  double v[1] = {1.0};
  const bool passed = group_reduce<BS, 1>(g, v, 0u);
  const uint64_t t1 = globaltimer_ns();
  if (threadIdx.x == 0) {
    const bool got = spin_geq(flag, 1ull, timeout_ns, err2);
    const uint64_t t2 = globaltimer_ns();
    out[0] = passed ? 1ull : 0ull;
    out[1] = got ? 1ull : 0ull;
    out[2] = t1 - t0;
    out[3] = t2 - t1;
  }
}

}  // namespace pdhcg

using namespace pdhcg;

extern "C" int pdhcg_selftest_bounded_wait(int32_t timeout_us, double* waited_seconds) {
  if (timeout_us < 1 || timeout_us > 10000000) {
    set_error("selftest_bounded_wait: timeout_us must be in [1, 1e7]");
    return PDHCG_E_INVALID;
  }
  constexpr int BS = 128;
  const size_t bar_bytes = kBarBytes, part_bytes = sizeof(double) * 2 * kSlots * 2;
  const size_t words = 4 + 4 + 2;  // out[4], flag + pad, err, err2 (8-byte words)
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, bar_bytes + part_bytes + words * 8);
  if (e != cudaSuccess) return cuda_fail(e, "selftest_bounded_wait: cudaMalloc");
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(buf);
  double* part = reinterpret_cast<double*>(buf + bar_bytes);
  unsigned long long* out = reinterpret_cast<unsigned long long*>(buf + bar_bytes + part_bytes);
  unsigned long long* flag = out + 4;
  int32_t* err = reinterpret_cast<int32_t*>(out + 8);
  int32_t* err2 = reinterpret_cast<int32_t*>(out + 9);
  unsigned long long h[4] = {0, 0, 0, 0};
  e = cudaMemset(buf, 0, bar_bytes + part_bytes + words * 8);
  if (e == cudaSuccess) {
    bounded_wait_kernel<BS><<<2, BS>>>(bar, part, err, err2, flag, uint64_t(timeout_us) * 1000ull, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
  int32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "selftest_bounded_wait");
  if (waited_seconds) *waited_seconds = double(h[2] + h[3]) * 1e-9;
  if (h[0] != 0 || h[1] != 0 || herr != 1) {
    set_error("selftest_bounded_wait: a wait on a flag that nothing sets did not report giving up");
    return PDHCG_E_CUDA;
  }
  set_error("selftest_bounded_wait: both bounded waits gave up after the limit, as designed");
  return PDHCG_E_DEVICE_TIMEOUT;
}
