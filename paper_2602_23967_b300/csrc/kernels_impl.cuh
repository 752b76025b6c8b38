// kernels_impl.cuh — launch wrappers, included once per precision.
#pragma once
#include "launch.h"
#include "setup_kernel.cuh"
#include "solve_kernel.cuh"

#include <algorithm>

namespace pdhcg {

template <class MatT, class VecT>
cudaError_t set_solve_attrs(size_t extra = 0) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // dynamic shared memory: the instance vectors of pool solves (group launches use none)
  size_t want = extra;
  const size_t static_part = 8192;  // group_reduce / row-engine shared arrays
  if (want + static_part > size_t(optin)) want = size_t(optin) - static_part;
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)solve_kernel<kGroupBS, MatT, VecT, false>,
                        (const void*)solve_kernel<kGroupBS, MatT, VecT, true>,
                        (const void*)solve_kernel<kPoolBS, MatT, VecT, false>,
                        (const void*)solve_kernel<kPoolBS, MatT, VecT, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(want));
  return e;
}

template <class MatT, class VecT>
int pool_blocks_per_sm(size_t smem_vec_bytes) {
  int nb = 0, nr = 0;
  if (set_solve_attrs<MatT, VecT>(smem_vec_bytes) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<kPoolBS, MatT, VecT, false>, kPoolBS,
                                                    smem_vec_bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, solve_kernel<kPoolBS, MatT, VecT, true>, kPoolBS,
                                                    smem_vec_bytes) != cudaSuccess)
    return 0;
  nb = std::min(nb, nr);
  if (PDHCG_POOL_MAX_PER_SM > 0) nb = std::min(nb, int(PDHCG_POOL_MAX_PER_SM));
  return nb;
}

template <class MatT, class VecT>
int group_blocks_per_sm(size_t smem_vec_bytes) {
  int nb = 0, nr = 0;
  if (set_solve_attrs<MatT, VecT>(smem_vec_bytes) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<kGroupBS, MatT, VecT, false>, kGroupBS,
                                                    smem_vec_bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, solve_kernel<kGroupBS, MatT, VecT, true>, kGroupBS,
                                                    smem_vec_bytes) != cudaSuccess)
    return 0;
  return std::min(nb, nr);
}

template <class MatT, class VecT>
cudaError_t kernel_limits(KernelLimits* out) {
  int dev = 0, sms = 0, nb = 0, nr = 0, ns = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = set_solve_attrs<MatT, VecT>();
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_kernel<kGroupBS, MatT, VecT, false>, kGroupBS, 0);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, solve_kernel<kGroupBS, MatT, VecT, true>, kGroupBS, 0);
  if (e != cudaSuccess) return e;
  nb = std::min(nb, nr);  // a cooperative launch of either variant must fit
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ns, setup_kernel<kGroupBS, MatT, VecT>, kGroupBS, 0);
  if (e != cudaSuccess) return e;
  out->max_coresident_group = sms * nb;
  out->max_coresident_setup = sms * ns;
  return cudaSuccess;
}

template <class MatT, class VecT>
cudaError_t launch_setup(const SetupArgs<MatT, VecT>& a, int nblk, unsigned long long* bar,
                         double* part, int32_t* err, uint64_t timeout_ns, cudaStream_t s) {
  SetupArgs<MatT, VecT> aa = a;
  if (nblk <= 1) {
    setup_kernel<kGroupBS, MatT, VecT><<<1, kGroupBS, 0, s>>>(aa, bar, part, err, timeout_ns);
    return cudaGetLastError();
  }
  void* args[] = {&aa, &bar, &part, &err, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void*)setup_kernel<kGroupBS, MatT, VecT>, dim3(nblk),
                                     dim3(kGroupBS), args, 0, s);
}

template <class MatT, class VecT>
cudaError_t launch_solve(const Inst<MatT, VecT>* d_insts, const LaunchPlan& plan, int grid,
                         cudaStream_t s) {
  LaunchPlan p = plan;
  const Inst<MatT, VecT>* di = d_insts;
  // dynamic shared memory: the vectors of pool instances (a cooperative launch
  // with pool CTAs beside its groups gives it to every CTA; groups ignore it)
  const size_t extra = size_t(plan.smem_vec_bytes);
  cudaError_t e = set_solve_attrs<MatT, VecT>(extra);
  if (e != cudaSuccess) return e;
  const size_t smem = extra;
  const bool r = plan.structured != 0;
  if (plan.group_blocks == 0) {
    if (r)
      solve_kernel<kPoolBS, MatT, VecT, true><<<grid, kPoolBS, smem, s>>>(di, p);
    else
      solve_kernel<kPoolBS, MatT, VecT, false><<<grid, kPoolBS, smem, s>>>(di, p);
    return cudaGetLastError();
  }
  void* args[] = {&di, &p};
  return cudaLaunchCooperativeKernel(r ? (const void*)solve_kernel<kGroupBS, MatT, VecT, true>
                                       : (const void*)solve_kernel<kGroupBS, MatT, VecT, false>,
                                     dim3(grid), dim3(kGroupBS), args, smem, s);
}

template <class MatT, class VecT>
cudaError_t launch_setup_pool(const SetupArgs<MatT, VecT>* d_args, int count, int* next, int32_t* err,
                              uint64_t timeout_ns, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, sms = 0, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, setup_pool_kernel<kGroupBS, MatT, VecT>, kGroupBS, 0);
  const int grid = std::max(1, std::min(count, std::max(nb, 1) * sms));
  setup_pool_kernel<kGroupBS, MatT, VecT><<<grid, kGroupBS, 0, s>>>(d_args, count, next, err, timeout_ns);
  return cudaGetLastError();
}

#define PDHCG_INSTANTIATE(MatT, VecT)                                                          \
  template cudaError_t kernel_limits<MatT, VecT>(KernelLimits*);                               \
  template cudaError_t launch_setup<MatT, VecT>(const SetupArgs<MatT, VecT>&, int,             \
                                                unsigned long long*, double*, int32_t*,        \
                                                uint64_t, cudaStream_t);                       \
  template int pool_blocks_per_sm<MatT, VecT>(size_t);                                          \
  template int group_blocks_per_sm<MatT, VecT>(size_t);                                         \
  template cudaError_t launch_setup_pool<MatT, VecT>(const SetupArgs<MatT, VecT>*, int, int*,   \
                                                     int32_t*, uint64_t, cudaStream_t);           \
  template cudaError_t launch_solve<MatT, VecT>(const Inst<MatT, VecT>*, const LaunchPlan&, int, \
                                                cudaStream_t);

}  // namespace pdhcg
