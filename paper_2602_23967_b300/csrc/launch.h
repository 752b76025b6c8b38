// launch.h — typed launch entry points of the setup and solve kernels (one
// explicit instantiation per precision in kernels_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "pdhcg_internal.h"

namespace pdhcg {

template <class MatT, class VecT>
struct SetupArgs;

// CTA sizes: multi-CTA groups (one large instance) and pooled single-CTA
// solves.  Pool CTAs come in two widths (pdhcg_params.pool_threads): 256
// threads (the default; the group kernel's own code, two CTAs per SM), or 128
// threads compiled for four CTAs per SM, which runs more instances at once
// when their vectors fit a quarter of the SM's shared memory.
constexpr int kGroupBS = 256;
#ifndef PDHCG_POOL_BS
#define PDHCG_POOL_BS 128
#endif
constexpr int kPoolBS = PDHCG_POOL_BS;  // the narrow pool width
// Upper bound on resident pool CTAs per SM (0: as many as fit).
#ifndef PDHCG_POOL_MAX_PER_SM
#define PDHCG_POOL_MAX_PER_SM 0
#endif

struct KernelLimits {
  int max_coresident_group;  // CTAs of the solve kernel resident at once (SMs x occupancy)
  int max_coresident_setup;
};

template <class MatT, class VecT>
cudaError_t kernel_limits(KernelLimits* out);

// Setup of one instance on nblk co-resident CTAs (cooperative when nblk > 1).
template <class MatT, class VecT>
cudaError_t launch_setup(const SetupArgs<MatT, VecT>& a, int nblk, unsigned long long* bar,
                         double* part, int32_t* err, uint64_t timeout_ns, cudaStream_t s);

// Resident pool CTAs of `bs` threads (kPoolBS or kGroupBS) per SM when each
// keeps smem_vec_bytes of vectors on chip.
template <class MatT, class VecT>
int pool_blocks_per_sm(size_t smem_vec_bytes, int bs);

// Largest dynamic shared memory per pool CTA of `bs` threads (16-byte multiple)
// with which per_sm of them fit on one SM; 0 if the runtime cannot say.
template <class MatT, class VecT>
size_t pool_smem_for(int per_sm, int bs);

// Resident CTAs per SM of the group-size solve kernel (both variants) with
// smem_vec_bytes of dynamic shared memory per CTA: the bound of a cooperative
// launch that mixes multi-CTA groups with pool CTAs.
template <class MatT, class VecT>
int group_blocks_per_sm(size_t smem_vec_bytes);

// Solve launch; cooperative when plan.group_blocks > 0.
template <class MatT, class VecT>
cudaError_t launch_solve(const Inst<MatT, VecT>* d_insts, const LaunchPlan& plan, int grid,
                         cudaStream_t s);

// Pipeline form of one large instance (pipeline_kernel.cuh): the iteration as
// a CUDA graph of ordinary kernels with device-driven conditional nodes, grid
// CTAs each (the row partition of d_inst must be for grid CTAs).  state: a
// device PipeState (its tickets zeroed before each launch), part: kSlots * grid
// doubles.  On success *exec_out is the instantiated graph, launched once per
// solve after the state and descriptor are uploaded.
template <class MatT, class VecT>
cudaError_t pipeline_build(const Inst<MatT, VecT>* d_inst, int grid, int method, void* state, double* part,
                           cudaGraphExec_t* exec_out);
template <class MatT, class VecT>
int pipeline_blocks_per_sm();
constexpr size_t kPipeStateBytes = 1024;  // >= sizeof(PipeState), checked where it is defined
// The leading timer fields of PipeState (PDHCG_PIPE_TIMERS builds), as the host reads them.
struct PipeClockView {
  unsigned long long neg_first[12], ns_busy[12], count[12], t_last_end, ns_gap;
};

// Setup of count instances in one launch (one CTA per instance at a time).
template <class MatT, class VecT>
cudaError_t launch_setup_pool(const SetupArgs<MatT, VecT>* d_args, int count, int* next, int32_t* err,
                              uint64_t timeout_ns, cudaStream_t s);

}  // namespace pdhcg
