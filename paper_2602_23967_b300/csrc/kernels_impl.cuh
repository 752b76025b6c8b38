// kernels_impl.cuh — launch wrappers, included once per precision.
#pragma once
#include "launch.h"
#include "pipeline_kernel.cuh"
#include "setup_kernel.cuh"
#include "solve_kernel.cuh"

#include <algorithm>
#include <mutex>

namespace pdhcg {

// Kernel attributes (dynamic shared-memory limit, carveout hint) belong to the
// function and the process; every reader or writer of them holds this lock.
inline std::mutex& attr_mutex() {
  static std::mutex m;
  return m;
}

// Sets the dynamic shared-memory limit of the six solve kernels and their
// carveout hint to the largest shared-memory share, so that occupancy queries
// report what a launch can get; a launch then narrows the hint of the kernel it
// issues (launch_solve).  The caller holds attr_mutex().
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
                        (const void*)solve_kernel<kGroupBS, MatT, VecT, false, true>,
                        (const void*)solve_kernel<kPoolBS, MatT, VecT, false>,
                        (const void*)solve_kernel<kPoolBS, MatT, VecT, true>,
                        (const void*)solve_kernel<kPoolBS, MatT, VecT, false, true>})
    if (e == cudaSuccess) {
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(want));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    }
  return e;
}

// The three pool variants (plain, structured, closed form) of one width.
template <class MatT, class VecT>
void pool_kernels(int bs, const void* (&f)[3]) {
  if (bs == kGroupBS) {
    f[0] = (const void*)solve_kernel<kGroupBS, MatT, VecT, false>;
    f[1] = (const void*)solve_kernel<kGroupBS, MatT, VecT, true>;
    f[2] = (const void*)solve_kernel<kGroupBS, MatT, VecT, false, true>;
  } else {
    f[0] = (const void*)solve_kernel<kPoolBS, MatT, VecT, false>;
    f[1] = (const void*)solve_kernel<kPoolBS, MatT, VecT, true>;
    f[2] = (const void*)solve_kernel<kPoolBS, MatT, VecT, false, true>;
  }
}

template <class MatT, class VecT>
int pool_blocks_per_sm(size_t smem_vec_bytes, int bs) {
  std::lock_guard<std::mutex> lock(attr_mutex());
  if (set_solve_attrs<MatT, VecT>(smem_vec_bytes) != cudaSuccess) return 0;
  const void* f[3];
  pool_kernels<MatT, VecT>(bs, f);
  int nb = 1 << 30;
  for (const void* k : f) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, bs, smem_vec_bytes) != cudaSuccess) return 0;
    nb = std::min(nb, b);
  }
  if (PDHCG_POOL_MAX_PER_SM > 0) nb = std::min(nb, int(PDHCG_POOL_MAX_PER_SM));
  return nb;
}

// Shared-memory carveout hint of kernel k: just what per_sm resident CTAs with
// smem bytes of dynamic shared memory each need; the rest of the SM's
// L1/shared storage stays L1, which caches the matrix streams and gathers.
// The hint belongs to the function, and one function serves pool launches
// (vectors in shared memory) and group launches (almost none), so every launch
// sets it right before it is issued (launch_solve, under attr_mutex()).
inline void set_carveout(const void* k, size_t smem, int per_sm) {
  int dev = 0, max_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess || max_sm <= 0) return;
  const size_t need = size_t(std::max(per_sm, 1)) * (smem + fa.sharedSizeBytes + 1024);
  const int pct = int(std::min<size_t>(100, (need * 100 + size_t(max_sm) - 1) / size_t(max_sm)));
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <class MatT, class VecT>
size_t pool_smem_for(int per_sm, int bs) {
  std::lock_guard<std::mutex> lock(attr_mutex());
  if (set_solve_attrs<MatT, VecT>(~size_t(0) >> 1) != cudaSuccess) return 0;  // the opt-in maximum
  const void* f[3];
  pool_kernels<MatT, VecT>(bs, f);
  size_t best = ~size_t(0);
  for (const void* k : f) {
    size_t b = 0;
    if (cudaOccupancyAvailableDynamicSMemPerBlock(&b, k, std::max(per_sm, 1), bs) != cudaSuccess) return 0;
    best = std::min(best, b);
  }
  return best & ~size_t(15);
}

template <class MatT, class VecT>
int group_blocks_per_sm(size_t smem_vec_bytes) {
  int nb = 0, nr = 0;
  std::lock_guard<std::mutex> lock(attr_mutex());
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
  std::lock_guard<std::mutex> lock(attr_mutex());
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
  const size_t smem = size_t(plan.smem_vec_bytes);
  std::lock_guard<std::mutex> lock(attr_mutex());  // set the attributes and launch as one
  cudaError_t e = set_solve_attrs<MatT, VecT>(smem);
  if (e != cudaSuccess) return e;
  const bool r = plan.structured != 0;
  const bool coop = plan.group_blocks != 0;
  const int bs = coop || plan.pool_bs == kGroupBS ? kGroupBS : kPoolBS;
  const void* fn;
  if (bs == kGroupBS)
    fn = r ? (const void*)solve_kernel<kGroupBS, MatT, VecT, true>
           : (!coop && plan.diag_only) ? (const void*)solve_kernel<kGroupBS, MatT, VecT, false, true>
                                       : (const void*)solve_kernel<kGroupBS, MatT, VecT, false>;
  else
    fn = r ? (const void*)solve_kernel<kPoolBS, MatT, VecT, true>
           : plan.diag_only ? (const void*)solve_kernel<kPoolBS, MatT, VecT, false, true>
                            : (const void*)solve_kernel<kPoolBS, MatT, VecT, false>;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the CTAs per SM this grid needs resident (all of them, for a cooperative launch)
  set_carveout(fn, smem, (grid + std::max(sms, 1) - 1) / std::max(sms, 1));
  void* args[] = {&di, &p};
  if (coop) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kGroupBS), args, smem, s);
  return cudaLaunchKernel(fn, dim3(grid), dim3(bs), args, smem, s);
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

// ---- the pipeline graph of one large instance (pipeline_kernel.cuh) ----
namespace {
struct GraphBuilder {
  cudaError_t err = cudaSuccess;
  cudaGraphNode_t kernel(cudaGraph_t g, cudaGraphNode_t dep, const void* fn, int grid, void* args) {
    cudaGraphNode_t n = nullptr;
    if (err != cudaSuccess) return n;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3(unsigned(grid));
    kp.blockDim = dim3(kPipeBS);
    kp.sharedMemBytes = 0;
    void* params[] = {args};
    kp.kernelParams = params;
    err = cudaGraphAddKernelNode(&n, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
    return n;
  }
  // A conditional node (IF or WHILE) after dep; *body receives its body graph.
  cudaGraphNode_t cond(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType t,
                       cudaGraph_t* body) {
    cudaGraphNode_t n = nullptr;
    if (err != cudaSuccess) return n;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = t;
    np.conditional.size = 1;
    err = cudaGraphAddNode(&n, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &np);
    if (err == cudaSuccess) *body = np.conditional.phGraph_out[0];
    return n;
  }
  cudaGraphConditionalHandle handle(cudaGraph_t g, unsigned dflt) {
    cudaGraphConditionalHandle h{};
    if (err == cudaSuccess) err = cudaGraphConditionalHandleCreate(&h, g, dflt, cudaGraphCondAssignDefault);
    return h;
  }
};
}  // namespace

template <class MatT, class VecT>
cudaError_t pipeline_build(const Inst<MatT, VecT>* d_inst, int grid, int method, void* state, double* part,
                           cudaGraphExec_t* exec_out) {
  *exec_out = nullptr;
  cudaGraph_t root = nullptr;
  cudaError_t e = cudaGraphCreate(&root, 0);
  if (e != cudaSuccess) return e;
  GraphBuilder B;
  PipeArgs a{};
  a.inst = d_inst;
  a.ps = static_cast<PipeState*>(state);
  a.part = part;
  // conditional nodes first (a handle is made in the graph that holds its
  // node), so that every kernel node gets the complete set of handles
  cudaGraph_t body = nullptr, inner = nullptr, chk = nullptr, rst = nullptr, out = nullptr;
  a.h.outer = B.handle(root, 1u);
  const cudaGraphNode_t c_outer = B.cond(root, nullptr, a.h.outer, cudaGraphCondTypeWhile, &body);
  cudaGraphNode_t c_inner = nullptr, c_check = nullptr, c_rst = nullptr, c_out = nullptr;
  if (method != PDHCG_INNER_DIAG) {
    a.h.inner = B.handle(body, 0u);
    c_inner = B.cond(body, nullptr, a.h.inner, cudaGraphCondTypeWhile, &inner);
  }
  a.h.check = B.handle(body, 0u);
  c_check = B.cond(body, nullptr, a.h.check, cudaGraphCondTypeIf, &chk);
  a.h.restart = B.handle(chk, 0u);
  c_rst = B.cond(chk, nullptr, a.h.restart, cudaGraphCondTypeIf, &rst);
  a.h.out = B.handle(chk, 0u);
  c_out = B.cond(chk, nullptr, a.h.out, cudaGraphCondTypeIf, &out);
  // kernels, each after the node before it
  auto dep = [&](cudaGraph_t g, cudaGraphNode_t from, cudaGraphNode_t to) {
    if (B.err == cudaSuccess && from && to) B.err = cudaGraphAddDependencies(g, &from, &to, nullptr, 1);
  };
  const cudaGraphNode_t k_init = B.kernel(root, nullptr, (const void*)pipe_init<MatT, VecT>, grid, &a);
  dep(root, k_init, c_outer);
  const cudaGraphNode_t k_p1 = B.kernel(body, nullptr, (const void*)pipe_phase1<MatT, VecT>, grid, &a);
  const cudaGraphNode_t k_xbar = B.kernel(body, nullptr, (const void*)pipe_xbar<MatT, VecT>, grid, &a);
  const cudaGraphNode_t k_p2 = B.kernel(body, nullptr, (const void*)pipe_phase2<MatT, VecT>, grid, &a);
  if (c_inner) {
    dep(body, k_p1, c_inner);
    dep(body, c_inner, k_xbar);
    const bool cg = method == PDHCG_INNER_CG;
    const cudaGraphNode_t i1 =
        B.kernel(inner, nullptr, cg ? (const void*)pipe_cg_a<MatT, VecT> : (const void*)pipe_bb_b<MatT, VecT>, grid, &a);
    const cudaGraphNode_t i2 =
        B.kernel(inner, nullptr, cg ? (const void*)pipe_cg_b<MatT, VecT> : (const void*)pipe_bb_a<MatT, VecT>, grid, &a);
    dep(inner, i1, i2);
  } else {
    dep(body, k_p1, k_xbar);
  }
  dep(body, k_xbar, k_p2);
  dep(body, k_p2, c_check);
  const cudaGraphNode_t k_chk = B.kernel(chk, nullptr, (const void*)pipe_check<MatT, VecT>, grid, &a);
  dep(chk, k_chk, c_rst);
  dep(chk, c_rst, c_out);
  B.kernel(rst, nullptr, (const void*)pipe_restart<MatT, VecT>, grid, &a);
  const cudaGraphNode_t k_rays = B.kernel(out, nullptr, (const void*)pipe_rays<MatT, VecT>, grid, &a);
  const cudaGraphNode_t k_write = B.kernel(out, nullptr, (const void*)pipe_write<MatT, VecT>, grid, &a);
  dep(out, k_rays, k_write);
  if (B.err == cudaSuccess) B.err = cudaGraphInstantiate(exec_out, root, 0);
  cudaGraphDestroy(root);
  if (B.err != cudaSuccess) *exec_out = nullptr;
  return B.err;
}

// Resident CTAs per SM of the pipeline's row kernels (the smallest of them).
template <class MatT, class VecT>
int pipeline_blocks_per_sm() {
  int lo = 1 << 30;
  for (const void* f : {(const void*)pipe_phase1<MatT, VecT>, (const void*)pipe_phase2<MatT, VecT>,
                        (const void*)pipe_bb_a<MatT, VecT>, (const void*)pipe_cg_a<MatT, VecT>,
                        (const void*)pipe_check<MatT, VecT>}) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kPipeBS, 0) != cudaSuccess) return 0;
    lo = std::min(lo, nb);
  }
  return lo;
}

#define PDHCG_INSTANTIATE(MatT, VecT)                                                          \
  template cudaError_t kernel_limits<MatT, VecT>(KernelLimits*);                               \
  template cudaError_t launch_setup<MatT, VecT>(const SetupArgs<MatT, VecT>&, int,             \
                                                unsigned long long*, double*, int32_t*,        \
                                                uint64_t, cudaStream_t);                       \
  template int pool_blocks_per_sm<MatT, VecT>(size_t, int);                                     \
  template size_t pool_smem_for<MatT, VecT>(int, int);                                          \
  template int group_blocks_per_sm<MatT, VecT>(size_t);                                         \
  template cudaError_t launch_setup_pool<MatT, VecT>(const SetupArgs<MatT, VecT>*, int, int*,   \
                                                     int32_t*, uint64_t, cudaStream_t);           \
  template cudaError_t launch_solve<MatT, VecT>(const Inst<MatT, VecT>*, const LaunchPlan&, int, \
                                                cudaStream_t);                                   \
  template cudaError_t pipeline_build<MatT, VecT>(const Inst<MatT, VecT>*, int, int, void*, double*, \
                                                  cudaGraphExec_t*);                              \
  template int pipeline_blocks_per_sm<MatT, VecT>();

}  // namespace pdhcg
