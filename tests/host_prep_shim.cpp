// host_prep_shim.cpp — test-only C entry points over the library's host-side
// SELL-C-sigma packing (build_sell in paper_2602_23967_b300/csrc/host_prep.cpp),
// so that a CPU test can check the layout the kernels read.  Built by
// tests/test_host_prep_cpu.py with g++; not part of the library.
#include <cstring>
#include <vector>

#include "host_problem.h"

namespace {
pdhcg::SellHost g_sell;
std::vector<int32_t> g_rp[2], g_ci[2];
}  // namespace

extern "C" {

// Pack a row space of nrows rows from one or two CSR matrices (rp2 == NULL for
// one).  rp*: nrows + 1 row pointers; ci*: column indices.  Returns 0.
int shim_build_sell(int32_t nrows, const int32_t* rp1, const int32_t* ci1, const int32_t* rp2,
                    const int32_t* ci2) {
  const int nmat = rp2 ? 2 : 1;
  const int32_t* rps[2] = {rp1, rp2};
  const int32_t* cis[2] = {ci1, ci2};
  const std::vector<int32_t>* rp[2] = {nullptr, nullptr};
  const std::vector<int32_t>* ci[2] = {nullptr, nullptr};
  for (int k = 0; k < nmat; ++k) {
    g_rp[k].assign(rps[k], rps[k] + nrows + 1);
    g_ci[k].assign(cis[k], cis[k] + rps[k][nrows]);
    rp[k] = &g_rp[k];
    ci[k] = &g_ci[k];
  }
  pdhcg::build_sell(nrows, nmat, rp, ci, &g_sell);
  return 0;
}

// sizes[0..5]: nslices, longs, huges, columns of matrix 0, of matrix 1, nmat-1 slots used.
void shim_sizes(int64_t* sizes) {
  sizes[0] = g_sell.nslices;
  sizes[1] = int64_t(g_sell.longs.size());
  sizes[2] = int64_t(g_sell.huges.size());
  sizes[3] = int64_t(g_sell.col[0].size());
  sizes[4] = int64_t(g_sell.col[1].size());
  sizes[5] = int64_t(g_sell.ptr[1].size());
}

// Copy the layout out; buffers sized by shim_sizes (ptr*: nslices + 1).
void shim_copy(int32_t* perm, int32_t* longs, int32_t* huges, int64_t* ptr0, int64_t* ptr1, int32_t* col0,
               int32_t* col1) {
  std::memcpy(perm, g_sell.perm.data(), sizeof(int32_t) * g_sell.perm.size());
  std::memcpy(longs, g_sell.longs.data(), sizeof(int32_t) * g_sell.longs.size());
  std::memcpy(huges, g_sell.huges.data(), sizeof(int32_t) * g_sell.huges.size());
  std::memcpy(ptr0, g_sell.ptr[0].data(), sizeof(int64_t) * g_sell.ptr[0].size());
  std::memcpy(ptr1, g_sell.ptr[1].data(), sizeof(int64_t) * g_sell.ptr[1].size());
  std::memcpy(col0, g_sell.col[0].data(), sizeof(int32_t) * g_sell.col[0].size());
  std::memcpy(col1, g_sell.col[1].data(), sizeof(int32_t) * g_sell.col[1].size());
}

}  // extern "C"
