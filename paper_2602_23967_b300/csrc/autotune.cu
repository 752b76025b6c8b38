// autotune.cu — pdhcg_autotune: picks the row layout and launch shape of the
// solve kernel by timing candidates on the device.
//
// Knobs:
//   * row layout (read at create): the SELL sort window sell_sigma, and the
//     row lengths above which a row gets a warp (long_row) or a CTA (huge_row);
//   * launch shape: for a single solve, the pipeline form against the
//     persistent multi-CTA kernel at several group sizes (group_blocks); for
//     a batched launch, the pool CTA width (256 or 128 threads) and the cap on
//     resident pool CTAs per SM.
// Search: coordinate descent from the defaults, launch shape first (no
// re-creation needed), then the layout with the best shape.  Each candidate
// runs kSteps PDHG steps (a warm-up solve, then a timed one) between two CUDA
// events on the handles' stream; the measure is device seconds per step.
// pick_fastest() keeps the defaults unless a candidate wins by more than 3 %.
// Choices are cached per shape class for the life of the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host_problem.h"

namespace pdhcg {

int cuda_fail(cudaError_t e, const char* where);

namespace {

constexpr int kSteps = 64;            // PDHG steps per timing (one check period)
constexpr double kMargin = 0.03;      // a candidate must beat the defaults by this much

struct Knobs {
  int32_t sigma = 0, long_row = 0, huge_row = 0, group_blocks = 0, pool_cap = 0, pipeline = 0, pool_threads = 0;
};

std::mutex g_mu;
std::map<std::string, pdhcg_tuning> g_cache;

int bucket_log2(double v) { return v < 1.0 ? 0 : int(std::floor(std::log2(v))); }

// Histogram signature of row lengths: shares (in tenths) of rows of length
// 1-4, 5-16, 17-64, 65-2047 and 2048 or more.
std::string row_signature(const pdhcg_csr* M) {
  if (!M || M->nrows <= 0) return "-";
  int64_t cnt[5] = {0, 0, 0, 0, 0};
  for (int32_t r = 0; r < M->nrows; ++r) {
    const int64_t l = M->rowptr[r + 1] - M->rowptr[r];
    cnt[l <= 4 ? 0 : l <= 16 ? 1 : l <= 64 ? 2 : l < 2048 ? 3 : 4]++;
  }
  std::string s;
  for (int64_t c : cnt) s += std::to_string(int(10.0 * double(c) / double(M->nrows) + 0.5)) + ".";
  return s;
}

// Shape class: precision, batch or single, inner solver class, size buckets
// and the row-length signatures of Q and A (taken from the first problem).
std::string shape_key(int count, const pdhcg_problem_data* pr, const pdhcg_params& prm) {
  const pdhcg_problem_data& p = pr[0];
  bool diag = true, box = false;
  if (p.Q)
    for (int32_t r = 0; r < p.Q->nrows && diag; ++r)
      for (int64_t k = p.Q->rowptr[r]; k < p.Q->rowptr[r + 1]; ++k)
        if (p.Q->col[k] != r && p.Q->val[k] != 0.0) {
          diag = false;
          break;
        }
  const int32_t n = p.A->ncols;
  for (int32_t j = 0; j < n && !box; ++j) box = std::isfinite(p.lv[j]) || std::isfinite(p.uv[j]);
  double mean_n = 0.0;
  for (int i = 0; i < count; ++i) mean_n += double(pr[i].A->ncols) / count;
  return std::to_string(prm.precision) + "|" + (count > 1 ? "batch" : "single") + "|" + std::to_string(prm.inner) +
         (diag ? "d" : "q") + (box ? "b" : "f") + "|n" + std::to_string(bucket_log2(mean_n)) + "|m" +
         std::to_string(bucket_log2(double(p.A->nrows))) + "|Q" + row_signature(p.Q) + "|A" +
         row_signature(p.A);
}

void apply(const Knobs& k, pdhcg_params* p) {
  p->sell_sigma = k.sigma;
  p->long_row = k.long_row;
  p->huge_row = k.huge_row;
  p->group_blocks = k.group_blocks;
  p->pool_ctas_per_sm = k.pool_cap;
  p->pipeline = k.pipeline;
  p->pool_threads = k.pool_threads;
}

// Device seconds per PDHG step of one configuration (<= 0: it failed).
double time_config(int count, const pdhcg_problem_data* pr, const pdhcg_params& base, const Knobs& k,
                   cudaStream_t s) {
  pdhcg_params p = base;
  apply(k, &p);
  p.max_iter = kSteps;
  p.eps_tol = 1e-300;  // no early stop: every candidate runs the same steps
  p.time_limit_s = 1e9;
  std::vector<pdhcg_t*> h(static_cast<size_t>(count), nullptr);
  int rc = count > 1 ? pdhcg_create_batch(count, pr, &p, s, h.data())
                     : pdhcg_create(pr[0].Q, pr[0].A, pr[0].c, pr[0].lc, pr[0].uc, pr[0].lv, pr[0].uv, &p, s,
                                    h.data());
  if (rc) return -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double sec = -1.0;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    std::vector<pdhcg_result> res(static_cast<size_t>(count));
    for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
      cudaEventRecord(e0, s);
      rc = count > 1 ? pdhcg_solve_batch(h.data(), count, res.data(), nullptr, nullptr)
                     : pdhcg_solve_dev(h[0], nullptr, nullptr, res.data(), nullptr, nullptr);
      cudaEventRecord(e1, s);
      if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
        sec = -1.0;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      int64_t steps = 0;
      for (const auto& r : res) steps = std::max<int64_t>(steps, r.iterations);
      sec = steps > 0 ? double(ms) * 1e-3 / double(steps) : -1.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (auto* q : h) pdhcg_destroy(q);
  return sec;
}

}  // namespace
}  // namespace pdhcg

using namespace pdhcg;

extern "C" int pdhcg_autotune(int count, const pdhcg_problem_data* problems, pdhcg_params* params,
                              void* cuda_stream, pdhcg_tuning* out) {
  if (count < 1 || !problems || !params || !out || !problems[0].A) {
    set_error("autotune: bad arguments");
    return PDHCG_E_INVALID;
  }
  int rc = check_params_c(params);
  if (rc) return rc;
  *out = pdhcg_tuning{};
  const std::string key = shape_key(count, problems, *params);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      out->from_cache = 1;
      out->candidates = 0;
      Knobs k{out->sell_sigma, out->long_row, out->huge_row, out->group_blocks, out->pool_ctas_per_sm,
              out->pipeline, out->pool_threads};
      apply(k, params);
      return PDHCG_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Knobs best;  // the defaults
  best.group_blocks = count > 1 ? 0 : params->group_blocks;
  int timed = 0;
  double t_default = -1.0;
  auto search = [&](const std::vector<Knobs>& cands) {
    std::vector<double> t(cands.size(), -1.0);
    for (size_t i = 0; i < cands.size(); ++i) {
      t[i] = time_config(count, problems, *params, cands[i], s);
      ++timed;
    }
    if (t_default < 0.0) t_default = t[0];
    const int b = pick_fastest(t, kMargin);
    if (b >= 0) best = cands[size_t(b)];
    return b >= 0 ? t[size_t(b)] : -1.0;
  };
  double t_best = -1.0;
  // 1. launch shape (candidate 0: the current best, i.e. the defaults)
  {
    std::vector<Knobs> c{best};
    if (count > 1) {
      Knobs k = best;
      k.pool_threads = 128;  // narrow CTAs, as many per SM as fit
      c.push_back(k);
      k = best;
      k.pool_cap = 1;
      c.push_back(k);
    } else {
      // the persistent multi-CTA kernel at several group sizes (the default
      // may be the pipeline form for a large problem)
      for (int g : {sms, 3 * sms / 2, 2 * sms}) {
        Knobs k = best;
        k.group_blocks = g;
        k.pipeline = -1;
        c.push_back(k);
      }
    }
    t_best = search(c);
  }
  // 2. row layout with that shape
  {
    std::vector<Knobs> c{best};
    for (int sg : {128, 8192}) {
      Knobs k = best;
      k.sigma = sg;
      c.push_back(k);
    }
    for (int lr : {32, 128}) {
      Knobs k = best;
      k.long_row = lr;
      c.push_back(k);
    }
    Knobs k = best;
    k.huge_row = 8192;
    c.push_back(k);
    const double t = search(c);
    if (t > 0.0) t_best = t;
  }
  if (!(t_best > 0.0)) {
    set_error("autotune: no candidate configuration ran");
    return PDHCG_E_CUDA;
  }
  out->sell_sigma = best.sigma;
  out->long_row = best.long_row;
  out->huge_row = best.huge_row;
  out->group_blocks = best.group_blocks;
  out->pool_ctas_per_sm = best.pool_cap;
  out->pipeline = best.pipeline;
  out->pool_threads = best.pool_threads;
  out->candidates = timed;
  out->from_cache = 0;
  out->seconds_per_step = t_best;
  out->default_seconds_per_step = t_default;
  apply(best, params);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = *out;
  return PDHCG_OK;
}
