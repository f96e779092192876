// Several independent problems solved concurrently: meshes of uneven size, each with its own
// material, boundary data, options and frequency list (one context each).  A pool of host
// workers takes the problems largest first (work ~ ne^2 x frequencies) and drives each through
// bem_solve_frequencies on its context's own stream, so the GPU runs the kernels of the small
// problems beside those of the large ones instead of one problem after another; within each
// problem all frequencies are batched and retired individually as before.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "bem_internal.cuh"

extern "C" int bem_solve_batch(bem_batch_item* items, int32_t n, int32_t max_workers) {
  if (!items || n < 1 || max_workers < 0) return BEM_ERR_INVALID_ARG;
  for (int32_t a = 0; a < n; ++a) {
    if (!items[a].ctx || !items[a].s || items[a].ns < 1) return BEM_ERR_INVALID_ARG;
    for (int32_t b = 0; b < a; ++b)
      if (items[a].ctx == items[b].ctx) return BEM_ERR_INVALID_ARG;  // one problem per context
    items[a].status = BEM_ERR_INVALID_ARG;
  }
  // largest problems first: they bound the makespan
  std::vector<int32_t> order(n);
  std::vector<double> work(n);
  for (int32_t a = 0; a < n; ++a) {
    order[a] = a;
    const double ne = (double)items[a].ctx->mesh.ne;
    work[a] = ne * ne * (double)items[a].ns;
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
  std::atomic<int32_t> next{0};
  auto worker = [&] {
    for (;;) {
      const int32_t k = next.fetch_add(1);
      if (k >= n) return;
      bem_batch_item& it = items[order[k]];
      it.status = bem_solve_frequencies(it.ctx, it.s, it.ns, it.x_out, it.stats);
    }
  };
  const int32_t nw = std::min<int32_t>(n, max_workers > 0 ? max_workers : n);
  std::vector<std::thread> pool;
  pool.reserve(nw);
  try {
    for (int32_t w = 0; w < nw; ++w) pool.emplace_back(worker);
  } catch (...) {
    // could not start every worker: the ones running (or this thread) finish the list
  }
  if (pool.empty()) worker();
  for (auto& t : pool) t.join();
  int rc = BEM_OK;
  for (int32_t a = 0; a < n; ++a) {
    const int s = items[a].status;
    if (s == BEM_OK) continue;
    if (rc == BEM_OK || (rc == BEM_ERR_NOT_CONVERGED && s != BEM_ERR_NOT_CONVERGED)) rc = s;
  }
  return rc;
}
