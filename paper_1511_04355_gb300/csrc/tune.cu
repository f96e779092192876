// Launch-shape tuning of the FP32 far-field operator (bem_autotune, bem_set_tuning,
// bem_load_tuning, bem_launch_shape).  The paper has no counterpart; the shape of the hot launch
// (frequencies per CTA, source tiles per CTA before the FP64 atomic add, grid waves) is chosen per
// mesh size and per number of frequencies in a launch from a table, which the autotuner fills by
// timing every candidate shape on the context's own mesh.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>

#include "bem_internal.cuh"

namespace bem {

namespace {

constexpr int kFts[] = {1, 4, 8, 12};  // 1 only for launches of at most 2 frequencies
constexpr int kTiles[] = {1, 2, 4};
constexpr int kWaves[] = {2, 4, 8};

void check_entry(const bem_tune_entry& e) {
  BEM_REQUIRE(e.ft == 1 || e.ft == 4 || e.ft == 8 || e.ft == 12, "tuning entry: ft must be 1, 4, 8 or 12");
  BEM_REQUIRE(e.tiles >= 1 && e.tiles <= 64, "tuning entry: tiles must be in [1, 64]");
  BEM_REQUIRE(e.waves >= 1 && e.waves <= 64, "tuning entry: waves must be in [1, 64]");
  BEM_REQUIRE(e.ne_max >= 1 && e.nfl_max >= 1, "tuning entry: ne_max and nfl_max must be >= 1");
}

// deterministic source vector for the timing runs (any non-zero values do)
__global__ void fill_kernel(cx<float>* x, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t h = (uint32_t)(t * 2654435761u) ^ (uint32_t)(t >> 7);
  x[t] = mk((float)(h & 0xffff) * 1.5e-5f - 0.5f, (float)(h >> 16) * 1.5e-5f - 0.5f);
}

}  // namespace

FarShape far32_shape(bem_ctx* ctx, int64_t nfl) {
  if (ctx->tune_forced) return ctx->tune_force;
  FarShape sh;
  const std::vector<bem_tune_entry>& t = ctx->tune;
  if (t.empty()) return sh;
  const int64_t ne = ctx->mesh.ne;
  // the mesh bucket: smallest ne_max >= ne, else the largest ne_max
  int64_t bucket = -1, largest = -1;
  for (const auto& e : t) {
    largest = std::max(largest, e.ne_max);
    if (e.ne_max >= ne && (bucket < 0 || e.ne_max < bucket)) bucket = e.ne_max;
  }
  if (bucket < 0) bucket = largest;
  // within it: smallest nfl_max >= nfl, else the largest nfl_max
  const bem_tune_entry* pick = nullptr;
  const bem_tune_entry* top = nullptr;
  for (const auto& e : t) {
    if (e.ne_max != bucket) continue;
    if (!top || e.nfl_max > top->nfl_max) top = &e;
    if (e.nfl_max >= nfl && (!pick || e.nfl_max < pick->nfl_max)) pick = &e;
  }
  if (!pick) pick = top;
  sh.ft = pick->ft;
  sh.tiles = pick->tiles;
  sh.waves = pick->waves;
  return sh;
}

}  // namespace bem

using namespace bem;

extern "C" {

int bem_set_tuning(bem_ctx* ctx, const bem_tune_entry* table, int32_t n) {
  return guarded_call(ctx, [&] {
    BEM_REQUIRE(n >= 0 && (n == 0 || table), "bad table");
    std::vector<bem_tune_entry> t(table, table + n);
    for (const auto& e : t) check_entry(e);
    ctx->tune = t;
  });
}

int bem_load_tuning(bem_ctx* ctx, const char* path) {
  return guarded_call(ctx, [&] {
    BEM_REQUIRE(path, "null path");
    std::ifstream in(path);
    BEM_REQUIRE(in.good(), std::string("cannot read tuning table ") + path);
    std::vector<bem_tune_entry> t;
    std::string line;
    int lineno = 0;
    while (std::getline(in, line)) {
      ++lineno;
      const size_t hash = line.find('#');
      if (hash != std::string::npos) line.resize(hash);
      std::istringstream ls(line);
      bem_tune_entry e{};
      long long ne_max = 0;
      if (!(ls >> ne_max)) continue;  // blank or comment line
      e.ne_max = ne_max;
      if (!(ls >> e.nfl_max >> e.ft >> e.tiles >> e.waves))
        throw Error(BEM_ERR_INVALID_ARG, std::string(path) + ":" + std::to_string(lineno) + ": need 5 fields");
      if (!(ls >> e.ms)) e.ms = 0.0;
      if (!(ls >> e.ms_fixed)) e.ms_fixed = 0.0;
      check_entry(e);
      t.push_back(e);
    }
    ctx->tune = t;
  });
}

int bem_launch_shape(bem_ctx* ctx, int64_t nfl, int32_t* ft, int32_t* tiles, int32_t* waves) {
  return guarded_call(ctx, [&] {
    BEM_REQUIRE(nfl >= 1, "nfl must be >= 1");
    const FarShape sh = far32_shape(ctx, nfl);
    if (ft) *ft = sh.ft;
    if (tiles) *tiles = sh.tiles;
    if (waves) *waves = sh.waves;
  });
}

int bem_autotune(bem_ctx* ctx, const double* s, int64_t ns, const int32_t* nfl, int32_t n_nfl,
                 bem_tune_entry* out) {
  return guarded_call(ctx, [&] {
    need_problem(ctx);
    BEM_REQUIRE(s && nfl && out && ns >= 1 && n_nfl >= 1, "bad arguments");
    for (int32_t j = 0; j < n_nfl; ++j) BEM_REQUIRE(nfl[j] >= 1 && nfl[j] <= ns, "nfl[j] must be in [1, ns]");
    std::vector<double> sh(2 * ns);
    copy_out(ctx, sh.data(), s, sizeof(double) * 2 * ns);
    prepare_frequencies(ctx, sh.data(), ns);
    const int64_t N = 3 * ctx->mesh.ne;
    DevBuf x, y;
    x.reserve(sizeof(cx<float>) * ns * N);
    y.reserve(sizeof(cx<float>) * ns * N);
    fill_kernel<<<grid_for(ns * N, 256), 256, 0, ctx->stream>>>(x.as<cx<float>>(), ns * N);
    BEM_LAUNCHED();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BEM_CUDA(cudaEventCreate(&e0));
    BEM_CUDA(cudaEventCreate(&e1));
    std::vector<bem_tune_entry> found;
    try {
      for (int32_t j = 0; j < n_nfl; ++j) {
        std::vector<int32_t> flist(nfl[j]);
        for (int32_t f = 0; f < nfl[j]; ++f) flist[f] = f;
        bem_tune_entry best{};
        best.ms = -1;
        for (int ft : kFts)
          for (int tiles : kTiles)
            for (int waves : kWaves) {
              if (ft == 1 && nfl[j] > 2) continue;
              ctx->tune_forced = true;
              ctx->tune_force.ft = ft;
              ctx->tune_force.tiles = tiles;
              ctx->tune_force.waves = waves;
              apply_operator32(ctx, x.as<cx<float>>(), y.as<cx<float>>(), BEM_APPLY_A, &flist);  // warm-up
              float tmin = 0;
              for (int rep = 0; rep < 2; ++rep) {
                BEM_CUDA(cudaEventRecord(e0, ctx->stream));
                apply_operator32(ctx, x.as<cx<float>>(), y.as<cx<float>>(), BEM_APPLY_A, &flist);
                BEM_CUDA(cudaEventRecord(e1, ctx->stream));
                BEM_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                BEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (rep == 0 || ms < tmin) tmin = ms;
              }
              if (ft == 12 && tiles == 2 && waves == 4) best.ms_fixed = tmin;
              if (best.ms < 0 || tmin < best.ms) {
                best.ne_max = ctx->mesh.ne;
                best.nfl_max = nfl[j];
                best.ft = ft;
                best.tiles = tiles;
                best.waves = waves;
                best.ms = tmin;
              }
            }
        found.push_back(best);
        out[j] = best;
      }
    } catch (...) {
      ctx->tune_forced = false;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    ctx->tune_forced = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // install: replace this mesh size's entries
    std::vector<bem_tune_entry> t;
    for (const auto& e : ctx->tune)
      if (e.ne_max != ctx->mesh.ne) t.push_back(e);
    t.insert(t.end(), found.begin(), found.end());
    ctx->tune = t;
  });
}

}  // extern "C"
