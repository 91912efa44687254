// Autotuner of the generic kernel's launch shape.
//
// Candidates: threads in {128, 256} x points per thread R in {4, 8, 16}, each
// with the split-K the wave model prefers and its halved/doubled neighbours.
// Each candidate is timed with CUDA events on the plan's own device buffers
// (the kernel's speed does not depend on the atom values).  The winner is
// cached in a JSON-lines file keyed by path, S layout, size buckets, number
// of species and GPU, so later plans of the same shape skip the timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "launch.h"
#include "tuner.h"

namespace scatter {

namespace {

std::string cache_key(const scatter_plan_s* p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, p->device);
  char buf[512];
  const int nb = (int)std::lround(std::log2((double)std::max<int64_t>(p->n_slots, 1)) * 2);
  const int mb = (int)std::lround(std::log2((double)std::max<int64_t>(p->n_s, 1)) * 2);
  const int n2 = p->s_kind == SCATTER_S_GRID ? (int)p->n_axis[2] : 0;
  snprintf(buf, sizeof(buf), "generic|kind%d|n2_%d|N%d|M%d|sp%d|%s|sm%d", (int)p->s_kind, n2, nb, mb,
           p->n_species, prop.name, p->n_sm);
  for (char* c = buf; *c; ++c)
    if (*c == '"') *c = '\'';
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, Tiling* t) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  const std::string pat = "\"key\": \"" + key + "\"";
  while (fgets(line, sizeof(line), f)) {
    if (!strstr(line, pat.c_str())) continue;
    int th = 0, r = 0, k = 0;
    const char* a = strstr(line, "\"threads\":");
    const char* b = strstr(line, "\"R\":");
    const char* c = strstr(line, "\"split_k\":");
    if (a && b && c && sscanf(a, "\"threads\": %d", &th) == 1 && sscanf(b, "\"R\": %d", &r) == 1 &&
        sscanf(c, "\"split_k\": %d", &k) == 1) {
      Tiling cand;
      cand.threads = th;
      cand.R = r;
      cand.split_k = k;
      const char* d = strstr(line, "\"atom_k\":");  // absent in older caches: S-parallel
      int ak = 0;
      if (d && sscanf(d, "\"atom_k\": %d", &ak) == 1 && ak >= 0 && ak <= 16) cand.atom_k = ak;
      if (generic_tiling_supported(cand) && k >= 1 && k <= 256) {
        *t = cand;
        found = true;
      }
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const Tiling& t, double ms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"threads\": %d, \"R\": %d, \"split_k\": %d, \"atom_k\": %d, \"ms\": %.4f}\n",
          key.c_str(), t.threads, t.R, t.split_k, t.atom_k, ms);
  fclose(f);
}

// Split-K minimising waves x (work per CTA + fixed cost) for a shape.
int best_split(const scatter_plan_s* p, const Tiling& shape) {
  const int64_t tiles = generic_num_tiles(p, shape);
  const int bps = std::max(1, generic_blocks_per_sm(p, shape));
  const double cap = (double)p->n_sm * bps;
  const double n = (double)std::max<int64_t>(p->n_slots, 1);
  double best = 1e300;
  int best_k = 1;
  for (int k = 1; k <= 64; ++k) {
    if (k > 1 && n / k < 256) break;
    const double waves = std::ceil((double)tiles * k / cap);
    const double cost = waves * (n / k + 512.0) + (k > 1 ? 0.02 * k * (double)p->n_s / cap : 0.0);
    if (cost < best * 0.995) {
      best = cost;
      best_k = k;
    }
  }
  return best_k;
}

double time_tiling(scatter_plan_s* p, const Tiling& t, int reps) {
  if (apply_tiling(p, t) != SCATTER_OK) return 1e30;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  if (launch_generic(p, p->d.amp, nullptr, nullptr) != SCATTER_OK) best = -1;  // warm-up
  for (int i = 0; i < reps && best >= 0; ++i) {
    cudaEventRecord(e0, nullptr);
    launch_generic(p, p->d.amp, nullptr, nullptr);
    cudaEventRecord(e1, nullptr);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      best = -1;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || best < 0) return 1e30;
  return best;
}

}  // namespace

Tiling heuristic_tiling(const scatter_plan_s* p) {
  Tiling t;
  t.threads = 256;
  t.R = 8;
  // lists carry three S components per point (24 registers at R = 8): four
  // points per thread measured ~7 % faster there, single plans and batches
  if (p->s_kind == SCATTER_S_LIST || (p->s_kind == SCATTER_S_GRID && p->n_axis[2] < 8)) t.R = 4;
  t.split_k = best_split(p, t);
  // short S lists: parallelise over the atoms instead (atompar.cu)
  if (atompar_preferred(p, t)) t.atom_k = atompar_choose_k(p);
  return t;
}

scatter_status autotune_generic(scatter_plan_s* p, const char* cache_path) {
  if (p->n_s == 0) return SCATTER_OK;
  const std::string key = cache_key(p);
  Tiling t;
  if (cache_lookup(cache_path, key, &t)) {
    if (log_enabled()) fprintf(stderr, "[scatter] autotune cache hit %s\n", key.c_str());
    return apply_tiling(p, t);
  }
  const Tiling start = p->tiling;
  std::vector<Tiling> cands;
  auto add = [&](Tiling c) {
    if (!generic_tiling_supported(c) || c.split_k < 1) return;
    for (const Tiling& o : cands)
      if (o.threads == c.threads && o.R == c.R && o.split_k == c.split_k && o.atom_k == c.atom_k) return;
    cands.push_back(c);
  };
  add(start);
  for (int th : {128, 256})
    for (int r : {4, 8, 16}) {
      Tiling c;
      c.threads = th;
      c.R = r;
      c.split_k = best_split(p, c);
      add(c);
      Tiling lo = c, hi = c;
      lo.split_k = std::max(1, c.split_k / 2);
      hi.split_k = c.split_k * 2;
      if ((double)p->n_slots / hi.split_k >= 256) add(hi);
      add(lo);
    }
  if (atompar_applicable(p))
    for (int K : {1, 2, 4, 8, 16}) {
      Tiling c;
      c.split_k = 1;
      c.atom_k = K;
      add(c);
    }
  double best_ms = 1e30;
  Tiling best = start;
  const double first = time_tiling(p, start, 1);
  // large problems: a single timed launch per candidate keeps tuning short
  const int reps = first > 50.0 ? 1 : 2;
  for (size_t i = 0; i < cands.size(); ++i) {
    const double ms = i == 0 ? first : time_tiling(p, cands[i], reps);
    if (log_enabled())
      fprintf(stderr, "[scatter] autotune threads=%d R=%d split=%d atom_k=%d: %.3f ms\n", cands[i].threads,
              cands[i].R, cands[i].split_k, cands[i].atom_k, ms);
    if (ms < best_ms) {
      best_ms = ms;
      best = cands[i];
    }
    if (first > 2000.0) break;  // seconds per launch: keep the heuristic
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "autotune");
  cache_store(cache_path, key, best, best_ms);
  return apply_tiling(p, best);
}

scatter_status autotune_batch(scatter_plan_s* p, const char* cache_path) {
  if (p->n_s == 0 || p->n_slots == 0) return SCATTER_OK;
  std::string key = cache_key(p);
  key.replace(0, 7, "batch");
  char extra[64];
  snprintf(extra, sizeof(extra), "|B%d", p->batch);
  key += extra;
  Tiling t;
  if (cache_lookup(cache_path, key, &t) && batch_blocks_per_sm(t.R, t.threads) > 0) {
    p->tiling = t;
    return prepare_batch(p);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 1e30;
  Tiling best = p->tiling;
  for (int th : {128, 256})
    for (int r : {4, 8, 16}) {
      Tiling c;
      c.threads = th;
      c.R = r;
      c.split_k = 1;
      p->tiling = c;
      if (prepare_batch(p) != SCATTER_OK) continue;
      enqueue_batch_kernels(p, p->d.amp, nullptr, nullptr);  // warm-up
      cudaEventRecord(e0, nullptr);
      enqueue_batch_kernels(p, p->d.amp, nullptr, nullptr);
      cudaEventRecord(e1, nullptr);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (log_enabled()) fprintf(stderr, "[scatter] autotune batch threads=%d R=%d: %.3f ms\n", th, r, ms);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "autotune batch");
  cache_store(cache_path, key, best, best_ms);
  p->tiling = best;
  return prepare_batch(p);
}

}  // namespace scatter
