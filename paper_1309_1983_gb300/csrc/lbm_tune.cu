// lbm_tune.cu - launch-shape autotuning for single lattices, and the text
// cache shared with the batch tuner (lbm_batch_capi.cu).
//
// A candidate is timed on the handle's bound stream with CUDA events over
// whole lbm_step calls, after warm-up steps; the fastest is applied. The
// cache is a text file of "key<TAB>a<TAB>b<TAB>ms" lines keyed by GPU name,
// SM count and problem; a hit applies the stored shape without timing, and a
// miss rewrites the file (temporary file + rename) with the new line added.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tune.h"

namespace lbm {

std::string device_key(int device) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown";
  std::string name(p.name);
  for (char &c : name)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return name + "/sm" + std::to_string(p.multiProcessorCount);
}

bool tune_cache_lookup(const char *path, const std::string &key, int *a, int *b, float *ms) {
  if (!path) return false;
  FILE *fh = std::fopen(path, "r");
  if (!fh) return false;
  char line[1024];
  bool hit = false;
  while (std::fgets(line, sizeof line, fh)) {
    char *tab = std::strchr(line, '\t');
    if (!tab || (size_t)(tab - line) != key.size() || key.compare(0, key.size(), line, key.size()))
      continue;
    int va, vb;
    float vm;
    if (std::sscanf(tab + 1, "%d\t%d\t%f", &va, &vb, &vm) == 3) {
      *a = va;
      *b = vb;
      *ms = vm;
      hit = true;  // the last line for a key wins
    }
  }
  std::fclose(fh);
  return hit;
}

int tune_cache_store(const char *path, const std::string &key, int a, int b, float ms) {
  if (!path) return 0;
  std::string old;
  if (FILE *fh = std::fopen(path, "r")) {
    char line[1024];
    while (std::fgets(line, sizeof line, fh)) {
      const char *tab = std::strchr(line, '\t');
      if (tab && (size_t)(tab - line) == key.size() && !key.compare(0, key.size(), line, key.size()))
        continue;  // replaced below
      old += line;
    }
    std::fclose(fh);
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE *fh = std::fopen(tmp.c_str(), "w");
  if (!fh) return -1;
  std::fputs(old.c_str(), fh);
  std::fprintf(fh, "%s\t%d\t%d\t%.6f\n", key.c_str(), a, b, ms);
  const bool ok = std::fclose(fh) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return -1;
  }
  return 0;
}

}  // namespace lbm

// ---- single lattices ----------------------------------------------------------

int lbm_autotune(lbm_t *h, const char *cache_path, int steps, int *bx_out, int *by_out,
                 float *ms_out) {
  if (!h) return lbm::set_error(LBM_EINVAL, "NULL handle");
  if (!h->bound) return lbm::set_error(LBM_EUNBOUND, "handle not bound");
  if (steps < 1 || steps > 100000) return lbm::set_error(LBM_EINVAL, "steps in [1, 100000]");
  const bool pair =
      h->kernel == LBM_KERNEL_PAIR || h->kernel == LBM_KERNEL_X2 || h->kernel == LBM_KERNEL_X4;
  char geo[160];
  std::snprintf(geo, sizeof geo, "lattice/%dx%dx%d/flags%u/kernel%d/walls%d", h->nx, h->ny,
                h->nz, h->flags, h->kernel, h->wall_mode);
  const std::string key = lbm::device_key(h->device) + "/" + geo;
  int a = 0, b = 0;
  float best_ms = 0.f;
  if (lbm::tune_cache_lookup(cache_path, key, &a, &b, &best_ms)) {
    const int rc = pair ? lbm_set_pair_block(h, a, b) : lbm_set_block(h, a, b);
    if (rc == LBM_OK) {
      if (bx_out) *bx_out = a;
      if (by_out) *by_out = b;
      if (ms_out) *ms_out = best_ms;
      return LBM_OK;
    }
  }
  // x-dominant shapes (Sec. 6): 32..256 threads along x (no wider than the
  // rounded-up row), 1..8 rows, 64..256 threads per block
  const int width = pair ? (h->nx + 1) / 2 : h->nx;
  const int xmax = ((width + 31) / 32) * 32;
  std::vector<std::pair<int, int>> cand;
  for (int x = 32; x <= 256; x *= 2) {
    if (x > (xmax < 32 ? 32 : xmax)) continue;
    for (int y = 1; y <= 8; y *= 2)
      if (x * y >= 64 && x * y <= 256) cand.push_back({x, y});
  }
  if (cand.empty()) cand.push_back({32, 2});
  int best_a = 0, best_b = 0;
  best_ms = 0.f;
  for (auto &c : cand) {
    int rc = pair ? lbm_set_pair_block(h, c.first, c.second) : lbm_set_block(h, c.first, c.second);
    if (rc) return rc;
    float ms = 0.f;
    rc = lbm::time_calls(h->stream, 1, [&]() { return lbm_step(h, steps); }, &ms);
    if (rc) return rc;
    ms /= steps;
    if (!best_a || ms < best_ms) {
      best_a = c.first;
      best_b = c.second;
      best_ms = ms;
    }
  }
  const int rc = pair ? lbm_set_pair_block(h, best_a, best_b) : lbm_set_block(h, best_a, best_b);
  if (rc) return rc;
  if (lbm::tune_cache_store(cache_path, key, best_a, best_b, best_ms))
    return lbm::set_error(LBM_EINVAL, "autotune cache not writable");
  if (bx_out) *bx_out = best_a;
  if (by_out) *by_out = best_b;
  if (ms_out) *ms_out = best_ms;
  return LBM_OK;
}
