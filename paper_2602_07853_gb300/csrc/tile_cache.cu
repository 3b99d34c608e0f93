// Process-wide cache of autotuned launch shapes of the standalone FP32 HVP
// (host code only).  Key: tangent format (25-number compressed or 45-number
// packed) and floor(log2(active cell bricks)); value: the fastest shape and its
// mean milliseconds.  Text form, one entry per line: "format log2_bricks tile ms".
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "mpml_internal.cuh"

namespace mpml {
namespace {

struct Entry {
  int tile;
  float ms;
};

std::mutex g_mu;
std::map<std::pair<int, int>, Entry> g_cache;

int size_class(int64_t ncb) {
  int k = 0;
  while (ncb > 1) {
    ncb >>= 1;
    ++k;
  }
  return k;
}

int format_of(int compressed) { return compressed ? NQC : 45; }

}  // namespace

int tile_cache_lookup(int compressed, int64_t ncb) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find({format_of(compressed), size_class(ncb)});
  return it == g_cache.end() ? -1 : it->second.tile;
}

void tile_cache_store(int compressed, int64_t ncb, int tile, float ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[{format_of(compressed), size_class(ncb)}] = Entry{tile, ms};
}

void tile_cache_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}

int tile_cache_save(const char* path) {
  if (!path) return MPML_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return MPML_ERR_ARG;
  for (const auto& kv : g_cache)
    std::fprintf(f, "%d %d %d %.6g\n", kv.first.first, kv.first.second, kv.second.tile, (double)kv.second.ms);
  return std::fclose(f) == 0 ? MPML_OK : MPML_ERR_ARG;
}

int tile_cache_load(const char* path) {
  if (!path) return MPML_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return MPML_ERR_ARG;
  std::vector<std::pair<std::pair<int, int>, Entry>> got;
  char line[256];
  bool bad = false;
  while (std::fgets(line, sizeof line, f)) {
    int fmt, cls, tile, used = 0;
    double ms;
    // skip blank lines
    bool blank = true;
    for (const char* q = line; *q; ++q)
      if (*q != ' ' && *q != '\t' && *q != '\n' && *q != '\r') blank = false;
    if (blank) continue;
    if (std::sscanf(line, "%d %d %d %lf %n", &fmt, &cls, &tile, &ms, &used) != 4 || line[used] != '\0' ||
        (fmt != NQC && fmt != 45) || cls < 0 || cls > 62 || tile < 0 || tile >= HVP_TILES || !(ms >= 0.0)) {
      bad = true;
      break;
    }
    got.push_back({{fmt, cls}, Entry{tile, (float)ms}});
  }
  std::fclose(f);
  if (bad) return MPML_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto& e : got) g_cache[e.first] = e.second;
  return MPML_OK;
}

}  // namespace mpml
