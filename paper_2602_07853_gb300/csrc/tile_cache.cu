// Process-wide cache of autotuned launch shapes (host code only).  Key: format
// and floor(log2(active cell bricks)); value: the fastest shape and its
// milliseconds.  Formats 25 / 45: the standalone FP32 HVP on the compressed /
// 45-number tangent (shapes 0 .. HVP_TILES-1); 125 / 145: the persistent solver
// on the same two tangents (shapes 0 .. MPML_PCG_SHAPES-1).  Text form, one
// entry per line: "format log2_bricks tile ms".
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

bool shape_ok(int fmt, int tile) {
  if (fmt == NQC || fmt == 45) return tile >= 0 && tile < HVP_TILES;
  if (fmt == 100 + NQC || fmt == 145) return tile >= 0 && tile < MPML_PCG_SHAPES;
  return false;
}

}  // namespace

int tile_cache_lookup_fmt(int fmt, int64_t ncb) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find({fmt, size_class(ncb)});
  return it == g_cache.end() ? -1 : it->second.tile;
}

void tile_cache_store_fmt(int fmt, int64_t ncb, int tile, float ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[{fmt, size_class(ncb)}] = Entry{tile, ms};
}

int tile_cache_lookup(int compressed, int64_t ncb) { return tile_cache_lookup_fmt(format_of(compressed), ncb); }

void tile_cache_store(int compressed, int64_t ncb, int tile, float ms) {
  tile_cache_store_fmt(format_of(compressed), ncb, tile, ms);
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
        !shape_ok(fmt, tile) || cls < 0 || cls > 62 || !(ms >= 0.0)) {
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
