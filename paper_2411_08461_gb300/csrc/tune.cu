// Tune cache of the dslash variants: process-wide map, optionally mirrored in the
// text file named by WCL_TUNE_CACHE (one line per configuration:
// "<variant> <block> <ms> <key>").  Entries are keyed by the device's name and
// SM count as well, so one file can serve several GPU types.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "context.cuh"

namespace wcl {

namespace {
std::mutex g_mu;
std::map<std::string, TuneChoice> g_cache;
bool g_loaded = false;

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "dev?";
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "/" + std::to_string(prop.multiProcessorCount);
}

void load_file() {
  g_loaded = true;
  const char* path = std::getenv("WCL_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    int v = 0, b = 0, n = 0;
    float ms = 0;
    if (std::sscanf(line, "%d %d %f %n", &v, &b, &ms, &n) != 3 || n <= 0) continue;
    std::string key = line + n;
    while (!key.empty() && (key.back() == '\n' || key.back() == '\r')) key.pop_back();
    if (v < V_THREAD || v > V_TMA_TILE || b <= 0 || b > 1024 || key.empty()) continue;
    g_cache[key] = TuneChoice{v, b};
  }
  std::fclose(f);
}
}  // namespace

bool tune_lookup(const std::string& key, TuneChoice* out) {
  const std::string k = device_tag() + " " + key;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_file();
  auto it = g_cache.find(k);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string& key, TuneChoice c, float ms) {
  const std::string k = device_tag() + " " + key;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_file();
  g_cache[k] = c;
  const char* path = std::getenv("WCL_TUNE_CACHE");
  if (!path || !*path) return;
  if (FILE* f = std::fopen(path, "a")) {
    std::fprintf(f, "%d %d %.5f %s\n", c.variant, c.block, ms, k.c_str());
    std::fclose(f);
  }
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
  g_loaded = true;  // do not reread the file either
}

}  // namespace wcl
