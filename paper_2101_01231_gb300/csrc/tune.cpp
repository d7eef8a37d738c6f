// The autotuner's process-wide cache of launch choices (see tune.h).
#include "tune.h"

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace ridg {
namespace {

std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_env_loaded = false;

bool load_locked(const char* path) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  while (std::getline(f, line)) {
    // "key value", the key may hold spaces: the value is the last field
    const size_t sp = line.find_last_of(' ');
    if (sp == std::string::npos || sp == 0) continue;
    char* end = nullptr;
    const long v = std::strtol(line.c_str() + sp + 1, &end, 10);
    if (end == line.c_str() + sp + 1) continue;
    g_cache[line.substr(0, sp)] = (int)v;
  }
  return true;
}

void ensure_env_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* p = std::getenv("RIDG_TUNE_CACHE");
  if (p && *p) load_locked(p);
}

}  // namespace

int tune_get(const std::string& key, int dflt) {
  std::lock_guard<std::mutex> lock(g_mu);
  ensure_env_locked();
  auto it = g_cache.find(key);
  return it == g_cache.end() ? dflt : it->second;
}

void tune_put(const std::string& key, int value) {
  std::lock_guard<std::mutex> lock(g_mu);
  ensure_env_locked();
  g_cache[key] = value;
}

bool tune_save(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  std::ofstream f(path, std::ios::trunc);
  if (!f) return false;
  for (const auto& kv : g_cache) f << kv.first << ' ' << kv.second << '\n';
  return (bool)f;
}

bool tune_load(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  ensure_env_locked();
  return load_locked(path);
}

}  // namespace ridg
