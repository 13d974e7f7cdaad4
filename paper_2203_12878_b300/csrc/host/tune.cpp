// Tuning cache (see tune.h).  File format, one entry per line:
//   <signature> <granularity> <radix_items> <path> <specialized> <milliseconds>
#include "tune.h"

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace drf {
namespace {

std::mutex g_mu;
std::map<std::string, PlanConfig> g_cache;
bool g_loaded = false;

const char *cache_path()
{
    const char *p = std::getenv("DRF_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const char *path = cache_path();
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string key, extra;
        PlanConfig c;
        double ms;
        if ((in >> key >> c.granularity >> c.radix_items >> c.path >> c.jit >> ms) && !(in >> extra)) g_cache[key] = c;
    }
}

}  // namespace

bool tune_lookup(const std::string &key, PlanConfig &out)
{
    std::lock_guard<std::mutex> g(g_mu);
    load_locked();
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    out = it->second;
    return true;
}

void tune_store(const std::string &key, const PlanConfig &cfg, double ms)
{
    std::lock_guard<std::mutex> g(g_mu);
    load_locked();
    g_cache[key] = cfg;
    const char *path = cache_path();
    if (!path) return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %u %u %u %u %.4f\n", key.c_str(), cfg.granularity, cfg.radix_items, cfg.path, cfg.jit, ms);
        std::fclose(f);
    }
}

}  // namespace drf
