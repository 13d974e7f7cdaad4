// Tuning cache (see tune.h).  File format, one entry per line:
//   <signature> <granularity> <radix_items> <path> <specialized> <radix_bits> <milliseconds>
// (lines without the digit width, from earlier files, read as width 0)
#include "tune.h"

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <stdexcept>
#include <vector>

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
        std::vector<std::string> tok;
        std::string t;
        while (in >> t) tok.push_back(t);
        if (tok.size() != 6 && tok.size() != 7) continue;
        try {
            PlanConfig c;
            c.granularity = (uint32_t)std::stoul(tok[1]);
            c.radix_items = (uint32_t)std::stoul(tok[2]);
            c.path = (uint32_t)std::stoul(tok[3]);
            c.jit = (uint32_t)std::stoul(tok[4]);
            if (tok.size() == 7) c.radix_bits = (uint32_t)std::stoul(tok[5]);
            g_cache[tok[0]] = c;
        } catch (const std::exception &) {
        }
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
        std::fprintf(f, "%s %u %u %u %u %u %.4f\n", key.c_str(), cfg.granularity, cfg.radix_items, cfg.path, cfg.jit,
                     cfg.radix_bits, ms);
        std::fclose(f);
    }
}

}  // namespace drf
