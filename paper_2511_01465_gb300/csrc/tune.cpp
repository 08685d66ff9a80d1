// tune.cpp -- the launch-shape autotuner's cache.
//
// Kernel families time a few candidate launch shapes on the caller's own
// workload the first time a (family, system, size bucket) key is seen while
// tuning is enabled, and store the fastest here.  With PITN_TUNE_CACHE set
// to a file path the cache is read from that file on first use and written
// back after every new entry (one "key a b" line per entry), so later
// processes start tuned.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "pitn.h"
#include "solver.h"

namespace pitn_host {

namespace {
std::mutex g_mu;
std::map<std::string, std::pair<int, int>> g_cache;
bool g_loaded = false;
bool g_enabled = false;

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = std::getenv("PITN_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char key[128];
    int a = 0, b = 0;
    while (std::fscanf(f, "%127s %d %d", key, &a, &b) == 3) g_cache[key] = {a, b};
    std::fclose(f);
}

void save_locked() {
    const char* path = std::getenv("PITN_TUNE_CACHE");
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto& kv : g_cache) std::fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}
}  // namespace

bool tune_enabled() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_enabled;
}

bool tune_lookup(const char* key, int* a, int* b) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    *a = it->second.first;
    *b = it->second.second;
    return true;
}

void tune_store(const char* key, int a, int b) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_cache[key] = {a, b};
    save_locked();
}

int tune_bucket(long long n) {
    int k = 0;
    while (n > 1) {
        n >>= 1;
        ++k;
    }
    return k;
}

}  // namespace pitn_host

extern "C" {

int pitn_tune_enable(int on) {
    std::lock_guard<std::mutex> lk(pitn_host::g_mu);
    pitn_host::g_enabled = on != 0;
    return PITN_OK;
}

int pitn_tune_clear(void) {
    std::lock_guard<std::mutex> lk(pitn_host::g_mu);
    pitn_host::g_cache.clear();
    pitn_host::g_loaded = true;  // an explicit clear also ignores the cache file
    return PITN_OK;
}

int pitn_tune_get(const char* key, int* a, int* b) {
    if (!key || !a || !b) return PITN_EINVAL;
    return pitn_host::tune_lookup(key, a, b) ? PITN_OK : PITN_EINVAL;
}

int pitn_tune_set(const char* key, int a, int b) {
    if (!key || !key[0] || std::strlen(key) >= 128) return PITN_EINVAL;
    // threads per CTA: whole warps; b = 0 only in a batch key (the per-IVP path)
    const bool batch = std::strncmp(key, "batch:", 6) == 0;
    if (a < 32 || a > 1024 || a % 32 != 0 || b < 0 || (b == 0 && !batch)) return PITN_EINVAL;
    pitn_host::tune_store(key, a, b);
    return PITN_OK;
}

}  // extern "C"
