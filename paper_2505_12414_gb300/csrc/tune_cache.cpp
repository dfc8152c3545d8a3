// tune_cache.cpp -- autotune results kept across processes.  With GBNLL_TUNE_CACHE naming a
// file, nll_autotune and nll_batch_autotune look up their workload's key there before timing
// anything, and append what they measured otherwise.  The file is plain text, one result per
// line: "<key> <a> <b> <c>" (three integers whose meaning the caller defines); the last line of
// a key wins, and lines that do not parse are skipped, so a damaged file only costs a new
// measurement.
#include "tune_cache.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

namespace gbnll {
namespace {
std::mutex g_tune_mutex;

const char* cache_path()
{
    const char* p = getenv("GBNLL_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}
}  // namespace

bool tune_cache_lookup(const std::string& key, int out[3])
{
    const char* path = cache_path();
    if (!path || key.empty() || key.find(' ') != std::string::npos) return false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE* f = fopen(path, "r");
    if (!f) return false;
    bool found = false;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char k[400];
        int a, b, c;
        if (sscanf(line, "%399s %d %d %d", k, &a, &b, &c) == 4 && key == k) {
            out[0] = a;
            out[1] = b;
            out[2] = c;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void tune_cache_store(const std::string& key, const int v[3])
{
    const char* path = cache_path();
    if (!path || key.empty() || key.size() >= 400 || key.find(' ') != std::string::npos) return;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE* f = fopen(path, "a");
    if (!f) return;  // an unwritable cache only loses the result
    fprintf(f, "%s %d %d %d\n", key.c_str(), v[0], v[1], v[2]);
    fclose(f);
}

std::string tune_cache_key(const char* device_name, int sm_count, const char* what, long long a, long long b,
                           long long c, long long d)
{
    std::string name = device_name ? device_name : "device";
    for (char& ch : name)
        if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    char buf[400];
    snprintf(buf, sizeof buf, "%s|sm%d|%s|%lld|%lld|%lld|%lld", name.c_str(), sm_count, what, a, b, c, d);
    return buf;
}

}  // namespace gbnll
