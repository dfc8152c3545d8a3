// tune_cache.h -- autotune results kept across processes (see tune_cache.cpp).
#pragma once

#include <string>

namespace gbnll {

// Key of a tuned workload: the device (name, SM count), what was tuned and four integers
// that identify the workload (model, variant, weights, size class...).
std::string tune_cache_key(const char* device_name, int sm_count, const char* what, long long a, long long b,
                           long long c, long long d);
// The last stored result of `key` in the file named by GBNLL_TUNE_CACHE; false without one.
bool tune_cache_lookup(const std::string& key, int out[3]);
// Appends `key` and its result to that file (nothing without GBNLL_TUNE_CACHE).
void tune_cache_store(const std::string& key, const int v[3]);

}  // namespace gbnll
