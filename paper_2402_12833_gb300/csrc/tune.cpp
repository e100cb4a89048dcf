// Launch-shape table of the autotuner (host code, no CUDA calls).
//
// The launchers ask this table for their grid shapes before falling back to
// the fixed rules (stream_blocks, spmm_blocks, gram_chunks, the narrow
// Jacobi switch).  mg_autotune fills it by timing candidate shapes on a
// hierarchy (api.cu); the table can be written to and read from a small JSON
// file tagged with the device name and SM count, so that later processes
// skip the timing.  A shape is keyed by (tunable, arithmetic, grid points,
// problems in the batch, columns): the same grid in another precision or
// with another column count is tuned on its own.
#include <atomic>
#include <map>
#include <mutex>
#include <stdio.h>
#include <string.h>
#include <string>
#include <tuple>
#include <vector>

#include "tune.h"

namespace mpcg {
namespace tune {

namespace {

using Key = std::tuple<int, int, long long, int, int>;
std::mutex g_mu;
std::map<Key, int> g_table;
std::atomic<int> g_size{0};

const char* const kNames[kNumTunables] = {"stream_blocks", "spmm_blocks", "gram_chunks", "jacobi_narrow"};

int fn_of(const char* name) {
  for (int i = 0; i < kNumTunables; ++i)
    if (strcmp(name, kNames[i]) == 0) return i;
  return -1;
}

}  // namespace

int lookup(int fn, int kind, long long npts, int nb, int C, int dflt) {
  if (g_size.load(std::memory_order_acquire) == 0) return dflt;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(Key(fn, kind, npts, nb, C));
  return it == g_table.end() ? dflt : it->second;
}

bool find(int fn, int kind, long long npts, int nb, int C, int* value) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(Key(fn, kind, npts, nb, C));
  if (it == g_table.end()) return false;
  *value = it->second;
  return true;
}

void set(int fn, int kind, long long npts, int nb, int C, int value) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[Key(fn, kind, npts, nb, C)] = value;
  g_size.store((int)g_table.size(), std::memory_order_release);
}

void erase(int fn, int kind, long long npts, int nb, int C) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.erase(Key(fn, kind, npts, nb, C));
  g_size.store((int)g_table.size(), std::memory_order_release);
}

void clear() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
  g_size.store(0, std::memory_order_release);
}

int size() { return g_size.load(std::memory_order_acquire); }

// {"format": "mpcg-autotune-1", "device": "...", "sm_count": N, "entries": [
//   {"fn": "stream_blocks", "kind": -1, "npts": P, "nb": B, "C": C, "value": V}, ...]}
bool save(const char* path, const char* device, int sm_count) {
  std::vector<std::pair<Key, int>> rows;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    rows.assign(g_table.begin(), g_table.end());
  }
  FILE* f = fopen(path, "w");
  if (!f) return false;
  std::string dev;
  for (const char* c = device; *c; ++c)
    if (*c != '"' && *c != '\\') dev += *c;
  fprintf(f, "{\"format\": \"mpcg-autotune-1\", \"device\": \"%s\", \"sm_count\": %d, \"entries\": [", dev.c_str(),
          sm_count);
  for (size_t i = 0; i < rows.size(); ++i) {
    const Key& k = rows[i].first;
    fprintf(f, "%s\n  {\"fn\": \"%s\", \"kind\": %d, \"npts\": %lld, \"nb\": %d, \"C\": %d, \"value\": %d}",
            i ? "," : "", kNames[std::get<0>(k)], std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k),
            rows[i].second);
  }
  fprintf(f, "\n]}\n");
  return fclose(f) == 0;
}

int load(const char* path, const char* device, int sm_count) {
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
  fclose(f);
  if (text.find("\"format\": \"mpcg-autotune-1\"") == std::string::npos) return -2;
  // device and SM count must match: shapes tuned on another part do not apply
  const size_t d = text.find("\"device\": \"");
  if (d == std::string::npos) return -2;
  const size_t d0 = d + 11, d1 = text.find('"', d0);
  if (d1 == std::string::npos) return -2;
  std::string dev;
  for (const char* c = device; *c; ++c)
    if (*c != '"' && *c != '\\') dev += *c;
  if (text.compare(d0, d1 - d0, dev) != 0) return -3;
  const size_t s = text.find("\"sm_count\": ");
  int sms = -1;
  if (s == std::string::npos || sscanf(text.c_str() + s + 12, "%d", &sms) != 1 || sms != sm_count) return -3;
  std::vector<std::pair<Key, int>> rows;
  size_t pos = text.find("\"entries\": [");
  if (pos == std::string::npos) return -2;
  while ((pos = text.find("{\"fn\": \"", pos)) != std::string::npos) {
    char name[64] = {0};
    int kind, nb, C, value;
    long long npts;
    if (sscanf(text.c_str() + pos,
               "{\"fn\": \"%63[a-z_]\", \"kind\": %d, \"npts\": %lld, \"nb\": %d, \"C\": %d, \"value\": %d}", name,
               &kind, &npts, &nb, &C, &value) != 6)
      return -2;
    const int fn = fn_of(name);
    if (fn < 0 || npts < 1 || nb < 1 || C < 0 || value < 0) return -2;
    rows.push_back({Key(fn, kind, npts, nb, C), value});
    pos += 8;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& r : rows) g_table[r.first] = r.second;
  g_size.store((int)g_table.size(), std::memory_order_release);
  return (int)rows.size();
}

}  // namespace tune
}  // namespace mpcg
