// Online autotuner for launch geometry.
//
// A tuned launch site names a key (site, shape class) and a list of candidate geometries that
// all compute the same values -- only how the work is spread over CTAs, clusters or SMs
// changes.  The first launches of a key go round the candidates, each bracketed by CUDA events
// on its stream; when the calling ABI function synchronises, the event times are read and each
// candidate keeps its fastest sample.  Once every candidate has kTuneSamples samples, the key
// is settled on the fastest and later launches take it without events.  The table lives for the
// process and is shared by every context, problem and host thread (guarded by a mutex); the
// pending event pairs are per host thread, so concurrent calls on other threads (the serving
// workers) resolve only their own.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace ihsbin {
namespace {

constexpr int kTuneMaxCand = 8;
constexpr int kTuneSamples = 2;

struct TuneEntry {
  int ncand = 0;
  int values[kTuneMaxCand] = {};
  float best_ms[kTuneMaxCand] = {};
  int samples[kTuneMaxCand] = {};
  int next = 0;     // next candidate to try
  int chosen = -1;  // settled candidate (index), -1 while tuning
  std::string site;
};

struct Pending {
  uint64_t key;
  int cand;
  cudaEvent_t e0, e1;
};

std::mutex g_mu;
std::map<uint64_t, TuneEntry> g_table;
thread_local std::vector<Pending> g_pending;

}  // namespace

uint64_t tune_key(int site, int64_t a, int64_t b, int64_t c) {
  // site (8 bits) and three shape fields folded into one key (collisions only merge shape classes)
  uint64_t k = (uint64_t)(site & 0xFF);
  k = k * 0x9E3779B97F4A7C15ull ^ (uint64_t)a;
  k = k * 0x9E3779B97F4A7C15ull ^ (uint64_t)b;
  k = k * 0x9E3779B97F4A7C15ull ^ (uint64_t)c;
  return k;
}

int shape_class(int64_t n) {  // ceil(log2 n), n >= 1
  int c = 0;
  while (((int64_t)1 << c) < n) ++c;
  return c;
}

TuneLaunch tune_begin(uint64_t key, const char* site, const int* values, int ncand, cudaStream_t st) {
  TuneLaunch t;
  t.key = key;
  ncand = std::max(1, std::min(ncand, kTuneMaxCand));
  std::lock_guard<std::mutex> g(g_mu);
  TuneEntry& e = g_table[key];
  if (e.ncand == 0) {
    e.ncand = ncand;
    std::copy(values, values + ncand, e.values);
    e.site = site;
  }
  if (e.chosen >= 0 || e.ncand == 1) {
    t.cand = e.chosen >= 0 ? e.chosen : 0;
    t.value = e.values[t.cand];
    return t;
  }
  t.cand = e.next;
  e.next = (e.next + 1) % e.ncand;
  t.value = e.values[t.cand];
  if (cudaEventCreate(&t.e0) == cudaSuccess && cudaEventCreate(&t.e1) == cudaSuccess) {
    cudaEventRecord(t.e0, st);
    t.timed = true;
  }
  return t;
}

void tune_end(TuneLaunch& t, cudaStream_t st) {
  if (!t.timed) return;
  cudaEventRecord(t.e1, st);
  g_pending.push_back({t.key, t.cand, t.e0, t.e1});
  t.timed = false;
}

void tune_resolve() {
  if (g_pending.empty()) return;
  std::lock_guard<std::mutex> g(g_mu);
  for (const Pending& q : g_pending) {
    float ms = 0.f;
    const bool ok = cudaEventElapsedTime(&ms, q.e0, q.e1) == cudaSuccess;
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
    auto it = g_table.find(q.key);
    if (!ok || it == g_table.end()) continue;
    TuneEntry& e = it->second;
    if (e.chosen >= 0) continue;
    if (e.samples[q.cand] == 0 || ms < e.best_ms[q.cand]) e.best_ms[q.cand] = ms;
    ++e.samples[q.cand];
    bool done = true;
    for (int c = 0; c < e.ncand; ++c) done = done && e.samples[c] >= kTuneSamples;
    if (done) {
      int best = 0;
      for (int c = 1; c < e.ncand; ++c)
        if (e.best_ms[c] < e.best_ms[best]) best = c;
      e.chosen = best;
    }
  }
  g_pending.clear();
}

void tune_discard() {
  for (const Pending& q : g_pending) {
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
  }
  g_pending.clear();
}

std::string tune_report() {
  std::lock_guard<std::mutex> g(g_mu);
  std::string out;
  char line[256];
  for (const auto& kv : g_table) {
    const TuneEntry& e = kv.second;
    std::snprintf(line, sizeof(line), "%s key=%016llx chosen=%d", e.site.c_str(), (unsigned long long)kv.first,
                  e.chosen >= 0 ? e.values[e.chosen] : -1);
    out += line;
    for (int c = 0; c < e.ncand; ++c) {
      std::snprintf(line, sizeof(line), " [%d: %.4f ms x%d]", e.values[c], e.best_ms[c], e.samples[c]);
      out += line;
    }
    out += "\n";
  }
  return out;
}

void tune_reset() {
  std::lock_guard<std::mutex> g(g_mu);
  g_table.clear();
}

}  // namespace ihsbin
