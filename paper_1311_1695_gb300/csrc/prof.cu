// Kernel timing with CUDA events (see prof.h).  Single-threaded use.
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lapeig.h"
#include "prof.h"

namespace lapeig {

namespace {

struct Pending {
  int name;
  double bytes;
  cudaEvent_t a, b;
};

struct Totals {
  double ms = 0.0, bytes = 0.0;
  long long launches = 0;
};

struct Profiler {
  bool on = false;
  std::vector<std::string> names;
  std::map<std::string, int> index;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<Totals> totals;

  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int name_id(const char* n) {
    auto it = index.find(n);
    if (it != index.end()) return it->second;
    const int id = (int)names.size();
    names.emplace_back(n);
    index[n] = id;
    totals.emplace_back();
    return id;
  }
  void drain() {
    if (pending.empty()) return;
    cudaEventSynchronize(pending.back().b);
    for (auto& p : pending) {
      float ms = 0.f;
      cudaEventSynchronize(p.b);
      cudaEventElapsedTime(&ms, p.a, p.b);
      Totals& t = totals[p.name];
      t.ms += ms;
      t.bytes += p.bytes;
      t.launches += 1;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};

Profiler& P() {
  static Profiler p;
  return p;
}

}  // namespace

bool prof_on() { return P().on; }

namespace {
thread_local int g_prof_depth = 0;
}
bool prof_enter() { return g_prof_depth++ > 0; }
void prof_exit() { --g_prof_depth; }

int prof_begin(const char* name, double bytes, cudaStream_t s) {
  Profiler& p = P();
  if (p.pending.size() > 200000) p.drain();
  Pending r{p.name_id(name), bytes, p.ev(), p.ev()};
  cudaEventRecord(r.a, s);
  p.pending.push_back(r);
  return (int)p.pending.size() - 1;
}

void prof_end(int slot, cudaStream_t s) { cudaEventRecord(P().pending[slot].b, s); }

void prof_set_last_bytes(const char* name, double bytes) {
  Profiler& p = P();
  auto it = p.index.find(name);
  if (it == p.index.end()) return;
  for (size_t i = p.pending.size(); i-- > 0;)
    if (p.pending[i].name == it->second) { p.pending[i].bytes = bytes; return; }
}

}  // namespace lapeig

extern "C" {

int lap_profile_enable(int on) {
  lapeig::P().on = on != 0;
  return LAP_OK;
}

int lap_profile_read(int max, char* names, int name_len, double* ms, double* bytes, int64_t* launches, int* count) {
  lapeig::Profiler& p = lapeig::P();
  p.drain();
  const int n = (int)p.names.size();
  int c = 0;
  for (int i = 0; i < n && c < max; ++i) {
    if (p.totals[i].launches == 0) continue;
    if (names) {
      std::strncpy(names + (size_t)c * name_len, p.names[i].c_str(), name_len - 1);
      names[(size_t)c * name_len + name_len - 1] = 0;
    }
    if (ms) ms[c] = p.totals[i].ms;
    if (bytes) bytes[c] = p.totals[i].bytes;
    if (launches) launches[c] = p.totals[i].launches;
    ++c;
  }
  if (count) *count = c;
  for (auto& t : p.totals) t = lapeig::Totals{};
  return LAP_OK;
}

}  // extern "C"
