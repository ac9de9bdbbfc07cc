// Optional kernel timing: when enabled, every launcher brackets its launch
// with a pair of CUDA events on the launch stream and records the kernel's
// algorithmic bytes (what a perfect cache would move).  lap_profile_read()
// synchronises, converts the event pairs into per-kernel totals and clears.
// Off by default; the events cost a timestamp write each on the GPU.
#pragma once
#include <cuda_runtime.h>

namespace lapeig {

bool prof_on();
int prof_begin(const char* name, double bytes, cudaStream_t s);  // returns a slot or -1
void prof_end(int slot, cudaStream_t s);
// Replace the bytes of the most recent pending launch named `name` (for a
// kernel whose work is known only after it ran, e.g. a solve that stops early).
void prof_set_last_bytes(const char* name, double bytes);

// Scope nesting on the calling thread: prof_enter returns true when a scope
// is already open (the launches of a sequence timed as one are not timed
// again on their own).
bool prof_enter();
void prof_exit();

struct ProfScope {
  int slot;
  cudaStream_t s;
  // name nullptr, or a scope inside another: not timed
  ProfScope(const char* name, double bytes, cudaStream_t st) : slot(-1), s(st) {
    const bool nested = prof_enter();
    if (!nested && name && prof_on()) slot = prof_begin(name, bytes, st);
  }
  ~ProfScope() {
    if (slot >= 0) prof_end(slot, s);
    prof_exit();
  }
};

}  // namespace lapeig

#define LAP_PROF(name, bytes, stream) ::lapeig::ProfScope _lap_prof_scope((name), (bytes), (stream))
