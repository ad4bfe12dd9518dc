// Per-kernel CUDA-event timing of libevo launches (off unless evo_profile_begin
// was called).  Each host launch function opens one Prof scope naming its
// kernel, how many kernels it launches, and the algorithmic flops and bytes of
// the launch; the scope records an event pair on the launch stream.  With
// EVO_NVTX=1 in the environment every scope is also an NVTX push/pop range of
// that name, so a profiler can select the launches of one kernel class (the
// triangle einsum and outer-product GEMMs share the GEMM kernel with every
// other projection).
#pragma once
#include <cuda_runtime.h>

namespace evo {

bool prof_on();
// NVTX ranges around every launch scope (EVO_NVTX=1 at load time).
bool prof_nvtx();
void prof_nvtx_push(const char *name);
void prof_nvtx_pop();
// True while recording and name passes the evo_profile_only selection.
bool prof_wants(const char *name);
// True while profiling with per-shape names (EVO_PROFILE_DETAIL=1 in the
// environment at evo_profile_begin).
bool prof_detail();
// A stable copy of a printf-formatted name (lives until the process exits).
const char *prof_name(const char *fmt, ...);
void prof_record(const char *name, int launches, double flops, double bytes, cudaEvent_t a, cudaEvent_t b);
cudaEvent_t prof_event();

struct Prof {
  const char *name;
  int launches;
  double flops, bytes;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(const char *n, cudaStream_t st, double f = 0, double by = 0, int nl = 1)
      : name(n), launches(nl), flops(f), bytes(by), s(st) {
    if (prof_nvtx()) prof_nvtx_push(n);
    if (prof_wants(n)) {
      a = prof_event();
      b = prof_event();
      if (a) cudaEventRecord(a, s);
    }
  }
  ~Prof() {
    if (a && b) {
      cudaEventRecord(b, s);
      prof_record(name, launches, flops, bytes, a, b);
    }
    if (prof_nvtx()) prof_nvtx_pop();
  }
};

}  // namespace evo
