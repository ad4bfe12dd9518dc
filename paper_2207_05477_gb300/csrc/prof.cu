// Launch profiling of libevo (see prof.h) and its C entry points.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "evo.h"
#include "prof.h"

namespace evo {
namespace {

struct Rec {
  const char *name;
  int launches;
  double flops, bytes;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
bool g_detail = false;
bool g_paused = false;  // recording session open but launches not timed
std::string g_only;  // record only this kernel name ("" = all)
std::set<std::string> g_names;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;  // events handed out since the last begin
size_t g_next = 0;

}  // namespace

bool prof_on() { return g_on && !g_paused; }

bool prof_nvtx() {
  static const bool on = [] {
    const char *v = std::getenv("EVO_NVTX");
    return v && v[0] == '1';
  }();
  return on;
}
void prof_nvtx_push(const char *name) { nvtxRangePushA(name); }
void prof_nvtx_pop() { nvtxRangePop(); }

bool pdl_enabled() {
  static const bool on = [] {
    const char *v = std::getenv("EVO_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}
bool prof_wants(const char *name) {
  if (!g_on || g_paused) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  return g_only.empty() || g_only == name;
}
bool prof_detail() { return g_on && g_detail; }

const char *prof_name(const char *fmt, ...) {
  char buf[64];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::lock_guard<std::mutex> lk(g_mu);
  return g_names.insert(std::string(buf)).first->c_str();
}

cudaEvent_t prof_event() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_next == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_next++];
}

void prof_record(const char *name, int launches, double flops, double bytes, cudaEvent_t a, cudaEvent_t b) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(Rec{name, launches, flops, bytes, a, b});
}

}  // namespace evo

using namespace evo;

extern "C" {

int evo_profile_only(const char *kernel_name) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_only = kernel_name ? kernel_name : "";
  return EVO_OK;
}

int evo_profile_pause(int paused) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_paused = paused != 0;
  return EVO_OK;
}

int evo_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.clear();
  g_next = 0;
  const char *d = std::getenv("EVO_PROFILE_DETAIL");
  g_detail = d && d[0] == '1';
  g_on = true;
  return EVO_OK;
}

int evo_profile_end(evo_stream_t stream, evo_profile_entry *out, int cap) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EVO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  g_paused = false;
  g_only.clear();
  std::map<std::string, evo_profile_entry> agg;
  std::vector<std::string> order;
  for (const Rec &r : g_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return EVO_ERR_CUDA;
    auto it = agg.find(r.name);
    if (it == agg.end()) {
      evo_profile_entry e;
      std::memset(&e, 0, sizeof(e));
      std::strncpy(e.name, r.name, sizeof(e.name) - 1);
      it = agg.emplace(r.name, e).first;
      order.push_back(r.name);
    }
    it->second.launches += r.launches;
    it->second.calls += 1;
    it->second.total_ms += ms;
    it->second.flops += r.flops;
    it->second.bytes += r.bytes;
  }
  g_recs.clear();
  int n = 0;
  for (const std::string &k : order) {
    if (out && n < cap) out[n] = agg[k];
    ++n;
  }
  return n;
}

}  // extern "C"
