// GEMM tile autotuner (host side) and its C entry points.
//
// The tcgen05 GEMM has two free launch parameters that do not change its
// result: the output tile width BN (64, 128 or 256 columns per 128-row tile;
// it sets how many persistent-CTA tiles a launch has and how evenly they fill
// the 152 SMs), and, for a product whose epilogue adds into an fp32
// destination with atomics (the weight gradients), the number of K ranges the
// contraction is split into.  Between evo_tune_begin and evo_tune_end every
// GEMM launch of the library is keyed by its shape and epilogue; each run of
// n consecutive launches of a key tries each of the key's n candidates once
// (in a shuffled order), every launch bracketed by a CUDA event pair.
// evo_tune_end takes, per key, the candidate with the lowest median time;
// later launches of that key use it (graph captures included).
// While a stream is capturing a graph nothing is timed.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "evo.h"
#include "kernels.h"

namespace evo {
namespace {

using Key = std::array<int64_t, 12>;

struct Cand {
  int bn, splits;
};

struct Trial {
  int cand;
  cudaEvent_t a, b;
};

struct Entry {
  std::vector<Cand> cands;
  std::vector<Trial> trials;
  uint64_t calls = 0;
  int best = -1;  // index into cands once tuned
};

std::mutex g_mu;
bool g_tuning = false;
std::map<Key, Entry> g_table;
std::vector<cudaEvent_t> g_pool;
size_t g_next = 0;

Key key_of(const GemmOp &g) {
  const Epi &e = g.e;
  const int64_t flags = (e.partial ? 1 : 0) | (e.atomic ? 2 : 0) | (e.c_f32 ? 4 : 0) | (e.accumulate ? 8 : 0) |
                        (e.residual ? 16 : 0) | (e.gate ? 32 : 0) | (e.relu_ref ? 64 : 0) | (e.aux ? 128 : 0) |
                        (e.bias ? 256 : 0) | (e.row_scale ? 512 : 0) | ((int64_t)e.act << 10);
  const int64_t plain = e.map.mdiv >= (1ll << 31) && e.map.ndiv >= (1ll << 31) && e.map.s_n0 == 1;
  return Key{g.M, g.N, g.K, g.batch, g.a_mn, g.b_mn, g.splits, flags, plain, e.map.s_m0, e.map.ndiv, e.map.mdiv};
}

std::vector<Cand> candidates(const GemmOp &g, int default_bn) {
  std::vector<int> bns{default_bn};
  for (int bn : {256, 128, 64})
    if (bn != default_bn && (bn == 64 || g.N > bn / 2)) bns.push_back(bn);
  std::vector<int> sps{g.splits};
  if (g.e.atomic && g.batch == 1) {
    // every K range keeps at least four 64-deep k-tiles
    const int most = std::max<int64_t>(1, g.K / 256);
    if (g.splits * 2 <= most) sps.push_back(g.splits * 2);
    if (g.splits >= 2) sps.push_back(g.splits / 2);
    if (g.splits != 1 && g.splits / 2 != 1 && g.splits * 2 <= most) sps.push_back(1);
  }
  std::vector<Cand> out;
  for (int sp : sps)
    for (int bn : bns) out.push_back(Cand{bn, sp});
  return out;
}

// A table entry applies to a launch only if the tuner itself could have
// offered it (a loaded file is not trusted further).
bool allowed(const GemmOp &g, const Cand &c) {
  const bool bn_ok = c.bn == 64 || ((c.bn == 128 || c.bn == 256) && g.N > c.bn / 2);
  const bool sp_ok = c.splits == g.splits ||
                     (g.e.atomic && g.batch == 1 && c.splits >= 1 && c.splits <= std::max<int64_t>(1, g.K / 256));
  return bn_ok && sp_ok;
}

void apply_best(const GemmOp &g, const Entry &e, TuneChoice &c) {
  if (e.best < 0 || !allowed(g, e.cands[e.best])) return;
  c.bn = e.cands[e.best].bn;
  c.splits = e.cands[e.best].splits;
}

// One line per tuned key: the twelve key fields, the built-in tile width and
// split count, then the chosen ones.
bool save_table(const char *path) {
  FILE *f = std::fopen(path, "w");
  if (!f) return false;
  std::fprintf(f, "# libevo GEMM tile table v1: M N K batch a_mn b_mn splits flags plain s_m0 ndiv mdiv "
                  "default_bn default_splits bn splits\n");
  for (const auto &kv : g_table) {
    const Entry &e = kv.second;
    if (e.best < 0) continue;
    for (int64_t v : kv.first) std::fprintf(f, "%lld ", (long long)v);
    std::fprintf(f, "%d %d %d %d\n", e.cands[0].bn, e.cands[0].splits, e.cands[e.best].bn, e.cands[e.best].splits);
  }
  return std::fclose(f) == 0;
}

bool valid_bn(long long bn) { return bn == 64 || bn == 128 || bn == 256; }

// Replaces the table with the file's entries; false (table unchanged) on a
// malformed file.
bool load_table(const char *path) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  std::map<Key, Entry> t;
  char line[512];
  bool ok = true;
  while (ok && std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    long long v[16];
    int n = 0, used = 0;
    const char *p = line;
    while (n < 16 && std::sscanf(p, "%lld%n", &v[n], &used) == 1) {
      p += used;
      ++n;
    }
    if (n != 16 || !valid_bn(v[12]) || !valid_bn(v[14]) || v[13] < 1 || v[15] < 1 || v[15] > (1 << 16)) {
      ok = false;
      break;
    }
    Key k;
    for (int i = 0; i < 12; ++i) k[i] = v[i];
    Entry e;
    e.cands.push_back(Cand{(int)v[12], (int)v[13]});
    e.best = 0;
    if (v[14] != v[12] || v[15] != v[13]) {
      // a split count other than the built-in one only for an atomic epilogue
      if (v[15] != v[13] && !((k[7] & 2) && k[3] == 1)) {
        ok = false;
        break;
      }
      e.cands.push_back(Cand{(int)v[14], (int)v[15]});
      e.best = 1;
    }
    t[k] = e;
  }
  std::fclose(f);
  if (ok) g_table.swap(t);
  return ok;
}

// EVO_TUNE_CACHE names a table file: read once before the first GEMM launch,
// written by evo_tune_end.
const char *cache_path() {
  static const char *p = std::getenv("EVO_TUNE_CACHE");
  return p && p[0] ? p : nullptr;
}

void load_cache_once() {
  static bool done = false;
  if (done) return;
  done = true;
  if (cache_path()) load_table(cache_path());
}

// Candidate of the k-th launch of a key: every n consecutive launches run
// each of the n candidates once, in an order that changes from one group to
// the next, so that a candidate is not tied to one call site of a workload
// that launches the key several times per pass.
int cand_of_call(uint64_t k, uint32_t n) {
  const uint64_t group = k / n;
  uint32_t perm[16];
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t x = group * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
  for (uint32_t i = n - 1; i > 0; --i) {  // Fisher-Yates with a xorshift stream
    x ^= x << 13, x ^= x >> 7, x ^= x << 17;
    const uint32_t j = (uint32_t)(x % (i + 1));
    const uint32_t t = perm[i];
    perm[i] = perm[j], perm[j] = t;
  }
  return (int)perm[k % n];
}

cudaEvent_t pool_event() {
  if (g_next == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_next++];
}

}  // namespace

TuneChoice tune_choose(const GemmOp &g, int default_bn, cudaStream_t s) {
  TuneChoice c{default_bn, g.splits, nullptr, nullptr};
  std::lock_guard<std::mutex> lk(g_mu);
  load_cache_once();
  if (!g_tuning && g_table.empty()) return c;
  const Key k = key_of(g);
  auto it = g_table.find(k);
  if (!g_tuning) {
    if (it != g_table.end()) apply_best(g, it->second, c);
    return c;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    if (it != g_table.end()) apply_best(g, it->second, c);
    return c;
  }
  if (it == g_table.end()) {
    it = g_table.emplace(k, Entry{}).first;
    it->second.cands = candidates(g, default_bn);
  }
  Entry &e = it->second;
  const int ci = cand_of_call(e.calls++, (uint32_t)e.cands.size());
  c.bn = e.cands[ci].bn;
  c.splits = e.cands[ci].splits;
  c.a = pool_event();
  c.b = pool_event();
  if (c.a && c.b) {
    e.trials.push_back(Trial{ci, c.a, c.b});
    cudaEventRecord(c.a, s);
  } else {
    c.a = c.b = nullptr;
  }
  return c;
}

void tune_done(const TuneChoice &c, cudaStream_t s) {
  if (c.b) cudaEventRecord(c.b, s);
}

}  // namespace evo

using namespace evo;

extern "C" {

int evo_tune_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  g_next = 0;
  g_tuning = true;
  return EVO_OK;
}

int evo_tune_end(evo_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EVO_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return EVO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuning = false;
  int tuned = 0;
  for (auto &kv : g_table) {
    Entry &e = kv.second;
    std::vector<std::vector<float>> ms(e.cands.size());
    for (const Trial &t : e.trials) {
      float x = 0.f;
      if (cudaEventElapsedTime(&x, t.a, t.b) != cudaSuccess) return EVO_ERR_CUDA;
      ms[t.cand].push_back(x);
    }
    e.trials.clear();
    // the median time per candidate (robust to a cold first launch); a
    // candidate that never ran cannot win, and the default (index 0) stays
    // unless every candidate ran
    std::vector<float> med(e.cands.size(), 0.f);
    bool all = true;
    for (size_t i = 0; i < ms.size(); ++i) {
      all = all && !ms[i].empty();
      if (ms[i].empty()) continue;
      std::sort(ms[i].begin(), ms[i].end());
      med[i] = ms[i][ms[i].size() / 2];
    }
    e.best = 0;
    if (all) {
      for (size_t i = 1; i < med.size(); ++i)
        if (med[i] < med[e.best]) e.best = (int)i;
    }
    ++tuned;
  }
  if (cache_path() && !save_table(cache_path())) return EVO_ERR_INVALID_ARG;
  return tuned;
}

int evo_tune_save(const char *path) {
  if (!path) return EVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  return save_table(path) ? EVO_OK : EVO_ERR_INVALID_ARG;
}

int evo_tune_load(const char *path) {
  if (!path) return EVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  load_cache_once();
  if (g_tuning) return EVO_ERR_INVALID_ARG;
  return load_table(path) ? EVO_OK : EVO_ERR_INVALID_ARG;
}

int evo_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  g_tuning = false;
  return EVO_OK;
}

int evo_tune_entries(evo_tune_entry *out, int cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  int i = 0;
  for (const auto &kv : g_table) {
    const Entry &e = kv.second;
    if (out && i < cap) {
      evo_tune_entry &o = out[i];
      std::memset(&o, 0, sizeof(o));
      o.M = kv.first[0], o.N = kv.first[1], o.K = kv.first[2], o.batch = kv.first[3];
      o.default_bn = e.cands[0].bn, o.default_splits = e.cands[0].splits;
      const Cand &b = e.cands[e.best >= 0 ? e.best : 0];
      o.bn = b.bn, o.splits = b.splits;
      o.candidates = (int)e.cands.size();
    }
    ++i;
  }
  return i;
}

}  // extern "C"
