// evo_block_fwd_noalloc: the block forward with its scratch in a fixed,
// library-owned device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot allocate device memory at call time --
// for example a serving process whose memory pool was carved up once at
// start-up and must not grow, or a host callback / latency-critical loop in
// which cudaMalloc (which may synchronise the device) is not allowed -- and
// that also do not want to keep a workspace of their own alive.
//
// Cost: the array below (128 MiB) is reserved on every GPU that loads this
// part of the library and stays reserved until the process exits.
#include <mutex>

#include "block.h"

namespace {

constexpr size_t kScratchBytes = 128ull << 20;
constexpr int kMaxDevices = 64;

// Device scratch shared by every call.  Host code must not use its name as a
// device address: the address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
int scratch_on_current_device(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return EVO_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return EVO_OK;
}

bool aligned256(const void *p) { return p && ((uintptr_t)p & 255u) == 0; }

}  // namespace

extern "C" int evo_block_fwd_noalloc(const evo_dims *d, const float *params, const void *params_bf16,
                                     const void *m_in, const void *z_in, void *m_out, void *z_out,
                                     const float *msa_mask, const float *pair_mask, evo_stream_t stream) {
  const int v = evo::validate_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !m_in || !z_in || !m_out || !z_out || !msa_mask || !pair_mask || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, m_in, z_in, (const void *)m_out, (const void *)z_out,
                        (const void *)msa_mask, (const void *)pair_mask})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (evo::workspace_bytes(*d, EVO_MODE_FWD) > kScratchBytes) return EVO_ERR_WORKSPACE;
  void *ws = nullptr;
  const int r = scratch_on_current_device(&ws);
  if (r != EVO_OK) return r;
  // The forward writes every scratch byte it reads, so nothing needs clearing.
  return evo::block_forward(*d, params, (const bf16 *)params_bf16, m_in, z_in, m_out, z_out, msa_mask, pair_mask, ws,
                            kScratchBytes, (cudaStream_t)stream);
}
