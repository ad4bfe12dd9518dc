// evo_block_fwd_noalloc: the block forward with its scratch in a fixed,
// library-owned device array instead of a caller-provided workspace.
//
// Who needs it: callers that cannot allocate device memory at call time --
// for example a serving process whose memory pool was carved up once at
// start-up and must not grow, or a host callback / latency-critical loop in
// which cudaMalloc (which may synchronise the device) is not allowed -- and
// that also do not want to keep a workspace of their own alive.
//
// It runs the inference workspace plan (every sub-module's scratch in one
// shared region, two buffers per residual stream), the plan evo_block_fwd_infer
// uses, so the fixed array covers larger problems than the training plan
// would: with 128 MiB, N_res up to 198 (BF16) / 138 (FP32) at N_seq = 16 and
// up to 181 / 100 at N_seq = 128 (evo_workspace_size, EVO_MODE_INFER).
//
// Cost: the array below (128 MiB) is reserved on every GPU that loads this
// part of the library and stays reserved until the process exits.
#include <cuda.h>

#include <mutex>

#include "block.h"

namespace {

constexpr size_t kScratchBytes = 128ull << 20;
constexpr int kMaxDevices = 64;

// Device scratch shared by every call.  Host code must not use its name as a
// device address: the address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
struct ScratchAddr {
  CUcontext ctx;  // the context the address was looked up in
  void *addr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// The current context of the calling thread, through the driver entry point
// (no link against libcuda).  nullptr when the query is unavailable.
CUcontext current_context() {
  typedef CUresult (*GetCurrentFn)(CUcontext *);
  static GetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (GetCurrentFn)p;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch in the current device's current context,
// looked up once per (device, context): a symbol's address belongs to the
// context it was loaded in, so a new context on the same device (after
// cudaDeviceReset, or a non-primary context made current) is looked up again.
int scratch_on_current_device(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVO_ERR_CUDA;
  // make sure the runtime has a context on this device before asking for it
  if (cudaFree(nullptr) != cudaSuccess) return EVO_ERR_CUDA;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchAddr &s = g_scratch[dev];
  if (!s.addr || s.ctx != ctx) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return EVO_ERR_CUDA;
    s.addr = p;
    s.ctx = ctx;
  }
  *out = s.addr;
  return EVO_OK;
}

bool aligned256(const void *p) { return p && ((uintptr_t)p & 255u) == 0; }

}  // namespace

extern "C" int evo_block_fwd_noalloc(const evo_dims *d, const float *params, const void *params_bf16,
                                     const void *m_in, const void *z_in, void *m_out, void *z_out,
                                     const float *msa_mask, const float *pair_mask, evo_stream_t stream) {
  const int v = evo::validate_infer_dims(d);
  if (v != EVO_OK) return v;
  const bool bf = d->act_dtype == EVO_BF16;
  if (!params || !m_in || !z_in || !m_out || !z_out || !msa_mask || !pair_mask || (bf && !params_bf16))
    return EVO_ERR_INVALID_ARG;
  for (const void *p : {(const void *)params, m_in, z_in, (const void *)m_out, (const void *)z_out,
                        (const void *)msa_mask, (const void *)pair_mask})
    if (!aligned256(p)) return EVO_ERR_ALIGNMENT;
  if (bf && !aligned256(params_bf16)) return EVO_ERR_ALIGNMENT;
  if (evo::workspace_bytes(*d, EVO_MODE_INFER) > kScratchBytes) return EVO_ERR_WORKSPACE;
  void *ws = nullptr;
  const int r = scratch_on_current_device(&ws);
  if (r != EVO_OK) return r;
  // The inference forward writes every scratch byte before it reads it, so
  // nothing in the shared array needs clearing between calls.
  return evo::block_forward_infer(*d, params, (const bf16 *)params_bf16, m_in, z_in, m_out, z_out, msa_mask,
                                  pair_mask, ws, kScratchBytes, (cudaStream_t)stream);
}
