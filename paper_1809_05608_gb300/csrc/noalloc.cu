// mgfld_step_noalloc: the implicit step with its workspace in a fixed, file-scope device
// array instead of caller memory.
//
// Some callers cannot hand this library a workspace: a host code that links it as a
// black-box solver and owns no GPU allocator of its own, a process whose device memory
// is entirely pre-reserved by another framework's pool, or a time-critical loop where
// the device synchronisation implied by cudaMalloc/cudaFree is not acceptable.  For
// them this entry point takes no workspace and calls no allocating routine: the scratch
// lives in `g_scratch` below, which every GPU that loads this library keeps for the
// lifetime of the process.
#include "mgfld_internal.cuh"

namespace {

constexpr size_t kScratchBytes = MGFLD_NOALLOC_SCRATCH_BYTES;

// The scratch itself.  In host code `g_scratch` names a host-side shadow, not device
// memory, so its device address is looked up below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device, looked up on every call with that
// device current (cheap, and it allocates nothing).  Not cached: a context torn down and
// created again (cudaDeviceReset) reloads the module at another address.
mgfld_status scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return MGFLD_ECUDA;
  *out = p;
  return MGFLD_OK;
}

}  // namespace

extern "C" mgfld_status mgfld_step_noalloc(const mgfld_dims *dims, const mgfld_problem *prob,
                                           mgfld_state *state, const mgfld_step_opts *opts,
                                           mgfld_step_report *report, void *stream) {
  if (!dims || !opts) return MGFLD_EINVAL;
  if (opts->profile) return MGFLD_EINVAL;       // timing would create CUDA events
  const size_t need = (prob && prob->pair_coef) ? mgfld_workspace_bytes_pair(dims, opts->precision)
                                                 : mgfld_workspace_bytes(dims, opts->precision);
  if (need == 0) return MGFLD_EINVAL;
  if (need > kScratchBytes) return MGFLD_ENOMEM;
  void *ws = nullptr;
  const mgfld_status st = scratch_address(&ws);
  if (st != MGFLD_OK) return st;
  // Every buffer of the step is written before it is read (k_init resets the per-ray
  // bookkeeping, the counters are cleared on the stream), so the previous call's
  // contents need no clearing here.
  // The outer iteration runs from the host (one stream synchronisation per iteration): the graph
  // path of mgfld_step would instantiate a CUDA graph, which allocates.
  return mgfld::step_host_synchronised(dims, prob, state, opts, report, ws, kScratchBytes, stream);
}
