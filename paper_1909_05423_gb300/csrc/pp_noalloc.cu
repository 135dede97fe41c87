// pp_noalloc.cu -- the refined mixed-precision solve without any device allocation.
//
// pp_solve_refined() allocates, on its first call on a plan, a grid-sized buffer for the
// residual / correction and a small buffer for the partial sums of the mean.  Some callers
// cannot allocate at that point: time-stepping loops that must not allocate or risk an
// out-of-memory error mid-run, and host applications whose own memory manager owns the device
// memory.  pp_solve_refined_noalloc() gives them the
// same result with no allocation at all: its scratch is the file-scope device array below,
// which every GPU that loads this library holds until the process exits.
#include <cstdio>
#include <mutex>
#include <string>

#include "pp_internal.h"

namespace {

constexpr size_t kResidBytes = 16u << 20;                        // u0, then residual / correction (FP32)
constexpr long long kMaxPoints = 2097152;                        // cells
static_assert(2 * (size_t)kMaxPoints * sizeof(float) <= kResidBytes, "u0 and the residual of the largest grid fit");
constexpr size_t kMeanBytes = (pp::kMeanParts + 1) * sizeof(float2);        // partial sums + mean
constexpr size_t kScratchBytes = kResidBytes + kMeanBytes;

// Shared scratch of every pp_solve_refined_noalloc() call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Host code must not take the address of g_noalloc_scratch directly (on the host that name is a
// stand-in, not a device address); the device address is looked up once per device, with that
// device current.
pp_status scratch_address(void** out, std::string* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return PP_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { *err = "device ordinal out of range"; return PP_ERR_INTERNAL; }
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      *err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
      return PP_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return PP_OK;
}

}  // namespace

using pp::set_last_error;

extern "C" pp_status pp_solve_refined_noalloc(pp_plan* p, const void* f, void* u, pp_stream_t stream) {
  if (!p || !f || !u) return set_last_error(PP_ERR_INVALID_ARG, "NULL plan or pointer");
  if (p->dtype != PP_MIXED_F64IO)
    return set_last_error(PP_ERR_INVALID_ARG, "pp_solve_refined_noalloc needs a PP_MIXED_F64IO plan");
  if (f == u) return set_last_error(PP_ERR_INVALID_ARG, "u must not alias f for the refined solve");
  long long npts = (long long)p->nx * p->ny * p->nz;
  if (npts > kMaxPoints) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "pp_solve_refined_noalloc: grid of %lld cells exceeds the %lld cells of its fixed scratch; "
             "use pp_solve_refined for larger grids",
             npts, kMaxPoints);
    return set_last_error(PP_ERR_UNSUPPORTED_SIZE, msg);
  }
  std::string err;
  void* base = nullptr;
  pp_status s = scratch_address(&base, &err);
  if (s != PP_OK) return set_last_error(s, err.c_str());
  void* resid = base;                                            // u0, then residual / correction
  void* partials = static_cast<unsigned char*>(base) + kResidBytes;
  float2* mean = static_cast<float2*>(partials) + pp::kMeanParts;
  // Every value read is first written by this call (the residual by the residual kernel, each
  // partial sum by its block, the mean by the finishing block), so nothing needs clearing.
  return pp::solve_refined_core(p, f, u, resid, partials, mean, (cudaStream_t)stream);
}
