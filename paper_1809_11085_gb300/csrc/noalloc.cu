// noalloc.cu -- scqr3_factor_noalloc: shifted CholeskyQR3 for callers that
// cannot allocate device memory.
//
// scqr3_factor takes its scratch (per-CTA partial Gram matrices, the pass
// state, the per-pass factors) from a caller-provided workspace. Some callers
// have no way to provide one: a host application that owns every byte of
// device memory through its own pool and does not let plug-in code allocate,
// a caller that runs close to the memory limit where a late cudaMalloc could
// fail, or a plain C/Fortran code that is handed device pointers but has no
// allocator of its own. For them this entry point runs the same kernels with
// the scratch placed in a fixed array that this library owns.
//
// The array lives in this translation unit only, so it is reserved on a
// device when this file's module is first used there and held until the
// process exits; processes that never call scqr3_factor_noalloc do not load
// it. Its device address is looked up once per device (with that device
// current) on the first call there; make that first call before any stream
// capture. All calls share the one array: the pass state is cleared at the
// start of every call and every other scratch entry is written before it is
// read, but two calls whose work overlaps on the GPU (different streams,
// different host threads) race on the array.
#include <mutex>

#include "scqr3_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)SCQR3_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCQR3_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return SCQR3_E_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SCQR3_OK;
}

}  // namespace

extern "C" int scqr3_factor_noalloc(const double* X, int64_t m, int n, int64_t ldx, double* Q,
                                    int64_t ldq, double* R, scqr3_info* info, void* stream) {
  size_t need = 0;
  const int r = scqr3_workspace_bytes(m, n, nullptr, nullptr, &need);
  if (r != SCQR3_OK) return r;
  if (need > kScratchBytes) return SCQR3_E_SCRATCH_LIMIT;
  void* ws = nullptr;
  const int a = scratch_address(&ws);
  if (a != SCQR3_OK) return a;
  return scqr3_factor(X, m, n, ldx, nullptr, Q, ldq, R, nullptr, ws, kScratchBytes, nullptr, info,
                      stream);
}
