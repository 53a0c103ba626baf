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
// The array lives in this translation unit, so a device reserves it when this
// module is loaded there and holds it until the process exits. Under lazy
// module loading (CUDA's default) that happens on the first use of the module
// on that device; under eager loading (CUDA_MODULE_LOADING=EAGER) it happens
// when the context is created, so every process that loads the library then
// reserves the array on each device it uses. Its device address is looked up
// once per device (with that device current) on the first call there; make
// that first call before any stream capture. All calls share the one array:
// the pass state is cleared at the start of every call and every other
// scratch entry is written before it is read, but two calls whose work
// overlaps on the GPU (different streams, different host threads) race on the
// array.
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

// scqr3_factor numbers its arguments by its own prototype; this entry point
// reports them by the positions in its prototype instead (X 1, m 2, n 3,
// ldx 4, Q 5, ldq 6, R 7, info 8).
static int own_arg_code(int r) {
  switch (r) {
    case -6: return -5;   // Q
    case -7: return -6;   // ldq
    case -8: return -7;   // R
    case -13: return -8;  // info
    default: return r;    // X, m, n, ldx keep their positions; other codes are not argument codes
  }
}

extern "C" int scqr3_factor_noalloc(const double* X, int64_t m, int n, int64_t ldx, double* Q,
                                    int64_t ldq, double* R, scqr3_info* info, void* stream) {
  if (!X) return -1;
  if (ldx < n) return -4;
  if (!Q) return -5;
  if (ldq < n) return -6;
  if (!R) return -7;
  if (!info) return -8;
  size_t need = 0;
  const int r = scqr3_workspace_bytes(m, n, nullptr, nullptr, &need);
  if (r != SCQR3_OK) return own_arg_code(r);
  if (need > kScratchBytes) return SCQR3_E_SCRATCH_LIMIT;
  void* ws = nullptr;
  const int a = scratch_address(&ws);
  if (a != SCQR3_OK) return a;
  return own_arg_code(scqr3_factor(X, m, n, ldx, nullptr, Q, ldq, R, nullptr, ws, kScratchBytes, nullptr,
                                   info, stream));
}
