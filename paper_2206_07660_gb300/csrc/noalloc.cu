// Allocation-free variant of the screened solve (tilde_P_omega kernels).
//
// Some callers cannot allocate device memory at the point where they need the
// solve: code that runs inside a memory pool or arena it does not own, plugins
// whose host application forbids cudaMalloc after start-up, and code paths
// that must not trigger an allocator's implicit synchronisation.  This entry
// point takes the caller's input and output buffers and uses, as scratch, one
// file-scope device array of GW_NOALLOC_SCRATCH_BYTES that every GPU loading
// the library keeps until the process exits.
#include <mutex>
#include "gw_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;   // GW_NOALLOC_SCRATCH_BYTES
constexpr size_t kFlagBytes = 256;                    // status word, kept apart from the panels

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;             // guards the per-device address table
void* g_addr[128];          // device address of the array, per device ordinal
bool g_ready[128];
thread_local std::string g_err;   // last failure of this thread's calls ("" after a success)

}  // namespace

extern "C" const char* gw_noalloc_last_error(void) { return g_err.c_str(); }

static gw_status noalloc_fail(gw_status s, const std::string& m) {
  g_err = m;
  return s;
}

extern "C" gw_status gw_screened_solve_noalloc(const double* P0, double* P, int64_t n, int64_t count,
                                               void* stream) {
  using namespace gwk;
  if (!P0 || !P || n <= 0 || count < 0) return noalloc_fail(GW_ERR_ARG, "null pointer or non-positive size");
  if (count == 0) { g_err.clear(); return GW_OK; }
  const size_t per_sys = screened_work_bytes(n, 1);
  if (n > (int64_t)1 << 20 || per_sys + kFlagBytes > kScratchBytes)
    return noalloc_fail(GW_ERR_ARG, "matrix order too large for the fixed scratch (" +
                                        std::to_string(kScratchBytes) + " bytes)");
  if (count > (INT64_MAX / 16) / (n * n)) return noalloc_fail(GW_ERR_ARG, "count * n * n overflows");
  const size_t bytes = (size_t)n * n * count * sizeof(double2);
  if (P != P0) {   // distinct buffers must not overlap (an in-place solve passes P == P0)
    const uintptr_t a = (uintptr_t)P0, b = (uintptr_t)P;
    if (a < b + bytes && b < a + bytes)
      return noalloc_fail(GW_ERR_ARG, "P and P0 overlap without being the same buffer");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return noalloc_fail(GW_ERR_CUDA, "no current device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(GW_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_ready[dev] = true;
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* d_info = (int*)base;
  double2* work = (double2*)((unsigned char*)base + kFlagBytes);
  const size_t work_bytes = kScratchBytes - kFlagBytes;
  cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int), st);     // the array keeps the last call's flag
  if (!e && P != P0) e = cudaMemcpyAsync(P, P0, bytes, cudaMemcpyDeviceToDevice, st);
  if (!e) e = screened_inplace((double2*)P, n, count, work, work_bytes, d_info, st);
  int h_info = 0;
  if (!e) e = cudaMemcpyAsync(&h_info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return noalloc_fail(GW_ERR_CUDA, cudaGetErrorString(e));
  if (h_info) return noalloc_fail(GW_ERR_SINGULAR, "zero pivot in the screened solve");
  g_err.clear();
  return GW_OK;
}
