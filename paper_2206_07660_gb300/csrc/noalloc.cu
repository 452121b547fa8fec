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

std::mutex g_mu;
void* g_addr[128];          // device address of the array, per device ordinal
bool g_ready[128];
std::string g_err;

}  // namespace

extern "C" const char* gw_noalloc_last_error(void) { return g_err.c_str(); }

extern "C" gw_status gw_screened_solve_noalloc(const double* P0, double* P, int64_t n, int64_t count,
                                               void* stream) {
  using namespace gwk;
  if (!P0 || !P || n <= 0 || count < 0) { g_err = "null pointer or non-positive size"; return GW_ERR_ARG; }
  if (count == 0) return GW_OK;
  const size_t per_sys = screened_work_bytes(n, 1);
  if (per_sys + kFlagBytes > kScratchBytes) {
    g_err = "matrix order too large for the fixed scratch (" + std::to_string(kScratchBytes) + " bytes)";
    return GW_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) { g_err = "no current device"; return GW_ERR_CUDA; }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) { g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return GW_ERR_CUDA; }
      g_ready[dev] = true;
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* d_info = (int*)base;
  double2* work = (double2*)((unsigned char*)base + kFlagBytes);
  const size_t work_bytes = kScratchBytes - kFlagBytes;
  cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int), st);     // the array keeps the last call's flag
  if (!e && P != P0) e = cudaMemcpyAsync(P, P0, (size_t)n * n * count * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (!e) e = screened_inplace((double2*)P, n, count, work, work_bytes, d_info, st);
  int h_info = 0;
  if (!e) e = cudaMemcpyAsync(&h_info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) { g_err = cudaGetErrorString(e); return GW_ERR_CUDA; }
  if (h_info) { g_err = "zero pivot in the screened solve"; return GW_ERR_SINGULAR; }
  return GW_OK;
}
