// pdlp_solve_device_noalloc: pdlp_solve_device for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or unwelcome,
// for example a process whose device memory is owned by another allocator (a
// framework's pool that must see every byte), a latency-bound loop that must
// never reach the CUDA driver's allocator, or a caller that has no way to hand us
// a workspace.  Such a caller passes only its inputs and outputs.
//
// The scratch of the solve lives in one file-scope __device__ array of
// kNoAllocBytes.  Every GPU that loads this library holds that array until
// the process exits, whether or not it ever calls this function.  Host code
// cannot use the array's name as a device address (there it names a host-side
// stand-in), so the first call on each device, with that device current,
// looks its address up with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture begins.
//
// All calls share the one array, and it keeps whatever the last call left in
// it.  The solve writes every scratch buffer it reads (its device state is
// copied in at the start of each call), so nothing carries over from one call
// to the next; but two calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on the array
// and corrupt each other.  Serialise calls per device.
//
// The call itself makes no device allocation and creates no CUDA object: no
// cudaMalloc / cudaFree, no pinned host buffer, no stream, event or graph; it
// launches the same kernels as pdlp_solve_device one by one on the caller's
// stream and polls the termination flag once per check period.  The launch-shape
// autotuner times candidate shapes with its own stream, events and graphs, so a
// request for it (pdlp_params.autotune = 1) is refused here; the size heuristic
// and explicit lanes_A / lanes_AT work as usual.
//
// Every call synchronises the stream (input validation, the termination flag),
// so no call may be made while the stream is being captured into a graph.  The
// cached address belongs to the device's current context: after cudaDeviceReset
// it is stale, so a process that resets a device must not call this again.
#include <mutex>

#include "../../include/pdlp.h"
#include "internal.h"

namespace pdlp {
int solve_device_noalloc(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                         const double* l, const double* u, const pdlp_params* p, const double* x0,
                         const double* y0, double* x_out, double* y_out, pdlp_result* r,
                         const pdlp_diagnostics* dg, void* workspace, size_t ws_bytes,
                         cudaStream_t s);
int set_error(int code, const char* msg);
}  // namespace pdlp

namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int pdlp_solve_device_noalloc(const pdlp_csr* A, const double* b, const char* sense,
                                         const double* c, const double* l, const double* u,
                                         const pdlp_params* p, const double* x0, const double* y0,
                                         double* x_out, double* y_out, pdlp_result* r,
                                         const pdlp_diagnostics* diag, void* stream) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  if (!A) return pdlp::set_error(PDLP_ERR_INVALID_INPUT, "NULL problem");
  if (p->autotune != 0)
    return pdlp::set_error(PDLP_ERR_INVALID_INPUT,
                           "autotune = 1 needs its own stream, events and graphs; "
                           "pdlp_solve_device_noalloc creates none (use autotune = 0)");
  const size_t need = pdlp_workspace_size(A->m, A->n, A->nnz, p);
  if (need == 0) return pdlp::set_error(PDLP_ERR_INVALID_INPUT, "invalid sizes");
  if (need > kNoAllocBytes)
    return pdlp::set_error(PDLP_ERR_OOM,
                           "problem needs more scratch than the 64 MiB static array of "
                           "pdlp_solve_device_noalloc holds (see pdlp_workspace_size)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return pdlp::set_error(PDLP_ERR_CUDA, "cudaGetDevice failed or device index out of range");
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return pdlp::set_error(PDLP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_addr[dev] = ptr;
    }
    ws = g_addr[dev];
  }
  return pdlp::solve_device_noalloc(A, b, sense, c, l, u, p, x0, y0, x_out, y_out, r, diag, ws,
                                    kNoAllocBytes, (cudaStream_t)stream);
}
