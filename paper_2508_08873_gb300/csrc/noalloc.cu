// Allocation-free entry point of the batched tridiagonal propagator.
//
// Some callers cannot allocate device memory: real-time or embedded hosts that
// forbid allocation after start-up, frameworks that own every device byte
// through their own memory pool, and latency-sensitive callers that must not
// trigger cudaFree's device-wide synchronisation.  lrp_propagate_noalloc
// serves them: the caller passes the operator, inputs and outputs as device
// pointers, and the only scratch the propagator needs -- the factorisation of
// I + dt*A -- lives in a fixed file-scope device array instead of a
// cudaMalloc'd buffer.  All calls share that array (see include/lrp.h).
#include <mutex>

#include "internal.h"

namespace {

// Scratch for the factorisation; every GPU that loads the library holds it
// until the process exits.  Sized for n <= LRP_NOALLOC_MAX_N.
constexpr size_t kScratchBytes = 300 * 1024;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};   // device address of g_scratch, per device
int g_sms[kMaxDevices] = {};

// Makes `device` current for the call and gives the calling thread its
// previous current device back on every return path.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
    ok = cudaSetDevice(device) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

using namespace lrp;

extern "C" lrp_status lrp_propagate_noalloc(int device, void* stream, int n, const double* lo,
                                            const double* di, const double* up, double dt, int M,
                                            int adjoint, int nvec, const double* x_in,
                                            double* x_out, int Q, const double* g,
                                            const double* c, lrp_precision prec) {
  if (device < 0 || device >= kMaxDevices || !lo || !di || !up || !x_out || nvec < 0 || M < 0 ||
      !(dt > 0) || Q < 0 || n < 2)
    return LRP_EINVAL;
  if (n > LRP_NOALLOC_MAX_N) return LRP_EINVAL;          // beyond the fixed scratch
  if (adjoint && Q > 0) return LRP_EINVAL;
  if (Q > 0 && (!g || !c)) return LRP_EINVAL;
  if (tri_raw_scratch_bytes(n) > kScratchBytes) return LRP_EINVAL;
  DeviceGuard guard(device);
  if (!guard.ok) return LRP_ECUDA;
  void* scratch = nullptr;
  int sms = 0;
  {
    // one-time set-up per device, with that device current: the host-side
    // name g_scratch is only a stand-in, the kernels need its device address
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return LRP_ECUDA;
      }
      if (cudaDeviceGetAttribute(&g_sms[device], cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess)
        return LRP_ECUDA;
      g_addr[device] = p;
    }
    scratch = g_addr[device];
    sms = g_sms[device];
  }
  PropIn in;
  in.x = x_in;                 // NULL: zero initial values
  in.x_f64 = 1;
  in.ldx = n;
  PropOut out;
  out.y = x_out;
  out.y_f64 = 1;
  out.ldy = n;
  PropSrc src;
  src.Q = Q;
  src.g = g;
  src.c = c;
  src.cstride = (long)M * Q;
  return tri_raw_propagate((cudaStream_t)stream, sms, scratch, n, lo, di, up, dt, adjoint, M, nvec,
                           prec == LRP_PREC_MIXED ? 1 : 0, in, out, src);
}
