// Allocation-free application of the even-odd operator M-hat.
//
// Who needs it: callers that may not call cudaMalloc / cudaFree while they run -- a
// host callback or a real-time loop whose latency budget has no room for an
// allocation (cudaFree also synchronises the device), or a framework whose memory pool
// owns all device memory and forbids allocations behind its back.  pfmp_mhat() borrows
// the operator's own odd-site temporary, allocated when the operator was created; this
// variant takes its temporary from a fixed array that is part of the library image
// instead, so the call itself allocates nothing.
//
// The scratch array below is PFMP_NOALLOC_SCRATCH_BYTES (64 MiB) of device memory that
// every GPU on which the library is loaded holds until the process exits.  The host
// code cannot use the array's name as a device address (on the host it names a
// stand-in object), so its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
#include <mutex>

#include "context.h"

namespace pfmp {
void mhat_with_temp(pfmp_op* op, int prec, void* out, const void* in, bool dagger, void* temp);
}
using namespace pfmp;

static __device__ __align__(256) unsigned char g_noalloc_scratch[PFMP_NOALLOC_SCRATCH_BYTES];

static constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mutex;

// device address of the scratch array on device dev, which must be the current device
// (looked up once per device)
static void* scratch_address(int dev) {
  int cur = -1;
  PFMP_CUDA(cudaGetDevice(&cur));
  PFMP_REQUIRE(cur == dev, PFMP_E_INVALID,
               "pfmp_mhat_noalloc: the operator's device must be the current device");
  PFMP_REQUIRE(dev >= 0 && dev < kMaxDevices, PFMP_E_UNSUPPORTED, "device index beyond the scratch table");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    PFMP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    PFMP_REQUIRE(p != nullptr, PFMP_E_CUDA, "cudaGetSymbolAddress returned a null scratch address");
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

extern "C" int pfmp_mhat_noalloc(pfmp_op* op, int prec, void* out, const void* in, int dagger) {
  try {
    set_last_error("");
    PFMP_REQUIRE(op && out && in && out != in, PFMP_E_INVALID, "bad argument");
    PFMP_REQUIRE(prec == PFMP_F64 || prec == PFMP_F32, PFMP_E_INVALID,
                 "pfmp_mhat_noalloc: precision must be PFMP_F64 or PFMP_F32");
    const size_t need = spinor_bytes(op->ctx->g, prec);
    PFMP_REQUIRE(need <= (size_t)PFMP_NOALLOC_SCRATCH_BYTES, PFMP_E_INVALID,
                 "pfmp_mhat_noalloc: the odd-site temporary (" + std::to_string(need) +
                     " bytes) exceeds the fixed scratch of " + std::to_string((long long)PFMP_NOALLOC_SCRATCH_BYTES) +
                     " bytes; use pfmp_mhat");
    void* temp = scratch_address(op->ctx->device);
    mhat_with_temp(op, prec, out, in, dagger != 0, temp);
  } catch (const Err& e) {
    return e.code;
  } catch (...) {
    set_last_error("unexpected C++ exception");
    return PFMP_E_INVALID;
  }
  return PFMP_OK;
}
