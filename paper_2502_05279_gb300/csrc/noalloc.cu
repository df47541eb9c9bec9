// Allocation-free variant of the residual-norm entry point.
//
// bmg_residual needs scratch for its per-block partial sums and obtains it from
// the stream-ordered allocator on every call.  Some callers cannot allow that:
// code that runs while another framework owns the device memory pool and
// forbids foreign allocations, allocation-free real-time or signal-handler
// paths, and tools that check a region of work for allocator calls.  For them
// bmg_residual_noalloc keeps that scratch in a fixed device array compiled into
// the library: every GPU that loads the library holds it (8 KiB) until the
// process exits.
//
// The array holds up to kPartials partial sums plus the result.  kPartials is
// the residual kernel's own block limit (min(n, that limit) blocks), so every n
// the ABI accepts fits; a partial count beyond the array is still checked and
// rejected with BMG_EINVAL.
// Every call shares the one array, so calls whose work overlaps on the GPU
// (other streams, other host threads) race on it and must be serialised by
// the caller.  Each call writes every slot it later reads, so nothing left by
// an earlier call needs clearing.
//
// The device address of the array is looked up once per device and kept for
// the life of the process; a cudaDeviceReset on that device unloads the
// library's device code, after which this entry point must not be called
// again in the process.
#include <mutex>

#include "common.cuh"
#include "cycle_device.cuh"
#include "kernels.h"

namespace bmg {
void zero_ring(int n, double* r, cudaStream_t s);   // k_cycle.cu
}

using namespace bmg;

namespace {

constexpr int kPartials = dev::NORM_BLOCKS_MAX;
static_assert(kPartials >= dev::NORM_BLOCKS_MAX, "the static scratch must hold every partial sum of the norm");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kPartials + 1];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device.  The host-side symbol is
// only a stand-in; the address comes from the runtime once per device, the
// first time this entry point runs there.
int scratch_address(double** out) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "bmg_residual_noalloc: cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(BMG_EINVAL, "bmg_residual_noalloc: device %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "bmg_residual_noalloc: cudaGetSymbolAddress");
    if (rc) return rc;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return BMG_OK;
}

}  // namespace

extern "C" int bmg_residual_noalloc(int n, int kind, const double* coef, const double* x, const double* f, double* r,
                                    double* norm, void* stream) {
  if (n < 3 || ((n + 1) & n) != 0 || (kind != 5 && kind != 9) || !coef || !x || !f)
    return set_error(BMG_EINVAL, "bmg_residual_noalloc: bad argument");
  int np = n < norm_partials_max() ? n : norm_partials_max();
  if (np > kPartials)
    return set_error(BMG_EINVAL, "bmg_residual_noalloc: %d partial sums exceed the static scratch of %d", np,
                     kPartials);
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  size_t ps = plane_size(n);
  StencilView<double, double> v{coef, coef + ps, coef + 2 * ps, coef + 3 * ps, coef + 4 * ps, nullptr, n, n + 2};
  if (r) zero_ring(n, r, s);
  int got = launch_residual(v, kind, x, f, r, norm ? scratch : (double*)nullptr, (const int*)nullptr, s);
  if (norm) {
    launch_norm_finalize(scratch, got, nullptr, 0, scratch + kPartials, s);
    rc = cuda_check(cudaMemcpyAsync(norm, scratch + kPartials, sizeof(double), cudaMemcpyDeviceToHost, s),
                    "bmg_residual_noalloc: copy");
    if (rc) return rc;
  }
  rc = cuda_check(cudaGetLastError(), "bmg_residual_noalloc: launch");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(s), "bmg_residual_noalloc");
}
