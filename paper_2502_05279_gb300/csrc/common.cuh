// Device helpers shared by the BoxMG kernels: rounding-explicit arithmetic,
// stencil access through the symmetric five-plane storage, launch bookkeeping.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/bmg.h"

namespace bmg {

// ---- arithmetic with one rounding per operation (never contracted to FMA) ----
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }

// s + a b and s - a b: a rounded product then a rounded sum (FU = false), or
// one fused multiply-add rounded once (FU = true; -a is exact).  The cycle's
// kernels take FU from the hierarchy's arithmetic mode.
template <bool FU> __device__ __forceinline__ double madd(double s, double a, double b) {
  return FU ? __fma_rn(a, b, s) : radd(s, rmul(a, b));
}
template <bool FU> __device__ __forceinline__ double msub(double s, double a, double b) {
  return FU ? __fma_rn(-a, b, s) : rsub(s, rmul(a, b));
}
template <bool FU> __device__ __forceinline__ float madd(float s, float a, float b) {
  return FU ? __fmaf_rn(a, b, s) : radd(s, rmul(a, b));
}
template <bool FU> __device__ __forceinline__ float msub(float s, float a, float b) {
  return FU ? __fmaf_rn(-a, b, s) : rsub(s, rmul(a, b));
}

// ---- storage -> compute conversion (exact for every pair used) ----
template <typename T> __device__ __forceinline__ T cvt(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cvt(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T cvt(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

// Canonical neighbour order of every row sum: O, W, E, S, N, SW, NE, NW, SE.
__host__ __device__ constexpr int nbr_dx(int k) {
  return k == 1 ? -1 : k == 2 ? 1 : k == 5 ? -1 : k == 6 ? 1 : k == 7 ? -1 : k == 8 ? 1 : 0;
}
__host__ __device__ constexpr int nbr_dy(int k) {
  return k == 3 ? -1 : k == 4 ? 1 : k == 5 ? -1 : k == 6 ? 1 : k == 7 ? 1 : k == 8 ? -1 : 0;
}

// Five-plane stencil view: O, W, S, SW, NW (each ld * ld, plane stride ps).
template <typename S>
struct Planes {
  const S* O;
  const S* W;
  const S* Sp;
  const S* SW;
  const S* NW;
  // a(p, p + (dx, dy)) for the k-th canonical neighbour, p = linear index.
  template <int K>
  __device__ __forceinline__ S a(size_t p, int ld) const {
    if (K == 0) return O[p];
    if (K == 1) return W[p];
    if (K == 2) return W[p + 1];
    if (K == 3) return Sp[p];
    if (K == 4) return Sp[p + ld];
    if (K == 5) return SW[p];
    if (K == 6) return SW[p + ld + 1];
    if (K == 7) return NW[p];
    return NW[p + 1 - ld];
  }
};

template <typename S>
__host__ __device__ inline Planes<S> planes_at(const S* base, size_t ps) {
  return Planes<S>{base, base + ps, base + 2 * ps, base + 3 * ps, base + 4 * ps};
}

// ---- programmatic dependent launch ----
// Every kernel of the cycle is launched with programmatic stream serialization
// and opens with pdl_enter(): it waits for its predecessor to complete and its
// writes to be visible before it touches global memory, then lets the next
// kernel on the stream be scheduled once all of its own CTAs have got that
// far.  The next kernel's CTAs thus take the SMs this one leaves while it
// drains, instead of starting after it; waiting first keeps that overlap to one
// kernel deep (a chain of kernels each triggering before its wait would fill
// the SMs with waiting CTAs).  Launched without the attribute, both
// instructions return at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Interpolation plane indices (Fig. 2 labels).
enum { CI_LSW = 0, CI_LSE, CI_LNW, CI_LNE, CI_LL, CI_LR, CI_LB, CI_LA };

__host__ __device__ inline size_t plane_size(int n) { return (size_t)(n + 2) * (size_t)(n + 2); }

// Control block of one solve (device memory).  `done`: 0 running, 1 converged,
// 2 maxit reached, 3 NaN/Inf.
struct Ctl {
  int done;
  int it;
  int maxit;
  int pad;
  double tol;
  double scale_next;     // power-of-two scale for the next FP32 residual
  double scale_applied;  // the scale the current FP32 residual carries
  // flexible CG scalars
  double zq, pq, pr, pq_prev;
  double beta;           // -zq / pq_prev of the current step, formed once by the zq reduction
  int first;             // 1 until the first direction is formed
  int pad2;
  double hist[1];        // [maxit + 1] residual norms (allocated past the struct)
};

}  // namespace bmg

// ---- debug build: device bounds checks ------------------------------------------
// Compiled with -DBMG_DEBUG (libbmg_debug.so), the kernels check the index of
// each global store, and the source range of each asynchronous row copy,
// against the logical extent of the level array it addresses.  A failed check
// skips the store (a copy reads the array's first element instead, or is
// zero-filled, so that its transaction still completes) and records the first
// failure of the translation unit: site, index, extent.  Nothing traps.  The
// host collects the records (bmg_debug_take; bmg_solve returns BMG_EBOUNDS).
// Test hook (bmg_debug_shrink(k)): every check uses extent - k, so the last k
// elements of each array count as outside; the accesses there are skipped and
// none leaves its array.  Without BMG_DEBUG every check is the constant true.
namespace bmg {
enum DbgSite {
  DBG_GS_STORE = 1,      // point Gauss-Seidel (row, checkerboard and tail kernels)
  DBG_STRIP_STORE,       // one-pass / two-pass strip kernels
  DBG_STRIP64_COPY,      // FP64 strip row copies (cp.async sources)
  DBG_RING_COPY,         // FP32 strip row copies (bulk-copy sources)
  DBG_RESTRICT_STORE,    // coarse right-hand side and iterate written by the restriction
  DBG_INTERP_STORE,      // interpolation + correction
  DBG_RESIDUAL_STORE,    // residual and the norm's partial sums
  DBG_LINE_STORE,        // line relaxation
  DBG_REFINE_STORE,      // refinement residual and update, FCG vectors
  DBG_PERIODIC,          // kernels of periodic hierarchies (stores and row copies)
  DBG_SETUP_STORE,       // setup: stencil preparation, 1/a_O, Dendy weights, Galerkin operator
  DBG_SITES
};
struct DbgRecord {
  int hit, site;
  long long index, extent;
};
}  // namespace bmg

#ifdef BMG_DEBUG
namespace bmg {
namespace {
__device__ DbgRecord g_dbg;          // one record per translation unit (no relocatable device code)
__device__ long long g_dbg_shrink;
}  // namespace
__device__ __forceinline__ bool dbg_in(int site, long long idx, long long lo, long long hi) {
  hi -= g_dbg_shrink;
  if (idx >= lo && idx < hi) return true;
  if (atomicCAS(&g_dbg.hit, 0, 1) == 0) {
    g_dbg.site = site;
    g_dbg.index = idx;
    g_dbg.extent = hi;
  }
  return false;
}
// Host side: each translation unit registers the accessors of its record
// (bmg_api.cu keeps the list).
struct DbgHooks {
  cudaError_t (*take)(DbgRecord* out, bool clear);
  cudaError_t (*shrink)(long long k);
};
void dbg_register(DbgHooks h);
namespace {
cudaError_t dbg_take_here(DbgRecord* out, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_dbg, sizeof(DbgRecord));
  if (e == cudaSuccess && clear && out->hit) {
    const DbgRecord zero = {0, 0, 0, 0};
    e = cudaMemcpyToSymbol(g_dbg, &zero, sizeof(DbgRecord));
  }
  return e;
}
cudaError_t dbg_shrink_here(long long k) { return cudaMemcpyToSymbol(g_dbg_shrink, &k, sizeof(long long)); }
struct DbgRegistrar {
  DbgRegistrar() { dbg_register(DbgHooks{dbg_take_here, dbg_shrink_here}); }
};
DbgRegistrar g_dbg_registrar;
}  // namespace
}  // namespace bmg
#define BMG_IN(site, idx, extent) ::bmg::dbg_in((site), (long long)(idx), 0LL, (long long)(extent))
#define BMG_IN_RANGE(site, idx, lo, hi) ::bmg::dbg_in((site), (long long)(idx), (long long)(lo), (long long)(hi))
#else
#define BMG_IN(site, idx, extent) true
#define BMG_IN_RANGE(site, idx, lo, hi) true
#endif

// Host-side launch helpers (implemented in bmg_api.cu).
namespace bmg {
void count_launch();
int set_error(int code, const char* fmt, ...);
int cuda_check(cudaError_t e, const char* what);
// cudaMalloc / cudaMallocHost of the setup calls, with the test hook for
// out-of-memory paths: when the environment variable BMG_FAIL_ALLOC holds
// k > 0, the k-th such allocation (counted from when the variable last changed)
// fails with cudaErrorMemoryAllocation without reaching the driver.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t host_malloc(void** p, size_t bytes);
}  // namespace bmg
