// C ABI of the BoxMG solver: the hierarchy object, its level schedule (the
// V-cycle of Fig. 1 enqueued level by level), CUDA-graph replay of one cycle,
// device-side convergence control, and the stateless single-step entry points.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "cycle_device.cuh"
#include "kernels.h"
#include "learned.h"
#include "periodic.h"

#include <nvtx3/nvToolsExt.h>

namespace bmg {

static thread_local char g_err[512] = "";
static thread_local long long* g_counter = nullptr;
static long long g_free_launches = 0;

void count_launch() {
  if (g_counter)
    ++*g_counter;
  else
    ++g_free_launches;
}

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

// A named NVTX range around an entry point's host work (tools that record NVTX
// show the library's setup, solve and timing calls as ranges; without such a
// tool the calls cost a few nanoseconds).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

namespace {
// Line smoothers: BMG_SMOOTHER_LINE (x-lines), _LINE_Y, _LINE_XY (alternating).
bool is_line(int smoother) { return smoother >= BMG_SMOOTHER_LINE && smoother <= BMG_SMOOTHER_LINE_XY; }
int line_dir(int smoother) {
  return smoother == BMG_SMOOTHER_LINE_Y ? LINE_Y : smoother == BMG_SMOOTHER_LINE_XY ? LINE_XY : LINE_X;
}

bool alloc_fault() {
  static std::mutex mu;
  static std::string seen;
  static long count = 0;
  const char* e = getenv("BMG_FAIL_ALLOC");
  const std::string v = e ? e : "";
  std::lock_guard<std::mutex> guard(mu);
  if (v != seen) {
    seen = v;
    count = 0;
  }
  const long k = v.empty() ? 0 : strtol(v.c_str(), nullptr, 10);
  return k > 0 && ++count == k;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (alloc_fault()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t host_malloc(void** p, size_t bytes) {
  if (alloc_fault()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

// ---- debug builds: the bounds-check records of every translation unit ----
#ifdef BMG_DEBUG
std::vector<DbgHooks>& dbg_hooks() {
  static std::vector<DbgHooks> v;
  return v;
}
void dbg_register(DbgHooks h) { dbg_hooks().push_back(h); }

// The first failed check recorded by any translation unit (hit = 0: none);
// clear: reset every record.
static cudaError_t dbg_collect(DbgRecord* first, bool clear) {
  *first = DbgRecord{0, 0, 0, 0};
  for (const DbgHooks& h : dbg_hooks()) {
    DbgRecord r;
    const cudaError_t e = h.take(&r, clear);
    if (e != cudaSuccess) return e;
    if (r.hit && !first->hit) *first = r;
  }
  return cudaSuccess;
}
#endif

const char* dbg_site_name(int site) {
  static const char* names[DBG_SITES] = {"none",
                                         "point Gauss-Seidel store",
                                         "strip sweep store",
                                         "FP64 strip row copy",
                                         "FP32 strip row copy",
                                         "restriction store",
                                         "interpolation store",
                                         "residual store",
                                         "line relaxation store",
                                         "refinement / FCG store",
                                         "periodic-sides kernel",
                                         "setup store"};
  return site >= 0 && site < DBG_SITES ? names[site] : "unknown";
}

// BMG_EBOUNDS when a debug build's bounds check failed since the last
// bmg_debug_take (the record stays until it is taken); BMG_OK otherwise and
// always in release builds.
int debug_check(const char* where) {
#ifdef BMG_DEBUG
  DbgRecord r;
  if (cudaDeviceSynchronize() != cudaSuccess || dbg_collect(&r, false) != cudaSuccess)
    return set_error(BMG_ECUDA, "%s: reading the debug bounds records failed", where);
  if (r.hit)
    return set_error(BMG_EBOUNDS, "%s: debug bounds check failed: %s, index %lld outside [0, %lld)", where,
                     dbg_site_name(r.site), r.index, r.extent);
#else
  (void)where;
#endif
  return BMG_OK;
}

// BMG_ETIMEOUT when a one-pass sweep gave up on its bulk copies since the last check.
int timeout_check(const char* where) {
  if (strip_timeouts()) return set_error(BMG_ETIMEOUT, "%s: a one-pass sweep timed out waiting for its copies", where);
  return debug_check(where);
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BMG_OK;
  if (e == cudaErrorMemoryAllocation) return set_error(BMG_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(BMG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void zero_ring(int n, double* r, cudaStream_t s);   // k_cycle.cu
int mlp_level0_interp(const void* m, int n, const double* st, double* ci, cudaStream_t s);   // learned_api.cu

}  // namespace bmg

using namespace bmg;

#define CK(call)                                     \
  do {                                               \
    int _rc = cuda_check((call), #call);             \
    if (_rc != BMG_OK) return _rc;                   \
  } while (0)

namespace {

struct Level {
  int n = 0, kind = 9;
  double* st = nullptr;   // O, W, S, SW, NW, D
  double* ci = nullptr;   // 8 interpolation planes toward level + 1
  double* x = nullptr;    // levels >= 1
  double* f = nullptr;
  bool bf16 = false;      // FP32 cycle reads BF16 off-diagonals on this level
  int cl64 = 0, cl32 = 0; // row-kernel cluster sizes chosen by the autotuner (0 = default)
  float* st32 = nullptr;  // O, W, S, SW, NW, D in FP32
  __nv_bfloat16* off16 = nullptr;
  float* od32 = nullptr;  // O32, D32 of a BF16 level
  float* ci32 = nullptr;
  float* x32 = nullptr;
  float* f32 = nullptr;
  int tile32 = -1;        // FP32 sweeps: -1 row kernel (in place), else tile shape of the one-pass kernel
  int pair32 = -1;        // >= 0: pairs of sweeps run as one two-sweep launch of this shape (needs tile32 >= 0)
  double* lcp = nullptr;  // line relaxation: elimination multipliers (FP64 cycle)
  float* lcp32 = nullptr; // the same for the FP32 cycle
  float* x32b = nullptr;  // second iterate of a tile-swept level (sweeps alternate x32 <-> x32b)
  int fused = 0;          // 1: the cycle's multiply-adds on this level are fused (BMG_ARITH_FUSED)
  int tile64 = -1;        // FP64 sweeps: -1 row kernel (in place), else shape of the FP64 one-pass kernel
  double* x64b = nullptr; // second iterate of an FP64 level swept by the one-pass kernel
  float* pk32 = nullptr;  // the FP32 / BF16 stencil packed per point (StencilView::pk)
  int pair_rr = 0;        // 1: the two pre-smoothing sweeps, the residual and the restriction in one pass
};

StencilView<double, double> view64(const Level& L) {
  size_t ps = plane_size(L.n);
  return {L.st, L.st + ps, L.st + 2 * ps, L.st + 3 * ps, L.st + 4 * ps, L.st + 5 * ps, L.n, L.n + 2, L.fused};
}
StencilView<float, float> view32(const Level& L) {
  size_t ps = plane_stride32(L.n);
  return {L.st32, L.st32 + ps, L.st32 + 2 * ps, L.st32 + 3 * ps, L.st32 + 4 * ps, L.st32 + 5 * ps,
          L.n,    L.n + 2,       L.fused,         L.pk32};
}
StencilView<float, __nv_bfloat16> viewbf(const Level& L) {
  size_t ps = plane_stride32(L.n);
  return {L.od32, L.off16, L.off16 + ps, L.off16 + 2 * ps, L.off16 + 3 * ps, L.od32 + ps, L.n, L.n + 2, L.fused,
          L.pk32};
}

}  // namespace

struct bmg_hierarchy {
  int n = 0, nlev = 0, precision = BMG_FP64, nu1 = 2, nu2 = 1, inner = 1, use_graph = 1, coarsest = 3, krylov = 0;
  int interp = BMG_INTERP_DENDY, interp_used = BMG_INTERP_DENDY;
  int smoother = BMG_SMOOTHER_AUTO;
  int arith = BMG_ARITH_ROUNDED;
  int fuse_restrict = BMG_FUSE_AUTO;
  const void* mlp = nullptr;
  double factor_learned = 0.0, factor_dendy = 0.0;
  double* kr = nullptr;   // flexible CG vectors r, z, p, q (FP64, (n+2)^2 each)
  std::vector<Level> lv;
  cudaStream_t user = nullptr;   // caller stream (ordering only)
  cudaStream_t ws = nullptr;     // internal non-blocking work stream
  cudaEvent_t ev = nullptr;
  double* Lfac = nullptr;        // coarsest Cholesky factor (m x m)
  double* work = nullptr;        // m x m factor workspace, then m doubles for substitutions
  int m = 0;
  double* partials = nullptr;
  int* err = nullptr;            // device error word of setup kernels
  Ctl* ctl = nullptr;            // device control block (hist sized for maxit_cap + 1)
  Ctl* ctl_host = nullptr;       // pinned mirror of the header
  int maxit_cap = 0;
  float* r32_user_dummy = nullptr;
  // graph of one cycle, keyed by the caller buffers it was captured with
  cudaGraphExec_t gexec = nullptr;
  const double* g_rhs = nullptr;
  double* g_x = nullptr;
  long long g_kernels = 0;
  long long launches = 0;
  struct Mark {
    int level, kernel, fp32;
    long long launches;
    cudaEvent_t a, b;
  };
  std::vector<Mark>* prof = nullptr;   // non-null while bmg_profile records
  int last_hist = 0;
  std::vector<double> hist;
  // level-fused tail: levels >= tail_l run in one launch (-1: none)
  int tail_l = -1;
  void* d_tail = nullptr;   // TailDesc<double> or TailDesc<float> in device memory
  // a batch member that borrows the operator arrays (stencils, weights, Cholesky
  // factor and its workspace) of another hierarchy and owns only its state
  bool shared_ops = false;
  // general sizes: the caller's grid nx x ny, embedded in the n x n level 0; the
  // solve runs on the embedded right-hand side and iterate (NULL when nx = ny = n)
  int nx = 0, ny = 0;
  double* fpad = nullptr;
  double* xpad = nullptr;
  // periodic sides: the hierarchy of periodic.cu (nlev stays 0, lv empty)
  PerHier* per = nullptr;
};

namespace {

struct CounterScope {
  long long* prev;
  explicit CounterScope(long long* c) : prev(g_counter) { g_counter = c; }
  ~CounterScope() { g_counter = prev; }
};

// Run one step's launches, bracketed by CUDA events when profiling.
template <class F>
void step(bmg_hierarchy* h, int level, int kernel, int fp32, F&& f) {
  if (!h->prof) {
    f();
    return;
  }
  bmg_hierarchy::Mark m{level, kernel, fp32, 0, nullptr, nullptr};
  cudaEventCreate(&m.a);
  cudaEventCreate(&m.b);
  cudaEventRecord(m.a, h->ws);
  long long before = h->launches;
  f();
  m.launches = h->launches - before;
  cudaEventRecord(m.b, h->ws);
  h->prof->push_back(m);
}

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return BMG_OK;
  CK(dev_malloc((void**)p, count * sizeof(T)));
  return BMG_OK;
}

// dalloc, zeroed on stream s; nothing stays allocated when either step fails.
template <typename T>
int dalloc_zero(T** p, size_t count, cudaStream_t s) {
  int rc = dalloc(p, count);
  if (!rc && count) rc = cuda_check(cudaMemsetAsync(*p, 0, count * sizeof(T), s), "cudaMemsetAsync");
  if (rc) {
    cudaFree(*p);
    *p = nullptr;
  }
  return rc;
}

// FP32 / BF16 level arrays: `planes` planes of level size n, plane_stride32(n)
// elements apart, with STRIP_GUARD zeroed elements before the first and after
// every plane; *p is the first plane (256-byte aligned).  Freed by gfree.
template <typename T>
int galloc(T** p, int n, int planes, cudaStream_t s) {
  *p = nullptr;
  const size_t count = STRIP_GUARD + planes * plane_stride32(n);
  T* raw = nullptr;
  if (int e = dalloc_zero(&raw, count, s)) return e;
  *p = raw + STRIP_GUARD;
  return BMG_OK;
}

template <typename T>
void gfree(T* p) {
  if (p) cudaFree(p - STRIP_GUARD);
}

void vcycle64(bmg_hierarchy* h, int l, double* x, const double* f, const int* done) {
  Level& L = h->lv[l];
  cudaStream_t s = h->ws;
  if (l == h->tail_l) {
    step(h, l, BMG_K_TAIL, 0,
         [&] { launch_tail<double>((const TailDesc<double>*)h->d_tail, 1, L.n, done, s, L.fused); });
    return;
  }
  if (l == h->nlev - 1) {
    step(h, l, BMG_K_COARSE, 0, [&] { launch_coarse_solve<double>(L.n, h->Lfac, f, x, h->work, done, s); });
    return;
  }
  auto v = view64(L);
  Level& C = h->lv[l + 1];
  // One-pass level: each sweep reads *cur and writes the other of x / x64b;
  // the interpolation writes the array from which nu2 sweeps end in x.
  double* cur = x;
  auto relax64 = [&](int sweeps) {
    if (is_line(h->smoother))
      step(h, l, BMG_K_RELAX, 0,
           [&] { launch_line<double, double>(v, L.kind, f, x, L.lcp, sweeps, line_dir(h->smoother), done, s); });
    else if (L.tile64 >= 0)
      for (int k = 0; k < sweeps; ++k) {
        double* nxt = cur == x ? L.x64b : x;
        step(h, l, BMG_K_RELAX, 0, [&] { launch_gs_tile64(v, f, cur, nxt, L.tile64, done, s); });
        cur = nxt;
      }
    else
      step(h, l, BMG_K_RELAX, 0, [&] { launch_gs(v, L.kind, f, x, sweeps, done, s, L.cl64); });
  };
  relax64(h->nu1);
  step(h, l, BMG_K_RESID_RESTRICT, 0, [&] { launch_resid_restrict(v, L.kind, L.ci, cur, f, C.f, C.x, done, s); });
  vcycle64(h, l + 1, C.x, C.f, done);
  double* dst = L.tile64 >= 0 && (h->nu2 & 1) ? L.x64b : x;
  step(h, l, BMG_K_INTERP, 0, [&] { launch_interp_to<double>(L.n, L.ci, C.x, cur, dst, done, s, L.fused); });
  cur = dst;
  relax64(h->nu2);
}

// Sweeps of an FP32 level.  Row kernel: in place on x32.  One-pass tile kernel:
// each sweep reads *cur and writes the other of x32 / x32b, and *cur follows.
template <typename S>
void relax32(bmg_hierarchy* h, const StencilView<float, S>& v, int l, int sweeps, float** cur, const int* done) {
  Level& L = h->lv[l];
  if (is_line(h->smoother)) {
    step(h, l, BMG_K_RELAX, 1, [&] {
      launch_line<float, S>(v, L.kind, (const float*)L.f32, L.x32, L.lcp32, sweeps, line_dir(h->smoother), done,
                            h->ws);
    });
    return;
  }
  if (L.tile32 < 0) {
    step(h, l, BMG_K_RELAX, 1,
         [&] { launch_gs(v, L.kind, (const float*)L.f32, L.x32, sweeps, done, h->ws, L.cl32); });
    return;
  }
  const int pairs = L.pair32 >= 0 ? sweeps / 2 : 0;
  if (pairs)
    step(h, l, BMG_K_RELAX_PAIR, 1, [&] {
      for (int k = 0; k < pairs; ++k) {
        float* dst = *cur == L.x32 ? L.x32b : L.x32;
        launch_gs_pair(v, (const float*)L.f32, (const float*)*cur, dst, L.pair32, done, h->ws);
        *cur = dst;
      }
    });
  if (sweeps > 2 * pairs)
    step(h, l, BMG_K_RELAX, 1, [&] {
      for (int k = 2 * pairs; k < sweeps; ++k) {
        float* dst = *cur == L.x32 ? L.x32b : L.x32;
        launch_gs_tile(v, (const float*)L.f32, (const float*)*cur, dst, L.tile32, done, h->ws);
        *cur = dst;
      }
    });
}

// Launches of `sweeps` sweeps on a one-pass level (each moves the iterate to the other array).
int sweep_launches(const Level& L, int sweeps) { return L.pair32 >= 0 ? sweeps / 2 + sweeps % 2 : sweeps; }

template <typename S>
void restrict32(bmg_hierarchy* h, const StencilView<float, S>& v, int l, const float* x, const int* done) {
  Level& L = h->lv[l];
  Level& C = h->lv[l + 1];
  step(h, l, BMG_K_RESID_RESTRICT, 1,
       [&] { launch_resid_restrict(v, L.kind, (const float*)L.ci32, x, (const float*)L.f32, C.f32, C.x32, done,
                                   h->ws); });
}

// The FP32 cycle leaves every level's result in x32.  On a tile-swept level the
// interpolation writes the array from which nu2 alternating sweeps end in x32.
void vcycle32(bmg_hierarchy* h, int l, const int* done) {
  Level& L = h->lv[l];
  cudaStream_t s = h->ws;
  if (l == h->tail_l) {
    step(h, l, BMG_K_TAIL, 1,
         [&] { launch_tail<float>((const TailDesc<float>*)h->d_tail, 1, L.n, done, s, L.fused); });
    return;
  }
  if (l == h->nlev - 1) {
    step(h, l, BMG_K_COARSE, 1,
         [&] { launch_coarse_solve<float>(L.n, h->Lfac, (const float*)L.f32, L.x32, h->work, done, s); });
    return;
  }
  Level& C = h->lv[l + 1];
  float* cur = L.x32;
  auto pre = [&](const auto& v) {
    if (L.pair_rr && h->nu1 == 2) {   // temporal blocking: sweeps, residual and restriction in one pass
      float* dst = cur == L.x32 ? L.x32b : L.x32;
      step(h, l, BMG_K_PAIR_RESTRICT, 1, [&] {
        if (!launch_gs_pair_restrict(v, (const float*)L.f32, (const float*)cur, dst, (const float*)L.ci32, C.f32,
                                     C.x32, L.pair32 == 1 ? 1 : 0, done, s)) {
          launch_gs_pair(v, (const float*)L.f32, (const float*)cur, dst, L.pair32, done, s);
          launch_resid_restrict(v, L.kind, (const float*)L.ci32, (const float*)dst, (const float*)L.f32, C.f32,
                                C.x32, done, s);
        }
      });
      cur = dst;
      return;
    }
    relax32(h, v, l, h->nu1, &cur, done);
    restrict32(h, v, l, cur, done);
  };
  if (L.bf16)
    pre(viewbf(L));
  else
    pre(view32(L));
  vcycle32(h, l + 1, done);
  float* dst = L.tile32 >= 0 && (sweep_launches(L, h->nu2) & 1) ? L.x32b : L.x32;
  step(h, l, BMG_K_INTERP, 1, [&] { launch_interp_to<float>(L.n, L.ci32, C.x32, cur, dst, done, s, L.fused); });
  cur = dst;
  if (L.bf16)
    relax32(h, viewbf(L), l, h->nu2, &cur, done);
  else
    relax32(h, view32(L), l, h->nu2, &cur, done);
}

// Device milliseconds of fn(): the fastest of three timed calls after one
// untimed call (one sample alone lets noise decide between close candidates).
template <typename F>
int time_call(cudaStream_t s, F&& fn, float* ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  fn();
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    float t = 0;
    cudaEventRecord(e0, s);
    fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t, e0, e1);
    best = t < best ? t : best;
  }
  *ms = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  return BMG_OK;
}

// ---- the autotuner's record file ----------------------------------------------------
// With the environment variable BMG_TUNE_CACHE naming a file, every tuner
// decision is appended to it as one line
//   <device> <tuner key> <count> <value 1> ... <value count> <best ms>
// and a decision found there for this kind of device is reused instead of
// timed again, so a later process skips the timing.  Every candidate of every
// tuner computes the same bits, so a record changes only the speed; records
// whose values are out of range for their tuner are ignored.
struct TuneRecord {
  std::vector<int> v;
  float ms = 0.0f;
};

std::string device_tag() {
  static std::string tag;
  if (tag.empty()) {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
      tag = prop.name;
      for (char& c : tag)
        if (c == ' ') c = '_';
      tag += "/sm" + std::to_string(prop.multiProcessorCount);
    } else {
      tag = "unknown";
    }
  }
  return tag;
}

struct TuneFile {
  std::mutex mu;
  std::string path;
  std::map<std::string, TuneRecord> recs;
};

TuneFile& tune_file() {
  static TuneFile tf;
  return tf;
}

// (Re)load the records when BMG_TUNE_CACHE names another file than last time.
// Caller holds the lock.
void tune_file_sync(TuneFile& tf) {
  const char* e = getenv("BMG_TUNE_CACHE");
  const std::string path = e ? e : "";
  if (path == tf.path) return;
  tf.path = path;
  tf.recs.clear();
  if (path.empty()) return;
  FILE* fp = fopen(path.c_str(), "r");
  if (!fp) return;
  char line[512];
  while (fgets(line, sizeof line, fp)) {
    char dev[128], key[256];
    int count = 0, used = 0;
    if (sscanf(line, "%127s %255s %d%n", dev, key, &count, &used) != 3 || count < 1 || count > 8) continue;
    TuneRecord r;
    const char* q = line + used;
    bool ok = true;
    for (int k = 0; k < count && ok; ++k) {
      int val = 0, adv = 0;
      ok = sscanf(q, "%d%n", &val, &adv) == 1;
      r.v.push_back(val);
      q += adv;
    }
    if (!ok || sscanf(q, "%f", &r.ms) != 1) continue;
    tf.recs[std::string(dev) + " " + key] = r;
  }
  fclose(fp);
}

bool tune_file_get(const std::string& key, size_t count, TuneRecord* out) {
  TuneFile& tf = tune_file();
  std::lock_guard<std::mutex> guard(tf.mu);
  tune_file_sync(tf);
  if (tf.path.empty()) return false;
  auto it = tf.recs.find(device_tag() + " " + key);
  if (it == tf.recs.end() || it->second.v.size() != count) return false;
  *out = it->second;
  return true;
}

void tune_file_put(const std::string& key, const TuneRecord& r) {
  TuneFile& tf = tune_file();
  std::lock_guard<std::mutex> guard(tf.mu);
  tune_file_sync(tf);
  if (tf.path.empty()) return;
  tf.recs[device_tag() + " " + key] = r;
  FILE* fp = fopen(tf.path.c_str(), "a");
  if (!fp) return;
  fprintf(fp, "%s %s %zu", device_tag().c_str(), key.c_str(), r.v.size());
  for (int x : r.v) fprintf(fp, " %d", x);
  fprintf(fp, " %.6g\n", r.ms);
  fclose(fp);
}

std::string tune_key(const char* tuner, std::initializer_list<int> fields) {
  std::string k = tuner;
  for (int f : fields) k += ":" + std::to_string(f);
  return k;
}

// Autotuner of the solo hierarchy.  For every 9-point level with n >= 127 it
// times two Gauss-Seidel sweeps on scratch iterates with the level's real
// stencil: the row kernel for each admissible cluster size (1, 2, 4, 8 CTAs
// per row, at least a warp of pairs per CTA) and, for FP32 levels, the
// one-pass tile kernel for each tile shape; the fastest is kept.  Every
// candidate computes the same bits; only the speed differs.  Results are
// cached per (n, compute type, storage type, arithmetic mode) for the life of
// the process.
template <typename T, typename S>
int tune_rows(const StencilView<T, S>& v, cudaStream_t s, int* best_out, float* ms_out = nullptr) {
  static std::map<std::tuple<int, int, int, int>, std::pair<int, float>> cache;
  auto key = std::make_tuple(v.n, (int)sizeof(T), (int)sizeof(S), v.fused);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *best_out = it->second.first;
    if (ms_out) *ms_out = it->second.second;
    return BMG_OK;
  }
  const int base = rows_cluster<T>(v.n);
  const std::string fkey = tune_key("rows", {v.n, (int)sizeof(T), (int)sizeof(S), v.fused});
  TuneRecord fr;
  if (tune_file_get(fkey, 1, &fr)) {
    const int cl = fr.v[0];
    if ((cl == base || (cl > base && cl <= 8 && (cl & (cl - 1)) == 0 && ((v.n + 1) / 2 + cl - 1) / cl >= 32))) {
      cache[key] = {cl, fr.ms};
      *best_out = cl;
      if (ms_out) *ms_out = fr.ms;
      return BMG_OK;
    }
  }
  size_t ps = plane_size(v.n);
  T* scratch = nullptr;
  if (int e = dalloc_zero(&scratch, 2 * ps, s)) return e;
  float best = 1e30f;
  int best_cl = base, rc = BMG_OK;
  for (int cl = base; cl <= 8 && !rc; cl *= 2) {
    if (cl > base && ((v.n + 1) / 2 + cl - 1) / cl < 32) break;
    float ms = 0;
    rc = time_call(s, [&] { launch_gs(v, 9, (const T*)(scratch + ps), scratch, 2, (const int*)nullptr, s, cl); }, &ms);
    ms *= 0.5f;   // per sweep
    if (ms < best) {
      best = ms;
      best_cl = cl;
    }
  }
  cudaFree(scratch);
  if (rc) return rc;
  cache[key] = {best_cl, best};
  tune_file_put(fkey, TuneRecord{{best_cl}, best});
  *best_out = best_cl;
  if (ms_out) *ms_out = best;
  return BMG_OK;
}

template <typename S>
int tune_tile(const StencilView<float, S>& v, cudaStream_t s, int* best_out, float* ms_out) {
  static std::map<std::tuple<int, int, int>, std::pair<int, float>> cache;
  auto key = std::make_tuple(v.n, (int)sizeof(S), v.fused);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *best_out = it->second.first;
    *ms_out = it->second.second;
    return BMG_OK;
  }
  const std::string fkey = tune_key("tile", {v.n, (int)sizeof(S), v.fused});
  TuneRecord fr;
  if (tune_file_get(fkey, 1, &fr) && fr.v[0] >= 0 && fr.v[0] < GS_TILE_SHAPES) {
    cache[key] = {fr.v[0], fr.ms};
    *best_out = fr.v[0];
    *ms_out = fr.ms;
    return BMG_OK;
  }
  size_t ps = plane_stride32(v.n);
  float* scratch = nullptr;   // x, x', f laid out like a level's arrays
  int rc0 = galloc(&scratch, v.n, 3, s);
  if (rc0) return rc0;
  const float* f = scratch + 2 * ps;
  float best = 1e30f;
  int best_shape = 0, rc = BMG_OK;
  for (int shape = 0; shape < GS_TILE_SHAPES && !rc; ++shape) {
    float ms = 0;
    rc = time_call(s, [&] {
      launch_gs_tile(v, f, scratch, scratch + ps, shape, (const int*)nullptr, s);
      launch_gs_tile(v, f, scratch + ps, scratch, shape, (const int*)nullptr, s);
    }, &ms);
    ms *= 0.5f;   // per sweep
    if (ms < best) {
      best = ms;
      best_shape = shape;
    }
  }
  gfree(scratch);
  if (!rc && strip_timeouts()) rc = set_error(BMG_ETIMEOUT, "one-pass sweep: bulk copies did not complete");
  if (rc) return rc;
  cache[key] = {best_shape, best};
  tune_file_put(fkey, TuneRecord{{best_shape}, best});
  *best_out = best_shape;
  *ms_out = best;
  return BMG_OK;
}

template <typename S>
int tune_pair(const StencilView<float, S>& v, cudaStream_t s, int* best_out, float* ms_out) {
  static std::map<std::tuple<int, int, int>, std::pair<int, float>> cache;
  auto key = std::make_tuple(v.n, (int)sizeof(S), v.fused);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *best_out = it->second.first;
    *ms_out = it->second.second;
    return BMG_OK;
  }
  const std::string fkey = tune_key("pair", {v.n, (int)sizeof(S), v.fused});
  TuneRecord fr;
  if (tune_file_get(fkey, 1, &fr) && fr.v[0] >= -1 && fr.v[0] < GS_PAIR_SHAPES) {
    cache[key] = {fr.v[0], fr.ms};
    *best_out = fr.v[0];
    *ms_out = fr.ms;
    return BMG_OK;
  }
  size_t ps = plane_stride32(v.n);
  float* scratch = nullptr;   // x, x', f laid out like a level's arrays
  int rc = galloc(&scratch, v.n, 3, s);
  if (rc) return rc;
  const float* f = scratch + 2 * ps;
  float best = 1e30f;
  int best_shape = -1;
  for (int shape = 0; shape < GS_PAIR_SHAPES && !rc; ++shape) {
    float ms = 0;
    bool launched = true;
    rc = time_call(s, [&] {
      launched = launch_gs_pair(v, f, scratch, scratch + ps, shape, (const int*)nullptr, s) &&
                 launch_gs_pair(v, f, scratch + ps, scratch, shape, (const int*)nullptr, s);
    }, &ms);
    ms *= 0.5f;   // per pair of sweeps
    if (launched && ms < best) {
      best = ms;
      best_shape = shape;
    }
  }
  gfree(scratch);
  if (!rc && strip_timeouts()) rc = set_error(BMG_ETIMEOUT, "two-sweep pass: bulk copies did not complete");
  if (rc) return rc;
  cache[key] = {best_shape, best};
  tune_file_put(fkey, TuneRecord{{best_shape}, best});
  *best_out = best_shape;
  *ms_out = best;
  return BMG_OK;
}

// Row kernel vs one-pass tile kernel for an FP32 level; allocates the second
// iterate when the tile kernel wins, and then also weighs one two-sweep pass
// against two one-pass sweeps.
template <typename S>
int tune_level32(Level& L, const StencilView<float, S>& v, cudaStream_t s) {
  float ms_rows = 0, ms_tile = 0;
  int shape = 0, rc = tune_rows(v, s, &L.cl32, &ms_rows);
  if (!rc) rc = tune_tile(v, s, &shape, &ms_tile);
  if (rc) return rc;
  if (ms_tile < ms_rows) {
    if ((rc = galloc(&L.x32b, L.n, 1, s))) return rc;
    L.tile32 = shape;
    int pshape = -1;
    float ms_pair = 0;
    if ((rc = tune_pair(v, s, &pshape, &ms_pair))) return rc;
    if (pshape >= 0 && ms_pair < 2.0f * ms_tile) L.pair32 = pshape;
  }
  return BMG_OK;
}

// FP64 one-pass kernel: each shape timed over two sweeps on scratch iterates.
int tune_tile64(const StencilView<double, double>& v, cudaStream_t s, int* best_out, float* ms_out) {
  static std::map<std::pair<int, int>, std::pair<int, float>> cache;
  auto key = std::make_pair(v.n, v.fused);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *best_out = it->second.first;
    *ms_out = it->second.second;
    return BMG_OK;
  }
  const std::string fkey = tune_key("tile64", {v.n, v.fused});
  TuneRecord fr;
  if (tune_file_get(fkey, 1, &fr) && fr.v[0] >= 0 && fr.v[0] < GS_TILE64_SHAPES) {
    cache[key] = {fr.v[0], fr.ms};
    *best_out = fr.v[0];
    *ms_out = fr.ms;
    return BMG_OK;
  }
  const size_t ps = plane_size(v.n);
  double* scratch = nullptr;   // x, x', f
  if (int e = dalloc_zero(&scratch, 3 * ps, s)) return e;
  const double* f = scratch + 2 * ps;
  int best_shape = 0, rc = BMG_OK;
  float best = 1e30f;
  for (int shape = 0; shape < GS_TILE64_SHAPES && !rc; ++shape) {
    float ms = 0;
    rc = time_call(s, [&] {
      launch_gs_tile64(v, f, scratch, scratch + ps, shape, (const int*)nullptr, s);
      launch_gs_tile64(v, f, scratch + ps, scratch, shape, (const int*)nullptr, s);
    }, &ms);
    if (ms * 0.5f < best) {
      best = ms * 0.5f;
      best_shape = shape;
    }
  }
  cudaFree(scratch);
  if (rc) return rc;
  cache[key] = {best_shape, best};
  tune_file_put(fkey, TuneRecord{{best_shape}, best});
  *best_out = best_shape;
  *ms_out = best;
  return BMG_OK;
}

// Row kernel vs the one-pass kernel for an FP64 level (the second iterate is
// allocated when the one-pass kernel wins).
int tune_level64(Level& L, cudaStream_t s) {
  float ms_rows = 0, ms_tile = 0;
  int shape = 0, rc = tune_rows(view64(L), s, &L.cl64, &ms_rows);
  if (!rc) rc = tune_tile64(view64(L), s, &shape, &ms_tile);
  if (rc) return rc;
  if (ms_tile < ms_rows) {
    if ((rc = dalloc_zero(&L.x64b, plane_size(L.n), s))) return rc;
    L.tile64 = shape;
  }
  return BMG_OK;
}

// Level-fused tail of the solo hierarchy: the first level l (>= 1 for FP64, and
// not a BF16 level) with n <= tail_max_n and at least one level below it.
template <typename T>
int build_tail(bmg_hierarchy* h, int lmin) {
  int lt = -1;
  for (int l = lmin; l + 1 < h->nlev; ++l)
    if (h->lv[l].n <= tail_max_n<T>() && !h->lv[l].bf16) {
      lt = l;
      break;
    }
  if (lt < 0 || h->nlev - lt > TAIL_LEVELS) return BMG_OK;
  TailDesc<T> d{};
  d.nlev = h->nlev - lt;
  d.nu1 = h->nu1;
  d.nu2 = h->nu2;
  d.top_kind = h->lv[lt].kind;
  d.done = nullptr;
  for (int k = 0; k < d.nlev; ++k) {
    Level& L = h->lv[lt + k];
    Level* C = lt + k + 1 < h->nlev ? &h->lv[lt + k + 1] : nullptr;
    if constexpr (sizeof(T) == 8)
      d.lv[k] = LevelDesc<double, double>{view64(L), L.ci, L.x, L.f, C ? C->x : nullptr, C ? C->f : nullptr,
                                          nullptr, h->Lfac, h->work};
    else
      d.lv[k] = LevelDesc<float, float>{view32(L), L.ci32, L.x32, L.f32, C ? C->x32 : nullptr,
                                        C ? C->f32 : nullptr, nullptr, h->Lfac, h->work};
  }
  CK(dev_malloc((void**)&h->d_tail, sizeof(d)));
  CK(cudaMemcpy(h->d_tail, &d, sizeof(d), cudaMemcpyHostToDevice));
  h->tail_l = lt;
  return BMG_OK;
}

// BMG_SMOOTHER_TILE + s: the tile kernel with shape s on every 9-point level
// but the coarsest (levels that end up in the level-fused tail ignore it); on
// an FP64 hierarchy the FP64 one-pass kernel with shape s (s < 4).
int force_tile(bmg_hierarchy* h) {
  for (int l = 0; l + 1 < h->nlev; ++l) {
    Level& L = h->lv[l];
    if (L.kind != 9) continue;
    if (h->precision == BMG_FP64) {
      if (int rc = dalloc_zero(&L.x64b, plane_size(L.n), h->ws)) return rc;
      L.tile64 = h->smoother - BMG_SMOOTHER_TILE;
      continue;
    }
    int rc = galloc(&L.x32b, L.n, 1, h->ws);
    if (rc) return rc;
    if (h->smoother >= BMG_SMOOTHER_PAIR) {
      L.tile32 = 3;
      L.pair32 = h->smoother - BMG_SMOOTHER_PAIR;
    } else {
      L.tile32 = h->smoother - BMG_SMOOTHER_TILE;
    }
  }
  return BMG_OK;
}

// BMG_SMOOTHER_LINE / _LINE_Y / _LINE_XY: the multiplier scratch of every relaxed level.
int alloc_line(bmg_hierarchy* h) {
  for (int l = 0; l + 1 < h->nlev; ++l) {
    Level& L = h->lv[l];
    int rc = h->precision == BMG_FP64 ? dalloc(&L.lcp, plane_size(L.n)) : galloc(&L.lcp32, L.n, 1, h->ws);
    if (rc) return rc;
  }
  return BMG_OK;
}

// The tuners' result caches are process-wide; setups running on several host
// threads take turns through this lock.
std::mutex& tune_lock() {
  static std::mutex m;
  return m;
}

int autotune_solo(bmg_hierarchy* h) {
  std::lock_guard<std::mutex> guard(tune_lock());
  for (int l = 0; l + 1 < h->nlev; ++l) {
    Level& L = h->lv[l];
    if (L.kind != 9 || L.n < 127) continue;
    int rc = BMG_OK;
    if (h->precision == BMG_FP64)
      rc = h->smoother == BMG_SMOOTHER_AUTO ? tune_level64(L, h->ws)
           : L.tile64 >= 0                ? BMG_OK
                                          : tune_rows(view64(L), h->ws, &L.cl64);
    else if (h->smoother != BMG_SMOOTHER_AUTO)
      rc = L.tile32 >= 0 ? BMG_OK : L.bf16 ? tune_rows(viewbf(L), h->ws, &L.cl32) : tune_rows(view32(L), h->ws, &L.cl32);
    else if (L.bf16)
      rc = tune_level32(L, viewbf(L), h->ws);
    else
      rc = tune_level32(L, view32(L), h->ws);
    if (rc) return rc;
  }
  return BMG_OK;
}

// A level whose two pre-smoothing sweeps run as one two-sweep pass: the pass
// that also forms the residual and restricts it (temporal blocking) against
// the two-sweep pass plus the separate residual + restriction, timed on
// scratch iterates with the level's stencil; the coarse level's right-hand
// side and iterate are written by both (they are rewritten every cycle).
template <typename S>
int tune_pair_restrict(Level& L, Level& C, const StencilView<float, S>& v, cudaStream_t s) {
  const std::string fkey = tune_key("pair_restrict", {v.n, (int)sizeof(S), v.fused, L.pair32});
  TuneRecord fr;
  if (tune_file_get(fkey, 1, &fr) && (fr.v[0] == 0 || fr.v[0] == 1)) {
    L.pair_rr = fr.v[0];
    return BMG_OK;
  }
  size_t ps = plane_stride32(v.n);
  float* scratch = nullptr;   // x, x', f laid out like a level's arrays
  int rc = galloc(&scratch, v.n, 3, s);
  if (rc) return rc;
  const float* f = scratch + 2 * ps;
  // the two candidates timed alternately, twice each (the clocks may still be
  // rising during setup), the faster time of each kept
  float ms_sep = 1e30f, ms_fused = 1e30f;
  bool fused_ok = true;
  for (int round = 0; round < 2 && !rc; ++round) {
    float ms = 0;
    rc = time_call(s, [&] {
      launch_gs_pair(v, f, scratch, scratch + ps, L.pair32, (const int*)nullptr, s);
      launch_resid_restrict(v, L.kind, (const float*)L.ci32, (const float*)(scratch + ps), f, C.f32, C.x32,
                            (const int*)nullptr, s);
    }, &ms);
    ms_sep = std::min(ms_sep, ms);
    if (!rc)
      rc = time_call(s, [&] {
        fused_ok = launch_gs_pair_restrict(v, f, scratch, scratch + ps, (const float*)L.ci32, C.f32, C.x32,
                                           L.pair32 == 1 ? 1 : 0, (const int*)nullptr, s);
      }, &ms);
    ms_fused = std::min(ms_fused, ms);
  }
  gfree(scratch);
  if (!rc && strip_timeouts()) rc = set_error(BMG_ETIMEOUT, "two-sweep pass: bulk copies did not complete");
  if (rc) return rc;
  L.pair_rr = fused_ok && ms_fused < ms_sep ? 1 : 0;
  tune_file_put(fkey, TuneRecord{{L.pair_rr}, L.pair_rr ? ms_fused : ms_sep});
  return BMG_OK;
}

// Levels outside the level-fused tail whose two pre-smoothing sweeps are one
// two-sweep pass (nu1 = 2): the fused pass when forced, or when the tuner
// finds it faster (graphs on).
int choose_pair_restrict(bmg_hierarchy* h) {
  if (h->precision == BMG_FP64 || h->nu1 != 2 || h->fuse_restrict == BMG_FUSE_OFF) return BMG_OK;
  if (h->fuse_restrict == BMG_FUSE_AUTO && !h->use_graph) return BMG_OK;
  std::lock_guard<std::mutex> guard(tune_lock());
  for (int l = 0; l + 1 < h->nlev; ++l) {
    if (h->tail_l >= 0 && l >= h->tail_l) break;
    Level& L = h->lv[l];
    if (L.kind != 9 || L.tile32 < 0 || L.pair32 < 0) continue;
    if (h->fuse_restrict == BMG_FUSE_ON) {
      L.pair_rr = 1;
      continue;
    }
    int rc = L.bf16 ? tune_pair_restrict(L, h->lv[l + 1], viewbf(L), h->ws)
                    : tune_pair_restrict(L, h->lv[l + 1], view32(L), h->ws);
    if (rc) return rc;
  }
  return BMG_OK;
}

// One iteration of the solve loop: a V-cycle (or a refinement step) followed by
// the residual norm and the convergence test, all on the device.
// bmg_profile's brackets for the periodic hierarchy's steps (the marks of step()).
void per_mark_begin(void* ctx, int level, int kernel) {
  bmg_hierarchy* h = (bmg_hierarchy*)ctx;
  bmg_hierarchy::Mark m{level, kernel, 0, h->launches, nullptr, nullptr};
  cudaEventCreate(&m.a);
  cudaEventCreate(&m.b);
  cudaEventRecord(m.a, h->ws);
  h->prof->push_back(m);
}

void per_mark_end(void* ctx) {
  bmg_hierarchy* h = (bmg_hierarchy*)ctx;
  bmg_hierarchy::Mark& m = h->prof->back();
  m.launches = h->launches - m.launches;
  cudaEventRecord(m.b, h->ws);
}

void enqueue_iteration(bmg_hierarchy* h, const double* rhs, double* x) {
  if (h->per) {
    PerMarks mk;
    if (h->prof) {
      mk.ctx = h;
      mk.begin = per_mark_begin;
      mk.end = per_mark_end;
    }
    per_enqueue_iteration(h->per, rhs, x, h->partials, h->ctl, h->ws, h->prof ? &mk : nullptr);
    return;
  }
  const int* done = &h->ctl->done;
  Level& L0 = h->lv[0];
  int np = 0;
  if (h->krylov == BMG_KRYLOV_FCG) {
    size_t ps = plane_size(L0.n);
    double *r = h->kr, *z = h->kr + ps, *pv = h->kr + 2 * ps, *q = h->kr + 3 * ps;
    bool mixed = h->precision != BMG_FP64;
    if (mixed)
      for (int c = 0; c < h->inner; ++c) vcycle32(h, 0, done);
    else
      vcycle64(h, 0, z, r, done);
    step(h, 0, BMG_K_FCG, 0, [&] {
      launch_fcg_step(view64(L0), L0.kind, x, r, mixed ? nullptr : z, mixed ? L0.x32 : nullptr, pv, q,
                      mixed ? L0.f32 : nullptr, mixed ? L0.x32 : nullptr, mixed ? nullptr : z, h->partials, h->ctl,
                      h->ws, nullptr, nullptr);
    });
    np = L0.n < norm_partials_max() ? L0.n : norm_partials_max();
  } else if (h->precision == BMG_FP64) {
    vcycle64(h, 0, x, rhs, done);
    step(h, 0, BMG_K_NORM, 0, [&] {
      np = launch_residual(view64(L0), L0.kind, (const double*)x, rhs, (double*)nullptr, h->partials, done, h->ws);
    });
  } else {
    for (int c = 0; c < h->inner; ++c) vcycle32(h, 0, done);
    step(h, 0, BMG_K_IR_UPDATE, 0, [&] { launch_ir_update(L0.n, x, L0.x32, h->ctl, h->ws); });
    step(h, 0, BMG_K_IR_RESIDUAL, 0, [&] {
      np = launch_ir_residual(view64(L0), L0.kind, x, rhs, L0.f32, L0.x32, h->partials, h->ctl, h->ws);
    });
  }
  step(h, 0, BMG_K_FINALIZE, 0, [&] { launch_norm_finalize(h->partials, np, h->ctl, 1, nullptr, h->ws); });
}

int enqueue_initial(bmg_hierarchy* h, const double* rhs, double* x) {
  if (h->per) {
    per_enqueue_initial(h->per, rhs, x, h->partials, h->ctl, h->ws);
    return BMG_OK;
  }
  Level& L0 = h->lv[0];
  if (h->krylov == BMG_KRYLOV_FCG) {
    size_t ps = plane_size(L0.n);
    bool mixed = h->precision != BMG_FP64;
    int np = launch_fcg_init(view64(L0), L0.kind, x, rhs, h->kr, mixed ? nullptr : h->kr + ps,
                             mixed ? L0.f32 : nullptr, mixed ? L0.x32 : nullptr, h->partials, h->ctl, h->ws);
    launch_norm_finalize(h->partials, np, h->ctl, 0, nullptr, h->ws);
  } else if (h->precision == BMG_FP64) {
    int np = launch_residual(view64(L0), L0.kind, x, rhs, (double*)nullptr, h->partials, (const int*)nullptr, h->ws);
    launch_norm_finalize(h->partials, np, h->ctl, 0, nullptr, h->ws);
  } else {
    int np = launch_ir_residual(view64(L0), L0.kind, x, rhs, L0.f32, L0.x32, h->partials, h->ctl, h->ws);
    launch_norm_finalize(h->partials, np, h->ctl, 0, nullptr, h->ws);
  }
  return BMG_OK;
}

int capture_graph(bmg_hierarchy* h, const double* rhs, double* x) {
  if (h->gexec && h->g_rhs == rhs && h->g_x == x) return BMG_OK;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->ws, cudaStreamCaptureModeThreadLocal));
  long long before = h->launches;
  enqueue_iteration(h, rhs, x);
  h->g_kernels = h->launches - before;
  h->launches = before;
  CK(cudaStreamEndCapture(h->ws, &g));
  cudaError_t e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  h->g_rhs = rhs;
  h->g_x = x;
  return BMG_OK;
}

int order_after_user(bmg_hierarchy* h) {
  CK(cudaEventRecord(h->ev, h->user));
  CK(cudaStreamWaitEvent(h->ws, h->ev, 0));
  return BMG_OK;
}

int ensure_ctl(bmg_hierarchy* h, int maxit) {
  if (maxit <= h->maxit_cap && h->ctl) return BMG_OK;
  if (h->ctl) cudaFree(h->ctl);
  h->ctl = nullptr;
  int cap = maxit < 64 ? 64 : maxit;
  CK(dev_malloc((void**)&h->ctl, sizeof(Ctl) + sizeof(double) * (size_t)(cap + 1)));
  h->maxit_cap = cap;
  if (h->gexec) {   // the graph holds the old control block address
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return BMG_OK;
}

void free_level(Level& L, bool shared_ops = false) {
  if (shared_ops) {   // borrowed operator arrays stay with their owner
    L.st = nullptr;
    L.ci = nullptr;
    L.st32 = nullptr;
    L.off16 = nullptr;
    L.od32 = nullptr;
    L.ci32 = nullptr;
    L.pk32 = nullptr;
  }
  cudaFree(L.st);
  cudaFree(L.ci);
  cudaFree(L.x);
  cudaFree(L.f);
  cudaFree(L.lcp);
  gfree(L.lcp32);
  gfree(L.st32);
  gfree(L.off16);
  gfree(L.od32);
  gfree(L.pk32);
  cudaFree(L.ci32);
  gfree(L.x32);
  gfree(L.x32b);
  gfree(L.f32);
  cudaFree(L.x64b);
  L = Level{};
}

bool is_level_size(int n) { return n >= 3 && ((n + 1) & n) == 0; }

// The smallest n = 2^m - 1 >= max(nx, ny, 3): the level-0 size of an nx x ny problem.
int embed_size(int nx, int ny) {
  int n = 3;
  while (n < nx || n < ny) n = 2 * n + 1;
  return n;
}

int setup_impl(bmg_hierarchy* h, const bmg_stencil* A, int n, const bmg_opts* o) {
  cudaStream_t s = h->ws;
  // level sizes
  std::vector<int> sizes{n};
  while (sizes.back() > h->coarsest) sizes.push_back((sizes.back() - 1) / 2);
  h->nlev = (int)sizes.size();
  h->lv.resize(h->nlev);
  int rc;
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lv[l];
    L.n = sizes[l];
    L.kind = l == 0 ? A->kind : 9;
    L.fused = h->arith == BMG_ARITH_FUSED;
    size_t ps = plane_size(L.n);
    if ((rc = dalloc(&L.st, 6 * ps))) return rc;
    if (l + 1 < h->nlev)
      if ((rc = dalloc(&L.ci, 8 * plane_size(sizes[l + 1])))) return rc;
    if (l > 0) {
      if ((rc = dalloc(&L.x, ps))) return rc;
      if ((rc = dalloc(&L.f, ps))) return rc;
      CK(cudaMemsetAsync(L.x, 0, ps * sizeof(double), s));
      CK(cudaMemsetAsync(L.f, 0, ps * sizeof(double), s));
    }
  }
  h->m = h->coarsest * h->coarsest;
  if ((rc = dalloc(&h->Lfac, (size_t)h->m * h->m))) return rc;
  if ((rc = dalloc(&h->work, (size_t)h->m * h->m + h->m))) return rc;
  if ((rc = dalloc(&h->partials, 2 * (size_t)norm_partials_max()))) return rc;
  if (h->krylov == BMG_KRYLOV_FCG) {
    size_t ps = plane_size(n);
    if ((rc = dalloc(&h->kr, 4 * ps))) return rc;
    CK(cudaMemsetAsync(h->kr, 0, 4 * ps * sizeof(double), s));
  }
  if ((rc = dalloc(&h->err, 1))) return rc;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), s));

  launch_prepare(n, h->nx, h->ny, A->kind, A->coef, h->lv[0].st, h->err, s);
  if (h->nx != n || h->ny != n) {   // embedded problem: the solve's own f and x on the n x n grid
    if ((rc = dalloc(&h->fpad, plane_size(n)))) return rc;
    if ((rc = dalloc(&h->xpad, plane_size(n)))) return rc;
    CK(cudaMemsetAsync(h->fpad, 0, plane_size(n) * sizeof(double), s));
    CK(cudaMemsetAsync(h->xpad, 0, plane_size(n) * sizeof(double), s));
  }
  for (int l = 0; l + 1 < h->nlev; ++l) {
    Level& L = h->lv[l];
    Level& C = h->lv[l + 1];
    if (l == 0 && h->interp == BMG_INTERP_LEARNED) {
      if ((rc = mlp_level0_interp(h->mlp, L.n, L.st, L.ci, s))) return rc;
    } else {
      launch_dendy(L.n, L.st, L.ci, h->err, s);
    }
    launch_rap(L.n, L.st, L.ci, C.st, s);
    launch_dinv(C.n, C.st, h->err, s);
  }
  Level& Lc = h->lv[h->nlev - 1];
  launch_factor(Lc.n, Lc.st, h->Lfac, h->work, h->err, s);
  CK(cudaGetLastError());

  if (h->precision != BMG_FP64) {
    int nbf = h->precision == BMG_BF16_IR ? (o && o->bf16_levels > 0 ? o->bf16_levels : 2) : 0;
    for (int l = 0; l < h->nlev; ++l) {
      Level& L = h->lv[l];
      size_t ps = plane_size(L.n);
      L.bf16 = l < nbf && l + 1 < h->nlev;
      if (L.bf16) {
        if ((rc = galloc(&L.off16, L.n, 4, s))) return rc;
        if ((rc = galloc(&L.od32, L.n, 2, s))) return rc;
        launch_lower_bf16(L.n, L.st, L.off16, L.od32, s);
      } else {
        if ((rc = galloc(&L.st32, L.n, 6, s))) return rc;
      }
      if (l + 1 < h->nlev && (rc = dalloc(&L.ci32, 8 * plane_size(h->lv[l + 1].n)))) return rc;
      launch_lower32(L.n, L.bf16 ? nullptr : L.st, L.bf16 ? nullptr : L.st32, L.ci, L.ci32, s);
      if (l + 1 < h->nlev) {   // the packed copy the bulk-copy sweeps stream (guard band after it too)
        if ((rc = galloc(&L.pk32, L.n, L.bf16 ? PK_WORDS_BF16 : PK_WORDS_F32, s))) return rc;
        if (L.bf16)
          launch_pack_bf16(L.n, L.off16, L.od32, L.pk32, s);
        else
          launch_pack32(L.n, L.st32, L.pk32, s);
      }
      if ((rc = galloc(&L.x32, L.n, 1, s))) return rc;
      if ((rc = galloc(&L.f32, L.n, 1, s))) return rc;
    }
  }
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (herr) return set_error(BMG_ESINGULAR, "setup: non-positive %s",
                             herr == 1 ? "diagonal" : herr == 2 ? "interpolation denominator" : "Cholesky pivot");
  return BMG_OK;
}

}  // namespace

extern "C" int bmg_solve(bmg_hierarchy* h, const double* rhs, double* x, double tol, int maxit, int* iters,
                         double* relres);

namespace {
// V-cycle factor (r_8 / r_4)^(1/4) from a SplitMix64 uniform[-1,1) start
// (stream 0x5EED) with a zero right-hand side.
int measure_factor(bmg_hierarchy* h, double* out) {
  size_t ps = plane_size(h->n);
  double *x = nullptr, *f = nullptr;
  int rc0 = cuda_check(dev_malloc((void**)&x, ps * sizeof(double)), "factor measurement");
  if (!rc0) rc0 = cuda_check(dev_malloc((void**)&f, ps * sizeof(double)), "factor measurement");
  if (!rc0) rc0 = cuda_check(cudaMemset(x, 0, ps * sizeof(double)), "factor measurement");
  if (!rc0) rc0 = cuda_check(cudaMemset(f, 0, ps * sizeof(double)), "factor measurement");
  if (rc0) {
    cudaFree(x);
    cudaFree(f);
    return rc0;
  }
  launch_uniform_pm1(h->n, 0x5EEDull, x, nullptr);
  CK(cudaDeviceSynchronize());
  int it = 0;
  double rr = 0;
  // the stationary cycle, whatever solve mode the hierarchy has; a graph
  // captured in the other mode must not be replayed
  const int krylov = h->krylov;
  auto drop_graph = [&] {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_rhs = nullptr;
    h->g_x = nullptr;
  };
  drop_graph();
  h->krylov = BMG_KRYLOV_NONE;
  int rc = bmg_solve(h, f, x, 0.0, 15, &it, &rr);
  h->krylov = krylov;
  drop_graph();
  cudaFree(x);
  cudaFree(f);
  if (rc != BMG_OK && rc != BMG_ENOTCONV) return rc;
  // the asymptotic factor read off iterations 5 .. 15
  if (h->hist.size() < 16 || !(h->hist[5] > 0)) {
    *out = 0.0;
    return BMG_OK;
  }
  *out = std::pow(h->hist[15] / h->hist[5], 0.1);
  return BMG_OK;
}
}  // namespace

extern "C" {

const char* bmg_strerror(int code) {
  switch (code) {
    case BMG_OK: return "ok";
    case BMG_EINVAL: return "invalid argument";
    case BMG_ENOMEM: return "out of device memory";
    case BMG_ECUDA: return "CUDA error";
    case BMG_ESINGULAR: return "singular or indefinite operator";
    case BMG_ENAN: return "residual is NaN or Inf";
    case BMG_ENOTCONV: return "not converged within maxit";
    case BMG_ETIMEOUT: return "device wait timed out";
    case BMG_EBOUNDS: return "debug bounds check failed";
    default: return "unknown error";
  }
}

const char* bmg_last_error(void) { return g_err; }

namespace {
// Periodic sides (periodic.cu): FP64 stationary V-cycles with point Gauss-Seidel
// and Dendy interpolation; the solve loop, graph capture and control block are
// the Dirichlet hierarchy's.
int setup_periodic(bmg_hierarchy* h, const bmg_stencil* A, int nx, int ny, int periodic, bmg_hierarchy** out) {
  const char* why = nullptr;
  if (periodic & ~(BMG_PERIODIC_X | BMG_PERIODIC_Y)) why = "bad periodic flags";
  else if (h->precision != BMG_FP64) why = "periodic sides take FP64 cycles only";
  else if (h->interp != BMG_INTERP_DENDY) why = "periodic sides take Dendy interpolation only";
  else if (h->krylov != BMG_KRYLOV_NONE && h->krylov != BMG_KRYLOV_FCG) why = "bad krylov mode";
  else if (h->smoother != BMG_SMOOTHER_AUTO && h->smoother != BMG_SMOOTHER_ROWS && h->smoother != BMG_SMOOTHER_TILE)
    why = "periodic sides take point Gauss-Seidel (smoother AUTO, ROWS or TILE) only";
  else if (h->coarsest != 3) why = "periodic sides take the default coarsest level";
  else if (!per_levels_for(nx, ny, periodic))
    why = "a periodic axis needs 2^m points, a Dirichlet axis 2^m - 1, both axes the same m >= 2";
  if (why) {
    delete h;
    return set_error(BMG_EINVAL, "bmg_setup (periodic %d, %d x %d): %s", periodic, nx, ny, why);
  }
  h->n = 0;
  h->nlev = 0;
  CounterScope cs(&h->launches);
  int rc = cuda_check(cudaStreamCreateWithFlags(&h->ws, cudaStreamNonBlocking), "stream");
  if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming), "event");
  if (!rc) rc = cuda_check(host_malloc((void**)&h->ctl_host, sizeof(Ctl)), "pinned");
  if (!rc) rc = order_after_user(h);
  if (!rc) rc = dalloc(&h->partials, 2 * (size_t)norm_partials_max());
  if (!rc) rc = per_setup(&h->per, A->kind, A->coef, nx, ny, periodic, h->arith == BMG_ARITH_FUSED, h->nu1, h->nu2,
                          h->smoother == BMG_SMOOTHER_ROWS   ? PER_SWEEP_ROWS
                          : h->smoother == BMG_SMOOTHER_TILE ? PER_SWEEP_STRIP
                                                             : PER_SWEEP_AUTO,
                          h->krylov == BMG_KRYLOV_FCG, h->ws);
  if (!rc) rc = ensure_ctl(h, 64);
  if (rc) {
    bmg_free(h);
    return rc;
  }
  *out = h;
  return BMG_OK;
}
}  // namespace

int bmg_setup(const bmg_stencil* A, int nx, int ny, const bmg_opts* o, bmg_hierarchy** out) {
  Range nvtx("bmg_setup");
  if (!out) return set_error(BMG_EINVAL, "bmg_setup: out is NULL");
  *out = nullptr;
  if (!A || !A->coef) return set_error(BMG_EINVAL, "bmg_setup: stencil is NULL");
  if (A->kind != 5 && A->kind != 9) return set_error(BMG_EINVAL, "bmg_setup: kind %d is not 5 or 9", A->kind);
  if (nx < 1 || ny < 1 || nx > 65535 || ny > 65535)
    return set_error(BMG_EINVAL, "bmg_setup: grid %d x %d outside 1 .. 65535", nx, ny);
  const bool embedded = nx != ny || !is_level_size(nx);
  if (embedded && o && o->interp == BMG_INTERP_LEARNED)
    return set_error(BMG_EINVAL, "bmg_setup: learned interpolation needs nx = ny = 2^m - 1");
  bmg_hierarchy* h = new bmg_hierarchy();
  h->nx = nx;
  h->ny = ny;
  h->n = embed_size(nx, ny);
  if (o) {
    h->precision = o->precision;
    h->coarsest = o->coarsest ? o->coarsest : 3;
    if (o->nu1 || o->nu2) {
      h->nu1 = o->nu1;
      h->nu2 = o->nu2;
    }
    h->inner = o->inner_cycles > 0 ? o->inner_cycles : 1;
    h->use_graph = o->use_graph;
    h->krylov = o->krylov;
    h->interp = o->interp;
    h->mlp = o->mlp;
    h->user = (cudaStream_t)o->stream;
    h->smoother = o->smoother;
    h->arith = o->arith;
    h->fuse_restrict = o->fuse_restrict;
  }
  if (h->fuse_restrict < BMG_FUSE_AUTO || h->fuse_restrict > BMG_FUSE_ON) {
    int fr = h->fuse_restrict;
    delete h;
    return set_error(BMG_EINVAL, "bmg_setup: bad fuse_restrict %d", fr);
  }
  if (h->smoother < BMG_SMOOTHER_AUTO ||
      (h->smoother >= BMG_SMOOTHER_TILE + GS_TILE_SHAPES && h->smoother < BMG_SMOOTHER_PAIR) ||
      (h->smoother >= BMG_SMOOTHER_PAIR + GS_PAIR_SHAPES && !is_line(h->smoother))) {
    delete h;
    return set_error(BMG_EINVAL, "bmg_setup: bad smoother %d", h->smoother);
  }
  if (h->precision == BMG_FP64 && h->smoother >= BMG_SMOOTHER_TILE + GS_TILE64_SHAPES &&
      !is_line(h->smoother)) {
    int sm = h->smoother;
    delete h;
    return set_error(BMG_EINVAL, "bmg_setup: smoother %d has no FP64 kernel (tile0 .. tile3 do)", sm);
  }
  if (h->precision < BMG_FP64 || h->precision > BMG_BF16_IR || !is_level_size(h->coarsest) || h->coarsest > 15 ||
      h->nu1 < 0 || h->nu2 < 0 || h->interp < 0 || h->interp > 1 || (h->interp == BMG_INTERP_LEARNED && !h->mlp) ||
      h->krylov < 0 || h->krylov > 1 || h->arith < BMG_ARITH_ROUNDED || h->arith > BMG_ARITH_FUSED) {
    delete h;
    return set_error(BMG_EINVAL, "bmg_setup: bad options");
  }
  if (h->coarsest > h->n) h->coarsest = h->n;
  if (o && o->periodic) return setup_periodic(h, A, nx, ny, o->periodic, out);
  CounterScope cs(&h->launches);
  int rc = cuda_check(cudaStreamCreateWithFlags(&h->ws, cudaStreamNonBlocking), "stream");
  if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming), "event");
  if (!rc) rc = cuda_check(host_malloc((void**)&h->ctl_host, sizeof(Ctl)), "pinned");
  if (!rc) rc = order_after_user(h);
  if (!rc) rc = setup_impl(h, A, h->n, o);
  const bool line = is_line(h->smoother);
  if (!rc && line) rc = alloc_line(h);
  if (!rc && !line && h->smoother >= BMG_SMOOTHER_TILE) rc = force_tile(h);
  if (!rc && !line && h->use_graph) rc = autotune_solo(h);
  if (!rc && !line && h->use_graph)   // the level-fused tail relaxes by points
    rc = h->precision == BMG_FP64 ? build_tail<double>(h, 1) : build_tail<float>(h, 0);
  if (!rc && !line) rc = choose_pair_restrict(h);
  if (!rc) rc = ensure_ctl(h, 64);
  if (rc) {
    bmg_free(h);
    return rc;
  }
  h->interp_used = h->interp;
  if (h->interp == BMG_INTERP_LEARNED) {
    // Dendy is the fallback: build it too, measure both factors, keep the better.
    bmg_opts od = *o;
    od.interp = BMG_INTERP_DENDY;
    od.mlp = nullptr;
    bmg_hierarchy* hd = nullptr;
    rc = bmg_setup(A, nx, ny, &od, &hd);
    double fl = 0, fd = 0;
    if (!rc) rc = measure_factor(h, &fl);
    if (!rc) rc = measure_factor(hd, &fd);
    if (rc) {
      bmg_free(h);
      bmg_free(hd);
      return rc;
    }
    bmg_hierarchy* keep = fl <= fd ? h : hd;
    bmg_free(keep == h ? hd : h);
    keep->interp_used = keep == h ? BMG_INTERP_LEARNED : BMG_INTERP_DENDY;
    keep->factor_learned = fl;
    keep->factor_dendy = fd;
    h = keep;
  }
  *out = h;
  return BMG_OK;
}

int bmg_tuned_cluster(const bmg_hierarchy* h, int level) {
  if (h && h->per) {
    if (level < 0 || level >= per_num_levels(h->per)) return set_error(BMG_EINVAL, "bmg_tuned_cluster: bad level");
    const int k = per_level_sweep(h->per, level);
    return k == 2 ? BMG_TILE_SWEEP : k;
  }
  if (!h || level < 0 || level >= h->nlev) return set_error(BMG_EINVAL, "bmg_tuned_cluster: bad level");
  const Level& L = h->lv[level];
  if (h->precision != BMG_FP64 && L.tile32 >= 0) return BMG_TILE_SWEEP + L.tile32;
  if (h->precision == BMG_FP64 && L.tile64 >= 0) return BMG_TILE_SWEEP + L.tile64;
  return h->precision == BMG_FP64 ? L.cl64 : L.cl32;
}

int bmg_tuned_pair(const bmg_hierarchy* h, int level) {
  if (!h || level < 0 || level >= h->nlev) return set_error(BMG_EINVAL, "bmg_tuned_pair: bad level");
  return h->precision != BMG_FP64 ? h->lv[level].pair32 : -1;
}

int bmg_interp_info(const bmg_hierarchy* h, int* used, double* fl, double* fd) {
  if (!h) return set_error(BMG_EINVAL, "bmg_interp_info: NULL hierarchy");
  if (used) *used = h->interp_used;
  if (fl) *fl = h->factor_learned;
  if (fd) *fd = h->factor_dendy;
  return BMG_OK;
}

// General sizes: the embedded problem's right-hand side and iterate for the
// caller's rhs and x (nx x ny layout): their interiors copied into fpad / xpad.
// Without embedding, the caller's arrays themselves.
static void map_in(bmg_hierarchy* h, const double*& rhs, double*& x) {
  if (!h->fpad) return;
  launch_embed_vec(h->nx, h->ny, h->n, rhs, h->fpad, false, h->ws);
  launch_embed_vec(h->nx, h->ny, h->n, x, h->xpad, false, h->ws);
  rhs = h->fpad;
  x = h->xpad;
}

// The caller's x from the embedded iterate.
static void map_out(bmg_hierarchy* h, double* x_caller) {
  if (h->fpad) launch_embed_vec(h->nx, h->ny, h->n, h->xpad, x_caller, true, h->ws);
}

static int reset_ctl(bmg_hierarchy* h, double tol, int maxit) {
  int rc;
  if ((rc = ensure_ctl(h, maxit))) return rc;
  Ctl c0{};
  c0.maxit = maxit;
  c0.tol = tol;
  c0.scale_next = 1.0;
  c0.scale_applied = 1.0;
  *h->ctl_host = c0;
  CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, h->ws));
  return BMG_OK;
}

int bmg_time_cycles(bmg_hierarchy* h, const double* rhs, double* x, int cycles, double* ms) {
  Range nvtx("bmg_time_cycles");
  if (!h || !rhs || !x || !ms || cycles < 1) return set_error(BMG_EINVAL, "bmg_time_cycles: bad argument");
  CounterScope cs(&h->launches);
  int rc;
  if ((rc = order_after_user(h))) return rc;
  if ((rc = reset_ctl(h, 0.0, cycles))) return rc;
  double* x_caller = x;
  map_in(h, rhs, x);
  enqueue_initial(h, rhs, x);
  if (h->use_graph && (rc = capture_graph(h, rhs, x))) return rc;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, h->ws));
  for (int i = 0; i < cycles; ++i) {
    if (h->use_graph) {
      CK(cudaGraphLaunch(h->gexec, h->ws));
      h->launches += h->g_kernels;
    } else {
      enqueue_iteration(h, rhs, x);
    }
  }
  CK(cudaEventRecord(b, h->ws));
  map_out(h, x_caller);
  CK(cudaEventSynchronize(b));
  float t = 0;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CK(cudaStreamSynchronize(h->ws));
  *ms = t;
  if ((rc = timeout_check("bmg_time_cycles"))) return rc;
  return cuda_check(cudaGetLastError(), "bmg_time_cycles");
}

int bmg_profile(bmg_hierarchy* h, const double* rhs, double* x, int cycles, bmg_prof_row* rows, int cap) {
  Range nvtx("bmg_profile");
  if (!h || !rhs || !x || cycles < 1) return set_error(BMG_EINVAL, "bmg_profile: bad argument");
  CounterScope cs(&h->launches);
  int rc;
  if ((rc = order_after_user(h))) return rc;
  if ((rc = reset_ctl(h, 0.0, cycles))) return rc;
  double* x_caller = x;
  map_in(h, rhs, x);
  enqueue_initial(h, rhs, x);
  std::vector<bmg_hierarchy::Mark> marks;
  h->prof = &marks;
  for (int i = 0; i < cycles; ++i) enqueue_iteration(h, rhs, x);
  h->prof = nullptr;
  map_out(h, x_caller);
  rc = cuda_check(cudaStreamSynchronize(h->ws), "bmg_profile");
  std::vector<bmg_prof_row> acc;
  for (auto& m : marks) {
    float t = 0;
    if (!rc) cudaEventElapsedTime(&t, m.a, m.b);
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
    bool found = false;
    for (auto& r : acc)
      if (r.level == m.level && r.kernel == m.kernel && r.fp32 == m.fp32) {
        r.launches += (int)m.launches;
        r.ms += t;
        found = true;
      }
    if (!found) acc.push_back(bmg_prof_row{m.level, m.kernel, m.fp32, (int)m.launches, (double)t});
  }
  if (rc) return rc;
  for (size_t k = 0; k < acc.size() && (int)k < cap; ++k) rows[k] = acc[k];
  if ((rc = timeout_check("bmg_profile"))) return rc;
  return (int)acc.size();
}

int bmg_solve(bmg_hierarchy* h, const double* rhs, double* x, double tol, int maxit, int* iters, double* relres) {
  Range nvtx("bmg_solve");
  if (!h || !rhs || !x) return set_error(BMG_EINVAL, "bmg_solve: NULL argument");
  if (maxit < 0 || !(tol >= 0.0)) return set_error(BMG_EINVAL, "bmg_solve: bad tol or maxit");
  CounterScope cs(&h->launches);
  int rc;
  if ((rc = order_after_user(h))) return rc;
  if ((rc = reset_ctl(h, tol, maxit))) return rc;
  double* x_caller = x;
  map_in(h, rhs, x);
  enqueue_initial(h, rhs, x);
  CK(cudaGetLastError());
  if (h->use_graph && (rc = capture_graph(h, rhs, x))) return rc;
  const int chunk = 4;
  int launched = 0;
  for (;;) {
    CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->ws));
    CK(cudaStreamSynchronize(h->ws));
    if (h->ctl_host->done || launched >= maxit) break;
    int k = maxit - launched < chunk ? maxit - launched : chunk;
    for (int i = 0; i < k; ++i) {
      if (h->use_graph) {
        CK(cudaGraphLaunch(h->gexec, h->ws));
        h->launches += h->g_kernels;
      } else {
        enqueue_iteration(h, rhs, x);
      }
    }
    CK(cudaGetLastError());
    launched += k;
  }
  map_out(h, x_caller);
  CK(cudaStreamSynchronize(h->ws));
  Ctl& c = *h->ctl_host;
  int it = c.it;
  h->hist.assign((size_t)it + 1, 0.0);
  CK(cudaMemcpy(h->hist.data(), (char*)h->ctl + offsetof(Ctl, hist), sizeof(double) * (it + 1),
                cudaMemcpyDeviceToHost));
  if (iters) *iters = it;
  if (relres) *relres = h->hist[0] > 0 ? h->hist[it] / h->hist[0] : 0.0;
  if ((rc = timeout_check("bmg_solve"))) return rc;
  if (c.done == 3) return set_error(BMG_ENAN, "bmg_solve: residual norm is not finite at cycle %d", it);
  if (c.done == 2 || c.done == 0) return set_error(BMG_ENOTCONV, "bmg_solve: %d cycles, relres %g", it,
                                                   h->hist[0] > 0 ? h->hist[it] / h->hist[0] : 0.0);
  return BMG_OK;
}

int bmg_history(const bmg_hierarchy* h, double* out, int cap) {
  if (!h) return set_error(BMG_EINVAL, "bmg_history: NULL hierarchy");
  int cnt = (int)h->hist.size();
  if (out)
    for (int k = 0; k < cnt && k < cap; ++k) out[k] = h->hist[k];
  return cnt;
}

int bmg_num_levels(const bmg_hierarchy* h) {
  if (!h) return set_error(BMG_EINVAL, "NULL hierarchy");
  return h->per ? per_num_levels(h->per) : h->nlev;
}

int bmg_level_shape(const bmg_hierarchy* h, int l, int* nx, int* ny) {
  if (!h) return set_error(BMG_EINVAL, "bmg_level_shape: NULL hierarchy");
  if (h->per) return per_level_shape(h->per, l, nx, ny);
  if (l < 0 || l >= h->nlev) return set_error(BMG_EINVAL, "bmg_level_shape: bad level %d", l);
  if (nx) *nx = h->lv[l].n;
  if (ny) *ny = h->lv[l].n;
  return BMG_OK;
}

int bmg_level_size(const bmg_hierarchy* h, int l) {
  if (!h || l < 0 || l >= h->nlev) return set_error(BMG_EINVAL, "bmg_level_size: bad level");
  return h->lv[l].n;
}

int bmg_get_stencil(const bmg_hierarchy* h, int l, double* out) {
  if (h && out && h->per) return per_get_stencil(h->per, l, out, h->ws);
  if (!h || !out || l < 0 || l >= h->nlev) return set_error(BMG_EINVAL, "bmg_get_stencil: bad argument");
  CK(cudaMemcpyAsync(out, h->lv[l].st, 5 * plane_size(h->lv[l].n) * sizeof(double), cudaMemcpyDeviceToDevice,
                     h->ws));
  CK(cudaStreamSynchronize(h->ws));
  return BMG_OK;
}

int bmg_get_interp(const bmg_hierarchy* h, int l, double* out) {
  if (h && out && h->per) return per_get_interp(h->per, l, out, h->ws);
  if (!h || !out || l < 0 || l + 1 >= h->nlev) return set_error(BMG_EINVAL, "bmg_get_interp: bad argument");
  CK(cudaMemcpyAsync(out, h->lv[l].ci, 8 * plane_size(h->lv[l + 1].n) * sizeof(double), cudaMemcpyDeviceToDevice,
                     h->ws));
  CK(cudaStreamSynchronize(h->ws));
  return BMG_OK;
}

long long bmg_launch_count(const bmg_hierarchy* h) { return h ? h->launches : 0; }

void bmg_free(bmg_hierarchy* h) {
  if (!h) return;
  if (h->ws) cudaStreamSynchronize(h->ws);
  for (Level& L : h->lv) free_level(L, h->shared_ops);
  if (!h->shared_ops) {
    cudaFree(h->Lfac);
    cudaFree(h->work);
  }
  cudaFree(h->partials);
  cudaFree(h->kr);
  cudaFree(h->fpad);
  cudaFree(h->xpad);
  per_free(h->per);
  cudaFree(h->d_tail);
  cudaFree(h->err);
  cudaFree(h->ctl);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->ws) cudaStreamDestroy(h->ws);
  delete h;
}

int bmg_inner_cycle(bmg_hierarchy* h, const float* r32, float* e32) {
  if (!h || !r32 || !e32) return set_error(BMG_EINVAL, "bmg_inner_cycle: NULL argument");
  if (h->precision == BMG_FP64) return set_error(BMG_EINVAL, "bmg_inner_cycle: hierarchy has no FP32 cycle");
  CounterScope cs(&h->launches);
  int rc;
  if ((rc = order_after_user(h))) return rc;
  Level& L0 = h->lv[0];
  size_t bytes = plane_size(L0.n) * sizeof(float);
  CK(cudaMemcpyAsync(L0.f32, r32, bytes, cudaMemcpyDeviceToDevice, h->ws));
  CK(cudaMemsetAsync(L0.x32, 0, bytes, h->ws));
  for (int c = 0; c < h->inner; ++c) vcycle32(h, 0, nullptr);
  CK(cudaMemcpyAsync(e32, L0.x32, bytes, cudaMemcpyDeviceToDevice, h->ws));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->ws));
  return timeout_check("bmg_inner_cycle");
}

int bmg_wait_selftest(void) {
  strip_timeouts();   // clear
  launch_wait_selftest(nullptr);
  CK(cudaDeviceSynchronize());
  CK(cudaGetLastError());
  int rc = timeout_check("bmg_wait_selftest");
  return rc == BMG_ETIMEOUT ? BMG_OK : set_error(BMG_ECUDA, "bmg_wait_selftest: the bounded wait did not give up");
}

// ---- stateless steps -----------------------------------------------------------------

static StencilView<double, double> raw_view(int n, const double* coef, bool with_d) {
  size_t ps = plane_size(n);
  return {coef, coef + ps, coef + 2 * ps, coef + 3 * ps, coef + 4 * ps, with_d ? coef + 5 * ps : nullptr, n, n + 2};
}

static int step_done(cudaStream_t s, const char* what) {
  CK(cudaGetLastError());
  int rc = cuda_check(cudaStreamSynchronize(s), what);
  return rc ? rc : debug_check(what);
}

int bmg_dendy_interp(int n, const double* coef, double* ci, void* stream) {
  if (!is_level_size(n) || !coef || !ci) return set_error(BMG_EINVAL, "bmg_dendy_interp: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int* err = nullptr;
  CK(cudaMallocAsync((void**)&err, sizeof(int), s));
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  launch_dendy(n, coef, ci, err, s);
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(err, s));
  int rc = step_done(s, "bmg_dendy_interp");
  if (rc) return rc;
  return herr ? set_error(BMG_ESINGULAR, "bmg_dendy_interp: non-positive denominator") : BMG_OK;
}

int bmg_rap(int n, const double* coef, const double* ci, double* coarse, void* stream) {
  if (!is_level_size(n) || !coef || !ci || !coarse) return set_error(BMG_EINVAL, "bmg_rap: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  // the kernel writes six planes; give it room for the sixth
  int nc = (n - 1) / 2;
  double* tmp = nullptr;
  CK(cudaMallocAsync((void**)&tmp, 6 * plane_size(nc) * sizeof(double), s));
  launch_rap(n, coef, ci, tmp, s);
  CK(cudaMemcpyAsync(coarse, tmp, 5 * plane_size(nc) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaFreeAsync(tmp, s));
  return step_done(s, "bmg_rap");
}

int bmg_relax(int n, int kind, const double* coef, const double* f, double* x, int sweeps, void* stream) {
  if (!is_level_size(n) || (kind != 5 && kind != 9) || !coef || !f || !x || sweeps < 0)
    return set_error(BMG_EINVAL, "bmg_relax: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_gs(raw_view(n, coef, false), kind, f, x, sweeps, (const int*)nullptr, s);
  return step_done(s, "bmg_relax");
}

int bmg_relax_line(int n, int kind, const double* coef, const double* f, double* x, double* work, int sweeps,
                   void* stream) {
  if (!is_level_size(n) || (kind != 5 && kind != 9) || !coef || !f || !x || !work || sweeps < 0)
    return set_error(BMG_EINVAL, "bmg_relax_line: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_line<double, double>(raw_view(n, coef, false), kind, f, x, work, sweeps, LINE_X, (const int*)nullptr, s);
  return step_done(s, "bmg_relax_line");
}

int bmg_debug_build(void) {
#ifdef BMG_DEBUG
  return 1;
#else
  return 0;
#endif
}

int bmg_debug_take(int* site, long long* index, long long* extent) {
#ifdef BMG_DEBUG
  DbgRecord r;
  if (cudaDeviceSynchronize() != cudaSuccess || dbg_collect(&r, true) != cudaSuccess)
    return set_error(BMG_ECUDA, "bmg_debug_take: reading the records failed");
  if (site) *site = r.site;
  if (index) *index = r.index;
  if (extent) *extent = r.extent;
  return r.hit ? 1 : 0;
#else
  if (site) *site = 0;
  if (index) *index = 0;
  if (extent) *extent = 0;
  return 0;
#endif
}

const char* bmg_debug_site_name(int site) { return dbg_site_name(site); }

int bmg_debug_shrink(long long k) {
#ifdef BMG_DEBUG
  if (k < 0) return set_error(BMG_EINVAL, "bmg_debug_shrink: negative count");
  for (const DbgHooks& h : dbg_hooks())
    if (h.shrink(k) != cudaSuccess) return set_error(BMG_ECUDA, "bmg_debug_shrink: setting the extent failed");
  return BMG_OK;
#else
  (void)k;
  return set_error(BMG_EINVAL, "bmg_debug_shrink: not a debug build (BMG_DEBUG)");
#endif
}

int bmg_relax_line_y(int n, int kind, const double* coef, const double* f, double* x, double* work, int sweeps,
                     void* stream) {
  if (!is_level_size(n) || (kind != 5 && kind != 9) || !coef || !f || !x || !work || sweeps < 0)
    return set_error(BMG_EINVAL, "bmg_relax_line_y: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_line<double, double>(raw_view(n, coef, false), kind, f, x, work, sweeps, LINE_Y, (const int*)nullptr, s);
  return step_done(s, "bmg_relax_line_y");
}

int bmg_resid_restrict(int n, int kind, const double* coef, const double* ci, const double* x, const double* f,
                       double* fc, void* stream) {
  if (!is_level_size(n) || (kind != 5 && kind != 9) || !coef || !ci || !x || !f || !fc)
    return set_error(BMG_EINVAL, "bmg_resid_restrict: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(fc, 0, plane_size((n - 1) / 2) * sizeof(double), s));
  launch_resid_restrict(raw_view(n, coef, false), kind, ci, x, f, fc, (double*)nullptr, (const int*)nullptr, s);
  return step_done(s, "bmg_resid_restrict");
}

int bmg_interp_correct(int n, const double* ci, const double* ec, double* x, void* stream) {
  if (!is_level_size(n) || !ci || !ec || !x) return set_error(BMG_EINVAL, "bmg_interp_correct: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  launch_interp_correct<double>(n, ci, ec, x, (const int*)nullptr, s);
  return step_done(s, "bmg_interp_correct");
}

int bmg_residual(int n, int kind, const double* coef, const double* x, const double* f, double* r, double* norm,
                 void* stream) {
  if (!is_level_size(n) || (kind != 5 && kind != 9) || !coef || !x || !f)
    return set_error(BMG_EINVAL, "bmg_residual: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;   // partial sums + the norm
  if (norm) CK(cudaMallocAsync((void**)&scratch, (norm_partials_max() + 1) * sizeof(double), s));
  if (r) zero_ring(n, r, s);
  int np = launch_residual(raw_view(n, coef, false), kind, x, f, r, scratch, (const int*)nullptr, s);
  if (norm) {
    launch_norm_finalize(scratch, np, nullptr, 0, scratch + norm_partials_max(), s);
    CK(cudaMemcpyAsync(norm, scratch + norm_partials_max(), sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(scratch, s));
  }
  return step_done(s, "bmg_residual");
}

int bmg_coarse_factor(int n, const double* coef, double* L, void* stream) {
  if (!is_level_size(n) || n > 15 || !coef || !L) return set_error(BMG_EINVAL, "bmg_coarse_factor: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int m = n * n;
  double* work = nullptr;
  int* err = nullptr;
  CK(cudaMallocAsync((void**)&work, (size_t)m * m * sizeof(double), s));
  CK(cudaMallocAsync((void**)&err, sizeof(int), s));
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  launch_factor(n, coef, L, work, err, s);
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(work, s));
  CK(cudaFreeAsync(err, s));
  int rc = step_done(s, "bmg_coarse_factor");
  if (rc) return rc;
  return herr ? set_error(BMG_ESINGULAR, "bmg_coarse_factor: non-positive pivot") : BMG_OK;
}

int bmg_coarse_solve(int n, const double* L, const double* f, double* x, void* stream) {
  if (!is_level_size(n) || n > 15 || !L || !f || !x) return set_error(BMG_EINVAL, "bmg_coarse_solve: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* y = nullptr;
  CK(cudaMallocAsync((void**)&y, (size_t)n * n * sizeof(double), s));
  launch_coarse_solve<double>(n, L, f, x, y, (const int*)nullptr, s);
  CK(cudaFreeAsync(y, s));
  return step_done(s, "bmg_coarse_solve");
}

int bmg_measure_fp64_rate(double* out, void* stream) {
  if (!out) return set_error(BMG_EINVAL, "bmg_measure_fp64_rate: NULL");
  double r = measure_fp64_rate((cudaStream_t)stream);
  if (r <= 0) return set_error(BMG_ECUDA, "bmg_measure_fp64_rate failed");
  *out = r;
  return BMG_OK;
}

}  // extern "C"

// =====================================================================================
// Batched solver
// =====================================================================================
#include <array>
#include <map>
#include <tuple>

namespace {
// group slot = storage * 2 + (kind == 5): storage 0 double, 1 float, 2 bf16
constexpr int kGroups = 6;
}

struct bmg_batch {
  int nprob = 0, precision = BMG_FP64, nu1 = 2, nu2 = 1, inner = 1, use_graph = 1, arith = BMG_ARITH_ROUNDED;
  int smoother = BMG_SMOOTHER_AUTO;
  int rhs_block = BMG_RHS_BLOCK_AUTO;
  std::vector<bmg_hierarchy*> hs;
  cudaStream_t user = nullptr, ws = nullptr;
  cudaEvent_t ev = nullptr;
  int bmax = 0, maxn = 0;
  struct Group {
    int n = 0, count = 0, cl = 1, storage = 0, kind = 9;
    int tile = -1, pair = -1;   // one-pass / two-sweep shapes chosen for an FP32 group (-1: row kernel / none)
    int multi = 0;              // 2 or 4: one-pass sweeps with that many members per warp (shared operator)
    int dir = 0;                // while a cycle is enqueued: 0 = iterate in x, 1 = in x2
    size_t elem = 0;
    void* d = nullptr;
    std::vector<char> host;
  };
  std::vector<std::array<Group, kGroups>> stages;   // index b = levels above the coarsest
  std::vector<int> tuned_cl;                         // per stage, 0 = not tuned
  // level-fused tails, grouped by the stage they start at
  std::vector<int> tail_count;
  std::vector<int> tail_n;      // per stage: size of the first level of the tails starting there
  std::vector<std::vector<char>> tail_host;
  std::vector<void*> tail_dev;
  std::vector<TopDesc> top;
  TopDesc* d_top = nullptr;
  std::vector<int2> bmap;       // (problem, block) of the top-level residual launches
  int2* d_bmap = nullptr;
  char* ctls = nullptr;
  size_t ctl_stride = 0;
  int maxit_cap = 0;
  std::vector<char> ctl_host;
  int* d_alldone = nullptr;
  int* h_alldone = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const double*> g_rhs;
  std::vector<double*> g_x;
  long long g_kernels = 0, launches = 0;
  std::vector<std::vector<double>> hist;
};

namespace {

Ctl* batch_ctl(bmg_batch* B, int p) { return (Ctl*)(B->ctls + (size_t)p * B->ctl_stride); }

int group_slot(int storage, int kind) { return storage * 2 + (kind == 5 ? 1 : 0); }

template <typename T, typename S>
void append_desc(bmg_batch::Group& g, const LevelDesc<T, S>& d) {
  const char* c = (const char*)&d;
  g.host.insert(g.host.end(), c, c + sizeof(d));
}

// Fill every stage's descriptor tables and the top-level table for the caller
// buffers rhs/x and upload them (the device addresses never change, so a
// captured graph stays valid).  With rhs == NULL only the group sizes are set.
// First level of problem p that joins its level-fused tail (-1: none): the
// rule of the solo hierarchy (FP64 from level 1, n <= 15; FP32 from level 0,
// n <= 63, not BF16), only when graphs are in use.
int batch_tail_level(bmg_batch* B, bmg_hierarchy* h) {
  if (!B->use_graph) return -1;
  const bool f64 = B->precision == BMG_FP64;
  const int thr = f64 ? tail_max_n<double>() : tail_max_n<float>();
  for (int l = f64 ? 1 : 0; l + 1 < h->nlev; ++l)
    if (h->lv[l].n <= thr && !h->lv[l].bf16) return h->nlev - l <= TAIL_LEVELS ? l : -1;
  return -1;
}

template <typename T>
void append_tail(bmg_batch* B, bmg_hierarchy* h, int lt, const int* done, int b) {
  TailDesc<T> d{};
  d.nlev = h->nlev - lt;
  d.nu1 = B->nu1;
  d.nu2 = B->nu2;
  d.top_kind = h->lv[lt].kind;
  d.done = done;
  for (int k = 0; k < d.nlev; ++k) {
    Level& L = h->lv[lt + k];
    Level* C = lt + k + 1 < h->nlev ? &h->lv[lt + k + 1] : nullptr;
    if constexpr (sizeof(T) == 8)
      d.lv[k] = LevelDesc<double, double>{view64(L), L.ci, L.x, L.f, C ? C->x : nullptr, C ? C->f : nullptr,
                                          nullptr, h->Lfac, h->work};
    else
      d.lv[k] = LevelDesc<float, float>{view32(L), L.ci32, L.x32, L.f32, C ? C->x32 : nullptr,
                                        C ? C->f32 : nullptr, nullptr, h->Lfac, h->work};
  }
  const char* c = (const char*)&d;
  B->tail_host[b].insert(B->tail_host[b].end(), c, c + sizeof(d));
}

// Fill every stage's descriptor tables, the tails and the top-level table for
// the caller buffers rhs/x and upload them (the device addresses never change,
// so a captured graph stays valid).  With rhs == NULL only the sizes are set.
int build_batch_tables(bmg_batch* B, const double* const* rhs, double* const* x) {
  for (auto& st : B->stages)
    for (auto& g : st) {
      g.host.clear();
      if (!rhs) g.count = 0;
    }
  for (auto& t : B->tail_host) t.clear();
  if (!rhs) std::fill(B->tail_count.begin(), B->tail_count.end(), 0);
  B->top.clear();
  const size_t tail_elem = B->precision == BMG_FP64 ? sizeof(TailDesc<double>) : sizeof(TailDesc<float>);
  for (int p = 0; p < B->nprob; ++p) {
    bmg_hierarchy* h = B->hs[p];
    const int L = h->nlev;
    const int* done = &batch_ctl(B, p)->done;
    const int lt = batch_tail_level(B, h);
    if (lt >= 0) {
      const int bt = L - 1 - lt;
      B->tail_n[bt] = std::max(B->tail_n[bt], h->lv[lt].n);
      if (!rhs)
        ++B->tail_count[bt];
      else if (B->precision == BMG_FP64)
        append_tail<double>(B, h, lt, done, bt);
      else
        append_tail<float>(B, h, lt, done, bt);
    }
    for (int l = 0; l < L; ++l) {
      if (lt >= 0 && l >= lt) break;   // these levels run inside the tail
      Level& lv = h->lv[l];
      const int b = L - 1 - l;
      Level* C = l + 1 < L ? &h->lv[l + 1] : nullptr;
      int storage = B->precision == BMG_FP64 ? 0 : (lv.bf16 ? 2 : 1);
      bmg_batch::Group& g = B->stages[b][group_slot(storage, lv.kind)];
      g.n = lv.n;
      g.storage = storage;
      g.kind = lv.kind;
      if (!rhs) {
        ++g.count;
        g.elem = storage == 0 ? sizeof(LevelDesc<double, double>)
                              : storage == 1 ? sizeof(LevelDesc<float, float>) : sizeof(LevelDesc<float, __nv_bfloat16>);
        continue;
      }
      if (storage == 0) {
        LevelDesc<double, double> d{view64(lv), lv.ci, l == 0 ? x[p] : lv.x, l == 0 ? rhs[p] : lv.f,
                                    C ? C->x : nullptr, C ? C->f : nullptr, done, h->Lfac, h->work, lv.x64b};
        append_desc(g, d);
      } else if (storage == 2) {
        LevelDesc<float, __nv_bfloat16> d{viewbf(lv), lv.ci32, lv.x32, lv.f32, C ? C->x32 : nullptr,
                                          C ? C->f32 : nullptr, done, h->Lfac, h->work, lv.x32b};
        append_desc(g, d);
      } else {
        LevelDesc<float, float> d{view32(lv), lv.ci32, lv.x32, lv.f32, C ? C->x32 : nullptr, C ? C->f32 : nullptr,
                                  done, h->Lfac, h->work, lv.x32b};
        append_desc(g, d);
      }
    }
    if (rhs) {
      Level& l0 = h->lv[0];
      B->top.push_back(TopDesc{view64(l0), l0.kind, x[p], rhs[p], l0.f32, l0.x32, h->partials, batch_ctl(B, p)});
    }
  }
  if (!rhs) return BMG_OK;
  for (auto& st : B->stages)
    for (auto& g : st)
      if (g.count) {
        if (g.host.size() != g.elem * (size_t)g.count) return set_error(BMG_ECUDA, "batched: table size mismatch");
        CK(cudaMemcpyAsync(g.d, g.host.data(), g.host.size(), cudaMemcpyHostToDevice, B->ws));
      }
  for (size_t b = 0; b < B->tail_host.size(); ++b)
    if (B->tail_count[b]) {
      if (B->tail_host[b].size() != tail_elem * B->tail_count[b])
        return set_error(BMG_ECUDA, "batched: tail table size mismatch");
      CK(cudaMemcpyAsync(B->tail_dev[b], B->tail_host[b].data(), B->tail_host[b].size(), cudaMemcpyHostToDevice,
                         B->ws));
    }
  CK(cudaMemcpyAsync(B->d_top, B->top.data(), sizeof(TopDesc) * B->top.size(), cudaMemcpyHostToDevice, B->ws));
  return BMG_OK;
}

template <typename T, typename S>
const LevelDesc<T, S>* gdesc(const bmg_batch::Group& g) { return (const LevelDesc<T, S>*)g.d; }

// Sweeps of a group: the row kernel in place, or one-pass / two-sweep launches
// that move the iterate between x and x2 (g.dir follows it).
template <typename S>
void group_onepass(bmg_batch* B, bmg_batch::Group& g, int sweeps) {
  const LevelDesc<float, S>* d = gdesc<float, S>(g);
  int k = 0;
  if (g.multi) {
    for (; k < sweeps; ++k, g.dir ^= 1) launch_gs_tile_bk(d, g.count, g.n, g.multi, g.dir, B->ws, B->arith);
    return;
  }
  for (; g.pair >= 0 && k + 2 <= sweeps; k += 2, g.dir ^= 1)
    launch_gs_pair_b(d, g.count, g.n, g.pair, g.dir, B->ws, B->arith);
  for (; k < sweeps; ++k, g.dir ^= 1) launch_gs_tile_b(d, g.count, g.n, g.tile, g.dir, B->ws, B->arith);
}

int group_launches(const bmg_batch::Group& g, int sweeps) {
  if (g.tile < 0) return 0;
  return g.pair >= 0 && !g.multi ? sweeps / 2 + sweeps % 2 : sweeps;
}

void group_relax(bmg_batch* B, bmg_batch::Group& g, int sweeps) {
  if (!g.count || !sweeps) return;
  if (g.tile >= 0 && g.storage == 0)
    for (int k = 0; k < sweeps; ++k, g.dir ^= 1)
      launch_gs_tile64_b(gdesc<double, double>(g), g.count, g.n, g.tile, g.dir, B->ws, B->arith);
  else if (g.tile >= 0 && g.storage == 1) group_onepass<float>(B, g, sweeps);
  else if (g.tile >= 0 && g.storage == 2) group_onepass<__nv_bfloat16>(B, g, sweeps);
  else if (g.storage == 0)
    launch_gs_b(gdesc<double, double>(g), g.count, g.n, g.kind, sweeps, g.cl, B->ws, B->arith);
  else if (g.storage == 1)
    launch_gs_b(gdesc<float, float>(g), g.count, g.n, g.kind, sweeps, g.cl, B->ws, B->arith);
  else
    launch_gs_b(gdesc<float, __nv_bfloat16>(g), g.count, g.n, g.kind, sweeps, g.cl, B->ws, B->arith);
}

void group_restrict(bmg_batch* B, bmg_batch::Group& g) {
  if (!g.count) return;
  if (g.storage == 0)
    launch_resid_restrict_b(gdesc<double, double>(g), g.count, g.n, g.kind, B->ws, g.dir, B->arith);
  else if (g.storage == 1)
    launch_resid_restrict_b(gdesc<float, float>(g), g.count, g.n, g.kind, B->ws, g.dir, B->arith);
  else
    launch_resid_restrict_b(gdesc<float, __nv_bfloat16>(g), g.count, g.n, g.kind, B->ws, g.dir, B->arith);
}

// x (or x2) += P e: reads the array g.dir names and writes the one from which
// the post-smoothing launches end in x.
void group_interp(bmg_batch* B, bmg_batch::Group& g) {
  if (!g.count) return;
  const int din = g.dir, dout = group_launches(g, B->nu2) & 1;
  if (g.storage == 0) launch_interp_b(gdesc<double, double>(g), g.count, g.n, B->ws, din, dout, B->arith);
  else if (g.storage == 1) launch_interp_b(gdesc<float, float>(g), g.count, g.n, B->ws, din, dout, B->arith);
  else launch_interp_b(gdesc<float, __nv_bfloat16>(g), g.count, g.n, B->ws, din, dout, B->arith);
  g.dir = dout;
}

void group_coarse(bmg_batch* B, bmg_batch::Group& g) {
  if (!g.count) return;
  if (g.storage == 0) launch_coarse_b(gdesc<double, double>(g), g.count, B->ws);
  else if (g.storage == 1) launch_coarse_b(gdesc<float, float>(g), g.count, B->ws);
  else launch_coarse_b(gdesc<float, __nv_bfloat16>(g), g.count, B->ws);
}

// One V(nu1, nu2) cycle of every problem: down the stages (largest first), the
// coarsest solves, back up.
void batch_vcycle(bmg_batch* B) {
  for (int b = B->bmax; b >= 1; --b) {
    for (auto& g : B->stages[b]) {
      g.dir = 0;
      group_relax(B, g, B->nu1);
      group_restrict(B, g);
    }
    if (B->tail_count[b]) {   // problems whose remaining levels run in one level-fused launch
      if (B->precision == BMG_FP64)
        launch_tail<double>((const TailDesc<double>*)B->tail_dev[b], B->tail_count[b], B->tail_n[b], nullptr, B->ws,
                            B->arith);
      else
        launch_tail<float>((const TailDesc<float>*)B->tail_dev[b], B->tail_count[b], B->tail_n[b], nullptr, B->ws,
                           B->arith);
    }
  }
  for (auto& g : B->stages[0]) group_coarse(B, g);
  for (int b = 1; b <= B->bmax; ++b)
    for (auto& g : B->stages[b]) {
      group_interp(B, g);
      group_relax(B, g, B->nu2);
    }
}

void batch_iteration(bmg_batch* B) {
  if (B->precision == BMG_FP64) {
    batch_vcycle(B);
    launch_residual_b(B->d_top, B->d_bmap, (int)B->bmap.size(), B->ws, B->arith);
  } else {
    for (int c = 0; c < B->inner; ++c) batch_vcycle(B);
    launch_ir_update_b(B->d_top, B->nprob, B->maxn, B->ws);
    launch_ir_residual_b(B->d_top, B->d_bmap, (int)B->bmap.size(), B->ws, B->arith);
  }
  launch_finalize_b(B->d_top, B->nprob, 1, B->ws);
}

void batch_initial(bmg_batch* B) {
  if (B->precision == BMG_FP64)
    launch_residual_b(B->d_top, B->d_bmap, (int)B->bmap.size(), B->ws, B->arith);
  else
    launch_ir_residual_b(B->d_top, B->d_bmap, (int)B->bmap.size(), B->ws, B->arith);
  launch_finalize_b(B->d_top, B->nprob, 0, B->ws);
}

int batch_ensure_ctl(bmg_batch* B, int maxit) {
  if (B->ctls && maxit <= B->maxit_cap) return BMG_OK;
  int cap = maxit < 64 ? 64 : maxit;
  size_t stride = (sizeof(Ctl) + sizeof(double) * (size_t)(cap + 1) + 255) / 256 * 256;
  char* c = nullptr;
  CK(dev_malloc((void**)&c, stride * B->nprob));
  if (B->ctls) cudaFree(B->ctls);
  B->ctls = c;
  B->ctl_stride = stride;
  B->maxit_cap = cap;
  if (B->gexec) {   // tables and graph hold control-block addresses
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
  }
  B->g_rhs.clear();
  return BMG_OK;
}

int batch_reset(bmg_batch* B, double tol, int maxit) {
  int rc;
  if ((rc = batch_ensure_ctl(B, maxit))) return rc;
  B->ctl_host.assign(B->ctl_stride * B->nprob, 0);
  for (int p = 0; p < B->nprob; ++p) {
    Ctl* c = (Ctl*)(B->ctl_host.data() + (size_t)p * B->ctl_stride);
    c->maxit = maxit;
    c->tol = tol;
    c->scale_next = 1.0;
    c->scale_applied = 1.0;
  }
  CK(cudaMemcpyAsync(B->ctls, B->ctl_host.data(), B->ctl_host.size(), cudaMemcpyHostToDevice, B->ws));
  return BMG_OK;
}

int batch_prepare(bmg_batch* B, const double* const* rhs, double* const* x) {
  bool same = B->gexec && (int)B->g_rhs.size() == B->nprob;
  for (int p = 0; same && p < B->nprob; ++p) same = B->g_rhs[p] == rhs[p] && B->g_x[p] == x[p];
  int rc;
  if ((rc = build_batch_tables(B, rhs, x))) return rc;
  if (!B->use_graph || same) return BMG_OK;
  if (B->gexec) {
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(B->ws, cudaStreamCaptureModeThreadLocal));
  long long before = B->launches;
  batch_iteration(B);
  B->g_kernels = B->launches - before;
  B->launches = before;
  CK(cudaStreamEndCapture(B->ws, &g));
  cudaError_t e = cudaGraphInstantiate(&B->gexec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  B->g_rhs.assign(rhs, rhs + B->nprob);
  B->g_x.assign(x, x + B->nprob);
  return BMG_OK;
}

int batch_launch_iterations(bmg_batch* B, int k) {
  for (int i = 0; i < k; ++i) {
    if (B->use_graph) {
      CK(cudaGraphLaunch(B->gexec, B->ws));
      B->launches += B->g_kernels;
    } else {
      batch_iteration(B);
    }
  }
  return cuda_check(cudaGetLastError(), "batched iteration");
}

// Autotuner: for every stage of 9-point levels with n >= 127, time two sweeps
// of the row kernel for each admissible cluster size on scratch copies of the
// stage's iterates (the stencils are the real ones) and keep the fastest; for
// FP32 stages with n >= 255 also the one-pass kernel (shapes 0 and 3) and the
// two-sweep pass (shapes 0 and 3).  Every candidate computes the same bits.
struct GroupChoice {
  int cl, tile, pair, multi;
};
// (n, storage, count, kind, arith, shared operator) -> choice
static std::map<std::tuple<int, int, int, int, int, int>, GroupChoice> g_tuned;

// Whether the members of group g (stage b) share one operator -- a batch of
// right-hand sides, whose members borrow one hierarchy's level arrays.
bool group_shared(const bmg_batch* B, const bmg_batch::Group& g, int b) {
  const void* pk = nullptr;
  int cnt = 0;
  for (const bmg_hierarchy* h : B->hs) {
    const int l = h->nlev - 1 - b;
    if (l < 0) continue;
    const Level& lv = h->lv[l];
    const int storage = B->precision == BMG_FP64 ? 0 : (lv.bf16 ? 2 : 1);
    if (lv.n != g.n || lv.kind != g.kind || storage != g.storage) continue;
    if (!lv.pk32) return false;
    if (cnt++ == 0)
      pk = lv.pk32;
    else if (lv.pk32 != pk)
      return false;
  }
  return cnt >= 2;
}

// Allocates the second iterate of every problem's level in FP32 group g.
int group_alloc_x2(bmg_batch* B, const bmg_batch::Group& g, int b) {
  for (bmg_hierarchy* h : B->hs) {
    const int l = h->nlev - 1 - b;
    if (l < 0) continue;
    Level& lv = h->lv[l];
    const int storage = B->precision == BMG_FP64 ? 0 : (lv.bf16 ? 2 : 1);
    if (lv.n != g.n || lv.kind != g.kind || storage != g.storage || lv.x32b || lv.x64b) continue;
    int rc = BMG_OK;
    if (storage == 0) {
      rc = dalloc_zero(&lv.x64b, plane_size(lv.n), B->ws);
    } else {
      rc = galloc(&lv.x32b, lv.n, 1, B->ws);
    }
    if (rc) return rc;
  }
  return BMG_OK;
}

template <typename T, typename S>
int tune_group(bmg_batch* B, bmg_batch::Group& g, int b) {
  const bool shared = sizeof(T) == 4 && B->rhs_block != BMG_RHS_BLOCK_OFF && group_shared(B, g, b);
  auto key = std::make_tuple(g.n, g.storage, g.count, g.kind, B->arith, shared ? 1 : 0);
  auto it = g_tuned.find(key);
  const std::string fkey = tune_key("group", {g.n, g.storage, g.count, g.kind, B->arith, shared ? 1 : 0});
  TuneRecord fr;
  if (it == g_tuned.end() && tune_file_get(fkey, 4, &fr)) {
    const int base = rows_cluster<T>(g.n), cl = fr.v[0], tile = fr.v[1], pair = fr.v[2], multi = fr.v[3];
    const bool cl_ok = cl == base || (cl > base && cl <= 8 && (cl & (cl - 1)) == 0 && ((g.n + 1) / 2 + cl - 1) / cl >= 32);
    const bool tile_ok = tile >= -1 && tile <= 3;
    const bool pair_ok = pair == -1 || (sizeof(T) == 4 && pair >= 0 && pair <= 3);
    const bool multi_ok = multi == 0 || (shared && (multi == 2 || multi == 4) && g.count >= multi && tile >= 0);
    if (cl_ok && tile_ok && pair_ok && multi_ok) it = g_tuned.emplace(key, GroupChoice{cl, tile, pair, multi}).first;
  }
  if (it == g_tuned.end()) {
    const int base = rows_cluster<T>(g.n);
    const size_t ps = plane_stride32(g.n);   // scratch x, x2, f per problem, laid out like level arrays
    T* scratch = nullptr;
    int rc = galloc(&scratch, g.n, 3 * g.count, B->ws);
    if (rc) return rc;
    std::vector<LevelDesc<T, S>> d((const LevelDesc<T, S>*)g.host.data(),
                                   (const LevelDesc<T, S>*)g.host.data() + g.count);
    for (int k = 0; k < g.count; ++k) {
      d[k].x = scratch + 3 * ps * k;
      d[k].x2 = scratch + 3 * ps * k + ps;
      d[k].f = scratch + 3 * ps * k + 2 * ps;
      d[k].done = nullptr;
    }
    LevelDesc<T, S>* dd = nullptr;
    rc = cuda_check(dev_malloc((void**)&dd, sizeof(LevelDesc<T, S>) * g.count), "tuning descriptors");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(dd, d.data(), sizeof(LevelDesc<T, S>) * g.count, cudaMemcpyHostToDevice, B->ws),
                      "tuning descriptors");
    GroupChoice best{base, -1, -1, 0};
    float best_ms = 1e30f, tile_ms = 1e30f;
    for (int cl = base; cl <= 8 && !rc; cl *= 2) {
      if (cl > base && ((g.n + 1) / 2 + cl - 1) / cl < 32) break;   // fewer than a warp of pairs per CTA
      float ms = 0;
      rc = time_call(B->ws, [&] { launch_gs_b<T, S>(dd, g.count, g.n, 9, 2, cl, B->ws, B->arith); }, &ms);
      if (ms * 0.5f < best_ms) {
        best_ms = ms * 0.5f;
        best.cl = cl;
      }
    }
    if constexpr (sizeof(T) == 8) {
      if (!rc && g.n >= 255) {
        for (int shape : {0, 2}) {   // the one-wave heights with 4- and 6-row rings
          float ms = 0;
          rc = time_call(B->ws, [&] {
            launch_gs_tile64_b((const LevelDesc<double, double>*)dd, g.count, g.n, shape, 0, B->ws, B->arith);
            launch_gs_tile64_b((const LevelDesc<double, double>*)dd, g.count, g.n, shape, 1, B->ws, B->arith);
          }, &ms);
          if (rc) break;
          if (ms * 0.5f < tile_ms) {
            tile_ms = ms * 0.5f;
            if (tile_ms < best_ms) best.tile = shape;
          }
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (!rc && g.n >= 255) {
        for (int shape : {0, 3}) {
          float ms = 0;
          rc = time_call(B->ws, [&] {
            launch_gs_tile_b<S>(dd, g.count, g.n, shape, 0, B->ws, B->arith);
            launch_gs_tile_b<S>(dd, g.count, g.n, shape, 1, B->ws, B->arith);
          }, &ms);
          if (rc) break;
          if (ms * 0.5f < tile_ms) {
            tile_ms = ms * 0.5f;
            if (tile_ms < best_ms) best.tile = shape;
          }
        }
        if (!rc && best.tile >= 0) {
          best_ms = tile_ms;
          float pair_best = 1e30f;
          for (int shape : {0, 3}) {
            float ms = 0;
            rc = time_call(B->ws, [&] {
              launch_gs_pair_b<S>(dd, g.count, g.n, shape, 0, B->ws, B->arith);
              launch_gs_pair_b<S>(dd, g.count, g.n, shape, 1, B->ws, B->arith);
            }, &ms);
            if (rc) break;
            if (ms * 0.25f < pair_best) {   // per sweep: two launches of two sweeps
              pair_best = ms * 0.25f;
              if (pair_best < best_ms) best.pair = shape;
            }
          }
          if (pair_best < best_ms) best_ms = pair_best;
        }
        // members of one operator: sweeps with 2 or 4 of them per warp
        for (int k : {2, 4}) {
          if (rc || !shared || g.count < k) break;
          float ms = 0;
          rc = time_call(B->ws, [&] {
            launch_gs_tile_bk<S>((const LevelDesc<float, S>*)dd, g.count, g.n, k, 0, B->ws, B->arith);
            launch_gs_tile_bk<S>((const LevelDesc<float, S>*)dd, g.count, g.n, k, 1, B->ws, B->arith);
          }, &ms);
          if (!rc && ms * 0.5f < best_ms) {
            best_ms = ms * 0.5f;
            best.multi = k;
            best.pair = -1;
            if (best.tile < 0) best.tile = 0;
          }
        }
      }
    }
    cudaFree(dd);
    gfree(scratch);
    if (!rc && strip_timeouts_b()) rc = set_error(BMG_ETIMEOUT, "batched one-pass sweep: bulk copies did not complete");
    if (rc) return rc;
    it = g_tuned.emplace(key, best).first;
    tune_file_put(fkey, TuneRecord{{best.cl, best.tile, best.pair, best.multi}, best_ms});
  }
  g.cl = it->second.cl;
  g.tile = it->second.tile;
  g.pair = it->second.pair;
  g.multi = it->second.multi;
  if (g.tile >= 0) return group_alloc_x2(B, g, b);
  return BMG_OK;
}

// BMG_SMOOTHER_TILE + s / BMG_SMOOTHER_PAIR + s on a batch: every group of
// 9-point levels outside the tails sweeps with the one-pass kernel of shape s
// (s <= 3; FP64 groups use the FP64 one-pass kernel), or (FP32 only) runs pairs
// of sweeps as two-sweep passes of shape s.
int force_batch_onepass(bmg_batch* B) {
  for (int b = 1; b <= B->bmax; ++b)
    for (auto& g : B->stages[b]) {
      if (!g.count || g.kind != 9) continue;
      if (B->smoother >= BMG_SMOOTHER_PAIR) {
        g.tile = 3;
        g.pair = B->smoother - BMG_SMOOTHER_PAIR;
      } else {
        g.tile = B->smoother - BMG_SMOOTHER_TILE;
      }
      int rc = group_alloc_x2(B, g, b);
      if (rc) return rc;
    }
  return BMG_OK;
}

// rhs_block = 2 or 4: every FP32 group of a shared operator sweeps with that
// many members per warp (allocating the second iterates it needs).
int force_rhs_block(bmg_batch* B) {
  if (B->precision == BMG_FP64 || (B->rhs_block != 2 && B->rhs_block != 4)) return BMG_OK;
  for (int b = 1; b <= B->bmax; ++b)
    for (auto& g : B->stages[b]) {
      if (!g.count || g.kind != 9 || g.storage == 0 || !group_shared(B, g, b)) continue;
      g.multi = B->rhs_block;
      g.pair = -1;
      if (g.tile < 0) g.tile = 0;
      if (int rc = group_alloc_x2(B, g, b)) return rc;
    }
  return BMG_OK;
}

int autotune_batch(bmg_batch* B) {
  std::lock_guard<std::mutex> guard(tune_lock());
  // descriptor contents are needed: build the tables with the internal level
  // arrays standing in for the caller buffers of level 0
  std::vector<const double*> rhs(B->nprob);
  std::vector<double*> x(B->nprob);
  for (int p = 0; p < B->nprob; ++p) {
    rhs[p] = B->hs[p]->lv[0].st;   // any valid device address: tuning swaps in scratch iterates
    x[p] = B->hs[p]->lv[0].st;
  }
  int rc;
  if ((rc = build_batch_tables(B, rhs.data(), x.data()))) return rc;
  for (int b = 1; b <= B->bmax; ++b) {
    for (auto& g : B->stages[b]) {
      if (!g.count || g.kind != 9 || g.n < 127 || g.tile >= 0) continue;   // forced groups keep their kernel
      if (g.storage == 0) rc = tune_group<double, double>(B, g, b);
      else if (g.storage == 1) rc = tune_group<float, float>(B, g, b);
      else rc = tune_group<float, __nv_bfloat16>(B, g, b);
      if (rc) return rc;
      B->tuned_cl[b] = g.tile >= 0 ? BMG_TILE_SWEEP + g.tile : g.cl;
    }
  }
  return BMG_OK;
}

// Options and streams of a new batch; *so gets the options of its member
// hierarchies (plain launches, point smoother, the batch's stream).
int batch_init(bmg_batch* B, const bmg_opts* o, bmg_opts* so) {
  *so = bmg_opts{};
  if (o) *so = *o;
  so->use_graph = 0;
  so->smoother = BMG_SMOOTHER_AUTO;
  if (o) B->smoother = o->smoother;
  if (is_line(B->smoother))
    return set_error(BMG_EINVAL, "batched solves: line relaxation is available for single problems only");
  if (B->smoother < BMG_SMOOTHER_AUTO ||
      (B->smoother >= BMG_SMOOTHER_TILE + 4 && B->smoother < BMG_SMOOTHER_PAIR) ||
      B->smoother >= BMG_SMOOTHER_PAIR + GS_PAIR_SHAPES)
    return set_error(BMG_EINVAL, "batched solves: bad smoother %d", B->smoother);
  if (o) {
    B->precision = o->precision;
    if (o->nu1 || o->nu2) {
      B->nu1 = o->nu1;
      B->nu2 = o->nu2;
    }
    B->inner = o->inner_cycles > 0 ? o->inner_cycles : 1;
    B->use_graph = o->use_graph;
    B->user = (cudaStream_t)o->stream;
    B->arith = o->arith;
    B->rhs_block = o->rhs_block;
  }
  if (B->rhs_block != BMG_RHS_BLOCK_AUTO && B->rhs_block != BMG_RHS_BLOCK_OFF && B->rhs_block != 2 &&
      B->rhs_block != 4)
    return set_error(BMG_EINVAL, "batched solves: bad rhs_block %d", B->rhs_block);
  if (B->arith < BMG_ARITH_ROUNDED || B->arith > BMG_ARITH_FUSED)
    return set_error(BMG_EINVAL, "batched solves: bad arith %d", B->arith);
  if (B->precision == BMG_FP64 && B->smoother >= BMG_SMOOTHER_PAIR)
    return set_error(BMG_EINVAL, "batched solves: two-sweep passes are FP32 only");
  int rc = cuda_check(cudaStreamCreateWithFlags(&B->ws, cudaStreamNonBlocking), "stream");
  if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming), "event");
  if (!rc) rc = cuda_check(cudaEventRecord(B->ev, B->user), "event");
  if (!rc) rc = cuda_check(cudaStreamWaitEvent(B->ws, B->ev, 0), "event");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(B->ws), "sync");
  so->stream = (void*)B->ws;
  return rc;
}

// A member hierarchy for one more right-hand side of h0's operator: it borrows
// h0's stencils, weights and Cholesky factor and owns zeroed iterates,
// right-hand sides and norm partials.
int clone_state(const bmg_hierarchy* h0, cudaStream_t s, bmg_hierarchy** out) {
  bmg_hierarchy* h = new bmg_hierarchy();
  h->shared_ops = true;
  h->n = h0->n;
  h->nlev = h0->nlev;
  h->precision = h0->precision;
  h->nu1 = h0->nu1;
  h->nu2 = h0->nu2;
  h->inner = h0->inner;
  h->coarsest = h0->coarsest;
  h->use_graph = 0;
  h->arith = h0->arith;
  h->m = h0->m;
  h->Lfac = h0->Lfac;
  h->work = h0->work;
  h->lv.resize(h0->lv.size());
  int rc = BMG_OK;
  for (size_t l = 0; l < h0->lv.size() && !rc; ++l) {
    const Level& S = h0->lv[l];
    Level& L = h->lv[l];
    L.n = S.n;
    L.kind = S.kind;
    L.bf16 = S.bf16;
    L.fused = S.fused;
    L.st = S.st;
    L.ci = S.ci;
    L.st32 = S.st32;
    L.pk32 = S.pk32;
    L.off16 = S.off16;
    L.od32 = S.od32;
    L.ci32 = S.ci32;
    const size_t ps = plane_size(L.n);
    if (l >= 1) {
      if (!(rc = dalloc(&L.x, ps))) rc = dalloc(&L.f, ps);
      if (!rc) rc = cuda_check(cudaMemsetAsync(L.x, 0, ps * sizeof(double), s), "clone");
      if (!rc) rc = cuda_check(cudaMemsetAsync(L.f, 0, ps * sizeof(double), s), "clone");
    }
    if (!rc && h->precision != BMG_FP64) {
      if (!(rc = galloc(&L.x32, L.n, 1, s))) rc = galloc(&L.f32, L.n, 1, s);
    }
  }
  if (!rc) rc = dalloc(&h->partials, 2 * (size_t)norm_partials_max());
  if (rc) {
    bmg_free(h);
    return rc;
  }
  *out = h;
  return BMG_OK;
}

// Stage tables, tails, control blocks and kernel choices of a batch whose
// member hierarchies are in B->hs.
int batch_finish(bmg_batch* B, int rc) {
  const int nprob = B->nprob;
  if (!rc) {
    B->stages.assign(B->bmax + 1, {});
    B->tuned_cl.assign(B->bmax + 1, 0);
    B->tail_count.assign(B->bmax + 1, 0);
    B->tail_n.assign(B->bmax + 1, 0);
    B->tail_host.assign(B->bmax + 1, {});
    B->tail_dev.assign(B->bmax + 1, nullptr);
    rc = build_batch_tables(B, nullptr, nullptr);   // group sizes
  }
  for (auto& st : B->stages)
    for (auto& g : st) {
      if (rc || !g.count) continue;
      g.cl = g.storage == 0 ? rows_cluster<double>(g.n) : rows_cluster<float>(g.n);
      rc = cuda_check(dev_malloc((void**)&g.d, g.elem * g.count), "batched tables");
    }
  for (size_t b = 0; !rc && b < B->tail_count.size(); ++b)
    if (B->tail_count[b])
      rc = cuda_check(dev_malloc((void**)&B->tail_dev[b], (B->precision == BMG_FP64 ? sizeof(TailDesc<double>)
                                                                             : sizeof(TailDesc<float>)) *
                                                      B->tail_count[b]),
                      "batched tails");
  if (!rc) rc = cuda_check(dev_malloc((void**)&B->d_top, sizeof(TopDesc) * nprob), "batched tables");
  if (!rc) {
    for (int p = 0; p < nprob; ++p) {
      const int G = B->hs[p]->n < norm_partials_max() ? B->hs[p]->n : norm_partials_max();
      for (int b = 0; b < G; ++b) B->bmap.push_back(make_int2(p, b));
    }
    rc = cuda_check(dev_malloc((void**)&B->d_bmap, sizeof(int2) * B->bmap.size()), "batched tables");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(B->d_bmap, B->bmap.data(), sizeof(int2) * B->bmap.size(), cudaMemcpyHostToDevice,
                                      B->ws),
                      "batched tables");
  }
  if (!rc) rc = cuda_check(dev_malloc((void**)&B->d_alldone, sizeof(int)), "batched flag");
  if (!rc) rc = cuda_check(host_malloc((void**)&B->h_alldone, sizeof(int)), "pinned");
  if (!rc) rc = batch_ensure_ctl(B, 64);
  if (!rc && B->smoother >= BMG_SMOOTHER_TILE) rc = force_batch_onepass(B);
  if (!rc && B->use_graph) rc = autotune_batch(B);
  if (!rc) rc = force_rhs_block(B);
  if (!rc) rc = cuda_check(cudaStreamSynchronize(B->ws), "batched setup");
  return rc;
}

}  // namespace

extern "C" {

int bmg_setup_batched(int nprob, const bmg_stencil* A, const int* n, const bmg_opts* o, bmg_batch** out) {
  Range nvtx("bmg_setup_batched");
  if (!out) return set_error(BMG_EINVAL, "bmg_setup_batched: out is NULL");
  *out = nullptr;
  if (nprob < 1 || !A || !n) return set_error(BMG_EINVAL, "bmg_setup_batched: bad argument");
  if (o && o->krylov != BMG_KRYLOV_NONE) return set_error(BMG_EINVAL, "bmg_setup_batched: stationary cycles only");
  for (int p = 1; p < nprob; ++p)
    if (A[p].kind != A[0].kind) return set_error(BMG_EINVAL, "bmg_setup_batched: problems differ in kind");
  for (int p = 0; p < nprob; ++p)
    if (!is_level_size(n[p])) return set_error(BMG_EINVAL, "bmg_setup_batched: n = %d is not 2^m - 1 >= 3", n[p]);
  bmg_batch* B = new bmg_batch();
  B->nprob = nprob;
  bmg_opts so{};
  CounterScope cs(&B->launches);
  int rc = batch_init(B, o, &so);
  for (int p = 0; p < nprob && !rc; ++p) {
    bmg_hierarchy* h = nullptr;
    rc = bmg_setup(&A[p], n[p], n[p], &so, &h);
    if (!rc) {
      B->hs.push_back(h);
      B->launches += h->launches;
      B->maxn = std::max(B->maxn, n[p]);
      B->bmax = std::max(B->bmax, h->nlev - 1);
    }
  }
  rc = batch_finish(B, rc);
  if (rc) {
    bmg_free_batched(B);
    return rc;
  }
  *out = B;
  return BMG_OK;
}

int bmg_batch_rhs(const bmg_hierarchy* h0, int k, const bmg_opts* o, bmg_batch** out) {
  Range nvtx("bmg_batch_rhs");
  if (!out) return set_error(BMG_EINVAL, "bmg_batch_rhs: out is NULL");
  *out = nullptr;
  if (!h0 || k < 1) return set_error(BMG_EINVAL, "bmg_batch_rhs: bad argument");
  if (h0->shared_ops) return set_error(BMG_EINVAL, "bmg_batch_rhs: h is itself a batch member");
  if (h0->fpad) return set_error(BMG_EINVAL, "bmg_batch_rhs: h holds an embedded (general-size) problem");
  if (h0->per) return set_error(BMG_EINVAL, "bmg_batch_rhs: h has periodic sides");
  if (o && o->krylov != BMG_KRYLOV_NONE) return set_error(BMG_EINVAL, "bmg_batch_rhs: stationary cycles only");
  if (o && o->precision != h0->precision)
    return set_error(BMG_EINVAL, "bmg_batch_rhs: precision %d differs from the hierarchy's %d", o->precision,
                     h0->precision);
  if (o && o->arith != h0->arith)
    return set_error(BMG_EINVAL, "bmg_batch_rhs: arith %d differs from the hierarchy's %d", o->arith, h0->arith);
  bmg_batch* B = new bmg_batch();
  B->nprob = k;
  bmg_opts so{};
  CounterScope cs(&B->launches);
  int rc = batch_init(B, o, &so);
  B->precision = h0->precision;
  B->arith = h0->arith;
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h0->ws), "bmg_batch_rhs");   // h0's setup has finished
  for (int p = 0; p < k && !rc; ++p) {
    bmg_hierarchy* h = nullptr;
    rc = clone_state(h0, B->ws, &h);
    if (!rc) {
      B->hs.push_back(h);
      B->maxn = h0->n;
      B->bmax = h0->nlev - 1;
    }
  }
  rc = batch_finish(B, rc);
  if (rc) {
    bmg_free_batched(B);
    return rc;
  }
  *out = B;
  return BMG_OK;
}

int bmg_solve_batched(bmg_batch* B, const double* const* rhs, double* const* x, double tol, int maxit, int* iters,
                      double* relres) {
  Range nvtx("bmg_solve_batched");
  if (!B || !rhs || !x) return set_error(BMG_EINVAL, "bmg_solve_batched: NULL argument");
  if (maxit < 0 || !(tol >= 0.0)) return set_error(BMG_EINVAL, "bmg_solve_batched: bad tol or maxit");
  for (int p = 0; p < B->nprob; ++p)
    if (!rhs[p] || !x[p]) return set_error(BMG_EINVAL, "bmg_solve_batched: NULL buffer of problem %d", p);
  CounterScope cs(&B->launches);
  int rc;
  CK(cudaEventRecord(B->ev, B->user));
  CK(cudaStreamWaitEvent(B->ws, B->ev, 0));
  if ((rc = batch_reset(B, tol, maxit))) return rc;
  if ((rc = batch_prepare(B, rhs, x))) return rc;
  batch_initial(B);
  const int chunk = 4;
  int launched = 0;
  for (;;) {
    launch_all_done(B->ctls, B->ctl_stride, B->nprob, B->d_alldone, B->ws);
    CK(cudaMemcpyAsync(B->h_alldone, B->d_alldone, sizeof(int), cudaMemcpyDeviceToHost, B->ws));
    CK(cudaStreamSynchronize(B->ws));
    if (*B->h_alldone || launched >= maxit) break;
    int k = maxit - launched < chunk ? maxit - launched : chunk;
    if ((rc = batch_launch_iterations(B, k))) return rc;
    launched += k;
  }
  B->ctl_host.resize(B->ctl_stride * B->nprob);
  CK(cudaMemcpy(B->ctl_host.data(), B->ctls, B->ctl_host.size(), cudaMemcpyDeviceToHost));
  B->hist.assign(B->nprob, {});
  int worst = BMG_OK;
  for (int p = 0; p < B->nprob; ++p) {
    const Ctl* c = (const Ctl*)(B->ctl_host.data() + (size_t)p * B->ctl_stride);
    B->hist[p].assign(c->hist, c->hist + c->it + 1);
    if (iters) iters[p] = c->it;
    if (relres) relres[p] = c->hist[0] > 0 ? c->hist[c->it] / c->hist[0] : 0.0;
    if (c->done == 3) worst = BMG_ENAN;
    else if (c->done != 1 && worst == BMG_OK) worst = BMG_ENOTCONV;
  }
  if (strip_timeouts_b()) return set_error(BMG_ETIMEOUT, "bmg_solve_batched: a one-pass sweep timed out");
  if ((rc = debug_check("bmg_solve_batched"))) return rc;
  if (worst == BMG_ENAN) return set_error(BMG_ENAN, "bmg_solve_batched: a residual norm is not finite");
  if (worst == BMG_ENOTCONV) return set_error(BMG_ENOTCONV, "bmg_solve_batched: not every problem converged");
  return BMG_OK;
}

int bmg_batched_history(const bmg_batch* B, int p, double* out, int cap) {
  if (!B || p < 0 || p >= B->nprob) return set_error(BMG_EINVAL, "bmg_batched_history: bad argument");
  if (p >= (int)B->hist.size()) return 0;
  int cnt = (int)B->hist[p].size();
  if (out)
    for (int k = 0; k < cnt && k < cap; ++k) out[k] = B->hist[p][k];
  return cnt;
}

int bmg_time_cycles_batched(bmg_batch* B, const double* const* rhs, double* const* x, int cycles, double* ms) {
  if (!B || !rhs || !x || !ms || cycles < 1) return set_error(BMG_EINVAL, "bmg_time_cycles_batched: bad argument");
  CounterScope cs(&B->launches);
  int rc;
  CK(cudaEventRecord(B->ev, B->user));
  CK(cudaStreamWaitEvent(B->ws, B->ev, 0));
  if ((rc = batch_reset(B, 0.0, cycles))) return rc;
  if ((rc = batch_prepare(B, rhs, x))) return rc;
  batch_initial(B);
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, B->ws));
  if ((rc = batch_launch_iterations(B, cycles))) return rc;
  CK(cudaEventRecord(b, B->ws));
  CK(cudaEventSynchronize(b));
  float t = 0;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t;
  if (strip_timeouts_b()) return set_error(BMG_ETIMEOUT, "bmg_time_cycles_batched: a one-pass sweep timed out");
  return BMG_OK;
}

long long bmg_batched_launch_count(const bmg_batch* B) { return B ? B->launches : 0; }

int bmg_batched_tuned_cluster(const bmg_batch* B, int stage) {
  if (!B || stage < 0 || stage > B->bmax) return set_error(BMG_EINVAL, "bmg_batched_tuned_cluster: bad stage");
  return B->tuned_cl[stage];
}

void bmg_free_batched(bmg_batch* B) {
  if (!B) return;
  if (B->ws) cudaStreamSynchronize(B->ws);
  for (auto* h : B->hs) bmg_free(h);
  for (auto& st : B->stages)
    for (auto& g : st) cudaFree(g.d);
  for (void* t : B->tail_dev) cudaFree(t);
  cudaFree(B->d_top);
  cudaFree(B->d_bmap);
  cudaFree(B->ctls);
  cudaFree(B->d_alldone);
  if (B->h_alldone) cudaFreeHost(B->h_alldone);
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->ws) cudaStreamDestroy(B->ws);
  delete B;
}

}  // extern "C"
