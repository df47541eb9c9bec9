// Batched V-cycle kernels: one launch per stage for many independent problems.
// Stages are levels counted from the coarsest (all problems reach the same
// coarsest size), so the problems of a stage share n and one grid shape; the
// problem index is the last grid dimension.  The bodies are those of the
// single-problem kernels (cycle_device.cuh), so every problem's arithmetic, and
// with it its residual history, is the same as in a solo solve.
#include "cycle_device.cuh"

namespace bmg {

using namespace dev;

namespace {

constexpr int BX = 32, BY = 8;

// FU: fused multiply-adds (BMG_ARITH_FUSED), as in the single-problem kernels.
template <typename T, typename S, int CL, bool FU>
__global__ void __launch_bounds__(rows_threads_max<T>(), sizeof(T) == 8 ? 2 : 1)
    k_gs_rows_b(const LevelDesc<T, S>* __restrict__ d, int pj) {
  pdl_enter();
  const LevelDesc<T, S> q = d[blockIdx.y];
  if (stopped(q.done)) return;   // uniform over the cluster: its CTAs share blockIdx.y
  gs_rows_body<T, S, CL, FU>(q.v, q.f, q.x, pj, blockIdx.x);
}

template <typename T, typename S, bool FU>
__global__ void k_gs_checker_b(const LevelDesc<T, S>* __restrict__ d, int c) {
  pdl_enter();
  const LevelDesc<T, S> q = d[blockIdx.z];
  if (stopped(q.done)) return;
  gs_checker_body<T, S, FU>(q.v, q.f, q.x, c, blockIdx.x, blockIdx.y);
}

template <typename T, typename S, bool NINE, bool FU>
__global__ void __launch_bounds__(TXC* TYC) k_resid_restrict_b(const LevelDesc<T, S>* __restrict__ d, int dir) {
  pdl_enter();
  const LevelDesc<T, S> q = d[blockIdx.z];
  if (stopped(q.done)) return;
  resid_restrict_body<T, S, NINE, FU>(q.v, q.ci, dir ? q.x2 : q.x, q.f, q.fc, q.xc, blockIdx.x, blockIdx.y);
}

template <typename T, typename S, bool FU>
__global__ void k_interp_b(const LevelDesc<T, S>* __restrict__ d, int din, int dout) {
  pdl_enter();
  const LevelDesc<T, S> q = d[blockIdx.z];
  if (stopped(q.done)) return;
  interp_body<T, FU>(q.v.n, q.ci, q.xc, din ? q.x2 : q.x, dout ? q.x2 : q.x,
                     blockIdx.x * blockDim.x + threadIdx.x + 1, blockIdx.y * blockDim.y + threadIdx.y + 1);
}

// One-pass sweeps of a group: warp g takes strip g % wpp of problem g / wpp.
constexpr int STRIP_WARPS_B = 4;
__device__ int g_strip_timeout_b = 0;

template <typename S, int TY, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS_B) k_gs_strip_ring_b(const LevelDesc<float, S>* __restrict__ d,
                                                                        int count, int n, int dir) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  const int nbx = (n + 55) / 56, wpp = nbx * ((n + TY - 1) / TY);
  const int w = threadIdx.x >> 5;
  const long g = (long)blockIdx.x * STRIP_WARPS_B + w;
  const int p = (int)(g / wpp), sidx = (int)(g % wpp);
  if (p >= count) return;                         // whole warps only
  const LevelDesc<float, S> q = d[p];
  if (stopped(q.done)) return;
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRing<S>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS_B * RING * StripRing<S>::SLOT) +
      w * RING;
  if (!gs_strip_ring_body<S, RING, FU>(q.v, q.f, dir ? q.x2 : q.x, dir ? q.x : q.x2, sidx % nbx, sidx / nbx, TY,
                                       ring, bars) &&
      (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout_b, 1);
}

// One sweep of a group whose members share one operator, K members per warp:
// warp g takes strip g % wpp of members K (g / wpp) .. K (g / wpp) + K - 1 (the
// last group padded with the last member, which it does not store).
template <typename S, int K, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS_B) k_gs_strip_ring_bk(const LevelDesc<float, S>* __restrict__ d,
                                                                         int count, int n, int dir, int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  const int nbx = (n + 55) / 56, wpp = nbx * ((n + ty - 1) / ty);
  const int w = threadIdx.x >> 5;
  const long g = (long)blockIdx.x * STRIP_WARPS_B + w;
  const int p0 = (int)(g / wpp) * K, sidx = (int)(g % wpp);
  if (p0 >= count) return;
  const float* fs[K];
  const float* xi[K];
  float* xo[K];
  unsigned active = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int p = p0 + q < count ? p0 + q : count - 1;
    const LevelDesc<float, S>& e = d[p];
    if (p0 + q < count && !stopped(e.done)) active |= 1u << q;
    fs[q] = e.f;
    xi[q] = dir ? e.x2 : e.x;
    xo[q] = dir ? e.x : e.x2;
  }
  if (!active) return;
  const StencilView<float, S> v = d[p0].v;
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRingK<S, K>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS_B * RING * StripRingK<S, K>::SLOT) +
      w * RING;
  if (!gs_strip_ring_k_body<S, K, RING, FU>(v, fs, xi, xo, active, sidx % nbx, sidx / nbx, ty, ring, bars) &&
      (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout_b, 1);
}

template <typename S, int TY, int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS_B) k_gs_strip2_ring_b(const LevelDesc<float, S>* __restrict__ d,
                                                                         int count, int n, int dir) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  const int nbx = (n + 47) / 48, wpp = nbx * ((n + TY - 1) / TY);
  const int w = threadIdx.x >> 5;
  const long g = (long)blockIdx.x * STRIP_WARPS_B + w;
  const int p = (int)(g / wpp), sidx = (int)(g % wpp);
  if (p >= count) return;
  const LevelDesc<float, S> q = d[p];
  if (stopped(q.done)) return;
  unsigned char* ring = strip_smem + (size_t)w * RING * StripRing<S>::SLOT;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(strip_smem + (size_t)STRIP_WARPS_B * RING * StripRing<S>::SLOT) +
      w * RING;
  if (!gs_strip2_ring_body<S, RING, FU>(q.v, q.f, dir ? q.x2 : q.x, dir ? q.x : q.x2, sidx % nbx, sidx / nbx, TY,
                                        ring, bars) &&
      (threadIdx.x & 31) == 0)
    atomicExch(&g_strip_timeout_b, 1);
}

// FP64 one-pass sweeps of a group (strips of 56 x ty, rows copied per lane; see
// gs_strip64_body): warp g takes strip g % wpp of problem g / wpp.
template <int RING, bool FU>
__global__ void __launch_bounds__(32 * STRIP_WARPS_B) k_gs_strip64_b(const LevelDesc<double, double>* __restrict__ d,
                                                                     int count, int n, int dir, int ty) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char strip_smem[];
  const int nbx = (n + 55) / 56, wpp = nbx * ((n + ty - 1) / ty);
  const int w = threadIdx.x >> 5;
  const long g = (long)blockIdx.x * STRIP_WARPS_B + w;
  const int p = (int)(g / wpp), sidx = (int)(g % wpp);
  if (p >= count) return;                         // whole warps only
  const LevelDesc<double, double> q = d[p];
  if (stopped(q.done)) return;
  gs_strip64_body<RING, FU>(q.v, q.f, dir ? q.x2 : q.x, dir ? q.x : q.x2, sidx % nbx, sidx / nbx, ty,
                            strip_smem + (size_t)w * RING * STRIP64_SLOT);
}

template <typename T, typename S>
__global__ void k_coarse_b(const LevelDesc<T, S>* __restrict__ d) {
  pdl_enter();
  const LevelDesc<T, S> q = d[blockIdx.x];
  if (stopped(q.done)) return;
  coarse_solve_body<T>(q.v.n, q.L, q.f, q.x, q.y);
}

// Top-level kernels: problems of different sizes in one grid; block b of a
// problem runs only when b < G = min(n, 1024) of that problem, so every
// problem keeps the reduction order of its solo solve.
template <bool FU>
// The residual-type kernels of the top levels run the blocks of every problem's
// canonical reduction (block b of G = min(n, 1024)) and no others: bmap[k] =
// (problem, b) for the k-th block of the launch.
__global__ void __launch_bounds__(NORM_THREADS) k_residual_b(const TopDesc* __restrict__ d,
                                                             const int2* __restrict__ bmap) {
  pdl_enter();
  const int2 m = bmap[blockIdx.x];
  const TopDesc& q = d[m.x];
  const int G = norm_blocks(q.v.n);
  if (q.ctl->done) return;
  if (q.kind == 9)
    residual_body<double, double, true, FU>(q.v, q.x, q.f, (double*)nullptr, q.partials, m.y, G);
  else
    residual_body<double, double, false, FU>(q.v, q.x, q.f, (double*)nullptr, q.partials, m.y, G);
}

__global__ void __launch_bounds__(NORM_THREADS) k_finalize_b(const TopDesc* __restrict__ d, int phase) {
  pdl_enter();
  const TopDesc q = d[blockIdx.x];
  finalize_body(q.partials, norm_blocks(q.v.n), q.ctl, phase, nullptr);
}

__global__ void k_ir_update_b(const TopDesc* __restrict__ d) {
  pdl_enter();
  const TopDesc q = d[blockIdx.z];
  if (q.ctl->done) return;
  ir_update_cols(q.v.n, q.x, q.e32, q.ctl->scale_applied, blockIdx.x * (BX * IRU_COLS) + threadIdx.x + 1,
                 blockIdx.y * blockDim.y + threadIdx.y + 1, BX);
}

template <bool FU>
__global__ void __launch_bounds__(NORM_THREADS) k_ir_residual_b(const TopDesc* __restrict__ d,
                                                                const int2* __restrict__ bmap) {
  pdl_enter();
  const int2 m = bmap[blockIdx.x];
  const TopDesc& q = d[m.x];
  const int G = norm_blocks(q.v.n);
  if (q.ctl->done) return;
  ir_residual_body<FU>(q.v, q.kind == 9, q.x, q.f, q.r32, q.e32, q.partials, q.ctl, m.y, G);
}

// One problem's level-fused tail per CTA.  The iterates and right-hand sides
// the tail writes live in shared memory for its duration (the top level's
// iterate is loaded at entry and written back at exit; the coarser levels' x
// and f exist only here), so a colour phase reads the previous phase's values
// from shared memory instead of L2; the read-only stencils, weights and the
// top level's right-hand side stay in global memory (cached in L1).
template <typename T>
__host__ __device__ inline size_t tail_smem_elems(int n0) {
  size_t e = (size_t)(n0 + 2) * (n0 + 2);
  for (int n = (n0 - 1) / 2; n >= 3; n = (n - 1) / 2) e += 2 * (size_t)(n + 2) * (n + 2);
  return e;
}

template <typename T, bool FU>
__global__ void __launch_bounds__(1024) k_tail(const TailDesc<T>* __restrict__ d, const int* done) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ TailDesc<T> q;
  const TailDesc<T>& g = d[blockIdx.x];
  if (stopped(done) || stopped(g.done)) return;
  T* sm = reinterpret_cast<T*>(tail_smem);
  const size_t ps0 = plane_size(g.lv[0].v.n);
  if (threadIdx.x == 0) {
    q = g;
    size_t off = ps0;
    for (int l = 1; l < g.nlev; ++l) {
      const size_t ps = plane_size(g.lv[l].v.n);
      q.lv[l].x = sm + off;
      q.lv[l].f = sm + off + ps;
      q.lv[l - 1].xc = sm + off;
      q.lv[l - 1].fc = sm + off + ps;
      off += 2 * ps;
    }
    q.lv[0].x = sm;
  }
  size_t total = ps0;
  for (int l = 1; l < g.nlev; ++l) total += 2 * plane_size(g.lv[l].v.n);
  for (size_t k = threadIdx.x; k < ps0; k += blockDim.x) sm[k] = g.lv[0].x[k];
  for (size_t k = ps0 + threadIdx.x; k < total; k += blockDim.x) sm[k] = T(0);
  __syncthreads();
  tail_body<T, FU>(q, q.top_kind);
  for (size_t k = threadIdx.x; k < ps0; k += blockDim.x) g.lv[0].x[k] = sm[k];
}

// 1 when every problem's control flag is set.
__global__ void k_all_done(const char* __restrict__ ctls, size_t stride, int count, int* out) {
  pdl_enter();
  __shared__ int any_running;
  if (threadIdx.x == 0) any_running = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < count; p += blockDim.x)
    if (((const Ctl*)(ctls + (size_t)p * stride))->done == 0) any_running = 1;
  __syncthreads();
  if (threadIdx.x == 0) *out = any_running ? 0 : 1;
}

template <typename T, typename S, int CL, bool FU>
void rows_b(const LevelDesc<T, S>* d, int count, int n, int threads, cudaStream_t s) {
  for (int pj = 1; pj >= 0; --pj) {
    const int rows = pj ? (n + 1) / 2 : (n - 1) / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(rows * CL), (unsigned)count);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = CL;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CL > 1 ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k_gs_rows_b<T, S, CL, FU>, d, pj);
    count_launch();
  }
}

}  // namespace

// cl: cluster size of the row kernel (>= rows_cluster<T>(n); the autotuner may
// pick a larger one, which splits each row over more, smaller CTAs).
template <typename T, typename S, bool FU>
static void gs_b(const LevelDesc<T, S>* d, int count, int n, int kind, int sweeps, int cl, cudaStream_t s) {
  if (kind == 9) {
    const int threads = rows_threads(n, cl);
    for (int k = 0; k < sweeps; ++k) {
      switch (cl) {
        case 1: rows_b<T, S, 1, FU>(d, count, n, threads, s); break;
        case 2: rows_b<T, S, 2, FU>(d, count, n, threads, s); break;
        case 4: rows_b<T, S, 4, FU>(d, count, n, threads, s); break;
        default: rows_b<T, S, 8, FU>(d, count, n, threads, s); break;
      }
    }
  } else {
    dim3 g(((n + 1) / 2 + BX - 1) / BX, (n + BY - 1) / BY, count);
    for (int k = 0; k < sweeps; ++k) {
      pdl_launch(k_gs_checker_b<T, S, FU>, g, dim3(BX, BY), 0, s, d, 0);
      count_launch();
      pdl_launch(k_gs_checker_b<T, S, FU>, g, dim3(BX, BY), 0, s, d, 1);
      count_launch();
    }
  }
}

template <typename T, typename S>
void launch_gs_b(const LevelDesc<T, S>* d, int count, int n, int kind, int sweeps, int cl, cudaStream_t s,
                 int fused) {
  if (count <= 0) return;
  if (fused)
    gs_b<T, S, true>(d, count, n, kind, sweeps, cl, s);
  else
    gs_b<T, S, false>(d, count, n, kind, sweeps, cl, s);
}

template <typename T, typename S>
void launch_resid_restrict_b(const LevelDesc<T, S>* d, int count, int n, int kind, cudaStream_t s, int dir,
                             int fused) {
  if (count <= 0) return;
  int nc = (n - 1) / 2;
  dim3 g((nc + TXC - 1) / TXC, (nc + TYC - 1) / TYC, count);
  const dim3 b(TXC, TYC);
  if (kind == 9 && fused)
    pdl_launch(k_resid_restrict_b<T, S, true, true>, g, b, 0, s, d, dir);
  else if (kind == 9)
    pdl_launch(k_resid_restrict_b<T, S, true, false>, g, b, 0, s, d, dir);
  else if (fused)
    pdl_launch(k_resid_restrict_b<T, S, false, true>, g, b, 0, s, d, dir);
  else
    pdl_launch(k_resid_restrict_b<T, S, false, false>, g, b, 0, s, d, dir);
  count_launch();
}

template <typename T, typename S>
void launch_interp_b(const LevelDesc<T, S>* d, int count, int n, cudaStream_t s, int din, int dout, int fused) {
  if (count <= 0) return;
  int nc = (n - 1) / 2;
  const dim3 g((nc + 1 + BX - 1) / BX, (nc + 1 + BY - 1) / BY, count);
  if (fused)
    pdl_launch(k_interp_b<T, S, true>, g, dim3(BX, BY), 0, s, d, din, dout);
  else
    pdl_launch(k_interp_b<T, S, false>, g, dim3(BX, BY), 0, s, d, din, dout);
  count_launch();
}

template <typename S, int TY, int RING, bool PAIR, bool FU>
static void strip_b_launch(const LevelDesc<float, S>* d, int count, int n, int dir, cudaStream_t s) {
  if (count <= 0) return;
  constexpr size_t bytes = (size_t)STRIP_WARPS_B * RING * (StripRing<S>::SLOT + 8);
  // the shared-memory limit is raised once per kernel (thread-safe static initialisation)
  static const bool attr = [] {
    if (PAIR)
      cudaFuncSetAttribute(k_gs_strip2_ring_b<S, TY, RING, FU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes);
    else
      cudaFuncSetAttribute(k_gs_strip_ring_b<S, TY, RING, FU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes);
    return true;
  }();
  (void)attr;
  const int width = PAIR ? 48 : 56;
  const long warps = (long)count * ((n + width - 1) / width) * ((n + TY - 1) / TY);
  const unsigned blocks = (unsigned)((warps + STRIP_WARPS_B - 1) / STRIP_WARPS_B);
  if (PAIR)
    pdl_launch(k_gs_strip2_ring_b<S, TY, RING, FU>, blocks, 32 * STRIP_WARPS_B, bytes, s, d, count, n, dir);
  else
    pdl_launch(k_gs_strip_ring_b<S, TY, RING, FU>, blocks, 32 * STRIP_WARPS_B, bytes, s, d, count, n, dir);
  count_launch();
}

template <typename S, bool FU>
static void gs_tile_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s) {
  switch (shape) {
    case 1: strip_b_launch<S, 8, 4, false, FU>(d, count, n, dir, s); break;
    case 2: strip_b_launch<S, 16, 4, false, FU>(d, count, n, dir, s); break;
    case 3: strip_b_launch<S, 32, 4, false, FU>(d, count, n, dir, s); break;
    default: strip_b_launch<S, 26, 4, false, FU>(d, count, n, dir, s); break;
  }
}

template <typename S, bool FU>
static void gs_pair_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s) {
  switch (shape) {
    case 1: strip_b_launch<S, 16, 4, true, FU>(d, count, n, dir, s); break;
    case 2: strip_b_launch<S, 32, 6, true, FU>(d, count, n, dir, s); break;
    case 3: strip_b_launch<S, 26, 4, true, FU>(d, count, n, dir, s); break;
    default: strip_b_launch<S, 32, 4, true, FU>(d, count, n, dir, s); break;
  }
}

// ty = 0: the smallest even strip height whose strips, over all `count`
// problems, fit into one wave of resident warps.
template <int RING, bool FU>
static void strip64_b_launch(const LevelDesc<double, double>* d, int count, int n, int dir, cudaStream_t s, int ty) {
  if (count <= 0) return;
  constexpr size_t bytes = (size_t)STRIP_WARPS_B * RING * STRIP64_SLOT;
  static const int resident_warps = [] {
    cudaFuncSetAttribute(k_gs_strip64_b<RING, FU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_strip64_b<RING, FU>, 32 * STRIP_WARPS_B, bytes);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * STRIP_WARPS_B;
  }();
  const long cols = (long)count * ((n + 55) / 56);
  if (ty <= 0) {
    const long nby_max = resident_warps / cols > 1 ? resident_warps / cols : 1;
    const long half = (n + 2 * nby_max - 1) / (2 * nby_max);
    ty = (int)(2 * (half > 1 ? half : 1));
  }
  const long warps = cols * ((n + ty - 1) / ty);
  pdl_launch(k_gs_strip64_b<RING, FU>, (unsigned)((warps + STRIP_WARPS_B - 1) / STRIP_WARPS_B), 32 * STRIP_WARPS_B,
             bytes, s, d, count, n, dir, ty);
  count_launch();
}

template <bool FU>
static void gs_tile64_b(const LevelDesc<double, double>* d, int count, int n, int shape, int dir, cudaStream_t s) {
  switch (shape) {
    case 1: strip64_b_launch<4, FU>(d, count, n, dir, s, 16); break;
    case 2: strip64_b_launch<6, FU>(d, count, n, dir, s, 0); break;
    case 3: strip64_b_launch<4, FU>(d, count, n, dir, s, 8); break;
    default: strip64_b_launch<4, FU>(d, count, n, dir, s, 0); break;
  }
}

void launch_gs_tile64_b(const LevelDesc<double, double>* d, int count, int n, int shape, int dir, cudaStream_t s,
                        int fused) {
  if (fused)
    gs_tile64_b<true>(d, count, n, shape, dir, s);
  else
    gs_tile64_b<false>(d, count, n, shape, dir, s);
}

template <typename S>
void launch_gs_tile_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s, int fused) {
  if (fused)
    gs_tile_b<S, true>(d, count, n, shape, dir, s);
  else
    gs_tile_b<S, false>(d, count, n, shape, dir, s);
}

// ty: the smallest even strip height whose strips, over all groups of K
// members, fit into one wave of resident warps.
template <typename S, int K, bool FU>
static void strip_bk_launch(const LevelDesc<float, S>* d, int count, int n, int dir, cudaStream_t s) {
  if (count <= 0) return;
  constexpr int RING = 4;
  constexpr size_t bytes = (size_t)STRIP_WARPS_B * RING * (StripRingK<S, K>::SLOT + 8);
  static const int resident_warps = [] {
    cudaFuncSetAttribute(k_gs_strip_ring_bk<S, K, RING, FU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_strip_ring_bk<S, K, RING, FU>, 32 * STRIP_WARPS_B,
                                                  bytes);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * STRIP_WARPS_B;
  }();
  const int groups = (count + K - 1) / K, nbx = (n + 55) / 56;
  const long cols = (long)groups * nbx;
  const int nby_max = resident_warps / cols > 1 ? (int)(resident_warps / cols) : 1;
  const int half = (n + 2 * nby_max - 1) / (2 * nby_max);
  const int ty = 2 * (half > 1 ? half : 1);
  const long warps = cols * ((n + ty - 1) / ty);
  const unsigned blocks = (unsigned)((warps + STRIP_WARPS_B - 1) / STRIP_WARPS_B);
  pdl_launch(k_gs_strip_ring_bk<S, K, RING, FU>, blocks, 32 * STRIP_WARPS_B, bytes, s, d, count, n, dir, ty);
  count_launch();
}

template <typename S>
bool launch_gs_tile_bk(const LevelDesc<float, S>* d, int count, int n, int k, int dir, cudaStream_t s, int fused) {
  if (k == 2) {
    if (fused)
      strip_bk_launch<S, 2, true>(d, count, n, dir, s);
    else
      strip_bk_launch<S, 2, false>(d, count, n, dir, s);
  } else if (k == 4) {
    if (fused)
      strip_bk_launch<S, 4, true>(d, count, n, dir, s);
    else
      strip_bk_launch<S, 4, false>(d, count, n, dir, s);
  } else {
    return false;
  }
  return true;
}
template bool launch_gs_tile_bk<float>(const LevelDesc<float, float>*, int, int, int, int, cudaStream_t, int);
template bool launch_gs_tile_bk<__nv_bfloat16>(const LevelDesc<float, __nv_bfloat16>*, int, int, int, int,
                                               cudaStream_t, int);

template <typename S>
void launch_gs_pair_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s, int fused) {
  if (fused)
    gs_pair_b<S, true>(d, count, n, shape, dir, s);
  else
    gs_pair_b<S, false>(d, count, n, shape, dir, s);
}
template void launch_gs_tile_b<float>(const LevelDesc<float, float>*, int, int, int, int, cudaStream_t, int);
template void launch_gs_tile_b<__nv_bfloat16>(const LevelDesc<float, __nv_bfloat16>*, int, int, int, int,
                                              cudaStream_t, int);
template void launch_gs_pair_b<float>(const LevelDesc<float, float>*, int, int, int, int, cudaStream_t, int);
template void launch_gs_pair_b<__nv_bfloat16>(const LevelDesc<float, __nv_bfloat16>*, int, int, int, int,
                                              cudaStream_t, int);

int strip_timeouts_b() {
  int h = 0, zero = 0;
  cudaMemcpyFromSymbol(&h, g_strip_timeout_b, sizeof(int));
  if (h) cudaMemcpyToSymbol(g_strip_timeout_b, &zero, sizeof(int));
  return h;
}

template <typename T, typename S>
void launch_coarse_b(const LevelDesc<T, S>* d, int count, cudaStream_t s) {
  if (count <= 0) return;
  pdl_launch(k_coarse_b<T, S>, count, 32, 0, s, d);
  count_launch();
}

void launch_residual_b(const TopDesc* d, const int2* bmap, int nblocks, cudaStream_t s, int fused) {
  if (fused)
    pdl_launch(k_residual_b<true>, nblocks, NORM_THREADS, 0, s, d, bmap);
  else
    pdl_launch(k_residual_b<false>, nblocks, NORM_THREADS, 0, s, d, bmap);
  count_launch();
}

void launch_finalize_b(const TopDesc* d, int count, int phase, cudaStream_t s) {
  pdl_launch(k_finalize_b, count, NORM_THREADS, 0, s, d, phase);
  count_launch();
}

void launch_ir_update_b(const TopDesc* d, int count, int maxn, cudaStream_t s) {
  pdl_launch(k_ir_update_b, dim3((maxn + BX * IRU_COLS - 1) / (BX * IRU_COLS), (maxn + BY - 1) / BY, count),
             dim3(BX, BY), 0, s, d);
  count_launch();
}

void launch_ir_residual_b(const TopDesc* d, const int2* bmap, int nblocks, cudaStream_t s, int fused) {
  if (fused)
    pdl_launch(k_ir_residual_b<true>, nblocks, NORM_THREADS, 0, s, d, bmap);
  else
    pdl_launch(k_ir_residual_b<false>, nblocks, NORM_THREADS, 0, s, d, bmap);
  count_launch();
}

template <typename T>
void launch_tail(const TailDesc<T>* d, int count, int top_n, const int* done_any, cudaStream_t s, int fused) {
  if (count <= 0) return;
  // tails start at n <= tail_max_n: at most 28.8 KB (FP32, n = 63) or 4 KB (FP64,
  // n = 15), inside the default 48 KB dynamic shared-memory limit
  const size_t bytes = tail_smem_elems<T>(top_n) * sizeof(T);
  if (fused)
    pdl_launch(k_tail<T, true>, count, 1024, bytes, s, d, done_any);
  else
    pdl_launch(k_tail<T, false>, count, 1024, bytes, s, d, done_any);
  count_launch();
}
template void launch_tail<double>(const TailDesc<double>*, int, int, const int*, cudaStream_t, int);
template void launch_tail<float>(const TailDesc<float>*, int, int, const int*, cudaStream_t, int);

void launch_all_done(const char* ctls, size_t stride, int count, int* out, cudaStream_t s) {
  pdl_launch(k_all_done, 1, 256, 0, s, ctls, stride, count, out);
  count_launch();
}

#define BMG_INST_B(T, S)                                                                                 \
  template void launch_gs_b<T, S>(const LevelDesc<T, S>*, int, int, int, int, int, cudaStream_t, int);       \
  template void launch_resid_restrict_b<T, S>(const LevelDesc<T, S>*, int, int, int, cudaStream_t, int, int); \
  template void launch_interp_b<T, S>(const LevelDesc<T, S>*, int, int, cudaStream_t, int, int, int);        \
  template void launch_coarse_b<T, S>(const LevelDesc<T, S>*, int, cudaStream_t);
BMG_INST_B(double, double)
BMG_INST_B(float, float)
BMG_INST_B(float, __nv_bfloat16)
#undef BMG_INST_B

}  // namespace bmg
