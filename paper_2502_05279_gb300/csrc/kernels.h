// Host-side launchers of the BoxMG kernels (one translation unit per family).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bmg {

// Stencil of one level as the kernels read it: diagonal O and reciprocal
// diagonal D in the compute type T, off-diagonal planes W, S, SW, NW in the
// storage type S (T itself, or bf16 under a float T).
template <typename T, typename S>
struct StencilView {
  const T* O;
  const S* W;
  const S* S_;
  const S* SW;
  const S* NW;
  const T* D;
  int n;
  int ld;
  int fused = 0;   // 1: the cycle's multiply-adds are fused (BMG_ARITH_FUSED)
  // FP32 / BF16 levels: the same stencil packed per point for the bulk-copy
  // sweeps, point p at pk[PK * p]: PK = 5 words d, w, s, sw, nw (FP32) or 3
  // words d, (w | s << 16), (sw | nw << 16) (BF16 halves); NULL if absent.
  const void* pk = nullptr;
};

// ---- setup (k_setup.cu), FP64 ----
// st: 6 planes O, W, S, SW, NW, D of (n+2)^2.  err: device int, set nonzero on
// a zero or negative diagonal / denominator / pivot.
// coef_in: the caller's planes on an nx x ny grid; st: level 0 of size n
// (n = nx = ny, or the embedding size; see k_prepare).
void launch_prepare(int n, int nx, int ny, int kind, const double* coef_in, double* st, int* err, cudaStream_t s);
// Interior of an nx x ny array into the n x n layout (back = false) or out of it.
void launch_embed_vec(int nx, int ny, int n, const double* in, double* out, bool back, cudaStream_t s);
void launch_dendy(int n, const double* st, double* ci, int* err, cudaStream_t s);
void launch_rap(int n, const double* st, const double* ci, double* stc, cudaStream_t s);
void launch_dinv(int n, double* st, int* err, cudaStream_t s);
void launch_factor(int n, const double* st, double* L, double* work, int* err, cudaStream_t s);
// st32 / off16 / od32: planes plane_stride32(n) elements apart.
void launch_lower32(int n, const double* st, float* st32, const double* ci, float* ci32, cudaStream_t s);
void launch_lower_bf16(int n, const double* st, __nv_bfloat16* off16, float* od32, cudaStream_t s);
// The packed stencil of an FP32 level (words d, w, s, sw, nw per point) or a
// BF16 level (words d, w|s, sw|nw) over all (n+2)^2 points, from its planes.
void launch_pack32(int n, const float* st32, float* pk, cudaStream_t s);
void launch_pack_bf16(int n, const __nv_bfloat16* off16, const float* od32, float* pk, cudaStream_t s);
constexpr int PK_WORDS_F32 = 5, PK_WORDS_BF16 = 3;

// ---- cycle (k_cycle.cu) ----
// `done`: device flag of the running solve (NULL = always run); every kernel
// returns at once when it is nonzero.
template <typename T, typename S>
void launch_gs(const StencilView<T, S>& v, int kind, const T* f, T* x, int sweeps, const int* done, cudaStream_t s,
               int cl = 0);   // cl: row-kernel cluster size, 0 = the smallest that covers a row
// Zebra line Gauss-Seidel sweeps: dir LINE_X (odd rows, then even rows, each
// solved exactly along x), LINE_Y (odd columns, then even columns, each solved
// exactly along y) or LINE_XY (an x-line sweep, then a y-line sweep); cp:
// scratch of the level's (n+2)^2 layout for the elimination multipliers.
enum { LINE_X = 0, LINE_Y = 1, LINE_XY = 2 };
template <typename T, typename S>
void launch_line(const StencilView<T, S>& v, int kind, const T* f, T* x, T* cp, int sweeps, int dir,
                 const int* done, cudaStream_t s);
// FP32 / BF16 level arrays are allocated with STRIP_GUARD zeroed elements
// before and after each array (plane), every array starting on a 256-byte
// boundary; planes of one level are plane_stride32(n) elements apart.  The
// bulk-copy form of the one-pass sweep relies on both.
constexpr int STRIP_GUARD = 128;
inline size_t plane_stride32(int n) { return (((size_t)(n + 2) * (n + 2) + STRIP_GUARD + 63) / 64) * 64; }
// Nonzero once a one-pass sweep gave up waiting for its bulk copies (then
// cleared): the sweep's result is invalid.
int strip_timeouts();
// One warp waits on an mbarrier phase that never completes (bounded wait).
void launch_wait_selftest(cudaStream_t s);
// One four-colour Gauss-Seidel sweep of a 9-point FP32 level in one launch:
// reads xin, writes every interior point of xout (xout != xin; the ghost ring
// of xout is not written).  One warp per strip of 56 x TY points: shapes
// 0 .. 3 stream rows by bulk copies into 4 row slots (TY = W, 8, 16, 32, W the
// smallest even height whose strips fit into one wave of resident warps),
// shapes 4, 5 load them into registers (TY 32, 16).  The bulk-copy
// shapes need the array layout above (else they run as shape 4).
constexpr int GS_TILE_SHAPES = 6;
template <typename S>
void launch_gs_tile(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s);
// Two four-colour sweeps of a 9-point FP32 level in one launch (temporal
// blocking): xin -> xout as two launch_gs_tile calls would give through an
// intermediate array.  One warp per strip of 48 x TY points, rows by bulk
// copies: shapes 0 .. 3 = TY W (one wave), 16, 32, 26 with 4, 4, 6, 4 row slots.  Needs
// the guarded, aligned array layout; returns false (nothing launched) without it.
constexpr int GS_PAIR_SHAPES = 4;
// The two pre-smoothing sweeps, the residual and its restriction in one pass
// (44-column strips): fc, xc are the next level's right-hand side and iterate
// (written / zeroed at its interior points).  Shape 0 or 1 (4- or 6-slot row
// rings).  Returns false when the arrays do not allow the bulk copies.
template <typename S>
bool launch_gs_pair_restrict(const StencilView<float, S>& v, const float* f, const float* xin, float* xout,
                             const float* ci, float* fc, float* xc, int shape, const int* done, cudaStream_t s);
template <typename S>
bool launch_gs_pair(const StencilView<float, S>& v, const float* f, const float* xin, float* xout, int shape,
                    const int* done, cudaStream_t s);
// One four-colour Gauss-Seidel sweep of a 9-point FP64 level in one launch,
// xin -> xout as launch_gs_tile (xout != xin, its ghost ring not written), for
// the plain FP64 layout (no guard band or alignment needed): warp strips of
// 56 x TY points, rows copied per lane into RING row slots; shapes 0 .. 3 =
// (TY, RING) = (one wave, 4), (16, 4), (one wave, 6), (8, 4), where "one
// wave" is the smallest even TY whose strips all fit into the resident warps.
// Needs v.D.
constexpr int GS_TILE64_SHAPES = 4;
void launch_gs_tile64(const StencilView<double, double>& v, const double* f, const double* xin, double* xout,
                      int shape, const int* done, cudaStream_t s);
template <typename T, typename S>
void launch_resid_restrict(const StencilView<T, S>& v, int kind, const T* ci, const T* x, const T* f, T* fc,
                           T* xc, const int* done, cudaStream_t s);
template <typename T>
void launch_interp_correct(int n, const T* ci, const T* ec, T* x, const int* done, cudaStream_t s, int fused = 0);
// xout = xin + P ec over every interior fine point (xin may equal xout).
template <typename T>
void launch_interp_to(int n, const T* ci, const T* ec, const T* xin, T* xout, const int* done, cudaStream_t s,
                      int fused = 0);
// r = f - A x (r may be NULL) with per-block partial sums of r^2 (partials may
// be NULL); returns the number of partials written.
template <typename T, typename S>
int launch_residual(const StencilView<T, S>& v, int kind, const T* x, const T* f, T* r, double* partials,
                    const int* done, cudaStream_t s);
template <typename T>
void launch_coarse_solve(int n, const double* L, const T* f, T* x, double* y, const int* done, cudaStream_t s);

int norm_partials_max();
// Sum partials in a fixed order and record the norm in ctl (phase 0 = initial
// residual, 1 = after a cycle).  Also writes the norm to out (may be NULL).
void launch_norm_finalize(const double* partials, int np, void* ctl, int phase, double* out, cudaStream_t s);

// Iterative refinement: x += scale_applied * e32 and the FP64 residual with
// its FP32 scaled copy (r32 = fl32(r / scale_next)), zeroing e32 for the next
// inner cycle.
void launch_ir_update(int n, double* x, const float* e32, void* ctl, cudaStream_t s);
int launch_ir_residual(const StencilView<double, double>& v, int kind, const double* x, const double* f,
                       float* r32, float* e32_zero, double* partials, void* ctl, cudaStream_t s);

// Flexible CG (FP64 outer loop).  z is the preconditioned residual: an FP64
// vector, or (z32 != NULL) scale_applied * z32.
int launch_fcg_init(const StencilView<double, double>& v, int kind, const double* x, const double* f, double* r,
                    double* z, float* r32, float* z32, double* partials, void* ctl, cudaStream_t s);
void launch_fcg_step(const StencilView<double, double>& v, int kind, double* x, double* r, const double* z,
                     const float* z32, double* p, double* q, float* r32, float* z32_zero, double* z_zero,
                     double* partials, void* ctl, cudaStream_t s, void (*mark)(void*, int), void* mark_arg);
// The step's scalar reductions over np partial sums in the canonical order:
// which = 0: z.q into ctl (and beta = -(z.q) / (p.q)_prev after the first
// step); which = 1: p.q and p.r (the second partial array NORM_BLOCKS_MAX
// entries after the first).
void launch_fcg_reduce(const double* partials, int np, void* ctl, int which, cudaStream_t s);

// FP64 throughput probe.
double measure_fp64_rate(cudaStream_t s);

}  // namespace bmg

// ---- batched (k_batched.cu) -----------------------------------------------------------
// Many independent problems, one launch per stage.  A stage is a level counted
// from the coarsest, so every problem in it has the same size n; each CTA reads
// its problem's descriptor (device array) from another grid dimension.
namespace bmg {

template <typename T, typename S>
struct LevelDesc {
  StencilView<T, S> v;
  const T* ci;        // weights toward the next coarser level (NULL at the coarsest)
  T* x;               // this level's iterate and right-hand side
  const T* f;
  T* xc;              // next coarser level's iterate and right-hand side
  T* fc;
  const int* done;    // the problem's control flag
  const double* L;    // coarsest level: Cholesky factor and substitution workspace
  double* y;
  T* x2 = nullptr;    // second iterate of a level swept by the one-pass kernels (else NULL)
};

// A problem's finest level, for the FP64 outer loop.
struct TopDesc {
  StencilView<double, double> v;
  int kind;
  double* x;
  const double* f;
  float* r32;         // mixed precision: level-0 FP32 right-hand side and iterate
  float* e32;
  double* partials;
  Ctl* ctl;
};

// fused (every batched launcher): 1 = the problems' hierarchies use BMG_ARITH_FUSED.
template <typename T, typename S>
void launch_gs_b(const LevelDesc<T, S>* d, int count, int n, int kind, int sweeps, int cl, cudaStream_t s,
                 int fused = 0);
template <typename T, typename S>
void launch_resid_restrict_b(const LevelDesc<T, S>* d, int count, int n, int kind, cudaStream_t s, int dir = 0,
                             int fused = 0);
template <typename T, typename S>
void launch_interp_b(const LevelDesc<T, S>* d, int count, int n, cudaStream_t s, int din = 0, int dout = 0,
                     int fused = 0);
// Batched one-pass sweeps of 9-point FP32 levels (all `count` problems share
// n): dir 0 reads x and writes x2, dir 1 the reverse (the residual +
// restriction reads, and the interpolation reads / writes, the array its dir
// flags name: 0 = x, 1 = x2).  Shapes as launch_gs_tile 0 .. 3 and
// launch_gs_pair; arrays in the guarded, aligned layout.
template <typename S>
void launch_gs_tile_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s,
                      int fused = 0);
// One sweep of a group whose members share one operator (a batch of
// right-hand sides), k = 2 or 4 members per warp: each stencil value is read
// once for the k members.  Needs the operator's packed stencil; false for
// another k.
template <typename S>
bool launch_gs_tile_bk(const LevelDesc<float, S>* d, int count, int n, int k, int dir, cudaStream_t s, int fused);
template <typename S>
void launch_gs_pair_b(const LevelDesc<float, S>* d, int count, int n, int shape, int dir, cudaStream_t s,
                      int fused = 0);
// Batched FP64 one-pass sweeps (dir as launch_gs_tile_b); shapes as
// launch_gs_tile64, with the one-wave height taken over all `count` problems.
void launch_gs_tile64_b(const LevelDesc<double, double>* d, int count, int n, int shape, int dir, cudaStream_t s,
                        int fused = 0);
int strip_timeouts_b();
template <typename T, typename S>
void launch_coarse_b(const LevelDesc<T, S>* d, int count, cudaStream_t s);
// bmap: (problem, block) of each of the nblocks blocks, every problem's
// min(n, 1024) canonical reduction blocks in turn.
void launch_residual_b(const TopDesc* d, const int2* bmap, int nblocks, cudaStream_t s, int fused = 0);
void launch_finalize_b(const TopDesc* d, int count, int phase, cudaStream_t s);
void launch_ir_update_b(const TopDesc* d, int count, int maxn, cudaStream_t s);
void launch_ir_residual_b(const TopDesc* d, const int2* bmap, int nblocks, cudaStream_t s, int fused = 0);
void launch_all_done(const char* ctls, size_t stride, int count, int* out, cudaStream_t s);
template <typename T>
int rows_cluster(int n);
int rows_threads(int n, int cl);

}  // namespace bmg

namespace bmg {
template <typename T>
struct TailDesc;
// The level-fused tail of `count` problems (one CTA each) whose first level
// has size top_n (the same for all); the tail's iterates and right-hand sides
// are held in dynamic shared memory, sized from top_n.
template <typename T>
void launch_tail(const TailDesc<T>* d, int count, int top_n, const int* done_any, cudaStream_t s, int fused = 0);
template <typename T>
constexpr int tail_max_n() { return sizeof(T) == 8 ? 15 : 63; }
}  // namespace bmg
