// Hierarchies with periodic sides (internal interface of periodic.cu).
//
// An axis is Dirichlet (N = 2^m - 1 points, zero ghost values) or periodic
// (N = 2^m points; point N + 1 is point 1, point 0 is point N), both axes
// sharing m.  Coarse point c sits on fine point 2c on either kind of axis, so a
// periodic axis of N points coarsens to a periodic axis of N / 2; the
// hierarchy stops at 3 (Dirichlet) / 4 (periodic) points per axis.  Arrays are
// (N_y + 2) x (N_x + 2) with zero ghost lines: the kernels wrap indices on
// the periodic axes instead of reading ghost copies.  The cycle is the FP64
// V(nu1, nu2) of the Dirichlet hierarchy (the same formulas, term orders and
// arithmetic modes); a 9-point sweep is one launch of the strip walk (or two
// row-parity launches), a 5-point one (level 0) one launch per colour.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace bmg {

struct PerHier;

// Sizes admissible for periodic flags (bit 0: x, bit 1: y); 0 when not.
int per_levels_for(int nx, int ny, int periodic);

// Build the hierarchy on stream s from the caller's planes (kind 5: O, W, S;
// kind 9: O, W, S, SW, NW; each (ny+2) x (nx+2)).  BMG_ESINGULAR for a
// non-positive diagonal or pivot or a zero interpolation denominator.  sweep
// says how 9-point levels are swept (the same bits either way): by the two
// row-parity launches in place (PER_SWEEP_ROWS), by the one-pass strip kernel
// into a second iterate (PER_SWEEP_STRIP), or per level by whichever of the
// two is faster, timed during setup (PER_SWEEP_AUTO).
// krylov: the solve runs flexible CG (FCG(1)) preconditioned by one V(nu1, nu2)
// cycle per step instead of stationary cycles.
enum { PER_SWEEP_AUTO = 0, PER_SWEEP_ROWS = 1, PER_SWEEP_STRIP = 2 };
int per_setup(PerHier** out, int kind, const double* coef, int nx, int ny, int periodic, int fused, int nu1,
              int nu2, int sweep, int krylov, cudaStream_t s);
void per_free(PerHier* P);

// Profiling brackets around each step's launches (begin: level and BMG_K_*
// kind of the step; end: after its last launch); NULL members are skipped.
struct PerMarks {
  void* ctx = nullptr;
  void (*begin)(void* ctx, int level, int kernel) = nullptr;
  void (*end)(void* ctx) = nullptr;
};

// The solve loop's device work: the initial residual norm (phase 0 of the
// control block), and one iteration = V-cycle + residual norm + convergence
// test (phase 1); with krylov, the initial step r = f - A x, z = 0 and one
// iteration = z = V(r) + FCG step (updated residual's norm, convergence
// test).  partials holds at least 2 x 1024 doubles.
void per_enqueue_initial(PerHier* P, const double* rhs, double* x, double* partials, Ctl* ctl, cudaStream_t s);
void per_enqueue_iteration(PerHier* P, const double* rhs, double* x, double* partials, Ctl* ctl, cudaStream_t s,
                           const PerMarks* marks = nullptr);

int per_num_levels(const PerHier* P);
// How level l is swept: 2 one-pass strip kernel, 1 row-parity pair (9-point)
// or one launch per colour (5-point), 0 not swept (the coarsest level).
int per_level_sweep(const PerHier* P, int l);
int per_level_shape(const PerHier* P, int l, int* nx, int* ny);
// Level l's five planes O, W, S, SW, NW ((ny+2) x (nx+2) each, ghost lines zero)
// and its eight interpolation planes toward level l + 1 ((ny_c+2) x (nx_c+2)).
int per_get_stencil(const PerHier* P, int l, double* out, cudaStream_t s);
int per_get_interp(const PerHier* P, int l, double* out, cudaStream_t s);

}  // namespace bmg
