"""Plain FP64 CPU oracle of the BoxMG hot path (setup and V(2,1) solve).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import or run anything under oracle/.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code with it; both sides receive their inputs from workloads/.

Modules:
  boxmg   -- FP64 stencil apply, Dendy interpolation, Galerkin RAP, Gauss-Seidel,
             residual + restriction, interpolation + correction, coarsest
             Cholesky, V(2,1) and the solve loop.
  mixed   -- FP32 / BF16-stencil V(2,1) inside FP64 iterative refinement
             (rounding emulated with numpy float32 and bit manipulation).
  learned -- the learned-interpolation network in FP64 with a hand-written
             backward pass, the learned prolongation built from it, and the
             training losses with their gradients.
  fused   -- element-wise fused multiply-add (C99 fma / fmaf from fma.c,
             compiled with gcc) for the fused arithmetic mode.

The paper (Nytko et al., "Teaching an old dog new tricks", arXiv 2502.05279)
states BoxMG through its kernel sequence (Fig. 1) and the restriction loop
(Fig. 2) and defers the rest to Dendy's black-box multigrid papers; the oracle
writes that published method out.  Every function names the passage or the
reading it follows.
"""
