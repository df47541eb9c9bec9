"""Learned operator-dependent interpolation: oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Pins (tests/test_learned_oracle.py): zero logits reproduce Dendy's weights;
any logits keep constants on zero-row-sum rows; the basis energy equals the
Galerkin diagonal; the test-vector energy is the dense quadratic form; the
gradients equal central finite differences.  What training gains over Dendy
has no number in the paper: parity unpinned for that claim.

The paper has no learned component; this follows the stated reading of the
extension:

* features (18 per coarse point c): for each of the 9 fine points q of the 3x3
  block centred on c (dy outer, dx inner), (a_W + a_E)/a_O and (a_S + a_N)/a_O
  at q;
* network: 18 -> 64 -> 64 -> 4, GELU (erf form) after the two hidden layers;
  outputs delta = (d_W, d_E, d_S, d_N), one logit per edge fine neighbour of c;
* interpolation: an edge fine point e between coarse points c1 and c2 keeps
  Dendy's total weight S_D = -(col_1 + col_2)/D (col_k the collapsed stencil
  toward c_k, D the collapsed centre), split as
      w_k = S_D u_k / (u_1 + u_2),  u_k = -col_k exp(delta of c_k for e),
  so delta = 0 gives Dendy's weights; centre points use Dendy's centre formula
  with these edge weights (the local row solve);
* training loss (weak approximation property): for K smooth test vectors v_k
  (random vectors after Gauss-Seidel sweeps with a zero right-hand side, which
  leaves the slowly converging error the coarse grid must represent),
      L = (1/K) sum_k E_k / E_k^D,   E_k = || v_k - P (v_k restricted to C) ||_A^2,
  E_k^D the same with delta = 0 (Dendy).  Its gradient is local: with
  g = -2 A (v - P R v) / (K E^D), dL/dw(p -> c) = g(p) v(c), chained through
  Dendy's centre formula to the edge weights and through the split to delta.
* basis_energy / loss_and_grad: the coarse basis energy (P^T A P)_cc relative
  to Dendy's, an alternative loss kept with its gradient for comparison.
"""
from __future__ import annotations

import math

import numpy as np

from . import boxmg as bx
from .boxmg import LA, LB, LL, LNE, LNW, LR, LSE, LSW

N_IN, N_HID, N_OUT = 18, 64, 4
PARAM_SHAPES = (("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
                ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Parameter vector -> named arrays (row-major, in PARAM_SHAPES order)."""
    out, k = {}, 0
    for name, shape in PARAM_SHAPES:
        m = int(np.prod(shape))
        out[name] = theta[k:k + m].reshape(shape)
        k += m
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([p[name].reshape(-1) for name, _ in PARAM_SHAPES])


# ---------------------------------------------------------------------------
# Features
# ---------------------------------------------------------------------------

def features(planes: np.ndarray) -> np.ndarray:
    """(M, 18) features of the interior coarse points, row-major (jc outer)."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    aO = bx.coupling(planes, 0, 0)
    fx = (bx.coupling(planes, -1, 0) + bx.coupling(planes, 1, 0)) / aO
    fy = (bx.coupling(planes, 0, -1) + bx.coupling(planes, 0, 1)) / aO
    cols = []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            # fine point (2ic+dx, 2jc+dy) -> interior index (2jc+dy-1, 2ic+dx-1)
            sl = (slice(1 + dy, 2 * nc + dy, 2), slice(1 + dx, 2 * nc + dx, 2))
            cols.append(fx[sl].reshape(-1))
            cols.append(fy[sl].reshape(-1))
    return np.stack(cols, axis=1)


# ---------------------------------------------------------------------------
# Network (FP64) with a hand-written backward pass
# ---------------------------------------------------------------------------

def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta: np.ndarray, X: np.ndarray):
    p = unpack(theta)
    z1 = X @ p["W1"] + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = gelu(z2)
    out = h2 @ p["W3"] + p["b3"]
    return out, (X, z1, h1, z2, h2)


def backward(theta: np.ndarray, cache, d_out: np.ndarray) -> np.ndarray:
    p = unpack(theta)
    X, z1, h1, z2, h2 = cache
    g = {"W3": h2.T @ d_out, "b3": d_out.sum(0)}
    dz2 = (d_out @ p["W3"].T) * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"].T) * gelu_grad(z1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return pack(g)


# ---------------------------------------------------------------------------
# Learned interpolation weights
# ---------------------------------------------------------------------------

def _delta_grid(delta: np.ndarray, nc: int) -> np.ndarray:
    """(4, nc+2, nc+2) with the outputs of the interior coarse points, 0 on ghosts."""
    g = np.zeros((4, nc + 2, nc + 2))
    g[:, 1:nc + 1, 1:nc + 1] = delta.T.reshape(4, nc, nc)
    return g


def edge_split(planes: np.ndarray, delta: np.ndarray):
    """Edge weights and the pieces of their derivative.  Returns ci with the
    edge planes (LL, LR, LB, LA) filled, plus for every x-edge and y-edge point
    the Dendy sum S_D and the share q of the first (west / south) coarse point."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    a = {d: bx.coupling(planes, *d) for d in bx.NBR}
    dg = _delta_grid(delta, nc)
    ci = np.zeros((8, nc + 2, nc + 2))
    # x-edge points i = 2ic-1 (ic = 1..nc+1), j = 2jc (jc = 1..nc) between
    # (ic-1, jc) [its E output, index 1] and (ic, jc) [its W output, index 0]
    X = (slice(1, n - 1, 2), slice(0, n, 2))
    colW = (a[(-1, -1)][X] + a[(-1, 0)][X]) + a[(-1, 1)][X]
    colE = (a[(1, -1)][X] + a[(1, 0)][X]) + a[(1, 1)][X]
    D = (a[(0, -1)][X] + a[(0, 0)][X]) + a[(0, 1)][X]
    SDx = -((colW + colE) / D)
    uW = -colW * np.exp(dg[1, 1:nc + 1, 0:nc + 1])
    uE = -colE * np.exp(dg[0, 1:nc + 1, 1:nc + 2])
    qx = uW / (uW + uE)
    ci[bx.LL, 1:nc + 1, 1:nc + 2] = SDx * qx
    ci[bx.LR, 1:nc + 1, 1:nc + 2] = SDx * (1.0 - qx)
    # y-edge points i = 2ic (ic = 1..nc), j = 2jc-1 (jc = 1..nc+1) between
    # (ic, jc-1) [its N output, index 3] and (ic, jc) [its S output, index 2]
    Y = (slice(0, n, 2), slice(1, n - 1, 2))
    rowS = (a[(-1, -1)][Y] + a[(0, -1)][Y]) + a[(1, -1)][Y]
    rowN = (a[(-1, 1)][Y] + a[(0, 1)][Y]) + a[(1, 1)][Y]
    D = (a[(-1, 0)][Y] + a[(0, 0)][Y]) + a[(1, 0)][Y]
    SDy = -((rowS + rowN) / D)
    uS = -rowS * np.exp(dg[3, 0:nc + 1, 1:nc + 1])
    uN = -rowN * np.exp(dg[2, 1:nc + 2, 1:nc + 1])
    qy = uS / (uS + uN)
    ci[bx.LB, 1:nc + 2, 1:nc + 1] = SDy * qy
    ci[bx.LA, 1:nc + 2, 1:nc + 1] = SDy * (1.0 - qy)
    return ci, (SDx, qx, SDy, qy)


def centre_weights(planes: np.ndarray, ci: np.ndarray) -> np.ndarray:
    """Fill the centre planes with Dendy's centre formula (local row solve)
    from the edge planes already in ci (in place; returns ci)."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    a = {d: bx.coupling(planes, *d) for d in bx.NBR}
    C = (slice(0, n, 2), slice(0, n, 2))
    lb_w, la_w = ci[bx.LB, 1:nc + 2, 0:nc + 1], ci[bx.LA, 1:nc + 2, 0:nc + 1]
    lb_e, la_e = ci[bx.LB, 1:nc + 2, 1:nc + 2], ci[bx.LA, 1:nc + 2, 1:nc + 2]
    ll_s, lr_s = ci[bx.LL, 0:nc + 1, 1:nc + 2], ci[bx.LR, 0:nc + 1, 1:nc + 2]
    ll_n, lr_n = ci[bx.LL, 1:nc + 2, 1:nc + 2], ci[bx.LR, 1:nc + 2, 1:nc + 2]
    o = a[(0, 0)][C]
    ci[bx.LSW, 1:nc + 2, 1:nc + 2] = -(((a[(-1, -1)][C] + a[(-1, 0)][C] * lb_w) + a[(0, -1)][C] * ll_s) / o)
    ci[bx.LSE, 1:nc + 2, 1:nc + 2] = -(((a[(1, -1)][C] + a[(1, 0)][C] * lb_e) + a[(0, -1)][C] * lr_s) / o)
    ci[bx.LNW, 1:nc + 2, 1:nc + 2] = -(((a[(-1, 1)][C] + a[(-1, 0)][C] * la_w) + a[(0, 1)][C] * ll_n) / o)
    ci[bx.LNE, 1:nc + 2, 1:nc + 2] = -(((a[(1, 1)][C] + a[(1, 0)][C] * la_e) + a[(0, 1)][C] * lr_n) / o)
    return ci


def learned_interp(planes: np.ndarray, delta: np.ndarray) -> np.ndarray:
    ci, _ = edge_split(planes, delta)
    return centre_weights(planes, ci)


# ---------------------------------------------------------------------------
# Training loss and its gradient with respect to the outputs
# ---------------------------------------------------------------------------

EDGE_OFFSETS = ((-1, 0), (1, 0), (0, -1), (0, 1))   # W, E, S, N edge fine points of c


def basis_energy(planes: np.ndarray, ci: np.ndarray):
    """Per interior coarse point: O_c = phi_c^T A phi_c and (A phi_c) at its
    four edge fine points (order W, E, S, N).  Shapes (nc, nc) and (4, nc, nc)."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    phi = bx.basis(ci)[:, :, 1:nc + 1, 1:nc + 1]
    A = {d: bx.coupling(planes, *d) for d in bx.NBR}

    def a_phi(ux, uy):
        """(A phi_c)(2c + u) over all c."""
        rows = slice(1 + uy, 2 * nc + uy, 2)
        cols = slice(1 + ux, 2 * nc + ux, 2)
        acc = np.zeros((nc, nc))
        for (vx, vy) in bx.NBR:
            ox, oy = ux + vx, uy + vy
            if abs(ox) <= 1 and abs(oy) <= 1:
                acc = acc + A[(vx, vy)][rows, cols] * phi[oy + 1, ox + 1]
        return acc

    energy = np.zeros((nc, nc))
    for (ux, uy) in bx.BLOCK:
        energy = energy + phi[uy + 1, ux + 1] * a_phi(ux, uy)
    edges = np.stack([a_phi(ux, uy) for (ux, uy) in EDGE_OFFSETS])
    return energy, edges


def loss_and_grad(planes: np.ndarray, delta: np.ndarray, energy_ref: np.ndarray):
    """L(delta) and dL/d delta, shape (M, 4)."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    M = nc * nc
    ci, (SDx, qx, SDy, qy) = edge_split(planes, delta)
    centre_weights(planes, ci)
    energy, aphi_edges = basis_energy(planes, ci)
    L = float(np.sum(energy / energy_ref)) / M
    G = np.zeros((4, nc + 2, nc + 2))                 # dL/dw(edge toward c), ghosts 0
    G[:, 1:nc + 1, 1:nc + 1] = 2.0 * aphi_edges / energy_ref / M
    dg = np.zeros((4, nc + 2, nc + 2))
    # x-edge between cW = (ic-1, jc) (its E edge, G index 1) and cE = (ic, jc) (its W edge, G index 0)
    diff = G[1, 1:nc + 1, 0:nc + 1] - G[0, 1:nc + 1, 1:nc + 2]
    t = diff * SDx * qx * (1.0 - qx)
    dg[1, 1:nc + 1, 0:nc + 1] += t
    dg[0, 1:nc + 1, 1:nc + 2] -= t
    # y-edge between cS = (ic, jc-1) (its N edge, index 3) and cN = (ic, jc) (its S edge, index 2)
    diff = G[3, 0:nc + 1, 1:nc + 1] - G[2, 1:nc + 2, 1:nc + 1]
    t = diff * SDy * qy * (1.0 - qy)
    dg[3, 0:nc + 1, 1:nc + 1] += t
    dg[2, 1:nc + 2, 1:nc + 1] -= t
    grad = dg[:, 1:nc + 1, 1:nc + 1].reshape(4, M).T
    return L, grad


def reference_energy(planes: np.ndarray) -> np.ndarray:
    """O_c of Dendy's interpolation (delta = 0), the loss normaliser."""
    nc = (bx.size_of(planes) - 1) // 2
    return basis_energy(planes, learned_interp(planes, np.zeros((nc * nc, 4))))[0]


def model_loss_grad(theta: np.ndarray, planes: np.ndarray, energy_ref=None):
    """Loss of the network on one problem and its gradient w.r.t. theta."""
    if energy_ref is None:
        energy_ref = reference_energy(planes)
    X = features(planes)
    out, cache = forward(theta, X)
    L, d_out = loss_and_grad(planes, out, energy_ref)
    return L, backward(theta, cache, d_out)


def init_params(normals: np.ndarray) -> np.ndarray:
    """Initial parameters from a vector of standard normals (drawn by the
    caller): W1, W2 He-scaled, biases 0, W3 = b3 = 0 (so delta = 0: Dendy)."""
    p = {name: np.zeros(shape) for name, shape in PARAM_SHAPES}
    k = N_IN * N_HID
    p["W1"] = normals[:k].reshape(N_IN, N_HID) * math.sqrt(2.0 / N_IN)
    p["W2"] = normals[k:k + N_HID * N_HID].reshape(N_HID, N_HID) * math.sqrt(2.0 / N_HID)
    return pack(p)


# ---------------------------------------------------------------------------
# Test-vector (approximation-property) loss
# ---------------------------------------------------------------------------

def inject_interp(ci: np.ndarray, v: np.ndarray):
    """(P R v, R v): R takes the values at coarse points."""
    n = v.shape[0] - 2
    nc = (n - 1) // 2
    ec = np.zeros((nc + 2, nc + 2))
    ec[1:nc + 1, 1:nc + 1] = v[2:2 * nc + 1:2, 2:2 * nc + 1:2]
    x = np.zeros_like(v)
    bx.interp_correct(ci, ec, x)
    return x, ec


def tv_energies(planes: np.ndarray, ci: np.ndarray, vecs) -> np.ndarray:
    """E_k = || v_k - P R v_k ||_A^2 for every test vector."""
    out = []
    for v in vecs:
        pv, _ = inject_interp(ci, v)
        e = v - pv
        out.append(bx.dot(e, bx.apply(planes, e)))
    return np.array(out)


def _add_outer(dW: np.ndarray, g: np.ndarray, ec: np.ndarray) -> None:
    """dW += the derivative of <g, P ec> with respect to the weight planes:
    for every weight w(p -> c) of P, g(p) ec(c), in the label layout."""
    nc = dW.shape[-1] - 2
    A, B, Bm = slice(1, nc + 1), slice(1, nc + 2), slice(0, nc + 1)
    even, odd = slice(2, 2 * nc + 1, 2), slice(1, 2 * nc + 2, 2)
    dW[LL, A, B] += g[even, odd] * ec[A, Bm]
    dW[LR, A, B] += g[even, odd] * ec[A, B]
    dW[LB, B, A] += g[odd, even] * ec[Bm, A]
    dW[LA, B, A] += g[odd, even] * ec[B, A]
    dW[LSW, B, B] += g[odd, odd] * ec[Bm, Bm]
    dW[LSE, B, B] += g[odd, odd] * ec[Bm, B]
    dW[LNW, B, B] += g[odd, odd] * ec[B, Bm]
    dW[LNE, B, B] += g[odd, odd] * ec[B, B]


def _weights_grad_to_delta(planes: np.ndarray, dW: np.ndarray, split) -> np.ndarray:
    """dL/d delta, shape (M, 4), from dL/dw of the eight weight planes:
    through Dendy's centre formula (linear in the edge weights) to the edge
    weights, then through the split w1 = S_D q, w2 = S_D (1 - q)."""
    SDx, qx, SDy, qy = split
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    B, Bm = slice(1, nc + 2), slice(0, nc + 1)
    dW = dW.copy()
    a = {d: bx.coupling(planes, *d) for d in bx.NBR}
    C = (slice(0, n, 2), slice(0, n, 2))
    o = a[(0, 0)][C]
    cW, cE, cS, cN = a[(-1, 0)][C] / o, a[(1, 0)][C] / o, a[(0, -1)][C] / o, a[(0, 1)][C] / o
    gsw, gse, gnw, gne = (dW[k, B, B].copy() for k in (LSW, LSE, LNW, LNE))
    dW[LB, B, Bm] += -cW * gsw
    dW[LL, Bm, B] += -cS * gsw
    dW[LB, B, B] += -cE * gse
    dW[LR, Bm, B] += -cS * gse
    dW[LA, B, Bm] += -cW * gnw
    dW[LL, B, B] += -cN * gnw
    dW[LA, B, B] += -cE * gne
    dW[LR, B, B] += -cN * gne
    dg = np.zeros((4, nc + 2, nc + 2))
    t = (dW[LL, 1:nc + 1, 1:nc + 2] - dW[LR, 1:nc + 1, 1:nc + 2]) * SDx * qx * (1.0 - qx)
    dg[1, 1:nc + 1, 0:nc + 1] += t
    dg[0, 1:nc + 1, 1:nc + 2] -= t
    t = (dW[LB, 1:nc + 2, 1:nc + 1] - dW[LA, 1:nc + 2, 1:nc + 1]) * SDy * qy * (1.0 - qy)
    dg[3, 0:nc + 1, 1:nc + 1] += t
    dg[2, 1:nc + 2, 1:nc + 1] -= t
    return dg[:, 1:nc + 1, 1:nc + 1].reshape(4, nc * nc).T


def tv_loss_grad(planes: np.ndarray, delta: np.ndarray, vecs, e_ref: np.ndarray):
    """L(delta) of the test-vector loss and dL/d delta, shape (M, 4)."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    K = len(vecs)
    ci, split = edge_split(planes, delta)
    centre_weights(planes, ci)
    dW = np.zeros((8, nc + 2, nc + 2))
    L = 0.0
    for v, er in zip(vecs, e_ref):
        pv, ec = inject_interp(ci, v)
        err = v - pv
        Ae = bx.apply(planes, err)
        L += bx.dot(err, Ae) / er / K
        _add_outer(dW, -2.0 * Ae / (er * K), ec)     # dL / d(P R v)(p) times v(c)
    return L, _weights_grad_to_delta(planes, dW, split)


def smooth_vectors(planes: np.ndarray, randoms, sweeps: int = 10):
    """Test vectors: each random vector (ghost ring zero) after `sweeps`
    Gauss-Seidel sweeps of A x = 0 (four colours), scaled to unit Euclidean norm."""
    lev = bx.Level(bx.size_of(planes), 9, np.array(planes, dtype=np.float64))
    out = []
    for r in randoms:
        v = np.array(r, dtype=np.float64)
        f = np.zeros_like(v)
        for _ in range(sweeps):
            bx.gs_sweep(9, lev.planes, lev.dinv, v, f)
        out.append(v / math.sqrt(bx.dot(v, v)))
    return out


def model_tv_loss_grad(theta, planes, vecs, e_ref):
    X = features(planes)
    out, cache = forward(theta, X)
    L, d_out = tv_loss_grad(planes, out, vecs, e_ref)
    return L, backward(theta, cache, d_out)


# ---------------------------------------------------------------------------
# Two-grid loss: the A-energy of the two-grid error propagation
#   E = S^nu2 (I - P A_c^{-1} P^T A) S^nu1,   A_c = P^T A P,
# the measured quantity the learned interpolation is trained to reduce.
# ---------------------------------------------------------------------------

def error_sweep(planes: np.ndarray, dinv: np.ndarray, e: np.ndarray) -> None:
    """One four-colour Gauss-Seidel sweep of A e = 0, in place: the error
    propagation S = M_4 M_3 M_2 M_1 of a sweep, M_c = I - J_c D^{-1} A (J_c
    keeps the points of colour c)."""
    bx.gs_sweep(9, planes, dinv, e, np.zeros_like(e))


def error_sweep_adjoint(planes: np.ndarray, dinv: np.ndarray, y: np.ndarray) -> None:
    """y <- S^T y, in place.  A is symmetric, so M_c^T = I - A D^{-1} J_c, and
    S^T = M_1^T M_2^T M_3^T M_4^T applies the colours in reverse order: for each,
    z = D^{-1} y on the colour's points (zero elsewhere), then y = y - A z."""
    for pi, pj in reversed(bx.COLOURS9):
        c = bx.colour(pi, pj)
        z = np.zeros_like(y)
        bx.at(z, 0, 0)[c] = bx.at(y, 0, 0)[c] * bx.at(dinv, 0, 0)[c]
        y -= bx.apply(planes, z)


def _dinv(planes: np.ndarray) -> np.ndarray:
    d = np.zeros_like(planes[0])
    bx.at(d, 0, 0)[...] = 1.0 / bx.at(planes[0], 0, 0)
    return d


def coarse_operator(planes: np.ndarray, ci: np.ndarray) -> np.ndarray:
    """The dense Galerkin operator A_c = P^T A P (interior coarse unknowns,
    lexicographic)."""
    return bx.dense_matrix(bx.rap(planes, ci))


def _coarse_solve(Ac: np.ndarray, fc: np.ndarray) -> np.ndarray:
    """A_c^{-1} fc for an (nc+2)^2 coarse array (any exact solve: numpy's)."""
    nc = fc.shape[-1] - 2
    u = np.zeros_like(fc)
    u[1:nc + 1, 1:nc + 1] = np.linalg.solve(Ac, fc[1:nc + 1, 1:nc + 1].reshape(-1)).reshape(nc, nc)
    return u


def two_grid(planes: np.ndarray, ci: np.ndarray, e: np.ndarray, Ac: np.ndarray, nu1: int = 2, nu2: int = 1):
    """E e for one error vector e (ghost ring zero) and the vectors on the way:
    e1 = S^nu1 e; u = A_c^{-1} P^T A e1; e2 = e1 - P u; e3 = S^nu2 e2."""
    dinv = _dinv(planes)
    e1 = np.array(e, dtype=np.float64)
    for _ in range(nu1):
        error_sweep(planes, dinv, e1)
    u = _coarse_solve(Ac, bx.restrict(ci, bx.apply(planes, e1)))
    e2 = e1.copy()
    bx.interp_correct(ci, -u, e2)
    e3 = e2.copy()
    for _ in range(nu2):
        error_sweep(planes, dinv, e3)
    return e1, u, e2, e3


def two_grid_energies(planes: np.ndarray, ci: np.ndarray, vecs, nu1: int = 2, nu2: int = 1) -> np.ndarray:
    """||E e_k||_A^2 for every vector."""
    Ac = coarse_operator(planes, ci)
    out = []
    for e in vecs:
        e3 = two_grid(planes, ci, e, Ac, nu1, nu2)[3]
        out.append(bx.dot(e3, bx.apply(planes, e3)))
    return np.array(out)


def two_grid_loss_grad(planes: np.ndarray, delta: np.ndarray, vecs, e_ref: np.ndarray, nu1: int = 2,
                       nu2: int = 1, weight: float = 1.0):
    """L = weight/K sum_k ||E e_k||_A^2 / e_ref_k and dL/d delta, shape (M, 4).

    With g2 = S^{nu2 T} (dL/d e3) and the adjoint coarse solve
    v = A_c^{-1} P^T g2, every term of E through P (the restriction P^T, the
    coarse operator P^T A P and the interpolation P) gives
        dL/dP = (A P v - g2) u^T - (A e2) v^T,
    taken on P's sparsity pattern, then chained to delta."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    K = len(vecs)
    ci, split = edge_split(planes, delta)
    centre_weights(planes, ci)
    Ac = coarse_operator(planes, ci)
    dinv = _dinv(planes)
    dW = np.zeros((8, nc + 2, nc + 2))
    L = 0.0
    for e, er in zip(vecs, e_ref):
        _, u, e2, e3 = two_grid(planes, ci, e, Ac, nu1, nu2)
        Ae3 = bx.apply(planes, e3)
        L += weight * bx.dot(e3, Ae3) / (K * er)
        g = 2.0 * weight / (K * er) * Ae3                # dL/d e3
        for _ in range(nu2):
            error_sweep_adjoint(planes, dinv, g)          # dL/d e2
        v = _coarse_solve(Ac, bx.restrict(ci, g))
        pv = np.zeros_like(e2)
        bx.interp_correct(ci, v, pv)
        _add_outer(dW, bx.apply(planes, pv) - g, u)
        _add_outer(dW, -bx.apply(planes, e2), v)
    return L, _weights_grad_to_delta(planes, dW, split)


def two_grid_reference(planes: np.ndarray, vecs, nu1: int = 2, nu2: int = 1) -> np.ndarray:
    """The loss normalisers: Dendy's two-grid energies (delta = 0)."""
    nc = (bx.size_of(planes) - 1) // 2
    return two_grid_energies(planes, learned_interp(planes, np.zeros((nc * nc, 4))), vecs, nu1, nu2)


def model_two_grid_loss_grad(theta: np.ndarray, crops, nu1: int = 2, nu2: int = 1):
    """Loss of the network over a batch of crops (planes, vectors, e_ref):
    the mean over crops of their two-grid losses, and its gradient w.r.t. theta."""
    C = len(crops)
    L = 0.0
    g = np.zeros_like(theta)
    for planes, vecs, e_ref in crops:
        out, cache = forward(theta, features(planes))
        l, d_out = two_grid_loss_grad(planes, out, vecs, e_ref, nu1, nu2, weight=1.0 / C)
        L += l
        g += backward(theta, cache, d_out)
    return L, g
