"""Pins of the learned-interpolation oracle: delta = 0 reproduces Dendy's
weights; the basis energy equals the Galerkin diagonal of the oracle's
stencil-form RAP; hand-written gradients equal central finite differences."""
import numpy as np
import pytest

import workloads as w
from oracle import boxmg as bx
from oracle import learned as ln


def hc_planes(n=31, seed=6, block=4):
    return w.fe9_from_cells(w.binary_blocks(n, block, 1.0, 1e6, seed))


def test_zero_output_is_dendy():
    planes = hc_planes(63)
    nc = 31
    ci = ln.learned_interp(planes, np.zeros((nc * nc, 4)))
    ref = bx.dendy_interp(planes)
    assert np.abs(ci - ref).max() <= 1e-14 * np.abs(ref).max()


def test_basis_energy_is_galerkin_diagonal():
    planes = hc_planes(31)
    nc = 15
    delta = w.normal(3, nc * nc * 4).reshape(nc * nc, 4) * 0.5
    ci = ln.learned_interp(planes, delta)
    energy, _ = ln.basis_energy(planes, ci)
    diag = bx.rap(planes, ci)[0, 1:nc + 1, 1:nc + 1]
    assert np.abs(energy - diag).max() <= 1e-12 * np.abs(diag).max()


def test_features_shape_and_constant_coefficients():
    n = 31
    X = ln.features(w.fe9_from_cells(np.ones((n + 1, n + 1))))
    assert X.shape == (15 * 15, 18)
    # interior constant FE stencil: (a_W + a_E)/a_O = (-1/3 - 1/3)/(8/3) = -1/4
    inner = X.reshape(15, 15, 18)[2:-2, 2:-2]
    assert np.allclose(inner, -0.25, rtol=0, atol=1e-15)


def test_loss_gradient_matches_finite_differences():
    planes = hc_planes(15, seed=8, block=2)
    nc = 7
    ref = ln.reference_energy(planes)
    delta = w.normal(4, nc * nc * 4).reshape(nc * nc, 4) * 0.3
    L0, g = ln.loss_and_grad(planes, delta, ref)
    assert abs(ln.loss_and_grad(planes, np.zeros_like(delta), ref)[0] - 1.0) <= 1e-13
    h = 1e-6
    for idx in [(0, 0), (10, 1), (24, 2), (30, 3), (48, 0), (17, 3)]:
        dp = delta.copy()
        dp[idx] += h
        dm = delta.copy()
        dm[idx] -= h
        fd = (ln.loss_and_grad(planes, dp, ref)[0] - ln.loss_and_grad(planes, dm, ref)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-6), idx


def test_network_gradient_matches_finite_differences():
    planes = hc_planes(15, seed=9, block=2)
    theta = ln.init_params(w.normal(11, ln.N_IN * ln.N_HID + ln.N_HID * ln.N_HID))
    p = ln.unpack(theta)
    p["W3"][...] = w.normal(12, ln.N_HID * ln.N_OUT).reshape(ln.N_HID, ln.N_OUT) * 0.1
    p["b1"][...] = w.normal(13, ln.N_HID) * 0.1
    theta = ln.pack(p)
    ref = ln.reference_energy(planes)
    L, g = ln.model_loss_grad(theta, planes, ref)
    assert g.shape == (ln.N_PARAMS,)
    rng_idx = (w.uniform01(14, 12) * ln.N_PARAMS).astype(int)
    h = 1e-4   # the loss is smooth; a smaller step only adds cancellation noise
    for k in list(rng_idx) + [ln.N_PARAMS - 1, ln.N_PARAMS - 5]:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (ln.model_loss_grad(tp, planes, ref)[0] - ln.model_loss_grad(tm, planes, ref)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-4), k


def test_initial_network_is_dendy_and_descent_lowers_the_loss():
    planes = hc_planes(31, seed=10, block=4)
    theta = ln.init_params(w.normal(15, ln.N_IN * ln.N_HID + ln.N_HID * ln.N_HID))
    ref = ln.reference_energy(planes)
    L0, g = ln.model_loss_grad(theta, planes, ref)
    assert abs(L0 - 1.0) <= 1e-13
    eps = 1e-5 / float(g @ g)                    # -g is a descent direction, first-order decrease eps |g|^2
    L1, _ = ln.model_loss_grad(theta - eps * g, planes, ref)
    assert L1 < L0 and abs((L0 - L1) - eps * float(g @ g)) <= 0.3 * eps * float(g @ g)


def tv_setup(n=15, seed=21, K=3):
    planes = w.fe9_from_cells(w.binary_blocks(n, 2, 1.0, 1e6, seed))
    vecs = ln.smooth_vectors(planes, [w.rhs_uniform(n, 300 + k) for k in range(K)])
    nc = (n - 1) // 2
    e_ref = ln.tv_energies(planes, ln.learned_interp(planes, np.zeros((nc * nc, 4))), vecs)
    return planes, vecs, e_ref


def test_tv_loss_at_dendy_is_one_and_gradient_matches_fd():
    planes, vecs, e_ref = tv_setup()
    nc = 7
    assert abs(ln.tv_loss_grad(planes, np.zeros((nc * nc, 4)), vecs, e_ref)[0] - 1.0) <= 1e-12
    delta = w.normal(31, nc * nc * 4).reshape(nc * nc, 4) * 0.3
    L, g = ln.tv_loss_grad(planes, delta, vecs, e_ref)
    h = 1e-5
    for idx in [(3, 0), (10, 1), (24, 2), (30, 3), (45, 1)]:
        dp, dm = delta.copy(), delta.copy()
        dp[idx] += h
        dm[idx] -= h
        fd = (ln.tv_loss_grad(planes, dp, vecs, e_ref)[0] - ln.tv_loss_grad(planes, dm, vecs, e_ref)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-4), idx


def test_tv_energy_is_a_quadratic_form():
    """E = (v - P R v)^T A (v - P R v) checked against the assembled dense A and P."""
    planes, vecs, _ = tv_setup(n=7, K=2)
    ci = bx.dendy_interp(planes)
    A = bx.dense_matrix(planes)
    for v in vecs:
        pv, _ = ln.inject_interp(ci, v)
        e = (v - pv)[1:8, 1:8].reshape(-1)
        assert abs(ln.tv_energies(planes, ci, [v])[0] - e @ A @ e) <= 1e-12 * abs(e @ A @ e)


def test_tv_network_gradient_matches_fd():
    planes, vecs, e_ref = tv_setup(seed=22)
    theta = ln.init_params(w.normal(41, ln.N_IN * ln.N_HID + ln.N_HID * ln.N_HID))
    p = ln.unpack(theta)
    p["W3"][...] = w.normal(42, ln.N_HID * ln.N_OUT).reshape(ln.N_HID, ln.N_OUT) * 0.1
    theta = ln.pack(p)
    L, g = ln.model_tv_loss_grad(theta, planes, vecs, e_ref)
    h = 1e-4
    for k in [0, 37, 1200, 3000, 5500, ln.N_PARAMS - 1]:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (ln.model_tv_loss_grad(tp, planes, vecs, e_ref)[0] - ln.model_tv_loss_grad(tm, planes, vecs, e_ref)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-4), k


@pytest.mark.parametrize("scale", [0.5, 3.0])
def test_learned_weights_keep_constants_for_any_logits(scale):
    """For a zero-row-sum operator, any logits keep each edge point's Dendy
    weight sum (1 there) and the centre rows solve their local equation, so
    interpolating a constant gives that constant at every fine point whose
    row is zero-sum and sees only interior coarse points, while the weights
    themselves differ from Dendy's."""
    n, nc = 63, 31
    planes = hc_planes(n, seed=9, block=4)
    delta = w.normal(12, nc * nc * 4).reshape(nc * nc, 4) * scale
    ci = ln.learned_interp(planes, delta)
    assert np.abs(ci - bx.dendy_interp(planes)).max() > 1e-2
    ec = np.zeros((nc + 2, nc + 2))
    ec[1:nc + 1, 1:nc + 1] = 1.0
    x = np.zeros((n + 2, n + 2))
    bx.interp_correct(ci, ec, x)
    assert np.abs(x[3:n - 1, 3:n - 1] - 1.0).max() <= 1e-12


# ---- the two-grid loss ---------------------------------------------------------------------

def _dense_two_grid(planes, ci, nu1=2, nu2=1):
    """E = S^nu2 (I - P (P^T A P)^{-1} P^T A) S^nu1 from dense matrices built
    from their definitions, independently of the oracle's sweeps and
    transfers: A entry by entry from the stencil planes and their symmetry;
    P column by column from the eight weight labels (the coarse point's own
    fine point 1, edge points toward it, centre points toward it); S as the
    product over the colours of I - J_c D^{-1} A."""
    n = bx.size_of(planes)
    nc = (n - 1) // 2
    m, mc = n * n, nc * nc
    O, W, S, SW, NW = planes
    A = np.zeros((m, m))
    idx = lambda i, j: (j - 1) * n + (i - 1)
    for j in range(1, n + 1):
        for i in range(1, n + 1):
            p = idx(i, j)
            A[p, p] = O[j, i]
            for di, dj, val in ((-1, 0, W[j, i]), (1, 0, W[j, i + 1]), (0, -1, S[j, i]), (0, 1, S[j + 1, i]),
                                (-1, -1, SW[j, i]), (1, 1, SW[j + 1, i + 1]), (-1, 1, NW[j, i]),
                                (1, -1, NW[j - 1, i + 1])):
                if 1 <= i + di <= n and 1 <= j + dj <= n:
                    A[p, idx(i + di, j + dj)] = val
    P = np.zeros((m, mc))
    for jc in range(1, nc + 1):
        for ic in range(1, nc + 1):
            c = (jc - 1) * nc + (ic - 1)
            I, J = 2 * ic, 2 * jc
            P[idx(I, J), c] = 1.0
            # edge points: x-edge (I-1, J) of cell (ic, jc) toward its east point LR; (I+1, J) of cell (ic+1, jc)
            # toward its west point LL; y-edges likewise with LA (cell (ic, jc)) and LB (cell (ic, jc+1))
            P[idx(I - 1, J), c] = ci[bx.LR, jc, ic]
            P[idx(I + 1, J), c] = ci[bx.LL, jc, ic + 1]
            P[idx(I, J - 1), c] = ci[bx.LA, jc, ic]
            P[idx(I, J + 1), c] = ci[bx.LB, jc + 1, ic]
            # centre points of the four cells around the coarse point
            P[idx(I - 1, J - 1), c] = ci[bx.LNE, jc, ic]
            P[idx(I + 1, J - 1), c] = ci[bx.LNW, jc, ic + 1]
            P[idx(I - 1, J + 1), c] = ci[bx.LSE, jc + 1, ic]
            P[idx(I + 1, J + 1), c] = ci[bx.LSW, jc + 1, ic + 1]
    Sm = np.eye(m)
    Dinv = np.diag(1.0 / np.diag(A))
    for pi, pj in bx.COLOURS9:
        J = np.zeros((m, m))
        for j in range(1, n + 1):
            for i in range(1, n + 1):
                if i % 2 == pi and j % 2 == pj:
                    J[idx(i, j), idx(i, j)] = 1.0
        Sm = (np.eye(m) - J @ Dinv @ A) @ Sm
    Ac = P.T @ A @ P
    CGC = np.eye(m) - P @ np.linalg.solve(Ac, P.T @ A)
    return np.linalg.matrix_power(Sm, nu2) @ CGC @ np.linalg.matrix_power(Sm, nu1), A, Sm


def _interior(v):
    return v[1:-1, 1:-1].reshape(-1)


def test_two_grid_is_the_dense_error_propagation():
    """E e from the oracle's sweeps, transfers and coarse solve equals the
    dense two-grid matrix applied to e, and the loss's energies equal
    e^T E^T A E e, for Dendy's and for learned weights."""
    planes = hc_planes(15, seed=9, block=2)
    nc = 7
    vecs = [w.rhs_uniform(15, 300 + k) for k in range(3)]
    for delta in (np.zeros((nc * nc, 4)), w.normal(5, nc * nc * 4).reshape(nc * nc, 4) * 0.7):
        ci = ln.learned_interp(planes, delta)
        E, A, _ = _dense_two_grid(planes, ci)
        Ac = ln.coarse_operator(planes, ci)
        energies = ln.two_grid_energies(planes, ci, vecs)
        for e, en in zip(vecs, energies):
            want = E @ _interior(e)
            got = _interior(ln.two_grid(planes, ci, e, Ac)[3])
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
            assert abs(en - want @ A @ want) <= 1e-12 * abs(en)


def test_two_grid_is_the_two_level_vcycle_and_its_spectral_radius():
    """With Dendy's weights the two-grid operator is the oracle's own V(2,1)
    on a two-level hierarchy (coarsest = (n-1)/2) applied to e with f = 0, and
    the solve on that hierarchy converges at the dense operator's spectral
    radius (measured asymptotic factor within 5 %)."""
    n, nc = 15, 7
    planes = hc_planes(n, seed=10, block=2)
    levels = bx.setup(9, planes, coarsest=nc)
    assert len(levels) == 2
    ci = levels[0].ci
    Ac = ln.coarse_operator(planes, ci)
    for k in range(3):
        e = w.rhs_uniform(n, 400 + k)
        x = e.copy()
        bx.vcycle(levels, 0, x, np.zeros_like(e))
        got = ln.two_grid(planes, ci, e, Ac)[3]
        assert np.abs(got - x).max() <= 1e-12 * np.abs(x).max()
    E, _, _ = _dense_two_grid(planes, ci)
    rho = max(abs(np.linalg.eigvals(E)))
    _, hist = bx.solve(levels, w.rhs_uniform(n, 5), tol=1e-300, maxit=15)
    measured = (hist[15] / hist[5]) ** 0.1                  # iterations 5 .. 15, above the rounding floor
    assert abs(measured - rho) <= 0.05 * rho, (measured, rho)


def test_error_sweep_adjoint_is_the_transpose():
    planes = hc_planes(15, seed=11, block=2)
    d = np.zeros_like(planes[0])
    bx.at(d, 0, 0)[...] = 1.0 / bx.at(planes[0], 0, 0)
    _, _, Sm = _dense_two_grid(planes, bx.dendy_interp(planes))
    for k in range(3):
        x, y = w.rhs_uniform(15, 500 + k), w.rhs_uniform(15, 600 + k)
        sx = x.copy()
        ln.error_sweep(planes, d, sx)
        sty = y.copy()
        ln.error_sweep_adjoint(planes, d, sty)
        assert np.abs(_interior(sx) - Sm @ _interior(x)).max() <= 1e-12 * np.abs(_interior(sx)).max()
        assert np.abs(_interior(sty) - Sm.T @ _interior(y)).max() <= 1e-12 * np.abs(_interior(sty)).max()
        assert abs(bx.dot(sx, y) - bx.dot(x, sty)) <= 1e-12 * abs(bx.dot(sx, y))


def test_two_grid_gradient_matches_finite_differences():
    n, nc = 15, 7
    planes = hc_planes(n, seed=12, block=2)
    vecs = [w.rhs_uniform(n, 700 + k) for k in range(3)]
    ref = ln.two_grid_reference(planes, vecs)
    L0, _ = ln.two_grid_loss_grad(planes, np.zeros((nc * nc, 4)), vecs, ref)
    assert abs(L0 - 1.0) <= 1e-12
    delta = w.normal(13, nc * nc * 4).reshape(nc * nc, 4) * 0.4
    L, g = ln.two_grid_loss_grad(planes, delta, vecs, ref)
    h = 1e-6
    for idx in [(0, 0), (8, 1), (24, 2), (31, 3), (48, 0), (17, 1), (40, 2)]:
        dp, dm = delta.copy(), delta.copy()
        dp[idx] += h
        dm[idx] -= h
        fd = (ln.two_grid_loss_grad(planes, dp, vecs, ref)[0] - ln.two_grid_loss_grad(planes, dm, vecs, ref)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-8 * np.abs(g).max(), (idx, fd, g[idx])


def test_model_two_grid_gradient_matches_finite_differences():
    n, nc = 15, 7
    crops = []
    for s in range(2):
        planes = hc_planes(n, seed=20 + s, block=2)
        vecs = [w.rhs_uniform(n, 800 + 10 * s + k) for k in range(2)]
        crops.append((planes, vecs, ln.two_grid_reference(planes, vecs)))
    theta = ln.init_params(w.normal(21, ln.N_IN * ln.N_HID + ln.N_HID * ln.N_HID))
    p = ln.unpack(theta)
    p["W3"][...] = w.normal(22, ln.N_HID * ln.N_OUT).reshape(ln.N_HID, ln.N_OUT) * 0.1
    theta = ln.pack(p)
    L, g = ln.model_two_grid_loss_grad(theta, crops)
    h = 1e-6
    off_w3 = ln.N_IN * ln.N_HID + ln.N_HID + ln.N_HID * ln.N_HID + ln.N_HID
    for k in (0, 100, ln.N_IN * ln.N_HID + 3, off_w3 + 5, off_w3 + 200, ln.N_PARAMS - 2):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (ln.model_two_grid_loss_grad(tp, crops)[0] - ln.model_two_grid_loss_grad(tm, crops)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * abs(fd) + 1e-8 * np.abs(g).max(), (k, fd, g[k])


def test_training_crops_are_dirichlet_problems_of_the_family():
    crops = w.training_crops(4, crops_per_problem=2)
    assert len(crops) == 8
    for planes, vecs in crops:
        assert planes.shape == (5, 33, 33) and vecs.shape == (4, 33, 33)
        k = -3.0 * planes[3][2:-1, 2:-1]                       # SW = -k/3 of the cell below-left
        assert set(np.unique(np.round(k, 6))) <= {1.0, 1e6}
        assert not vecs[:, 0].any() and not vecs[:, -1].any()
