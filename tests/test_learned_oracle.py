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
