"""Pins of the FP64 oracle of the learned orientation proposal: convolution
against scipy's correlate2d, every backward pass against central finite
differences of its forward, Gram-Schmidt and the symmetric loss against their
closed forms and invariances, Adam against its closed-form first step."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import synth

K = 8


def test_param_count(orc):
    ch = [1, 32, 64, 64, 128, 128]
    conv = sum(ch[i + 1] * ch[i] * 9 + ch[i + 1] for i in range(5))
    assert orc.cnn_num_params(K) == conv + 256 * 128 + 256 + 6 * K * 256 + 6 * K
    assert orc.cnn_num_params(1) == conv + 256 * 128 + 256 + 6 * 256 + 6


def test_standardise(orc):
    x = np.random.default_rng(0).normal(3.0, 2.0, 4096)
    y = orc.cnn_standardise(x)
    assert abs(y.mean()) < 1e-12 and abs(y.std() - 1.0) < 1e-12
    assert np.all(orc.cnn_standardise(np.full(64, 5.0)) == 0.0)


@pytest.mark.parametrize("ci,co,s", [(1, 3, 8), (4, 2, 6), (3, 5, 16)])
def test_conv_matches_correlate2d(orc, ci, co, s):
    rng = np.random.default_rng(ci * 10 + co)
    x = rng.normal(size=(ci, s, s))
    w = rng.normal(size=(co, ci, 3, 3))
    b = rng.normal(size=co)
    y = orc.conv3x3s2(x, w, b)
    ref = np.empty_like(y)
    for o in range(co):
        acc = sum(correlate2d(np.pad(x[i], 1), w[o, i], mode="valid") for i in range(ci))
        ref[o] = acc[::2, ::2] + b[o]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def _rand_rot(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q) * np.sign(q[0])


def test_gram_schmidt_closed_forms(orc):
    R = orc.gram_schmidt([3.0, 0, 0, 2.0, 5.0, 0])
    np.testing.assert_allclose(R, np.eye(3), atol=1e-15)
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = rng.normal(size=6)
        R = orc.gram_schmidt(a)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
        np.testing.assert_allclose(R[:, 0], a[:3] / np.linalg.norm(a[:3]), atol=1e-14)
        # invariant under scaling of a1 and shearing of a2 along a1
        a2 = np.r_[2.5 * a[:3], a[3:] + 0.7 * a[:3]]
        np.testing.assert_allclose(orc.gram_schmidt(a2), R, atol=1e-12)
        # a rotation's first two columns give back the rotation
        Q = orc.quat_to_matrix(_rand_rot(rng))
        np.testing.assert_allclose(orc.gram_schmidt(np.r_[Q[:, 0], Q[:, 1]]), Q, atol=1e-12)


def test_gram_schmidt_backward_finite_differences(orc):
    rng = np.random.default_rng(2)
    for _ in range(10):
        a, G = rng.normal(size=6), rng.normal(size=(3, 3))
        ga = orc.gram_schmidt_backward(a, G)
        h = 1e-6
        fd = np.array([(np.sum(G * orc.gram_schmidt(a + h * e)) - np.sum(G * orc.gram_schmidt(a - h * e))) / (2 * h)
                       for e in np.eye(6)])
        np.testing.assert_allclose(ga, fd, rtol=1e-6, atol=1e-8)


def test_cubic_matrices_are_the_cubic_group(orc):
    S = orc.cubic_matrices()
    assert len({tuple(m.round().astype(int).ravel()) for m in S}) == 24
    keys = {tuple(m.round().astype(int).ravel()) for m in S}
    for a in S:
        np.testing.assert_allclose(a @ a.T, np.eye(3), atol=0)
        assert round(np.linalg.det(a)) == 1
        for b in S:
            assert tuple((a @ b).round().astype(int).ravel()) in keys
    # the same group as the quaternion operators of the disorientation
    qs = {tuple(orc.quat_to_matrix(q).round().astype(int).ravel()) for q in orc.cubic_ops()}
    assert qs == keys


def _out6_of(R):
    return np.r_[R[:, 0], R[:, 1]]


def test_head_loss_zero_symmetric_and_winner(orc):
    rng = np.random.default_rng(3)
    S = orc.cubic_matrices()
    for _ in range(5):
        q = _rand_rot(rng)
        Rg = orc.quat_to_matrix(q)
        out = rng.normal(size=6 * K)
        out[18:24] = _out6_of(S[7] @ Rg) * 1.7   # head 3 encodes an equivalent orientation
        loss, g, h, s = orc.cnn_head_loss(out, K, q)
        assert loss < 1e-24 and h == 3 and s == 7
        np.testing.assert_allclose(g, 0, atol=1e-12)
        # loss(q) = loss(S q) for every operator: S Rg is Rg's symmetric equivalent
        out = rng.normal(size=6 * K)
        l0 = orc.cnn_head_loss(out, K, q, False)[0]
        for qs in orc.cubic_ops():
            l1 = orc.cnn_head_loss(out, K, orc.qmul(qs, q), False)[0]
            assert abs(l1 - l0) < 1e-10
        # the closed form |R - T|^2 = 6 - 2 tr(R^T T) at the winner
        l, _, h, s = orc.cnn_head_loss(out, K, q)
        R = orc.gram_schmidt(out[6 * h:6 * h + 6])
        assert abs(l - (6 - 2 * np.trace(R.T @ S[s] @ Rg))) < 1e-12


def test_head_loss_gradient_finite_differences(orc):
    rng = np.random.default_rng(4)
    q = _rand_rot(rng)
    out = rng.normal(size=6 * K)
    _, g, _, _ = orc.cnn_head_loss(out, K, q)
    h = 1e-6
    fd = np.array([(orc.cnn_head_loss(out + h * e, K, q, False)[0] - orc.cnn_head_loss(out - h * e, K, q, False)[0])
                   / (2 * h) for e in np.eye(6 * K)])
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8)


def test_matrix_to_quat_round_trip(orc):
    rng = np.random.default_rng(5)
    qs = [_rand_rot(rng) for _ in range(20)]
    for i in range(4):   # each component dominant in turn
        e = np.full(4, 0.1)
        e[i] = 1.0
        qs.append(e / np.linalg.norm(e))
    for q in qs:
        q = q * np.sign(q[0]) if q[0] != 0 else q
        np.testing.assert_allclose(orc.matrix_to_quat(orc.quat_to_matrix(q)), q, atol=1e-12)


def test_adam_closed_form(orc):
    rng = np.random.default_rng(6)
    n = 50
    g = rng.normal(size=n)
    p0 = rng.normal(size=n)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    orc.adam(p, g, m, v, 1, lr=1e-2)
    np.testing.assert_allclose(p, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    orc.adam(p, g, m, v, 2, lr=1e-2)   # constant gradient: the same step again
    np.testing.assert_allclose(p, p0 - 2e-2 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def _init_params(k=K, seed=0):
    return synth.cnn_init_params(k, seed)


def _images(B, seed):
    rng = np.random.default_rng(seed)
    return rng.gamma(2.0, 20.0, size=(B, 128, 128))


def test_forward_composes_the_layers(orc):
    """The flat parameter layout: the network equals its pinned layers composed."""
    p = _init_params()
    x = _images(2, 7)
    out = orc.cnn_forward(p, x, K)
    ch = [1, 32, 64, 64, 128, 128]
    o = 0
    for b in range(2):
        a = orc.cnn_standardise(x[b])[None]
        o = 0
        for l in range(5):
            nw = ch[l + 1] * ch[l] * 9
            w = p[o:o + nw].astype(np.float64).reshape(ch[l + 1], ch[l], 3, 3)
            bias = p[o + nw:o + nw + ch[l + 1]].astype(np.float64)
            o += nw + ch[l + 1]
            a = np.maximum(orc.conv3x3s2(a, w, bias), 0.0)
        pool = a.mean(axis=(1, 2))
        W1 = p[o:o + 256 * 128].astype(np.float64).reshape(256, 128)
        b1 = p[o + 256 * 128:o + 256 * 129].astype(np.float64)
        o += 256 * 129
        h1 = np.maximum(W1 @ pool + b1, 0.0)
        W2 = p[o:o + 6 * K * 256].astype(np.float64).reshape(6 * K, 256)
        b2 = p[o + 6 * K * 256:].astype(np.float64)
        np.testing.assert_allclose(out[b], W2 @ h1 + b2, rtol=1e-10, atol=1e-12)
    assert o + 6 * K * 256 + 6 * K == len(p)


def test_network_gradient_finite_differences(orc):
    p = _init_params(seed=1)
    x = _images(2, 8)
    q = np.stack([_rand_rot(np.random.default_rng(9 + i)) for i in range(2)])
    loss, grad, win = orc.cnn_loss_grad(p, x, q, K)
    assert grad.shape == p.shape and np.all((win[:, 0] >= 0) & (win[:, 0] < K))
    n = len(p)
    ch = [1, 32, 64, 64, 128, 128]
    starts, o = [], 0
    for l in range(5):
        starts += [o + 4, o + ch[l + 1] * ch[l] * 9 + 1]     # a weight and a bias of every conv layer
        o += ch[l + 1] * ch[l] * 9 + ch[l + 1]
    starts += [o + 300, o + 256 * 128 + 3, n - 6 * K * 256 - 6 * K + 100, n - 2]
    for i in starts:
        pp, pm = p.copy(), p.copy()
        pp[i] += np.float32(2e-5)   # small enough that no ReLU changes side
        pm[i] -= np.float32(2e-5)
        d = float(pp[i]) - float(pm[i])
        fd = (orc.cnn_loss_grad(pp, x, q, K, False)[0] - orc.cnn_loss_grad(pm, x, q, K, False)[0]) / d
        assert abs(fd - grad[i]) <= 1e-5 * abs(grad[i]) + 1e-9, (i, fd, grad[i])


def test_proposals_are_the_heads(orc):
    rng = np.random.default_rng(10)
    out = rng.normal(size=(3, 6 * K))
    q = orc.cnn_proposals(out, K)
    for b in range(3):
        for h in range(K):
            np.testing.assert_allclose(orc.quat_to_matrix(q[b, h]), orc.gram_schmidt(out[b, 6 * h:6 * h + 6]),
                                       atol=1e-12)
            assert q[b, h, 0] >= 0


def test_bf16_form_rounds_only_the_later_convolutions():
    """The BF16 inference form differs from the FP64 forward by the BF16
    rounding of the inputs and weights of convolutions 2..5 only: close to it
    (BF16 keeps 8 significant bits) but not equal; with those layers' weights
    zeroed it equals the FP64 forward exactly (nothing else is rounded)."""
    import oracle as orc
    p = synth.cnn_init_params(8, 9).astype(np.float32)
    x = np.random.default_rng(9).random((3, 128, 128))
    a, b = orc.cnn_forward(p, x, 8), orc.cnn_forward_bf16(p, x, 8)
    scale = np.abs(a).max()
    assert 0 < np.abs(a - b).max() <= 2e-2 * scale
    # zero the weights of convolutions 2..5: their outputs are their biases in both forms
    q = p.copy()
    o = 32 * 1 * 9 + 32
    for ci, co in ((32, 64), (64, 64), (64, 128), (128, 128)):
        q[o:o + co * ci * 9] = 0.0
        o += co * ci * 9 + co
    np.testing.assert_array_equal(orc.cnn_forward(q, x, 8), orc.cnn_forward_bf16(q, x, 8))
