"""Pins of the oracle's zero-shift screen (Eq. 1 is the correlation at zero
shift, Eq. 3) and of its BF16 input rounding."""
import numpy as np
import pytest


def test_bf16_round_half_even(orc):
    assert orc.bf16_round(1.0) == 1.0
    assert orc.bf16_round(1.0 + 2.0 ** -8) == 1.0                    # halfway: to the even mantissa
    assert orc.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # halfway: up to even
    assert orc.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert orc.bf16_round(-3.0) == -3.0


def test_bf16_round_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 3, 2000), [0.0, -0.0]])
    mine = np.array([orc.bf16_round(v) for v in x])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mine, ref)


def test_screen_is_zero_shift_correlation(orc):
    rng = np.random.default_rng(1)
    n = 32
    S, y, _ = orc.prep_many(rng.standard_normal((5, n, n)), want_spatial=True)
    sc = orc.screen(y[:2], y, bf16=False)
    for p in range(2):
        assert sc[p, p] == pytest.approx(1.0, abs=1e-12)
        for t in range(5):
            assert sc[p, t] == pytest.approx(orc.xcf_surface(S[t], S[p])[0, 0], abs=1e-12)
    # BF16 inputs move the scores by a few parts in 1e3 of their scale at most
    sb = orc.screen(y[:2], y, bf16=True)
    assert np.abs(sb - sc).max() < 1e-2 and np.abs(sb - sc).max() > 0
