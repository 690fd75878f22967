"""Pins of the oracle's single-edge BCA updates (Sec. 4, eqs. U, M, H).

Nothing here compares the oracle with itself: each check is a value printed in
the paper, a property the paper proves, or an equivalent formulation stated in
the paper but computed differently.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "prop3_counterexample.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def test_worked_example_printed_values(gold):
    """Appendix B, proof of Prop. 3: H on the printed costs gives the printed
    unaries, for both the original and the zeroed unaries."""
    tuv = np.asarray(gold["theta_uv"], float)
    u, v, res = oracle.update_edge("H", gold["theta_u"], gold["theta_v"], tuv)
    assert u.tolist() == gold["H"]["theta_u"]
    assert v.tolist() == gold["H"]["theta_v"]
    u2, v2, res2 = oracle.update_edge("H", gold["theta_u_prime"], gold["theta_v_prime"], tuv)
    assert u2.tolist() == gold["H_prime"]["theta_u"]
    assert v2.tolist() == gold["H_prime"]["theta_v"]
    d = gold["derived_by_hand_not_printed"]
    assert res.tolist() == d["H_residual"]
    assert res2.tolist() == d["H_prime_residual"]
    # H is not monotonous (Prop. 3): theta_u >= theta'_u but H[g]_u !>= H[g']_u
    assert not np.all(u >= u2)


def test_worked_example_M_U_by_hand(gold):
    tuv = np.asarray(gold["theta_uv"], float)
    d = gold["derived_by_hand_not_printed"]
    for rule in ("M", "U"):
        u, v, _ = oracle.update_edge(rule, gold["theta_u"], gold["theta_v"], tuv)
        assert u.tolist() == d[rule]["theta_u"] and v.tolist() == d[rule]["theta_v"]
        u, v, _ = oracle.update_edge(rule, gold["theta_u_prime"], gold["theta_v_prime"], tuv)
        assert u.tolist() == d[rule + "_prime"]["theta_u"] and v.tolist() == d[rule + "_prime"]["theta_v"]


def _random_edge(rng, Lu, Lv):
    return rng.random(Lu), rng.random(Lv), rng.standard_normal((Lu, Lv))


@pytest.mark.parametrize("Lu,Lv", [(1, 1), (1, 5), (4, 1), (3, 3), (7, 5), (16, 9)])
def test_H_residual_rows_and_cols_are_zero(Lu, Lv):
    """Eq. (H) pushes cost until every row-min and column-min of the residual
    pairwise table is 0 (text after eq. (H)); hence min theta_uv = 0 (Def. 1)."""
    rng = np.random.default_rng(Lu * 100 + Lv)
    for _ in range(20):
        tu, tv, tuv = _random_edge(rng, Lu, Lv)
        _, _, r = oracle.update_edge("H", tu, tv, tuv)
        assert np.allclose(r.min(axis=1), 0.0, atol=1e-12)
        assert np.allclose(r.min(axis=0), 0.0, atol=1e-12)


@pytest.mark.parametrize("rule", ["U", "M", "H"])
def test_block_optimality_and_restricted_dual(rule):
    """Prop. 1 / Def. 1: after a BCA update some (s,t) minimizes theta_u,
    theta_v and theta_uv jointly, and the restricted dual D_uv reaches its
    maximum min_{s,t} g (eq. restricted-dual); energies g(s,t) are preserved."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        Lu, Lv = rng.integers(1, 9, size=2)
        tu, tv, tuv = _random_edge(rng, Lu, Lv)
        g = tuv + tu[:, None] + tv[None, :]
        u, v, r = oracle.update_edge(rule, tu, tv, tuv)
        assert np.allclose(r + u[:, None] + v[None, :], g, atol=1e-12)
        assert abs(r.min() + u.min() + v.min() - g.min()) < 1e-12
        su = np.flatnonzero(u <= u.min() + 1e-12)
        sv = np.flatnonzero(v <= v.min() + 1e-12)
        sub = r[np.ix_(su, sv)]
        assert sub.min() <= r.min() + 1e-12


def test_H_equals_four_minimization_form():
    """Eq. (H) as printed (M update, then two push steps) equals the
    three-minimization form the text after eq. (H) states."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        Lu, Lv = rng.integers(1, 9, size=2)
        tu, tv, tuv = _random_edge(rng, Lu, Lv)
        g = tuv + tu[:, None] + tv[None, :]
        hu = 0.5 * g.min(axis=1)
        hv = 0.5 * g.min(axis=0)
        hv = hv + (g - hv[None, :] - hu[:, None]).min(axis=0)
        hu = hu + (g - hv[None, :] - hu[:, None]).min(axis=1)
        u, v, _ = oracle.update_edge("H", tu, tv, tuv)
        assert np.allclose(u, hu, atol=1e-12) and np.allclose(v, hv, atol=1e-12)


def test_dominance_H_M_U():
    """Prop. 2: H >= M >= U componentwise, for any g."""
    rng = np.random.default_rng(11)
    for _ in range(100):
        Lu, Lv = rng.integers(1, 10, size=2)
        tu, tv, tuv = _random_edge(rng, Lu, Lv)
        res = {r: oracle.update_edge(r, tu, tv, tuv) for r in "UMH"}
        for hi, lo in (("H", "M"), ("M", "U")):
            assert np.all(res[hi][0] >= res[lo][0] - 1e-12)
            assert np.all(res[hi][1] >= res[lo][1] - 1e-12)


def test_M_and_U_are_monotonous():
    """Prop. 3: theta_u >= theta'_u and theta_v >= theta'_v imply
    gamma[g] >= gamma[g'] for gamma in {U, M}."""
    rng = np.random.default_rng(5)
    for _ in range(100):
        Lu, Lv = rng.integers(1, 8, size=2)
        tu, tv, tuv = _random_edge(rng, Lu, Lv)
        tu2 = tu - rng.random(Lu)
        tv2 = tv - rng.random(Lv)
        for rule in "UM":
            a = oracle.update_edge(rule, tu, tv, tuv)
            b = oracle.update_edge(rule, tu2, tv2, tuv)
            assert np.all(a[0] >= b[0] - 1e-12) and np.all(a[1] >= b[1] - 1e-12)


def test_argmin_records_reproduce_values():
    """The recorded argmins of the three minimizations attain the minima."""
    rng = np.random.default_rng(9)
    tu, tv, tuv = _random_edge(rng, 6, 4)
    g = tuv + tu[:, None] + tv[None, :]
    u, v, _, (t1, s2, t3) = oracle.update_edge("H", tu, tv, tuv, record=True)
    a = 0.5 * g[np.arange(6), t1]
    assert np.allclose(a, 0.5 * g.min(axis=1))
    assert np.allclose(v, g[s2, np.arange(4)] - a[s2])
    assert np.allclose(u, g[np.arange(6), t3] - v[t3])
