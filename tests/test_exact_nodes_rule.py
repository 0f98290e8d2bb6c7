"""The point count of n_quad = EXACT_NODES (qts_exact_nodes, host logic) against
Thm 2 and the mathematics it rests on: an order-s integrand on a path with d
unique features has degree d - s, and n Gauss-Legendre points integrate degree
2n - 1 exactly but not degree 2n.  Pinned by the paper's worked example, by
monomials integrated with the oracle's own nodes, and by an oracle path whose
integrand has full degree, where one point fewer than the rule is inexact."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qts():
    from paper_2605_04497_gb300 import build as b

    b.build()
    import paper_2605_04497_gb300 as q

    return q


def test_paper_worked_example(qts):
    spec = json.load(open(os.path.join(HERE, "golden", "thm2_points.json")))
    for c in spec["cases"]:
        assert qts.exact_nodes(c["width"], c["order"]) == c["points"], c


def test_monomials_exact_and_minimal(qts):
    """n = exact_nodes(w, s) integrates t^(w-s) exactly with the oracle's
    nodes; n - 1 points cannot, because then w - s >= 2(n-1).  The error of
    n' points on t^(2n') is (n'!)^4 / ((2n'+1) ((2n')!)^2), 3.5e-10 at n' = 8
    and below rounding from n' = 14, so minimality is checked up to n' = 8."""
    for order in (1, 2, 3, 5):
        for width in range(1, 65):
            n = qts.exact_nodes(width, order)
            deg = max(width - order, 0)
            assert 1 <= n <= 32
            t, w = oracle.gl_nodes(n)
            assert abs(np.sum(w * t ** deg) - 1.0 / (deg + 1)) <= 1e-14, (width, order)
            if 1 < n <= 9:
                t, w = oracle.gl_nodes(n - 1)
                assert abs(np.sum(w * t ** deg) - 1.0 / (deg + 1)) > 1e-11, (width, order)


def test_out_of_range_arguments(qts):
    assert qts.exact_nodes(0, 1) == 0
    assert qts.exact_nodes(65, 1) == 0
    assert qts.exact_nodes(8, 0) == 0
    assert qts.exact_nodes(3, 5) == 1  # more interacting features than the path has


def _skewed_chain(d, F):
    """One tree: node k splits on feature k at 0 and continues to the right
    (edge weight 0.05) with a leaf on the left (0.95); the last split has two
    leaves.  A sample with every x_k > 0 reaches the deepest right leaf, whose
    path has o_j = 1 and z_j = 0.05 for all d features, so a_j(t) = 0.05 +
    0.95 t and its integrands have their full degree."""
    n = 2 * d + 1
    left = np.full(n, -1, np.int32)
    right = np.full(n, -1, np.int32)
    feature = np.zeros(n, np.int32)
    z = np.ones(n, np.float32)
    val = np.zeros(n, np.float32)
    for k in range(d):
        nxt = k + 1 if k + 1 < d else d
        left[k], right[k] = d + 1 + k, nxt
        feature[k] = k
        z[d + 1 + k], z[nxt] = 0.95, 0.05
    rng = np.random.default_rng(d)
    for v in range(n):
        if left[v] < 0:
            val[v] = rng.normal()
    return synth.Ensemble([0, n], left, right, feature, np.zeros(n, np.float32), np.ones(n, np.uint8),
                          z, val, np.ones(n), F)


@pytest.mark.parametrize("d", [4, 7, 10, 13])
def test_full_degree_path(qts, d):
    ens = _skewed_chain(d, d)
    X = np.ones((1, d), np.float32)
    ref = oracle.shap_exact(ens, X)
    n = qts.exact_nodes(d, 1)
    scale = np.abs(ref).max()
    assert np.abs(oracle.shap_quad(ens, X, n) - ref).max() <= 1e-13 * scale
    assert np.abs(oracle.shap_quad(ens, X, n - 1) - ref).max() > 1e-8 * scale


@pytest.mark.parametrize("d", [5, 7, 9])
def test_pairwise_diagonal_needs_the_first_order_count(qts, d):
    """On a full-degree path of odd width d, ceil((d - 1) / 2) points make the
    pair terms exact (Algorithm 1 with s = 2 against the exact expansion) but
    not the first-order values the interaction matrix's diagonal holds, which
    need ceil(d / 2): the pairwise call's rule is the first-order count."""
    ens = _skewed_chain(d, d)
    x = np.ones((1, d), np.float32)
    sii, phi = oracle.sii_exact(ens, x)
    n2, n1 = qts.exact_nodes(d, 2), qts.exact_nodes(d, 1)
    assert n1 == n2 + 1
    scale = np.abs(phi).max()
    assert np.abs(oracle.alg1(ens, x, 2, n2) - sii[0]).max() <= 1e-13 * scale
    assert np.abs(oracle.shap_quad(ens, x, n2) - phi).max() > 1e-8 * scale
    assert np.abs(oracle.shap_quad(ens, x, n1) - phi).max() <= 1e-13 * scale
