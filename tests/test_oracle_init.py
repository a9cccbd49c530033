"""Pins of the oracle's initialisation (Sec. 3.3, eq 23, Algorithm 1).

Eq (23) is a moment match of a skew-normal-type component: with delta the skewness
vector, the implied mean mu + sqrt(2/pi) delta and the implied variances
Sigma_aa + (1 - 2/pi) delta_a^2 reproduce the cluster's sample mean and sample
variances, the skewness takes the fraction (1 - alpha) of each variance, and
delta takes the sign of the third central moment.  These properties are checked
against numpy's moments of each cluster (not against the formula), and
Algorithm 1's selection against a brute-force maximum of the oracle's own
log-likelihood over the candidates.
"""
import math

import numpy as np
import pytest

from paper_1606_02054_gb300 import synth


@pytest.fixture(scope="module")
def data():
    w = synth.make_workload("flow_p4", n=600, with_init=False)
    return w


def _skew_vector(D, q, p):
    if q == 1:
        return D[:, 0].copy()
    d = np.zeros(p)
    for i in range(min(p, q)):
        d[i] = D[i, i]
    return d


def _skewed_clusters(p, g=3, n=3000, seed=0):
    """Clusters of independent gamma-skewed coordinates (nearly diagonal S, so
    Sigma^(0) stays positive definite for every alpha); labels are the clusters."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, g, n).astype(np.int32)
    shape = rng.uniform(1.5, 4.0, size=(g, p))
    sign = rng.choice([-1.0, 1.0], size=(g, p))
    y = sign[lab] * rng.gamma(shape[lab], 1.0) + 6.0 * lab[:, None]
    return y, lab


@pytest.mark.parametrize("p,q", [(4, 4), (4, 1), (4, 2), (6, 3), (2, 5)])
@pytest.mark.parametrize("alpha", [0.3, 0.6, 0.9])
def test_moment_start_matches_cluster_moments(oracle, p, q, alpha):
    y, lab = _skewed_clusters(p)
    n = y.shape[0]
    g = 3
    P, rc = oracle.moment_start(y, lab, g, q, alpha, nu0=10.0)
    assert rc == 0
    for h in range(g):
        yc = y[lab == h]
        ybar = yc.mean(0)
        S = np.cov(yc, rowvar=False)
        m3 = ((yc - ybar) ** 3).mean(0)
        d = _skew_vector(P["Delta"][h], q, p)
        skewed = np.ones(p, bool) if (q == 1 or q >= p) else (np.arange(p) < q)
        # implied mean = sample mean
        np.testing.assert_allclose(P["mu"][h] + math.sqrt(2 / math.pi) * d, ybar, rtol=0, atol=1e-12)
        # implied variances = sample variances; covariances untouched
        implied = np.diag(P["Sigma"][h]) + (1 - 2 / math.pi) * d ** 2
        np.testing.assert_allclose(implied, np.diag(S), rtol=1e-12)
        off = ~np.eye(p, dtype=bool)
        np.testing.assert_allclose(P["Sigma"][h][off], S[off], rtol=1e-12, atol=1e-14)
        # the skewness carries the fraction (1 - alpha) of each skewed variance
        np.testing.assert_allclose((1 - 2 / math.pi) * d[skewed] ** 2, (1 - alpha) * np.diag(S)[skewed],
                                   rtol=1e-12)
        assert np.all(d[~skewed] == 0)
        # sign of the third central moment
        assert np.all(np.sign(d[skewed]) == np.where(m3[skewed] >= 0, 1, -1))
        assert P["nu"][h] == 10.0
        assert abs(P["pi"][h] - len(yc) / n) < 1e-15


def test_moment_start_rejects_tiny_and_non_pd_clusters(oracle, data):
    y = data["y"]
    lab = np.zeros(len(y), dtype=np.int32)
    lab[0] = 1  # a cluster of one point has no covariance
    _, rc = oracle.moment_start(y, lab, 2, 4, 0.9)
    assert rc == 2
    # alpha -> 0 removes almost all of each variance from Sigma: not PD for correlated data
    lab = synth.kmeans(np.random.default_rng(3), y, 2)
    _, rc = oracle.moment_start(y, lab, 2, 4, 1e-9)
    assert rc != 0


def test_random_partition(oracle):
    a = oracle.random_partition(100000, 5, 1234, 0)
    b = oracle.random_partition(100000, 5, 1234, 0)
    c = oracle.random_partition(100000, 5, 1234, 1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() == 0 and a.max() == 4
    counts = np.bincount(a, minlength=5)
    chi2 = ((counts - 20000.0) ** 2 / 20000.0).sum()
    assert chi2 < 30.0  # 4 dof: far beyond the 1e-5 tail would be 28.5
    # first label from the published SplitMix64 output for key seed ^ (1 << 40) ^ 1
    u = oracle.splitmix64_u01(1234 ^ (1 << 40) ^ 1)
    assert a[0] == min(int(u * 5), 4)


def test_init_selects_the_best_candidate(oracle, data):
    y = data["y"]
    g, q = 3, 4
    spec = oracle.qmc(**data["qmc"])
    alphas = (0.5, 0.7, 0.9)
    best, ll, ib = oracle.init(y, g, q, spec, nstarts=3, seed=11, alphas=alphas)
    brute = np.full((3, len(alphas)), -np.inf)
    for s in range(3):
        lab = oracle.random_partition(len(y), g, 11, s)
        for a, al in enumerate(alphas):
            P, rc = oracle.moment_start(y, lab, g, q, al)
            if rc == 0:
                brute[s, a] = oracle.loglik(y, P, spec)
    np.testing.assert_array_equal(ll, brute)
    assert ib == int(np.argmax(brute))  # first maximum, start-major order
    s, a = divmod(ib, len(alphas))
    P, _ = oracle.moment_start(y, oracle.random_partition(len(y), g, 11, s), g, q, alphas[a])
    for k in P:
        np.testing.assert_array_equal(best[k], P[k])


def test_init_with_given_labels_prefers_the_true_partition(oracle):
    """Two well-separated components: the generating labels beat random partitions."""
    w = synth.make_workload("two_comp_p2", n=800, with_init=False)
    y, z = w["y"], w["z"]
    spec = oracle.qmc(**w["qmc"])
    rand = np.stack([oracle.random_partition(len(y), 2, 5, s) for s in range(2)])
    labels = np.concatenate([rand, z[None].astype(np.int32)])
    _, ll, ib = oracle.init(y, 2, 2, spec, nstarts=3, labels=labels)
    assert ib // ll.shape[1] == 2
    assert np.max(ll[2]) > np.max(ll[:2]) + 50.0


# ---- k-means partitions (Sec. 3.3: the initial clusterings of Algorithm 1) ----------
def _kmeans_start_indices(oracle, n, g, seed, start):
    """The starting centres' observation indices, from the stated SplitMix64 rule."""
    idx = []
    for h in range(g):
        a = 0
        while True:
            key = seed ^ ((start + 1) << 40) ^ (1 << 36) ^ (h + 1 + g * a)
            j = min(int(oracle.splitmix64_u01(key) * n), n - 1)
            if j not in idx:
                idx.append(j)
                break
            a += 1
    return idx


@pytest.mark.parametrize("name,n,g_over", [("flow_p4", 3000, None), ("wide_p16", 2000, None), ("two_comp_p2", 1000, 5)])
def test_kmeans_matches_sklearn_lloyd(oracle, name, n, g_over):
    """Pin: from the same starting centres, scikit-learn's Lloyd iteration (tol 0, one
    initialisation) reaches the same labels and centres."""
    sk = pytest.importorskip("sklearn.cluster")
    w = synth.make_workload(name, n=n, with_init=False)
    y, g = w["y"], g_over or w["g"]
    seed = 77
    labels, iters, cen = oracle.kmeans(y, g, nstarts=2, seed=seed, max_iter=300)
    for s in range(2):
        idx = _kmeans_start_indices(oracle, n, g, seed, s)
        km = sk.KMeans(n_clusters=g, init=y[idx], n_init=1, max_iter=300, tol=0.0, algorithm="lloyd").fit(y)
        assert iters[s] < 300  # converged: an assignment that changed nothing
        assert np.array_equal(labels[s], km.labels_)
        np.testing.assert_allclose(cen[s], km.cluster_centers_, rtol=1e-10, atol=1e-12)


def test_kmeans_fixed_point_and_first_tie(oracle):
    """At convergence every label is the nearest centre's and every centre is its
    cluster's mean; an observation equidistant from two centres takes the first."""
    w = synth.make_workload("flow_p4", n=1500, with_init=False)
    labels, iters, cen = oracle.kmeans(w["y"], 4, nstarts=1, seed=3, max_iter=500)
    d = ((w["y"][:, None, :] - cen[0][None]) ** 2).sum(-1)
    assert np.array_equal(labels[0], d.argmin(1))
    for h in range(4):
        np.testing.assert_allclose(cen[0][h], w["y"][labels[0] == h].mean(0), rtol=1e-12, atol=1e-12)
    # ties: two identical observations as the only points, g = 2 -> both centres equal
    y = np.array([[1.0, 2.0], [1.0, 2.0], [1.0, 2.0]])
    lab, _, _ = oracle.kmeans(y, 2, nstarts=1, seed=5, max_iter=10)
    assert np.all(lab == 0)
    with pytest.raises(ValueError):
        oracle.kmeans(y[:1], 2)
