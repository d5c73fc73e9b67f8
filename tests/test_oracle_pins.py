"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (the paper's worked example, brute force on tiny inputs,
closed forms, invariants, a library routine on a special case, finite
differences).  CPU only."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import inputs


def _rand_geno(n, m, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.05, 0.5, m)
    return ((rng.random((n, m)) < p).astype(np.int8) + (rng.random((n, m)) < p)).astype(np.int8)


def _golden(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "worked_example_3x2.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append([int(v) for v in vals])
    return {k: np.array(v, dtype=np.int64) for k, v in rows.items()}


# ---------------------------------------------------------------- distances

def test_worked_example_3x2(golden_dir):
    """Sec. IV-B worked example: 3 patients x 2 markers, hand-computed."""
    gold = _golden(golden_dir)
    patients = gold["G"].T.astype(np.int8)  # rows = patients a, b, c
    assert np.array_equal(oracle.sqdist(patients), gold["DT"])
    assert np.array_equal(oracle.sqdist(patients, method="gram"), gold["DT"])
    # the identity the example walks through, term by term, on the golden numbers
    assert np.array_equal(gold["D"] + gold["D"].T - 2 * gold["GTG"], gold["DT"])


def test_bruteforce_equals_gram_identity():
    for seed, (n1, n2, m) in enumerate([(1, 1, 1), (7, 5, 3), (33, 64, 300), (64, 17, 129)]):
        a = _rand_geno(n1, m, seed)
        b = _rand_geno(n2, m, seed + 100)
        d1 = oracle.sqdist(a, b)
        d2 = oracle.sqdist(a, b, method="gram")
        assert np.array_equal(d1, d2)


def test_distance_small_cases_by_hand():
    # one SNP differing by 1, by 2; nothing differing
    a = np.array([[0, 1, 2, 1]], dtype=np.int8)
    b = np.array([[0, 2, 2, 1], [2, 1, 0, 1], [0, 1, 2, 1]], dtype=np.int8)
    assert oracle.sqdist(a, b).tolist() == [[1, 8, 0]]


def test_distance_extremes_and_symmetry():
    m = 300
    z = np.zeros((1, m), np.int8)
    two = np.full((1, m), 2, np.int8)
    assert oracle.sqdist(z, two)[0, 0] == 4 * m  # max-value case
    g = _rand_geno(40, m, 3)
    d = oracle.sqdist(g)
    assert np.array_equal(d, d.T)
    assert np.all(np.diag(d) == 0)
    g[5] = g[9]
    assert oracle.sqdist(g)[5, 9] == 0


# ---------------------------------------------------------------- kernel

def test_gaussian_kernel_values():
    d = np.array([[0, 1, 3], [7, 100, 4]], dtype=np.int64)
    k = oracle.gaussian_kernel(d, 0.25)
    expect = [[1.0, math.exp(-0.25), math.exp(-0.75)], [math.exp(-1.75), math.exp(-25.0), math.exp(-1.0)]]
    assert np.allclose(k, expect, rtol=1e-15, atol=0)


def test_kernel_invariants_and_pd():
    g = _rand_geno(48, 64, 4)
    k = oracle.build_kernel(1 / 64, g)
    assert np.allclose(k, k.T, rtol=0, atol=0)
    assert np.all(np.diag(k) == 1.0)
    assert np.all((k > 0) & (k <= 1))
    # distinct rows -> Gaussian kernel is positive definite: Cholesky with lambda = 0
    assert len({r.tobytes() for r in g}) == len(g)
    l = oracle.cholesky(k)
    assert np.all(np.diag(l) > 0)
    # identical rows -> d = 0, K = 1, K singular: with rows 0 and 2 equal the
    # third pivot is exactly 1 - 1 - 0 = 0 and the factorisation must fail
    g2 = g[:3].copy()
    g2[2] = g2[0]
    k2 = oracle.build_kernel(1 / 64, g2)
    assert k2[2, 0] == 1.0
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky(k2)
    assert e.value.column == 2


# ---------------------------------------------------------------- factor

def test_cholesky_min_matrix_closed_form():
    # A_ij = min(i, j) (1-based) has the all-ones lower triangle as its factor
    n = 9
    i = np.arange(1, n + 1)
    a = np.minimum.outer(i, i).astype(np.float64)
    l = oracle.cholesky(a)
    assert np.array_equal(l, np.tril(np.ones((n, n))))


def test_cholesky_reconstruction_and_library():
    rng = np.random.default_rng(5)
    for n in (1, 2, 17, 128):
        x = rng.standard_normal((n, n))
        a = x @ x.T + n * np.eye(n)
        l = oracle.cholesky(a)
        assert np.array_equal(l, np.tril(l))
        err = np.linalg.norm(l @ l.T - a) / np.linalg.norm(a)
        assert err <= 10 * n * np.finfo(np.float64).eps
        assert np.allclose(l, np.linalg.cholesky(a), rtol=1e-12, atol=1e-12)


def test_cholesky_reports_first_bad_pivot():
    a = np.diag([4.0, 1.0, -1.0, 2.0])
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.cholesky(a)
    assert e.value.column == 2


# ---------------------------------------------------------------- solve

def test_substitution_on_known_triangle():
    l = np.array([[2.0, 0, 0], [1.0, 3.0, 0], [-1.0, 2.0, 4.0]])
    x = np.array([[1.0, -2.0], [0.5, 3.0], [2.0, 1.0]])
    y = l @ x
    assert np.allclose(oracle.forward_subst(l, y), x, rtol=1e-15, atol=1e-15)
    assert np.allclose(oracle.backward_subst(l, l.T @ x), x, rtol=1e-15, atol=1e-15)


def test_solve_gamma_zero_sherman_morrison():
    # gamma = 0: K = 1 1^T, A = (Y - 1 (1^T Y)/(lambda + N)) / lambda
    g = _rand_geno(50, 20, 6)
    y = np.random.default_rng(6).standard_normal((50, 3))
    lam = 0.37
    k = oracle.build_kernel(0.0, g)
    assert np.all(k == 1.0)
    a = oracle.associate(lam, k, y)
    expect = (y - np.ones((50, 1)) * y.sum(0, keepdims=True) / (lam + 50)) / lam
    assert np.allclose(a, expect, rtol=1e-10, atol=1e-12)


def test_solve_large_gamma_identity_kernel():
    g = _rand_geno(40, 30, 7)
    assert len({r.tobytes() for r in g}) == len(g)
    y = np.random.default_rng(7).standard_normal((40, 2))
    lam = 0.1
    k = oracle.build_kernel(1000.0, g)  # exp(-1000 d) underflows to 0 for d >= 1
    assert np.array_equal(k, np.eye(40))
    assert np.allclose(oracle.associate(lam, k, y), y / (1 + lam), rtol=1e-15, atol=0)


def test_solve_lambda_to_infinity():
    g = _rand_geno(60, 40, 8)
    y = np.random.default_rng(8).standard_normal((60, 2))
    k = oracle.build_kernel(1 / 40, g)
    knorm = np.linalg.norm(k, 2)
    for lam in (1e3, 1e6):
        a = oracle.associate(lam, k, y)
        assert np.linalg.norm(lam * a - y) / np.linalg.norm(y) <= knorm / lam


def test_solve_matches_library_solve():
    g = _rand_geno(64, 32, 9)
    y = np.random.default_rng(9).standard_normal((64, 4))
    k = oracle.build_kernel(1 / 32, g)
    a = oracle.associate(0.1, k, y)
    assert np.allclose(a, np.linalg.solve(k + 0.1 * np.eye(64), y), rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------- predict

def test_predict_identity_on_training_rows():
    # predicting the training rows gives K A = Y - lambda A
    g = _rand_geno(70, 50, 10)
    y = np.random.default_rng(10).standard_normal((70, 3))
    lam, gamma = 0.2, 1 / 50
    _, a, pr = oracle.krr(gamma, lam, g, y, g)
    assert np.allclose(pr, y - lam * a, rtol=1e-9, atol=1e-10)


def test_predict_matmul_by_hand():
    a = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    b = np.array([[1.0, -1.0, 0.5], [2.0, 0.0, 1.0]])
    assert np.array_equal(oracle.matmul(a, b), [[5.0, -1.0, 2.5], [11.0, -3.0, 5.5], [17.0, -5.0, 8.5]])


def test_kernel_rows_match_full_build():
    g = _rand_geno(30, 25, 11)
    t = _rand_geno(12, 25, 12)
    rows = np.array([0, 5, 11])
    assert np.allclose(oracle.kernel_rows(0.05, t, rows, g), oracle.build_kernel(0.05, t, g)[rows],
                       rtol=0, atol=0)


# ---------------------------------------------------------------- gradient

def test_gradient_matches_central_differences():
    g = _rand_geno(80, 64, 13)
    t = _rand_geno(24, 64, 14)
    rng = np.random.default_rng(13)
    y = rng.standard_normal((80, 2))
    yt = rng.standard_normal((24, 2))
    gamma, lam = 1 / 64, 0.1
    loss, dlg, dll = oracle.hyper_gradient(gamma, lam, g, y, t, yt)
    assert loss == pytest.approx(oracle.held_out_loss(gamma, lam, g, y, t, yt), rel=1e-12)
    h = 1e-3
    f = lambda lg, ll: oracle.held_out_loss(math.exp(lg), math.exp(ll), g, y, t, yt)
    lg0, ll0 = math.log(gamma), math.log(lam)
    fd_g = (f(lg0 + h, ll0) - f(lg0 - h, ll0)) / (2 * h)
    fd_l = (f(lg0, ll0 + h) - f(lg0, ll0 - h)) / (2 * h)
    assert dlg == pytest.approx(fd_g, rel=1e-5, abs=1e-12)
    assert dll == pytest.approx(fd_l, rel=1e-5, abs=1e-12)


def test_gradient_identity_kernel_closed_form():
    # K = I, K_t selects training rows: Yhat = Y_sel / (1 + lambda)
    g = _rand_geno(30, 40, 15)
    sel = np.array([2, 7, 19, 21])
    t = g[sel]
    rng = np.random.default_rng(15)
    y = rng.standard_normal((30, 2))
    yt = rng.standard_normal((4, 2))
    lam = 0.3
    loss, dlg, dll = oracle.hyper_gradient(1000.0, lam, g, y, t, yt)
    r = y[sel] / (1 + lam) - yt
    assert loss == pytest.approx((r * r).sum() / r.size, rel=1e-14)
    dl_dlam = (2 * r * (-y[sel] / (1 + lam) ** 2)).sum() / r.size
    assert dll == pytest.approx(lam * dl_dlam, rel=1e-12)
    assert dlg == 0.0


# ---------------------------------------------------------------- inputs recipe

def test_input_generator_recipe():
    prob = inputs.problem(200, 300, 3, 50, seed=1)
    g = prob["G"]
    assert g.dtype == torch.int8 and g.shape == (200, 300)
    assert set(torch.unique(g).tolist()) <= {0, 1, 2}
    p = inputs.allele_freqs(300, 1)
    assert float(p.min()) >= 0.05 and float(p.max()) <= 0.5
    assert prob["Y"].shape == (200, 3) and prob["Yt"].shape == (50, 3)
    assert prob["T"].shape == (50, 300)
    # deterministic for a fixed seed
    again = inputs.problem(200, 300, 3, 50, seed=1)
    assert torch.equal(again["G"], g) and torch.equal(again["Y"], prob["Y"])
    # mean genotype matches 2 p_j on a larger draw
    big = inputs.genotypes(4000, 64, seed=2).double()
    assert torch.allclose(big.mean(0), 2 * inputs.allele_freqs(64, 2), atol=0.08)


# ---------------------------------------------------------------- library-primitive methods

def test_blas_distances_equal_bruteforce():
    """The float64 Gram product gives the same integers as the term-by-term sum,
    including the largest value (all-0 against all-2 rows: 4 m)."""
    for seed, (n1, n2, m) in enumerate([(1, 1, 1), (7, 5, 3), (33, 64, 300), (64, 17, 129)]):
        a = _rand_geno(n1, m, seed + 200)
        b = _rand_geno(n2, m, seed + 300)
        assert np.array_equal(oracle.sqdist(a, b, method="blas"), oracle.sqdist(a, b))
        assert np.array_equal(oracle.sqdist(a, method="blas"), oracle.sqdist(a))
    m = 20000
    g = np.zeros((3, m), np.int8)
    g[1] = 2
    g[2, ::2] = 1
    d = oracle.sqdist(g, method="blas")
    assert d[1, 0] == 4 * m and d[0, 1] == 4 * m
    assert np.array_equal(d, oracle.sqdist(g))


def test_lapack_factor_and_solves_equal_plain_loops():
    rng = np.random.default_rng(31)
    for n in (1, 17, 200):
        x = rng.standard_normal((n, n))
        a = x @ x.T + n * np.eye(n)
        l0 = oracle.cholesky(a)
        l1 = oracle.cholesky(a, method="lapack")
        assert np.allclose(l1, l0, rtol=1e-12, atol=1e-12)
        y = rng.standard_normal((n, 3))
        z0 = oracle.forward_subst(l0, y)
        z1 = oracle.forward_subst(l0, y, method="lapack")
        assert np.allclose(z1, z0, rtol=1e-11, atol=1e-12)
        assert np.allclose(oracle.backward_subst(l0, z0, method="lapack"), oracle.backward_subst(l0, z0),
                           rtol=1e-11, atol=1e-12)
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.cholesky(np.diag([4.0, 1.0, -1.0, 2.0]), method="lapack")


def test_lapack_krr_and_gradient_equal_plain():
    g = _rand_geno(150, 90, 33)
    t = _rand_geno(40, 90, 34)
    rng = np.random.default_rng(33)
    y = rng.standard_normal((150, 3))
    yt = rng.standard_normal((40, 3))
    gamma, lam = 1 / 90, 0.1
    k0, a0, p0 = oracle.krr(gamma, lam, g, y, t)
    k1, a1, p1 = oracle.krr(gamma, lam, g, y, t, method="lapack")
    assert np.array_equal(k0, k1)
    assert np.allclose(a1, a0, rtol=1e-9, atol=1e-10)
    assert np.allclose(p1, p0, rtol=1e-9, atol=1e-10)
    r0 = oracle.hyper_gradient(gamma, lam, g, y, t, yt)
    r1 = oracle.hyper_gradient(gamma, lam, g, y, t, yt, method="lapack")
    assert np.allclose(r1, r0, rtol=1e-8, atol=1e-13)


# ---------------------------------------------------------------- IBS kernel (Alg. 5, second branch)

def test_ibs_hand_example_and_extremes():
    # loci: (0 vs 2) share 0 alleles, (1 vs 1) share 2, (2 vs 1) share 1 -> 3 of 6 alleles
    a = np.array([[0, 1, 2]], np.int8)
    b = np.array([[2, 1, 1], [0, 1, 2]], np.int8)
    assert oracle.ibs_count(a, b).tolist() == [[3, 6]]
    assert np.allclose(oracle.ibs_kernel(a, b), [[1.0, 2.0]], rtol=0, atol=0)
    m = 77
    z = np.zeros((1, m), np.int8)
    two = np.full((1, m), 2, np.int8)
    assert oracle.ibs_count(z, two)[0, 0] == 0
    g = _rand_geno(30, m, 41)
    k = oracle.ibs_kernel(g)
    assert np.array_equal(k, k.T) and np.all(np.diag(k) == 2.0)
    assert np.all((k >= 0) & (k <= 2))


def test_ibs_matches_allele_sharing_table_by_loops():
    # the definition spelled out allele by allele on tiny inputs: a genotype
    # is a pair of alleles (minor allele first), and the shared count is the
    # size of the multiset intersection
    def alleles(v):
        return [1] * int(v) + [0] * (2 - int(v))

    def shared(u, v):
        x, y = alleles(u), alleles(v)
        return sum(min(x.count(t), y.count(t)) for t in (0, 1))

    g1 = _rand_geno(6, 13, 42)
    g2 = _rand_geno(5, 13, 43)
    want = np.array([[sum(shared(g1[i, k], g2[j, k]) for k in range(13)) for j in range(5)] for i in range(6)])
    assert np.array_equal(oracle.ibs_count(g1, g2), want)
    assert np.array_equal(oracle.ibs_count(g1, g2, method="blas"), want)
    big1, big2 = _rand_geno(40, 500, 44), _rand_geno(33, 500, 45)
    assert np.array_equal(oracle.ibs_count(big1, big2, method="blas"), oracle.ibs_count(big1, big2))


def test_ibs_kernel_positive_semidefinite_and_solve():
    # each locus contributes E W E^T with the sharing table W positive
    # definite, so K is positive semidefinite and K + lambda I factorises
    g = _rand_geno(60, 40, 46)
    k = oracle.ibs_kernel(g)
    assert np.min(np.linalg.eigvalsh(k)) >= -1e-10
    y = np.random.default_rng(46).standard_normal((60, 2))
    _, w, pr = oracle.krr(0.0, 0.3, g, y, g, kernel="ibs")
    assert np.allclose(pr, y - 0.3 * w, rtol=1e-9, atol=1e-10)


# ---------------------------------------------------------------- confounders (Sec. IV-B, distance section)

def test_confounder_distances_by_hand_and_identity():
    c1 = np.array([[1.0, -2.0, 0.5]])
    c2 = np.array([[0.0, 1.0, 0.5], [1.0, -2.0, 0.5]])
    assert np.allclose(oracle.conf_sqdist(c1, c2), [[1.0 + 9.0, 0.0]], rtol=0, atol=0)
    rng = np.random.default_rng(51)
    a, b = rng.standard_normal((20, 7)), rng.standard_normal((11, 7))
    gram = (a * a).sum(1)[:, None] + (b * b).sum(1)[None, :] - 2 * a @ b.T
    assert np.allclose(oracle.conf_sqdist(a, b), gram, rtol=1e-12, atol=1e-12)
    # a common shift of every row leaves the distances unchanged
    assert np.allclose(oracle.conf_sqdist(a + 3.0, b + 3.0), oracle.conf_sqdist(a, b), rtol=1e-12, atol=1e-12)


def test_kernel_with_confounders_adds_before_exponential():
    g = _rand_geno(25, 30, 52)
    c = np.random.default_rng(52).standard_normal((25, 4))
    gamma = 1 / 30
    k0 = oracle.build_kernel(gamma, g)
    kc = oracle.build_kernel(gamma, g, c1=c)
    # exp(-gamma (d + dc)) = exp(-gamma d) exp(-gamma dc)
    assert np.allclose(kc, k0 * np.exp(-gamma * oracle.conf_sqdist(c)), rtol=1e-13, atol=0)
    assert np.allclose(oracle.build_kernel(gamma, g, c1=np.zeros((25, 4))), k0, rtol=4e-16, atol=0)
    assert np.all(np.diag(kc) == 1.0)


# ---------------------------------------------------------------- ridge regression (Sec. IV-A, Eq. 2)

def test_ridge_gram_is_integer_sum_and_optimality():
    g = _rand_geno(70, 40, 61)
    c = np.random.default_rng(61).standard_normal((70, 3))
    y = np.random.default_rng(62).standard_normal((70, 2))
    lam = 0.7
    gram, rhs, beta = oracle.ridge(lam, g, y, c)
    gi = g.astype(np.int64)
    # genotype block: exact integer sums over the patients
    assert np.array_equal(gram[:40, :40], np.einsum("pi,pj->ij", gi, gi).astype(np.float64))
    x = np.concatenate([g.astype(np.float64), c], axis=1)
    # first-order optimality of the ridge objective: X^T (Y - X beta) = lambda beta
    assert np.allclose(x.T @ (y - x @ beta), lam * beta, rtol=1e-9, atol=1e-9)
    assert np.allclose(beta, np.linalg.solve(x.T @ x + lam * np.eye(43), x.T @ y), rtol=1e-9, atol=1e-10)
    # lambda -> infinity: lambda beta -> X^T Y
    big = 1e9
    _, _, b2 = oracle.ridge(big, g, y, c)
    assert np.allclose(big * b2, rhs, rtol=1e-4, atol=1e-4)
    # library path = plain loops
    _, _, b3 = oracle.ridge(lam, g, y, c, method="lapack")
    assert np.allclose(b3, beta, rtol=1e-9, atol=1e-11)
    t = _rand_geno(9, 40, 63)
    ct = np.random.default_rng(63).standard_normal((9, 3))
    assert np.allclose(oracle.ridge_predict(t, beta, ct), np.concatenate([t, ct], axis=1) @ beta, rtol=1e-12,
                       atol=1e-12)
