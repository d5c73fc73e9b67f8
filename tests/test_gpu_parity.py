"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
* squared distances: bit-exact (integers);
* kernel entries: |K_gpu - K_ref| <= 4e-7 (FP32 storage + expf, a few ulp);
* mixed mode after refinement: ||Yt - Yt*||_F / ||Yt*||_F <= 1e-4 (the
  end-to-end accuracy target), relative residual <= 1e-5 (the floor of FP32
  storage of K and A is ~1e-6 at these sizes);
* plain FP32 mode (no refinement): ||Yt - Yt*|| / ||Yt*|| <= 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, KRRError, inputs
from paper_2409_01712_gb300 import krr as krrmod

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
MODES = ["fp32", "mixed"]


def _problem(n, m, p, n_test, seed):
    prob = inputs.problem(n, m, p, n_test, seed=seed)
    return {k: v.numpy() for k, v in prob.items()}


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,m,tile", [(700, 300, 256), (512, 128, 256), (1100, 1000, 512)])
def test_distances_bit_exact(mode, n, m, tile):
    prob = _problem(n, m, 1, 1, seed=11 + n)
    g = prob["G"]
    with KRR(tile=tile, mode=mode) as model:
        model.build_kernel(_to(g), 1.0 / m, keep_distances=True)
        d = model.distances().astype(np.int64)
        kgpu = model.kernel().astype(np.float64)
    dref = oracle.sqdist(g)
    nt = -(-n // tile)
    for i in range(nt):
        for j in range(i + 1):
            rs = slice(i * tile, min(n, (i + 1) * tile))
            cs = slice(j * tile, min(n, (j + 1) * tile))
            assert np.array_equal(d[rs, cs], dref[rs, cs]), (i, j)
            kref = oracle.gaussian_kernel(dref[rs, cs], 1.0 / m)
            assert np.max(np.abs(kgpu[rs, cs] - kref)) <= 4e-7, (i, j)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m", [4096, 16384])
def test_distance_extremes(mode, m):
    # all-0 vs all-2 rows: d = 4M and all-2 vs all-2: Gram entry 4M -- the
    # largest values the accumulator must hold exactly (M = 16384: 65536)
    g = np.zeros((300, m), np.int8)
    g[1::2] = 2
    g[7] = 1
    with KRR(tile=256, mode=mode) as model:
        model.build_kernel(_to(g), 1.0 / m, keep_distances=True)
        d = model.distances().astype(np.int64)
    dref = oracle.sqdist(g)
    tri = np.tril(np.ones((300, 300), bool))
    tri[:256, 256:] = False
    assert np.array_equal(d[tri], dref[tri])
    assert d[1, 0] == 4 * m
    assert d[3, 1] == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,m,p,tile", [(900, 256, 3, 256), (1536, 512, 1, 512), (2048, 512, 1, 1024)])
def test_fit_predict_matches_oracle(mode, n, m, p, tile):
    prob = _problem(n, m, p, 300, seed=5 + n)
    gamma, lam = 1.0 / m, 0.1
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"])
    with KRR(tile=tile, mode=mode) as model:
        model.build_kernel(_to(prob["G"]), gamma)
        finfo = model.factor(lam)
        a, sinfo = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a)
        pmap = model.precision_map()
    a = a.cpu().numpy().astype(np.float64)
    yt = yt.cpu().numpy().astype(np.float64)
    err_yt = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
    err_a = np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)
    nt = -(-n // tile)
    assert finfo["nt"] == nt
    assert pmap.shape == (nt, nt)
    print(f"\n{mode} n={n} tile={tile}: err_Yt={err_yt:.3e} err_A={err_a:.3e} residual={sinfo['rel_residual']:.3e}")
    if mode == "mixed":
        assert sinfo["converged"] in (1, 2), sinfo
        assert sinfo["rel_residual"] <= 1e-5, sinfo
        assert err_yt <= 1e-4, (err_yt, err_a, sinfo)
        # forward error in A: at most cond(K + lambda I) times the residual
        # (cond <= (0.5 n + lambda) / lambda, about 1e4 here); measured 2e-6 to
        # 3e-6 on these cases, stated bound 1e-4
        assert err_a <= 1e-4, (err_a, sinfo)
        assert finfo["tiles_fp32"] + finfo["tiles_fp16"] + finfo["tiles_e4m3"] == nt * (nt - 1) // 2
    else:
        assert err_yt <= 1e-3, (err_yt, err_a)
        assert np.all(pmap[np.tril_indices(nt, -1)] == 1)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("pinned", [False, True])
def test_host_buffers_and_multiple_rhs(mode, pinned):
    prob = _problem(600, 200, 4, 100, seed=77)
    gamma, lam = 1.0 / 200, 0.3
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"])
    with KRR(tile=256, mode=mode) as model:
        if pinned:  # page-locked host genotypes are read in place by the pack kernel
            model.build_kernel(torch.from_numpy(prob["G"]).pin_memory(), gamma)
        else:
            model.build_kernel(prob["G"], gamma)  # host numpy in (staged)
        model.factor(lam)
        a, _ = model.solve(prob["Y"])  # host in, host out
        assert isinstance(a, np.ndarray)
        yt = model.predict(prob["T"], a)
        # the factor is reused for a second phenotype set
        a2, _ = model.solve(prob["Y"][:, :2].copy())
    err = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
    assert err <= (1e-4 if mode == "mixed" else 1e-3)
    assert np.allclose(a2, a[:, :2], rtol=1e-4, atol=1e-4)


def test_closed_form_large_gamma():
    # distinct rows and a large gamma give K = I: A = Y / (1 + lambda)
    prob = _problem(512, 256, 2, 10, seed=3)
    lam = 0.25
    with KRR(tile=256, mode="mixed") as model:
        model.build_kernel(_to(prob["G"]), 50.0)
        model.factor(lam)
        a, info = model.solve(_to(prob["Y"]))
    assert np.allclose(a.cpu().numpy(), prob["Y"] / (1 + lam), rtol=1e-6, atol=1e-6)


def test_errors():
    prob = _problem(300, 64, 1, 10, seed=9)
    with KRR(tile=256, mode="mixed") as model:
        with pytest.raises(KRRError) as e:
            model.factor(0.1)
        assert e.value.status == krrmod.ESTATE
        with pytest.raises(KRRError) as e:
            model.build_kernel(_to(prob["G"]), -1.0)
        assert e.value.status == krrmod.EINVAL
        model.build_kernel(_to(prob["G"]), 1.0 / 64)
        with pytest.raises(KRRError) as e:
            model.solve(_to(prob["Y"]))
        assert e.value.status == krrmod.ESTATE
        # K - 1.5 I has negative eigenvalues (K_ii = 1): not positive definite
        with pytest.raises(KRRError) as e:
            model.factor(-1.5)
        assert e.value.status == krrmod.ENOTPD
        # the context stays usable afterwards
        model.factor(0.1)
        a, info = model.solve(_to(prob["Y"]))
        assert info["converged"]
    for bad_tile in (300, 768):  # a power of two in [256, 4096] only
        with pytest.raises(KRRError) as e:
            KRR(tile=bad_tile)
        assert e.value.status == krrmod.EINVAL


@pytest.mark.parametrize("mode", MODES)
def test_factor_backward_error(mode):
    """L L^T reconstructs K + lambda I: FP32 mode to FP32 rounding; mixed mode
    within the adaptive-precision budget (spectral error well below lambda,
    which keeps the refinement contracting)."""
    prob = _problem(1536, 512, 1, 10, seed=21)
    lam = 0.1
    with KRR(tile=256, mode=mode) as model:
        model.build_kernel(_to(prob["G"]), 1.0 / 512)
        model.factor(lam)
        k = model.kernel().astype(np.float64)
        l = model.factor_matrix().astype(np.float64)
        pmap = model.precision_map()
    k = np.tril(k) + np.tril(k, -1).T
    m = k + lam * np.eye(len(k))
    e = l @ l.T - m
    assert np.array_equal(l, np.tril(l))
    if mode == "fp32":
        assert np.linalg.norm(e) / np.linalg.norm(m) <= 1e-6
    else:
        assert np.linalg.norm(e, 2) <= 0.1 * lam
        # the mean component sits in tile column 0: it needs FP32; the rest FP16
        assert np.all(pmap[1:, 0] == 1), pmap
        assert np.all(pmap[np.tril_indices(len(pmap), -1)][len(pmap) - 1:] >= 1)


def test_fp64_diagonal_option():
    """The FP64 diagonal-tile Cholesky option gives the same answers."""
    prob = _problem(1100, 300, 2, 150, seed=51)
    gamma, lam = 1.0 / 300, 0.1
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"])
    with KRR(tile=256, mode="mixed", diag_fp64=True) as model:
        model.build_kernel(_to(prob["G"]), gamma)
        model.factor(lam)
        a, info = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a)
        pmap = model.precision_map()
    assert np.all(np.diag(pmap) == 0)  # diagonal tiles report FP64
    err = np.linalg.norm(yt.cpu().numpy() - yt_ref) / np.linalg.norm(yt_ref)
    assert err <= 1e-4, (err, info)


def test_empty_inputs_rejected():
    prob = _problem(300, 64, 2, 10, seed=9)
    with KRR(tile=256, mode="mixed") as model:
        with pytest.raises(KRRError) as e:
            model.build_kernel(_to(prob["G"][:0]), 1.0 / 64)  # no rows
        assert e.value.status == krrmod.EINVAL
        model.build_kernel(_to(prob["G"]), 1.0 / 64)
        model.factor(0.1)
        with pytest.raises(KRRError) as e:
            model.solve(_to(prob["Y"][:, :0]))  # no phenotypes
        assert e.value.status == krrmod.EINVAL
        a, _ = model.solve(_to(prob["Y"]))
        with pytest.raises(KRRError) as e:
            model.predict(_to(prob["T"][:0]), a)  # no held-out rows
        assert e.value.status == krrmod.EINVAL


@pytest.mark.parametrize("mode", MODES)
def test_single_row_closed_form(mode):
    # N = 1: K = [1], so A = Y / (1 + lambda) exactly; the other 255 rows of
    # the tile are padding (identity rows of K, zero right-hand side)
    g = np.zeros((1, 64), np.int8)
    g[0, ::3] = 2
    y = np.array([[2.0, -0.5]], np.float32)
    lam = 0.25
    with KRR(tile=256, mode=mode) as model:
        model.build_kernel(_to(g), 1.0 / 64)
        model.factor(lam)
        a, _ = model.solve(_to(y))
        yt = model.predict(_to(g), a)
    assert np.allclose(a.cpu().numpy(), y / (1 + lam), rtol=1e-6, atol=1e-7)
    # predicting the training row: K A = Y - lambda A
    assert np.allclose(yt.cpu().numpy(), y - lam * y / (1 + lam), rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n,m,p,tile", [(5000, 700, 2, 2048), (9000, 512, 2, 4096)])
def test_largest_tile_edges_match_oracle(n, m, p, tile):
    """The two largest tile edges the API accepts (2048, 4096: 32 and 64
    blocks of 64 in the diagonal step, 16 x 8 and 32 x 16 tensor-core blocks
    per tile), ragged N over three tiles, mixed mode with the lookahead,
    against the FP64 oracle (library Gram product and LAPACK factorisation)."""
    prob = _problem(n, m, p, 300, seed=11 + tile)
    gamma, lam = 1.0 / m, 0.1
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"], method="lapack")
    with KRR(tile=tile, mode="mixed") as model:
        model.build_kernel(_to(prob["G"]), gamma)
        finfo = model.factor(lam)
        a, sinfo = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a)
    a = a.cpu().numpy().astype(np.float64)
    yt = yt.cpu().numpy().astype(np.float64)
    err_yt = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
    err_a = np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)
    print(f"\nmixed n={n} tile={tile}: err_Yt={err_yt:.3e} err_A={err_a:.3e} residual={sinfo['rel_residual']:.3e}")
    assert finfo["nt"] == -(-n // tile)
    assert sinfo["converged"] in (1, 2), sinfo
    assert err_yt <= 1e-4, (err_yt, err_a, sinfo)
    assert err_a <= 1e-4, (err_a, sinfo)
