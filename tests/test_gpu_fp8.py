"""The FP8-dominant regime: structured cohorts (eight Balding-Nichols
subpopulations, F = 0.3) with a narrower kernel (gamma = 8/M), where most
off-diagonal factor tiles are small enough for E4M3 storage (the paper's FP8
precision heatmaps, Sec. V-C "Support for FP8" and "Precision Heatmaps").
Trailing-update blocks whose two factor tiles are both E4M3 run as
kind::f8f6f4 MMAs on the stored bytes.

Gates (the same as the uniform-genotype parity tests): Y_test within 1e-4 of
the FP64 oracle, relative residual <= 1e-5, the factor's backward error
||L L^T - (K + lambda I)||_2 <= 0.1 lambda, and E4M3 tiles at least a third
of the mosaic (most of it when the cohorts line up with the tiles).  The K-norm rule's map is checked against the rule evaluated on the
oracle's FP64 kernel tiles."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _structured(n, m, p, n_test, seed, fst=0.3):
    prob = inputs.structured_problem(n, m, p, n_test, seed=seed, populations=8, fst=fst)
    return {k: v.numpy() for k, v in prob.items()}


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("n,m,tile", [(4096, 2048, 256), (3000, 1500, 256), (6144, 2048, 512)])
def test_fp8_dominant_mosaic_matches_oracle(n, m, tile):
    prob = _structured(n, m, 3, 256, seed=90 + n)
    gamma, lam = 8.0 / m, 0.1
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"], method="lapack")
    with KRR(tile=tile, mode="mixed") as model:
        model.build_kernel(_to(prob["G"]), gamma)
        finfo = model.factor(lam)
        a, sinfo = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a)
        pmap = model.precision_map()
        k = model.kernel().astype(np.float64)
        l = model.factor_matrix().astype(np.float64)
    nt = -(-n // tile)
    noff = nt * (nt - 1) // 2
    assert finfo["tiles_fp32"] + finfo["tiles_fp16"] + finfo["tiles_e4m3"] == noff
    # cohorts of n / 8 rows do not line up with the tiles when n is ragged:
    # tiles that straddle two cohorts hold within-cohort entries and stay FP16
    assert finfo["tiles_e4m3"] >= noff // 3, finfo
    assert int((pmap[np.tril_indices(nt, -1)] == 3).sum()) == finfo["tiles_e4m3"]
    k = np.tril(k) + np.tril(k, -1).T
    e = l @ l.T - (k + lam * np.eye(n))
    assert np.linalg.norm(e, 2) <= 0.1 * lam
    yt = yt.cpu().numpy().astype(np.float64)
    a = a.cpu().numpy().astype(np.float64)
    err_yt = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
    err_a = np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)
    print(f"\nfp8 n={n} tile={tile}: e4m3 {finfo['tiles_e4m3']}/{noff} err_Yt={err_yt:.3e} err_A={err_a:.3e} "
          f"residual={sinfo['rel_residual']:.3e} iterations={sinfo['iterations']}")
    assert sinfo["converged"] in (1, 2), sinfo
    assert sinfo["rel_residual"] <= 1e-5, sinfo
    assert err_yt <= 1e-4, err_yt
    assert err_a <= 1e-3, err_a


def test_knorm_rule_map_matches_rule_on_oracle_kernel():
    """KRR_RULE_KNORM: tile (i, k) is E4M3 when 2^-4 ||K_ik||_F <= eps ||K||_F / NT,
    else FP16 when 2^-11 ||K_ik||_F <= eps ||K||_F / NT, else FP32.  The map is
    compared with the rule evaluated on the oracle's FP64 kernel (tiles whose
    norm lies within 1e-4 of a threshold are skipped: FP32 sums may round
    them either way).  Padding rows count as identity rows of K."""
    n, m, tile, eps = 3584, 1024, 256, 1e-3
    prob = _structured(n, m, 2, 64, seed=7, fst=0.2)
    gamma, lam = 10.0 / m, 0.1
    with KRR(tile=tile, mode="mixed", prec_rule="knorm", eps=eps) as model:
        model.build_kernel(_to(prob["G"]), gamma)
        finfo = model.factor(lam)
        a, sinfo = model.solve(_to(prob["Y"]))
        pmap = model.precision_map()
    kref = oracle.build_kernel(gamma, prob["G"], method="blas")
    nt = n // tile
    total = np.sqrt((kref ** 2).sum())
    thr = eps * total / nt
    checked = 0
    for i in range(nt):
        for k in range(i):
            w = np.linalg.norm(kref[i * tile:(i + 1) * tile, k * tile:(k + 1) * tile])
            ratios = (0.0625 * w / thr, 2.0 ** -11 * w / thr)
            if any(abs(r - 1.0) < 1e-4 for r in ratios):
                continue
            want = 3 if ratios[0] <= 1 else (2 if ratios[1] <= 1 else 1)
            assert pmap[i, k] == want, (i, k, pmap[i, k], want, ratios)
            checked += 1
    assert checked >= nt * (nt - 1) // 2 - 2
    assert finfo["tiles_e4m3"] > 0
    assert sinfo["converged"] in (1, 2) and sinfo["rel_residual"] <= 1e-5, sinfo
