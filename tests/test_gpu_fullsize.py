"""Parity at the benchmarked size, in the launch configuration the benchmark
times: N = 131072 training rows, M = 16384 SNPs, P = 20 phenotypes, 4096
held-out rows, tile 1024, mixed mode, gamma = 1/M, lambda = 0.1, the same
seeded generator.

The oracle cannot factor N = 131072 on the host, so it checks what it can
compute one entry or one row at a time, each from the definitions:
* kernel entries of 64 sampled training rows against all N columns
  (Alg. 5 on the brute-force distance): |K_gpu - K| <= 4e-7, as at small N;
* the residual of those rows, ||Y_S - lambda A_S - K_S A|| / ||Y_S|| with the
  oracle's K_S and the GPU's A: it must meet the refinement's stopping level
  (<= 2e-5; the device reports about 1e-5 for all rows);
* 32 sampled held-out predictions, K_test[S_t, :] A (Alg. 4) with the GPU's A.
  The floor is the FP32 kernel entry itself: each K_tj (FP32 expf, within a
  couple of ulp) carries a relative error up to about 2^-23, independent
  across j, so the sum over N = 131072 terms is off by about
  2^-23 sqrt(sum_j (K_tj A_j)^2) -- near 1e-5 of ||Yt|| here.  The gate is
  4 times that noise level (Frobenius norm over the sample), and the
  end-to-end bound 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

N, M, P, N_TEST, TILE = 131072, 16384, 20, 4096, 1024
SEED, LAM = 2409017120, 0.1


def test_fullsize_sampled_rows_match_oracle():
    gamma = 1.0 / M
    prob = inputs.problem(N, M, P, N_TEST, seed=SEED, device=DEV)
    g, y, t = prob["G"], prob["Y"], prob["T"]
    rng = np.random.default_rng(131072)
    rows = np.sort(rng.choice(N, 64, replace=False))
    trows = np.sort(rng.choice(N_TEST, 32, replace=False))
    with KRR(tile=TILE, mode="mixed") as model:
        model.build_kernel(g, gamma)
        finfo = model.factor(LAM)
        a, sinfo = model.solve(y)
        yt = model.predict(t, a)
        # K rows of the sample from the lower-triangle tiles (entry (i, j) with
        # tile(j) > tile(i) is stored as (j, i))
        kd = torch.empty((N, N), dtype=torch.float32, device=DEV)
        model.kernel(kd)
        ridx = torch.from_numpy(rows).to(DEV)
        lower = kd[ridx, :]
        upper = kd[:, ridx].t()
        del kd
    tcol = torch.arange(N, device=DEV) // TILE
    use_lower = tcol[None, :] <= (ridx // TILE)[:, None]
    k_gpu = torch.where(use_lower, lower, upper).double().cpu().numpy()
    assert sinfo["converged"] in (1, 2), sinfo
    assert finfo["tiles_fp32"] + finfo["tiles_fp16"] + finfo["tiles_e4m3"] == (N // TILE) * (N // TILE - 1) // 2

    g_h = g.cpu().numpy()
    k_ref = oracle.kernel_rows(gamma, g_h, rows, g_h)
    assert np.max(np.abs(k_gpu - k_ref)) <= 4e-7

    a_h = a.double().cpu().numpy()
    y_h = y.double().cpu().numpy()
    r = y_h[rows] - LAM * a_h[rows] - oracle.matmul(k_ref, a_h)
    rel = np.linalg.norm(r) / np.linalg.norm(y_h[rows])
    assert rel <= 2e-5, (rel, sinfo)

    kt_ref = oracle.kernel_rows(gamma, t.cpu().numpy(), trows, g_h)
    yt_ref = oracle.matmul(kt_ref, a_h)
    yt_s = yt.double().cpu().numpy()[trows]
    err = np.linalg.norm(yt_s - yt_ref) / np.linalg.norm(yt_ref)
    noise = 2.0 ** -23 * np.sqrt((kt_ref ** 2) @ (a_h ** 2))
    assert np.linalg.norm(yt_s - yt_ref) <= 4 * np.linalg.norm(noise), (err, np.linalg.norm(noise) / np.linalg.norm(yt_ref))
    assert err <= 1e-4, err


N_SUB = 16384


def test_c3_subproblem_matches_fp64_oracle():
    """The first 16384 rows of the N = 131072 workload (same seeded stream, M =
    16384, P = 20, the workload's 4096 held-out rows, tile 1024, mixed mode)
    against the full FP64 oracle solution of that subproblem (Alg. 1 with
    float64 library Gram products and factorisation, pinned against the
    plain loops on the CPU).

    Gates: squared distances bit-exact on a sample of tiles; the predictions
    ||Yt - Yt*||_F / ||Yt*||_F <= 1e-4 (the end-to-end target).  Reported and
    gated: ||A - A*||_F / ||A*||_F <= 1e-4 (the forward error in A grows with
    the condition number of K + lambda I, up to ||K|| / lambda, about 8e4
    here; measured 4.8e-6), and the FP64 relative residual of the GPU's A
    ||Y - (K + lambda I) A||_F / ||Y||_F <= 2e-5 (measured 3.7e-6).
    """
    gamma = 1.0 / M
    prob = inputs.problem(N, M, P, N_TEST, seed=SEED, device=DEV)
    g = prob["G"][:N_SUB].contiguous()
    y = prob["Y"][:N_SUB].contiguous()
    t = prob["T"]
    del prob
    with KRR(tile=TILE, mode="mixed") as model:
        model.build_kernel(g, gamma, keep_distances=True)
        finfo = model.factor(LAM)
        a, sinfo = model.solve(y)
        yt = model.predict(t, a)
        dd = torch.zeros((N_SUB, N_SUB), dtype=torch.int32, device=DEV)
        model.distances(dd)
    g_h, y_h, t_h = g.cpu().numpy(), y.double().cpu().numpy(), t.cpu().numpy()
    a_h, yt_h = a.double().cpu().numpy(), yt.double().cpu().numpy()
    # distances of three tiles (diagonal, first column, last row) against brute force
    rng = np.random.default_rng(16384)
    for ti, tj in ((5, 5), (9, 0), (15, 11)):
        rows = np.sort(rng.choice(TILE, 64, replace=False)) + ti * TILE
        dref = oracle.sqdist(g_h[rows], g_h[tj * TILE:(tj + 1) * TILE])
        dgpu = dd[torch.from_numpy(rows).to(DEV), tj * TILE:(tj + 1) * TILE].cpu().numpy().astype(np.int64)
        assert np.array_equal(dgpu, dref), (ti, tj)
    del dd
    k_ref, a_ref, yt_ref = oracle.krr(gamma, LAM, g_h, y_h, t_h, method="lapack")
    err_yt = np.linalg.norm(yt_h - yt_ref) / np.linalg.norm(yt_ref)
    err_a = np.linalg.norm(a_h - a_ref) / np.linalg.norm(a_ref)
    r = y_h - LAM * a_h - k_ref @ a_h
    rel_res = np.linalg.norm(r) / np.linalg.norm(y_h)
    print(f"\nc3 subproblem N={N_SUB}: err_Yt={err_yt:.3e} err_A={err_a:.3e} rel_residual_fp64={rel_res:.3e} "
          f"device_residual={sinfo['rel_residual']:.3e} iterations={sinfo['iterations']} "
          f"tiles fp32/fp16/e4m3={finfo['tiles_fp32']}/{finfo['tiles_fp16']}/{finfo['tiles_e4m3']}")
    assert sinfo["converged"] in (1, 2), sinfo
    assert err_yt <= 1e-4, err_yt
    assert rel_res <= 2e-5, rel_res
    assert err_a <= 1e-4, err_a
