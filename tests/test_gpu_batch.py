"""Batched problems under one captured CUDA graph (cross-validation style:
cohorts x lambdas of uneven size) against the CPU oracle, and run-to-run
identity of the graph replays.  Problems that pass the same genotype tensor
with the same gamma share one Build (the kernel matrix does not depend on
lambda).  Y_test tolerance 1e-4 (as the other parity tests)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRRBatch, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("autotune", [1, 2])
def test_batch_matches_oracle_and_replays(autotune):
    m, p = 300, 2
    sizes = [(700, 0.1), (700, 1.0), (1300, 0.1), (1300, 0.01), (1300, 1.0), (300, 0.1)]
    problems, refs, cohorts = [], [], {}
    for idx, (n, lam) in enumerate(sizes):
        prob = inputs.problem(n, m, p, 120, seed=900 + n)  # same n -> same cohort data
        g, y, t = prob["G"].numpy(), prob["Y"].numpy(), prob["T"].numpy()
        _, a_ref, yt_ref = oracle.krr(1.0 / m, lam, g, y.astype(np.float64), t)
        refs.append((a_ref, yt_ref))
        if n not in cohorts:  # one device copy per cohort: its lambdas share the Build
            cohorts[n] = {k: prob[k].to(DEV) for k in ("G", "Y", "T")}
        c = cohorts[n]
        problems.append({"G": c["G"], "Y": c["Y"], "T": c["T"], "gamma": 1.0 / m, "lam": lam})
    # autotune 2 also captures and times the whole batch for every candidate
    # assignment of tile edges (instantiating and releasing the graph each time)
    with KRRBatch(problems, ir_iters=3, autotune=autotune) as bt:
        res = bt.run()
        first = [yt.clone() for yt in bt.Yt]
        res2 = bt.run()
        for i, (a_ref, yt_ref) in enumerate(refs):
            assert res[i]["status"] == 0
            assert res[i]["tile"] in (256, 512, 1024)
            assert 0.0 < res[i]["rel_residual"] <= 1e-5, res[i]
            yt = bt.Yt[i].cpu().numpy().astype(np.float64)
            err = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
            assert err <= 1e-4, (i, err, res[i])
            assert torch.equal(bt.Yt[i], first[i])  # deterministic replay
            assert res2[i]["rel_residual"] == res[i]["rel_residual"]
