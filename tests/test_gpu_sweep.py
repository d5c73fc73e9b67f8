"""The substitution sweeps and the refinement residual (persistent dataflow
kernel) against FP64 references on the same stored factor.

With ir_max = 0 a solve is one forward and one backward sweep, so the
returned A must equal (L L^T)^-1 Y for the factor L the library stored (read
back densely), up to FP32 rounding: relative error <= 2e-5 here (FP32
products, FP32 accumulation over N = 1300 terms, L well conditioned).  The
reported relative residual must match ||Y - (K + lambda I) A|| / ||Y||
recomputed in FP64 from the oracle's K to 1e-3 of its value (the device
forms it from FP32 K tiles with FP64 row sums; for the 2^40-range case below,
where the residual is 20x smaller relative to the products, plus a floor of
2e-6 for the FP32 storage of K).

Cases: ragged N over several tiles; more than 32 right-hand sides (two
column chunks per sweep) with a leading dimension that is not a multiple of
4 (4-byte vector copies); a narrow kernel (gamma = 8 / M, off-diagonal K
around 4e-3) with an error bound loose enough for E4M3 factor tiles; blocks
of Y scaled by 2^20 and 2^-20, so that the scale each block predicts from
the block before it fails and the block is converted again with its exact
scale.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("p,eps,tile,gmul,jump", [(37, None, 256, 1.0, False), (40, None, 512, 1.0, False),
                                                  (5, 0.05, 256, 8.0, False), (6, None, 256, 1.0, True)])
def test_sweep_solve_and_residual_match_fp64(p, eps, tile, gmul, jump):
    n, m, lam = 1300, 300, 0.1
    gamma = gmul / m
    prob = inputs.problem(n, m, p, 1, seed=4242 + p)
    if jump:
        prob["Y"][tile:2 * tile] *= 2.0 ** 20
        prob["Y"][3 * tile:4 * tile] *= 2.0 ** -20
    g, y = prob["G"], prob["Y"].numpy().astype(np.float64)
    with KRR(tile=tile, mode="mixed", eps=eps, ir_max=0) as model:
        model.build_kernel(g.to(DEV), gamma)
        finfo = model.factor(lam)
        a, sinfo = model.solve(torch.from_numpy(prob["Y"].numpy()).to(DEV), raise_on_noconv=False)
        l_stored = model.factor_matrix().astype(np.float64)
    if eps is not None:
        assert finfo["tiles_e4m3"] > 0, finfo
    a = a.cpu().numpy().astype(np.float64)
    a_ref = oracle.backward_subst(l_stored, oracle.forward_subst(l_stored, y))
    err = np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref)
    assert err <= 2e-5, err
    k = oracle.build_kernel(gamma, g.numpy())
    r = y - k @ a - lam * a
    rel = np.linalg.norm(r) / np.linalg.norm(y)
    # the device forms the residual from FP32 K tiles: against the FP64 K that
    # is an error of about u32 |K| |A|, which only shows next to the small
    # residual of the 2^40-range case (a floor of 2e-6 ||Y||)
    floor = 2e-6 if jump else 1e-9
    assert abs(sinfo["rel_residual"] - rel) <= 1e-3 * rel + floor, (sinfo["rel_residual"], rel)
