"""Lookahead of the tile Cholesky (Alg. 3, Factorize): the diagonal step of
column k + 1 runs on a second stream, on a few CTAs, while the trailing update
of step k goes on (its diagonal target first).  Every tile still receives the
same updates in the same order, each update of a target tile is one
accumulation inside one launch, and the diagonal step orders its block
updates by counters, so the factor and the solution must be bit-identical to
the strictly sequential schedule (options.lookahead = 0).

The benchmarked size (N = 131072, tile 1024, 128 tile columns) is the one where
the update of a step is split in three launches: the diagonal target, the
targets beside the diagonal step, and the rest on every SM."""
import numpy as np
import pytest
import torch

from paper_2409_01712_gb300 import KRR, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _run(prob, m, tile, lookahead, want_factor):
    with KRR(tile=tile, mode="mixed", lookahead=lookahead) as model:
        model.build_kernel(prob["G"], 1.0 / m)
        finfo = model.factor(0.1)
        a, sinfo = model.solve(prob["Y"])
        pmap = model.precision_map()
        lf = model.factor_matrix() if want_factor else None
        torch.cuda.synchronize()
        return finfo, a.cpu().numpy(), sinfo, pmap, lf


@pytest.mark.parametrize("n,m,p,tile", [(1300, 700, 3, 256), (16384, 4096, 8, 1024)])
def test_lookahead_bit_identical_to_sequential(n, m, p, tile):
    prob = inputs.problem(n, m, p, 16, seed=77 + n, device=DEV)
    f0, a0, s0, m0, l0 = _run(prob, m, tile, False, True)
    f1, a1, s1, m1, l1 = _run(prob, m, tile, True, True)
    assert f0 == f1
    assert np.array_equal(m0, m1)
    assert np.array_equal(l0, l1)
    assert np.array_equal(a0, a1)
    assert s0["history"] == s1["history"]


def test_lookahead_bit_identical_at_benchmarked_size():
    n, m, p, tile = 131072, 16384, 20, 1024
    prob = inputs.problem(n, m, p, 16, seed=2409017120, device=DEV)
    f1, a1, s1, m1, _ = _run(prob, m, tile, True, False)
    f0, a0, s0, m0, _ = _run(prob, m, tile, False, False)
    assert s1["converged"] in (1, 2), s1
    assert f0 == f1
    assert np.array_equal(m0, m1)
    assert np.array_equal(a0, a1)
    assert s0["history"] == s1["history"]
