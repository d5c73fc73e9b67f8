"""Failure detection without a GPU fault: every device-side wait of the
library is bounded by the context's wait budget, and a wait that runs out
ends its kernel (after the kernel's own copies and MMAs in flight finish)
with KRR_ETIMEOUT, which the launching call returns; the context stays
usable.  The tests make the waits run out by giving them a budget of 1 ns
(no dependency between work items, copies or MMAs completes that fast), then
restore the budget and check that the same context computes the right
answer.  Also: refinement that cannot reach its tolerance (KRR_ENOCONV) and
an allocation larger than the device (KRR_ENOMEM), both recoverable."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, KRRError, inputs
from paper_2409_01712_gb300 import krr as krrmod

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
NORMAL = 2_000_000_000


def _case(seed=5, n=1300, m=400, p=2):
    prob = {k: v.numpy() for k, v in inputs.problem(n, m, p, 100, seed=seed).items()}
    _, a_ref, yt_ref = oracle.krr(1.0 / m, 0.1, prob["G"], prob["Y"].astype(np.float64), prob["T"])
    return prob, yt_ref


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _check(model, prob, yt_ref):
    a, info = model.solve(_to(prob["Y"]))
    yt = model.predict(_to(prob["T"]), a)
    err = np.linalg.norm(yt.cpu().numpy() - yt_ref) / np.linalg.norm(yt_ref)
    assert err <= 1e-4, (err, info)


def test_timeout_in_factor_then_recovery():
    # diagonal-step dataflow waits, the panel solve's and the trailing
    # update's (CTA pairs) barrier waits all run out
    prob, yt_ref = _case()
    with KRR(tile=256, mode="mixed") as model:
        model.build_kernel(_to(prob["G"]), 1.0 / 400)
        model.set_wait_budget(1)
        with pytest.raises(KRRError) as e:
            model.factor(0.1)
        assert e.value.status == krrmod.ETIMEOUT
        torch.cuda.synchronize()
        model.set_wait_budget(NORMAL)
        model.factor(0.1)
        _check(model, prob, yt_ref)


def test_timeout_in_solve_then_recovery():
    # the tensor-core substitution sweeps and the refinement residual
    prob, yt_ref = _case(seed=6)
    with KRR(tile=256, mode="mixed") as model:
        model.build_kernel(_to(prob["G"]), 1.0 / 400)
        model.factor(0.1)
        model.set_wait_budget(1)
        with pytest.raises(KRRError) as e:
            model.solve(_to(prob["Y"]))
        assert e.value.status == krrmod.ETIMEOUT
        torch.cuda.synchronize()
        model.set_wait_budget(NORMAL)
        _check(model, prob, yt_ref)  # the factor was not touched


def test_timeout_in_plain_fp32_path():
    # the CUDA-core sweeps of the comparison path wait on bounded counters too
    prob, yt_ref = _case(seed=7)
    with KRR(tile=256, mode="fp32") as model:
        model.build_kernel(_to(prob["G"]), 1.0 / 400)
        model.factor(0.1)
        model.set_wait_budget(1)
        with pytest.raises(KRRError) as e:
            model.solve(_to(prob["Y"]))
        assert e.value.status == krrmod.ETIMEOUT
        model.set_wait_budget(NORMAL)
        a, _ = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a)
    assert np.linalg.norm(yt.cpu().numpy() - yt_ref) / np.linalg.norm(yt_ref) <= 1e-3


def test_refinement_not_converged():
    # one refinement step cannot reach 1e-12: KRR_ENOCONV, with the best
    # iterate returned when asked for
    prob, yt_ref = _case(seed=8)
    with KRR(tile=256, mode="mixed", ir_max=1, ir_tol=1e-12) as model:
        model.build_kernel(_to(prob["G"]), 1.0 / 400)
        model.factor(0.1)
        with pytest.raises(KRRError) as e:
            model.solve(_to(prob["Y"]))
        assert e.value.status == krrmod.ENOCONV
        a, info = model.solve(_to(prob["Y"]), raise_on_noconv=False)
        assert info["iterations"] == 1 and info["converged"] == 0
        assert info["rel_residual"] < info["history"][0]
        yt = model.predict(_to(prob["T"]), a)
    assert np.linalg.norm(yt.cpu().numpy() - yt_ref) / np.linalg.norm(yt_ref) <= 1e-3


def test_allocation_failure_is_reported_and_recoverable():
    # 2^21 rows: the kernel tiles would need about 8.8 TB
    g = torch.zeros((1 << 21, 128), dtype=torch.int8, device=DEV)
    prob, yt_ref = _case(seed=9)
    with KRR(tile=1024, mode="mixed") as model:
        with pytest.raises(KRRError) as e:
            model.build_kernel(g, 1.0 / 128)
        assert e.value.status == krrmod.ENOMEM
        del g
        with pytest.raises(KRRError) as e:
            model.factor(0.1)  # nothing was built
        assert e.value.status == krrmod.ESTATE
        model.build_kernel(_to(prob["G"]), 1.0 / 400)
        model.factor(0.1)
        _check(model, prob, yt_ref)
