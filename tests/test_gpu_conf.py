"""Confounders (Sec. IV-B, distance section): the squared distances of
real-valued covariate columns join the exact genotype distances before the
exponential of the Gaussian kernel,
K_ij = exp(-gamma (||g_i - g_j||^2 + ||c_i - c_j||^2)).
On the GPU the covariate distance is summed term by term in FP32 inside the
build and predict epilogues.  Against the FP64 oracle: kernel entries within
1e-6 (FP32 confounder sums, FP32 storage), predictions within 1e-4 (mixed,
after refinement) or 1e-3 (plain FP32)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, KRRError, inputs
from paper_2409_01712_gb300 import krr as krrmod

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _case(n, m, p, n_test, nc, seed):
    prob = {k: v.numpy() for k, v in inputs.problem(n, m, p, n_test, seed=seed).items()}
    # covariates carrying about a tenth of the mean genotype distance (0.74 M)
    scale = float(np.sqrt(0.1 * 0.74 * m / (2 * nc)))
    c_all = inputs.confounders(n + n_test, nc, seed=seed, scale=scale).numpy()
    prob["C"], prob["Ct"] = c_all[:n].copy(), c_all[n:].copy()
    return prob


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
@pytest.mark.parametrize("n,m,nc,tile", [(700, 300, 3, 256), (1100, 1000, 16, 512)])
def test_kernel_with_confounders(mode, n, m, nc, tile):
    prob = _case(n, m, 1, 1, nc, seed=81 + n)
    gamma = 1.0 / m
    with KRR(tile=tile, mode=mode) as model:
        model.build_kernel(_to(prob["G"]), gamma, keep_distances=True, conf=_to(prob["C"]))
        d = model.distances().astype(np.int64)
        kgpu = model.kernel().astype(np.float64)
    dref = oracle.sqdist(prob["G"])
    kref = oracle.build_kernel(gamma, prob["G"], c1=prob["C"])
    nt = -(-n // tile)
    for i in range(nt):
        for j in range(i + 1):
            rs = slice(i * tile, min(n, (i + 1) * tile))
            cs = slice(j * tile, min(n, (j + 1) * tile))
            assert np.array_equal(d[rs, cs], dref[rs, cs]), (i, j)  # genotype distances stay exact
            assert np.max(np.abs(kgpu[rs, cs] - kref[rs, cs])) <= 1e-6, (i, j)


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
@pytest.mark.parametrize("n,m,p,nc,tile", [(900, 256, 3, 5, 256), (2048, 512, 20, 10, 512)])
def test_fit_predict_with_confounders(mode, n, m, p, nc, tile):
    prob = _case(n, m, p, 300, nc, seed=91 + n)
    gamma, lam = 1.0 / m, 0.1
    _, a_ref, yt_ref = oracle.krr(gamma, lam, prob["G"], prob["Y"].astype(np.float64), prob["T"],
                                  conf=prob["C"], conf_t=prob["Ct"])
    with KRR(tile=tile, mode=mode) as model:
        model.build_kernel(_to(prob["G"]), gamma, conf=_to(prob["C"]))
        model.factor(lam)
        a, sinfo = model.solve(_to(prob["Y"]))
        yt = model.predict(_to(prob["T"]), a, conf=_to(prob["Ct"]))
        with pytest.raises(KRRError) as e:  # the held-out confounders are required
            model.predict(_to(prob["T"]), a)
        assert e.value.status == krrmod.EINVAL
    err = np.linalg.norm(yt.cpu().numpy() - yt_ref) / np.linalg.norm(yt_ref)
    print(f"\nconfounders {mode} n={n} nc={nc}: err_Yt={err:.3e} residual={sinfo['rel_residual']:.3e}")
    assert err <= (1e-4 if mode == "mixed" else 1e-3), (err, sinfo)


def test_confounder_argument_checks():
    prob = _case(300, 64, 1, 10, 17, seed=5)
    with KRR(tile=256, mode="mixed") as model:
        with pytest.raises(KRRError) as e:  # at most 16 confounder columns
            model.build_kernel(_to(prob["G"]), 1.0 / 64, conf=_to(prob["C"]))
        assert e.value.status == krrmod.EINVAL
    with KRR(tile=256, mode="mixed", kernel="ibs") as model:
        with pytest.raises(KRRError) as e:  # confounders join the Gaussian kernel only
            model.build_kernel(_to(prob["G"]), 1.0, conf=_to(prob["C"][:, :4]))
        assert e.value.status == krrmod.EINVAL
