"""Ridge regression (Sec. IV-A, Eq. 2): beta = (X^T X + lambda I)^-1 X^T Y with
X = [G C], through krr_rr_build (the mixed-precision SYRK: G^T G exact on the
tensor cores, confounder columns in FP32), krr_rr_rhs (X^T Y), the same
krr_factor / krr_solve as KRR, and krr_rr_predict.  Against the FP64 oracle:
the genotype block of the Gram matrix bit-exact (integers below 2^24), the
confounder entries within the FP32 dot-product bound, the weights within 1e-3 and the
held-out predictions within 1e-4 (mixed, after refinement), or 1e-3 and 1e-3
(plain FP32, no refinement)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, KRRError, inputs
from paper_2409_01712_gb300 import krr as krrmod

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _to(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _case(n, m, p, n_test, nc, seed):
    prob = {k: v.numpy() for k, v in inputs.problem(n, m, p, n_test, seed=seed).items()}
    if nc:
        c_all = inputs.confounders(n + n_test, nc, seed=seed, scale=2.0).numpy()
        prob["C"], prob["Ct"] = c_all[:n].copy(), c_all[n:].copy()
    else:
        prob["C"] = prob["Ct"] = None
    return prob


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
@pytest.mark.parametrize("n,m,nc,p,tile", [(3000, 700, 0, 3, 256), (3000, 700, 5, 2, 256), (600, 1100, 3, 4, 512)])
def test_ridge_matches_oracle(mode, n, m, nc, p, tile):
    prob = _case(n, m, p, 200, nc, seed=101 + n + nc)
    lam = 10.0
    gram, rhs, beta_ref = oracle.ridge(lam, prob["G"], prob["Y"], prob["C"], method="lapack")
    yt_ref = oracle.ridge_predict(prob["T"], beta_ref, prob["Ct"])
    conf = None if prob["C"] is None else _to(prob["C"])
    with KRR(tile=tile, mode=mode) as model:
        model.rr_build(_to(prob["G"]), conf=conf)
        kg = model.kernel().astype(np.float64)
        b = model.rr_rhs(_to(prob["Y"]))
        model.factor(lam)
        beta, sinfo = model.solve(b)
        yt = model.rr_predict(_to(prob["T"]), beta, conf=None if prob["Ct"] is None else _to(prob["Ct"]))
        with pytest.raises(KRRError) as e:  # the KRR predict does not apply to a Gram matrix
            model.predict(_to(prob["T"]), beta)
        assert e.value.status == krrmod.EINVAL
    f = m + nc
    low = np.tril(np.ones((f, f), bool))
    nt = -(-f // tile)
    for i in range(nt):  # strictly-upper tiles are not stored
        low[i * tile:(i + 1) * tile, (i + 1) * tile:] = False
    # genotype block: exact integers; confounder rows: FP32 products
    gb = low.copy()
    gb[m:, :] = False
    assert np.array_equal(kg[gb], gram[gb])
    cb = low & ~gb
    if nc:
        # FP32 dot products over the patients: within the usual bound
        # gamma_K |x|^T |y| (K = the patients summed in one FP32 chunk, <= 2^11)
        x = np.concatenate([prob["G"].astype(np.float64), prob["C"].astype(np.float64)], axis=1)
        absgram = np.abs(x).T @ np.abs(x)
        assert np.all(np.abs(kg[cb] - gram[cb]) <= 2048 * 2.0 ** -24 * absgram[cb])
    assert np.allclose(b.cpu().numpy(), rhs, rtol=1e-5, atol=1e-4)
    beta = beta.cpu().numpy().astype(np.float64)
    yt = yt.cpu().numpy().astype(np.float64)
    err_b = np.linalg.norm(beta - beta_ref) / np.linalg.norm(beta_ref)
    err_y = np.linalg.norm(yt - yt_ref) / np.linalg.norm(yt_ref)
    print(f"\nridge {mode} n={n} m={m} nc={nc}: err_beta={err_b:.3e} err_Yt={err_y:.3e} "
          f"residual={sinfo['rel_residual']:.3e}")
    if mode == "mixed":
        assert sinfo["converged"] in (1, 2), sinfo
        assert err_b <= 1e-3 and err_y <= 1e-4, (err_b, err_y, sinfo)
    else:
        assert err_b <= 1e-3 and err_y <= 1e-3, (err_b, err_y)
