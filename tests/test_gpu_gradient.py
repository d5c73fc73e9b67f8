"""Hyperparameter gradient (adjoint reusing the Cholesky factor) against the
FP64 oracle's closed form and against central finite differences of the GPU
loss.  Tolerances: 2e-3 relative against the oracle (the GPU path carries
FP32 K and an FP32-floor refinement); 2e-2 against finite differences with
h = 1e-3 in log space (truncation ~h^2 plus the loss noise / h)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2409_01712_gb300 import KRR, held_out_loss, inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _prob(n, m, p, n_test, seed):
    prob = inputs.problem(n, m, p, n_test, seed=seed)
    return {k: v.numpy() for k, v in prob.items()}


def _gpu_grad(prob, gamma, lam, tile):
    to = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    with KRR(tile=tile, mode="mixed") as model:
        model.build_kernel(to(prob["G"]), gamma)
        model.factor(lam)
        a, _ = model.solve(to(prob["Y"]))
        return model.grad_hyper(to(prob["T"]), to(prob["Yt"]), a)


@pytest.mark.parametrize("n,m,p,n_test,tile", [(1024, 512, 2, 200, 256), (1300, 700, 3, 300, 512)])
def test_gradient_matches_oracle(n, m, p, n_test, tile):
    prob = _prob(n, m, p, n_test, seed=41 + n)
    gamma, lam = 1.0 / m, 0.1
    loss, dg, dl = _gpu_grad(prob, gamma, lam, tile)
    rloss, rdg, rdl = oracle.hyper_gradient(gamma, lam, prob["G"], prob["Y"], prob["T"], prob["Yt"])
    assert loss == pytest.approx(rloss, rel=1e-4)
    assert dl == pytest.approx(rdl, rel=2e-3)
    assert dg == pytest.approx(rdg, rel=2e-3, abs=2e-3 * abs(rloss))


def test_gradient_matches_finite_differences_and_autograd():
    prob = _prob(1024, 512, 2, 256, seed=7)
    to = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    g, y, t, yt = (to(prob[k]) for k in ("G", "Y", "T", "Yt"))
    lg = torch.tensor(math.log(1.0 / 512), dtype=torch.float64, requires_grad=True)
    ll = torch.tensor(math.log(0.1), dtype=torch.float64, requires_grad=True)
    loss = held_out_loss(lg, ll, g, y, t, yt, 256)
    loss.backward()
    h = 1e-3
    f = lambda a, b: float(held_out_loss(torch.tensor(a), torch.tensor(b), g, y, t, yt, 256))
    fd_g = (f(lg.item() + h, ll.item()) - f(lg.item() - h, ll.item())) / (2 * h)
    fd_l = (f(lg.item(), ll.item() + h) - f(lg.item(), ll.item() - h)) / (2 * h)
    assert lg.grad.item() == pytest.approx(fd_g, rel=2e-2, abs=1e-3 * float(loss))
    assert ll.grad.item() == pytest.approx(fd_l, rel=2e-2, abs=1e-3 * float(loss))


def test_gradient_at_differentiation_workload_size():
    """The differentiation workload: N_train = 16384, N_test = 4096, M = 8192,
    P = 8, gamma = 1/M, lambda = 0.1, tile 1024.  The adjoint gradient
    (reusing the Cholesky factor) against the FP64 oracle's closed form
    (float64 library Gram products and factorisation) and against central
    differences of the GPU loss with h = 1e-3 in log space."""
    n, n_test, m, p, tile = 16384, 4096, 8192, 8, 1024
    gamma, lam = 1.0 / m, 0.1
    prob = inputs.problem(n, m, p, n_test, seed=2409017125, device=DEV)
    g, y, t, yt = prob["G"], prob["Y"], prob["T"], prob["Yt"]
    with KRR(tile=tile, mode="mixed") as model:
        model.build_kernel(g, gamma)
        model.factor(lam)
        a, _ = model.solve(y)
        loss, dg, dl = model.grad_hyper(t, yt, a)

    def gpu_loss(log_g, log_l):
        with KRR(tile=tile, mode="mixed") as mdl:
            mdl.build_kernel(g, math.exp(log_g))
            mdl.factor(math.exp(log_l))
            aa, _ = mdl.solve(y)
            pr = mdl.predict(t, aa)
        return float(((pr.double() - yt.double()) ** 2).mean())

    h = 1e-3
    lg0, ll0 = math.log(gamma), math.log(lam)
    fd_g = (gpu_loss(lg0 + h, ll0) - gpu_loss(lg0 - h, ll0)) / (2 * h)
    fd_l = (gpu_loss(lg0, ll0 + h) - gpu_loss(lg0, ll0 - h)) / (2 * h)
    rloss, rdg, rdl = oracle.hyper_gradient(gamma, lam, g.cpu().numpy(), y.cpu().numpy(), t.cpu().numpy(),
                                            yt.cpu().numpy(), method="lapack")
    print(f"\ngradient N={n}: loss {loss:.6e} (oracle {rloss:.6e}); d/dlog gamma {dg:.6e} (oracle {rdg:.6e}, "
          f"fd {fd_g:.6e}); d/dlog lambda {dl:.6e} (oracle {rdl:.6e}, fd {fd_l:.6e})")
    assert loss == pytest.approx(rloss, rel=1e-4)
    assert dl == pytest.approx(rdl, rel=2e-3)
    assert dg == pytest.approx(rdg, rel=2e-3, abs=2e-3 * abs(rloss))
    assert dg == pytest.approx(fd_g, rel=2e-2, abs=1e-3 * rloss)
    assert dl == pytest.approx(fd_l, rel=2e-2, abs=1e-3 * rloss)
