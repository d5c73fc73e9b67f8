"""krr_predict_noalloc: prediction for callers that must not allocate device
memory at call time (a process whose device memory is reserved up front by
another allocator, or a latency-critical path that must not enter the
driver's allocator).  It keeps its working buffers in one fixed-size device
array of the library instead of cudaMalloc'd buffers.  Called here through
the C ABI and compared with krr_predict on two calls in a row; the free
device memory is the same before and after a call.

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test when it gets here."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_01712_gb300 import KRR, inputs
from paper_2409_01712_gb300 import krr as krrmod

pytestmark = pytest.mark.gpu

# Y_test tolerance the parity tests use (relative Frobenius error)
RTOL_YT = 1e-4


def _call(lib, model, t, a, out):
    return lib.krr_predict_noalloc(model._ctx, ctypes.c_void_p(t.data_ptr()), t.shape[0], t.stride(0),
                                   ctypes.c_void_p(a.data_ptr()), a.stride(0), a.shape[1],
                                   ctypes.c_void_p(out.data_ptr()), out.stride(0))


def test_predict_noalloc_matches_predict():
    lib = krrmod.load_library()
    dev = torch.device("cuda:0")
    n, m, p, n_test = 1000, 700, 3, 200  # ragged: not multiples of the tile or 128
    prob = inputs.problem(n, m, p, n_test, seed=31)
    g, y, t = prob["G"].to(dev), prob["Y"].to(dev), prob["T"].to(dev)
    with KRR(tile=256, mode="mixed") as model:
        model.build_kernel(g, 1.0 / m)
        model.factor(0.1)
        a, _ = model.solve(y)
        ref = model.predict(t, a)
        torch.cuda.synchronize()
        for _ in range(2):  # the second call reuses the array the first one left behind
            out = torch.full((n_test, p), float("nan"), device=dev)
            st = _call(lib, model, t, a, out)
            torch.cuda.synchronize()
            assert st == krrmod.OK, lib.krr_last_error(model._ctx)
            err = (torch.linalg.norm(out.double() - ref.double()) / torch.linalg.norm(ref.double())).item()
            assert err <= RTOL_YT, err
        # after a warm call (the array's address is looked up), a call takes
        # no device memory: cudaMalloc works in 2 MB pages, so any allocation
        # would show in the free bytes
        out = torch.empty((n_test, p), device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(lib, model, t, a, out)
        torch.cuda.synchronize()
        assert st == krrmod.OK
        assert torch.cuda.mem_get_info()[0] == free0
        # limits are checked, nothing is written on refusal
        big = torch.zeros((300, m), dtype=torch.int8, device=dev)
        out = torch.zeros((300, p), device=dev)
        assert _call(lib, model, big, a, out) == krrmod.EINVAL
        host_out = np.zeros((n_test, p), np.float32)
        st = lib.krr_predict_noalloc(model._ctx, ctypes.c_void_p(t.data_ptr()), n_test, m,
                                     ctypes.c_void_p(a.data_ptr()), p, p,
                                     ctypes.c_void_p(host_out.ctypes.data), p)
        assert st == krrmod.EINVAL
