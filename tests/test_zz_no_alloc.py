"""The allocation-free probe fit, sh_fit_static.

It exists for callers that cannot call cudaMalloc (a real-time frame loop
where an allocation would synchronise the device, or a host that owns all
device memory itself).  It must give the same probe as the ordinary sh_fit
entry point, call after call, even though every call reuses the one scratch
array compiled into the library.  This file is collected last so that a run
stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_01660_b300 import scenes

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _static_fit(nat, D, Y, w, lam, outs=None):
    """Call the C entry point directly through ctypes (device buffers from torch)."""
    if outs is None:
        outs = (torch.empty((3, 9), dtype=torch.float32, device="cuda"),
                torch.empty((3, 9), dtype=torch.float64, device="cuda"),
                torch.empty((1,), dtype=torch.int32, device="cuda"))
    sh, sh64, status = outs
    status.fill_(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = nat._lib.sh_fit_static(ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                ctypes.c_void_p(w.data_ptr()), D.shape[0], float(lam),
                                ctypes.c_void_p(sh.data_ptr()), ctypes.c_void_p(sh64.data_ptr()),
                                ctypes.c_void_p(status.data_ptr()), stream)
    assert rc == 0
    return sh, sh64, status


def test_static_fit_matches_sh_fit_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    nat = native()
    cases = [(scenes.cubemap_samples(64, seed=5), 1e-3), (scenes.cubemap_samples(16, seed=9), 0.2)]
    for (D, Y, w), lam in cases:
        D, Y, w = _dev(D), _dev(Y), _dev(w)
        ref, ref64 = nat.sh_fit(D, Y, w, lam=lam, want64=True)
        outs = None
        for call in range(2):  # the second call reuses the scratch the first one filled
            if call == 1:
                # the outputs already exist: the call itself must take no device memory
                torch.cuda.synchronize()
                free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            sh, sh64, status = outs = _static_fit(nat, D, Y, w, lam, outs)
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_allocated() == used0
            assert int(status.item()) == 0
            np.testing.assert_allclose(sh64.cpu().numpy(), ref64.cpu().numpy(), rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(sh.cpu().numpy(), ref.cpu().numpy(), rtol=1e-6, atol=1e-7)


def test_static_fit_rejects_too_many_samples_and_reports_not_spd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2601_01660_b300 import native
    nat = native()
    D = _dev(np.float32(np.tile([[0, 0, 1.0]], (10, 1))))
    Y = _dev(np.ones((10, 3), np.float32))
    w = _dev(np.ones(10, np.float32))
    sh, sh64, status = _static_fit(nat, D, Y, w, 0.0)   # rank-deficient, lambda = 0
    torch.cuda.synchronize()
    assert int(status.item()) == 6 and bool((sh == 0).all())
    big = 4 * 1024 * 1024 + 1
    rc = nat._lib.sh_fit_static(ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                ctypes.c_void_p(w.data_ptr()), big, 1e-3,
                                ctypes.c_void_p(sh.data_ptr()), None, None, None)
    assert rc == 3
