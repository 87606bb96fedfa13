"""tdse_populations_noalloc against tdse_populations.

The no-allocation variant serves callers that cannot allocate device memory
at the point of use (another framework's allocator owns all device memory, or
an allocation would synchronise the device inside a latency-critical loop).
It must give the same populations as the ordinary entry point, on repeated
calls that reuse its fixed scratch array.  This file sorts last so that a
failure here cannot hide failures elsewhere.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fn(tdse_lib):
    f = tdse_lib._lib.tdse_populations_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
    f.restype = ctypes.c_int
    return f


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_populations_match_the_ordinary_entry_point(tdse_lib):
    f = _fn(tdse_lib)
    lmax, n, B = 5, 300, 4
    N = (lmax + 1) * n
    E = inputs.energies(lmax, n)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(lmax, n, 2), lmax, n, "fp64")
    E_dev = torch.from_numpy(E).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):           # two calls in a row share the fixed scratch
        cs = np.stack([inputs.random_state(N, 100 * call + b) * (1 + b) for b in range(B)])
        c = torch.from_numpy(cs.reshape(-1)).cuda()
        ref = H.populations(c, B)
        ps = torch.empty(B, N, dtype=torch.float64, device="cuda")
        pl = torch.empty(B, lmax + 1, dtype=torch.float64, device="cuda")
        bound = torch.empty(B, dtype=torch.float64, device="cuda")
        ion = torch.empty(B, dtype=torch.float64, device="cuda")
        st = f(_p(c), _p(E_dev), lmax, n, B, _p(ps), _p(pl), _p(bound), _p(ion), stream)
        assert st == 0, tdse_lib._lib.tdse_last_error()
        torch.cuda.synchronize()
        # same kernels, same reduction order: equal to the ordinary entry point
        # (the tolerance the other population tests use is 1e-13 relative)
        for got, want in ((ps, ref["per_state"]), (pl, ref["per_l"]), (bound, ref["bound"]), (ion, ref["ionised"])):
            assert torch.allclose(got, want, rtol=1e-13, atol=0.0)
    H.close()


def test_noalloc_rejects_requests_beyond_its_fixed_scratch(tdse_lib):
    f = _fn(tdse_lib)
    lmax, n, B = 31, 4, 600          # 600 * 32 = 19200 (state, block) pairs > 16384
    c = torch.zeros(B * (lmax + 1) * n, dtype=torch.complex128, device="cuda")
    E = torch.zeros((lmax + 1) * n, dtype=torch.float64, device="cuda")
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    st = f(_p(c), _p(E), lmax, n, B, None, None, _p(out), None, None)
    assert st == tdse_lib.EINVAL
    assert b"exceeds" in tdse_lib._lib.tdse_last_error()
