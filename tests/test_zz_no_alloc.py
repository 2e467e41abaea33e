"""tilt_svt_noalloc: the allocation-free SVT entry point must give what tilt_svt gives, and
what the FP64 oracle gives, without allocating device memory.

Collected last on purpose: if it fails, a run that stops at the first failure has already
run every other test.  It creates its own context for the reference call, so it passes both
alone in a fresh process and after the other tests."""
import ctypes
import math

import numpy as np
import pytest

from oracle import tilt_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(seed, m, n):
    rng = np.random.default_rng(seed)
    r = min(m, n) // 6
    M = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) / math.sqrt(n)
         + 0.02 * rng.standard_normal((m, n))).astype(np.float32)
    eps = float(np.linalg.svd(M.astype(np.float64), compute_uv=False)[r] * 1.5)
    return M, eps


def test_svt_noalloc_matches_svt_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    L = tilt.lib()
    ctx = tilt.Context(0)
    try:
        # one call with the SVD buffers in shared memory, one with them in the scratch array
        for seed, m, n in ((1, 96, 72), (2, 200, 180)):
            M, eps = _case(seed, m, n)
            M_d = torch.from_numpy(tilt.to_long_layout(M)).cuda()
            A_ref, sig_ref, _ = ctx.svt(M_d, m, n, eps)
            A = torch.full_like(M_d, float("nan"))
            sig = torch.full((min(m, n),), float("nan"), device="cuda")
            rc = L.tilt_svt_noalloc(M_d.data_ptr(), m, n, ctypes.c_float(eps), A.data_ptr(), sig.data_ptr(), None)
            assert rc == 0, L.tilt_last_error(None)
            torch.cuda.synchronize()
            A_ref = A_ref.cpu().numpy().astype(np.float64)
            err = np.linalg.norm(A.cpu().numpy() - A_ref) / np.linalg.norm(A_ref)
            assert err <= 1e-5, (m, n, err)
            np.testing.assert_allclose(np.sort(sig.cpu().numpy()), np.sort(sig_ref), rtol=1e-5, atol=1e-6)
            # and the FP64 oracle's S_eps(M) (Eq. S_operator)
            A_or = O.svt(M.astype(np.float64), eps)[0]
            got = tilt.from_long_layout(A.cpu().numpy(), m, n)
            assert np.linalg.norm(got - A_or) <= 1e-5 * np.linalg.norm(A_or)
        # sizes beyond the scratch limit are rejected without a launch
        big = torch.zeros(300 * 10, device="cuda")
        assert L.tilt_svt_noalloc(big.data_ptr(), 300, 10, ctypes.c_float(0.1), big.data_ptr(), None, None) == \
            tilt.TILT_E_INVAL
    finally:
        ctx.close()


def test_svt_noalloc_allocates_nothing_and_runs_on_the_given_stream():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    L = tilt.lib()
    m, n = 150, 120
    M, eps = _case(3, m, n)
    M_d = torch.from_numpy(tilt.to_long_layout(M)).cuda()
    A = torch.empty_like(M_d)
    torch.cuda.synchronize()
    # the first call on a device does the one-time set-up (symbol address, kernel attributes)
    assert L.tilt_svt_noalloc(M_d.data_ptr(), m, n, ctypes.c_float(eps), A.data_ptr(), None, None) == 0
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    outs = [torch.full_like(M_d, float("nan")) for _ in range(5)]   # every buffer exists before
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for A2 in outs:
        rc = L.tilt_svt_noalloc(M_d.data_ptr(), m, n, ctypes.c_float(eps), A2.data_ptr(), None,
                                ctypes.c_void_p(st.cuda_stream))
        assert rc == 0, L.tilt_last_error(None)
    st.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    A_or = O.svt(M.astype(np.float64), eps)[0]
    for A2 in outs:
        got = tilt.from_long_layout(A2.cpu().numpy(), m, n)
        assert np.linalg.norm(got - A_or) <= 1e-5 * np.linalg.norm(A_or)
