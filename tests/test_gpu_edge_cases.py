"""Edge cases of the CUDA path through the C ABI: a window partly outside the image (clamped
samples, counted as in the oracle), degenerate windows (zero image: status -3; constant image:
singular J^T J + Q^T Q, status -2; a non-finite sample: status -1), the caller's stream, an
empty batch, and the largest window size end to end."""
import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    return tilt


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("ttype", [6, 8])
def test_window_partly_outside_the_image(T, ttype):
    # the window centre is moved to 10 px from the left edge: about 40 % of the samples clamp
    rng = np.random.default_rng(5)
    p = synth.make_patch(rng, 48, 64, kind="lowrank", rank=3, theta_deg=8.0, skew=0.05, ttype=ttype)
    tau = np.array(p.tau0, np.float64)
    tau[2] = 10.0
    with T.Context(0) as ctx:
        Dh_d, J_d, norm, oob = ctx.warp_jacobian(torch.from_numpy(p.img).cuda(), p.m, p.n, tau, ttype)
    Dref, Jref, sref, oref = O.warp_normalise_jacobian(p.img.astype(np.float64), tau, ttype, p.m, p.n)
    assert oref > 0.2 * p.m * p.n
    assert oob == oref
    assert abs(norm - sref) <= 1e-6 * sref
    assert rel(T.from_long_layout(Dh_d.cpu().numpy(), p.m, p.n), Dref) <= 1e-5
    assert rel(T.jacobian_to_rows(J_d.cpu().numpy(), p.m, p.n, ttype), Jref) <= 1e-5


def test_degenerate_windows_report_their_status(T):
    m, n = 40, 52
    tau0 = [1.0, 0.0, 60.0, 0.0, 1.0, 50.0]
    zero = np.zeros((100, 120), np.float32)
    flat = np.full((100, 120), 0.5, np.float32)
    with T.Context(0) as ctx:
        # one at a time (persistent workers) and as a grouped launch
        r0 = ctx.wait(ctx.submit(zero, m, n, tau0, 6), 60000)
        r1 = ctx.wait(ctx.submit(flat, m, n, tau0, 6), 60000)
        tk = ctx.submit_batch([(zero, m, n, tau0, 6), (flat, m, n, tau0, 6)], None)
        rb = [ctx.wait(t, 60000) for t in tk]
    for r in (r0, rb[0]):
        assert r["status"] == -3                       # ||D o tau|| = 0: nothing to normalise
        np.testing.assert_array_equal(r["tau"], tau0)
    for r in (r1, rb[1]):
        assert r["status"] == -2                       # zero image gradient: J = 0, G = Q^T Q is rank 3
        np.testing.assert_array_equal(r["tau"], tau0)


def test_non_finite_window_reports_status_minus_one(T):
    # a NaN written into the host image inside the window (host-side injection): the warp
    # sees a non-finite sample, both submit paths retire the problem with status -1 and
    # keep tau0; a problem in the same batch with a clean image is unaffected
    p = synth.small_affine(3)
    bad = p.img.copy()
    bad[bad.shape[0] // 2, bad.shape[1] // 2] = np.nan
    prm = T.default_params(max_outer=2)
    with T.Context(0) as ctx:
        r0 = ctx.wait(ctx.submit(bad, p.m, p.n, p.tau0, p.ttype, prm), 60000)
        tk = ctx.submit_batch([(bad, p.m, p.n, p.tau0, p.ttype), (p.img, p.m, p.n, p.tau0, p.ttype)], prm)
        rb = [ctx.wait(t, 60000) for t in tk]
    for r in (r0, rb[0]):
        assert r["status"] == -1
        np.testing.assert_array_equal(r["tau"], p.tau0)
    assert rb[1]["status"] >= 0
    ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=2))
    assert O.tau_error(rb[1]["tau"], ref.tau) <= 1e-3


def test_caller_stream_carries_the_context(T):
    # tilt_config.cuda_stream: grouped launches, copies and steps on the caller's stream give
    # the same results as the context's own streams (bit for bit: same kernels, same inputs)
    patches = [q for q in synth.mixed_affine_batch(12, first=40) if max(q.m, q.n) <= 80][:3]
    prm = T.default_params(max_outer=2)
    items = [(q.img, q.m, q.n, q.tau0, q.ttype) for q in patches]
    with T.Context(0) as ctx:
        want = [ctx.wait(t, 300000) for t in ctx.submit_batch(items, prm)]
    st = torch.cuda.Stream()
    with T.Context(0, cuda_stream=st.cuda_stream) as ctx:
        got = [ctx.wait(t, 300000) for t in ctx.submit_batch(items, prm)]
        Dh, J, norm, oob = ctx.warp_jacobian(torch.from_numpy(patches[0].img).cuda(), patches[0].m,
                                             patches[0].n, patches[0].tau0, 6)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g["tau"], w["tau"])
        assert g["inner_iters"] == w["inner_iters"]
    assert norm > 0


def test_empty_batch(T):
    with T.Context(0) as ctx:
        assert ctx.submit_batch([], None) == []
        # the context still works afterwards
        p = synth.small_affine(0)
        r = ctx.wait(ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, T.default_params(max_outer=1)), 60000)
        assert r["status"] in (0, 1, 2)


def test_largest_window_end_to_end(T):
    # 512 x 512 (no SVD buffer fits in shared memory): one outer step of a few inner iterations
    p = synth.multistart_batch(1)[0]
    prm = T.default_params(max_outer=1, max_inner=6)
    with T.Context(0) as ctx:
        r = ctx.wait(ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm), 600000)
    ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=1, max_inner=6))
    assert r["inner_iters"] == ref.inner_iters == 6
    assert O.tau_error(r["tau"], ref.tau) <= 1e-3
    assert r["rank"] == ref.rank
