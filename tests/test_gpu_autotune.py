"""The autotuner picks a Jacobi schedule (group width and pair ordering) per size bucket,
persists it, and solves under every schedule match the oracle."""
import time

import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_autotune_choices_persist_and_keep_parity(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    cache = str(tmp_path / "tune.txt")
    shapes = [(48, 40), (120, 100), (200, 200)]
    with tilt.Context(0, autotune_cache=cache) as ctx:
        chosen = ctx.autotune(shapes, tilt.AFFINE)
    assert all((w & 255) in (4, 8, 16) and (w >> 8) in (0, 1) for w in chosen)
    lines = open(cache).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 3
    with tilt.Context(0, autotune_cache=cache) as ctx:
        t0 = time.perf_counter()
        again = ctx.autotune(shapes, tilt.AFFINE)       # read from the cache: no timing runs
        assert time.perf_counter() - t0 < 0.05
        assert again == chosen
        patches = [p for p in synth.mixed_affine_batch(40, first=700) if max(p.m, p.n) <= 60][:2]
        ctx.autotune([(p.m, p.n) for p in patches], tilt.AFFINE)
        prm = tilt.default_params(max_outer=2)
        res = [ctx.wait(ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm), 300000) for p in patches]
    for p, r in zip(patches, res):
        ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=2))
        assert O.tau_error(r["tau"], ref.tau) <= 1e-3


@pytest.mark.parametrize("schedule", [4, 8, 16, 256 + 4, 256 + 8, 256 + 16])
def test_every_schedule_matches_oracle(tmp_path, schedule, _oracle_cache={}):
    """Each schedule, forced through a cache file, on windows with an odd and an even short
    side (a ragged last column block for the block-cyclic ordering)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    batch = synth.mixed_affine_batch(60, first=900)
    patches = [batch[9], batch[27], batch[32]]          # 47 x 42, 119 x 93, 111 x 112
    cache = tmp_path / "tune.txt"
    cache.write_text("".join("%d %d %d\n" % ((max(p.m, p.n) + 15) // 16, (min(p.m, p.n) + 15) // 16, schedule)
                             for p in patches))
    prm = tilt.default_params(max_outer=2)
    with tilt.Context(0, autotune_cache=str(cache)) as ctx:
        assert ctx.autotune([(p.m, p.n) for p in patches], tilt.AFFINE) == [schedule] * 3
        tickets = [ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm) for p in patches]
        res = [ctx.wait(t, 300000) for t in tickets]
    for q, (p, r) in enumerate(zip(patches, res)):
        if q not in _oracle_cache:
            _oracle_cache[q] = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=2))
        ref = _oracle_cache[q]
        assert O.tau_error(r["tau"], ref.tau) <= 1e-3, (schedule, p.m, p.n)
        assert r["rank"] == ref.rank, (schedule, p.m, p.n)
