"""The C-ABI library builds, loads without a GPU and exports every symbol the header declares."""
import os
import re
import subprocess

from paper_1205_5351_gb300 import build, tilt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tilt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(tilt_[a-z_]+)\s*\(", src))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (tilt_[a-z_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported
    assert declared == set(tilt.SIGNATURES), declared ^ set(tilt.SIGNATURES)
    L = tilt.lib()
    for name in declared:
        assert getattr(L, name) is not None


def test_default_params_match_oracle_readings():
    from oracle import tilt_oracle as O
    p = tilt.default_params()
    o = O.Params()
    assert (p.eps1, p.eps2, p.rho0, p.mu_max, p.max_inner, p.max_outer, p.outer_tol) == \
           (o.eps1, o.eps2, o.rho0, o.mu_max, o.max_inner, o.max_outer, o.outer_tol)
    assert p.lambda_ <= 0 and p.mu0 <= 0 and o.lam <= 0 and o.mu0 <= 0


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    try:
        tilt.Context(0)
    except tilt.TiltError as e:
        assert e.code in (tilt.TILT_E_INVAL, tilt.TILT_E_CUDA)
    else:
        raise AssertionError("context created without a GPU")
