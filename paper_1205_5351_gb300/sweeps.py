"""Range-of-convergence and corruption sweeps of Sec. 6.2 as batched workloads.

The checkerboard grid (rotation x skew) and the corruption levels (0-100 %) of the paper's
robustness experiment are solved as one grouped submission each through the C ABI
(``tilt.Context.submit_batch``); this module only scores the results.  A window counts as
rectified when the recovered linear part maps the window axes onto the texture's axes: with
L_G the rendering transform's linear part and L the recovered one, K = L_G^-1 L must be a
scaled signed permutation (axis-aligned scalings, axis swaps and flips leave a checkerboard
or a separable low-rank texture low-rank), to within ``tol`` in the ratio of its off-pattern
to its on-pattern entries.  tol = 0.05 admits about 3 degrees of residual rotation or skew.
"""
from __future__ import annotations

import numpy as np


def linear_part(tau) -> np.ndarray:
    t = np.asarray(tau, dtype=np.float64)
    return np.array([[t[0], t[1]], [t[3], t[4]]])


def misalignment(tau, tau_true) -> float:
    """Smallest off-pattern ratio of K = L_G^-1 L over the two axis assignments."""
    K = np.linalg.solve(linear_part(tau_true), linear_part(tau))
    a = np.abs(K)
    with np.errstate(divide="ignore", invalid="ignore"):
        diag = max(a[0, 1] / a[0, 0], a[1, 0] / a[1, 1])
        anti = max(a[0, 0] / a[0, 1], a[1, 1] / a[1, 0])
    r = min(diag, anti)
    return float(r) if np.isfinite(r) else float("inf")


def rectified(tau, tau_true, tol: float = 0.05) -> bool:
    return misalignment(tau, tau_true) < tol


def solve(ctx, patches, params=None, on_device: bool = False, timeout_ms: int = 600000):
    """One grouped submission of the patches; returns their result dicts in order."""
    items = [(p.img, p.m, p.n, p.tau0, p.ttype) for p in patches]
    tickets = ctx.submit_batch(items, params, on_device=on_device)
    return [ctx.wait(t, timeout_ms) for t in tickets]


def convergence_map(patches, results, tol: float = 0.05) -> dict:
    """Success over the (rotation, skew) grid of the range-of-convergence experiment."""
    thetas = sorted({p.meta["theta_deg"] for p in patches})
    skews = sorted({p.meta["skew"] for p in patches})
    grid = [[None] * len(skews) for _ in thetas]
    for p, r in zip(patches, results):
        ok = r["status"] >= 0 and rectified(r["tau"], p.tau_true, tol)
        grid[thetas.index(p.meta["theta_deg"])][skews.index(p.meta["skew"])] = int(ok)
    return {"theta_deg": thetas, "skew": skews, "rectified": grid,
            "rate": float(np.mean([v for row in grid for v in row if v is not None]))}


def corruption_rates(patches, results, tol: float = 0.05) -> dict:
    """Fraction of textures rectified at each corruption level of the robustness experiment."""
    levels = sorted({p.meta["corruption"] for p in patches})
    hits = {lv: [] for lv in levels}
    for p, r in zip(patches, results):
        hits[p.meta["corruption"]].append(int(r["status"] >= 0 and rectified(r["tau"], p.tau_true, tol)))
    return {"corruption": levels, "success_rate": [float(np.mean(hits[lv])) for lv in levels],
            "textures": len(hits[levels[0]]) if levels else 0}
