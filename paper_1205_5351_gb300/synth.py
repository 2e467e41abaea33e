"""Seeded synthetic TILT inputs: low-rank or checkerboard textures rendered under a
known affine or projective transform, with Gaussian noise and sparse corruption.

This module holds none of the solver's arithmetic.  It draws random numbers, evaluates
a continuous, periodic texture at inverse-mapped canvas points and writes images; the
CUDA path and the FP64 oracle both take its outputs as their inputs.

Texture model (Sec. 2.1 of the paper: a low-rank texture is a matrix of rank r << min(m, n)):

* ``lowrank``: T(u, v) = sum_k a_k(v) b_k(u), where a_k and b_k are periodic,
  piecewise-linear curves through N(0, 1) knots spaced ``cell`` pixels apart, rescaled to
  [0, 1].  Sampled on an axis-aligned grid it has rank <= r + 1 (the rescale adds a
  constant).
* ``checker``: T = 1/2 + 1/2 sq(u) sq(v) with sq a +-1 square wave of period ``period``
  and a one-pixel linear ramp at each edge (rank 2 on an axis-aligned grid).

The canvas pixel (x = column, y = row) shows T at tau_G^{-1}(x, y), where tau_G maps
centred window coordinates (u, v) to canvas coordinates with the homography
[[L11, L12, cx], [L21, L22, cy], [h7, h8, 1]] and L = R(theta) [[1, t], [0, 1]] (the
rotation/skew family of the paper's range-of-convergence experiment, Sec. 6.2).
Corruption replaces a fraction of canvas pixels by Uniform[0, 1] values (Sec. 6.2,
robustness experiment, with intensities scaled to [0, 1]).

Seeds: every patch draws from ``numpy.random.default_rng(config_index * 10**6 + index)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AFFINE = 6
PROJECTIVE = 8


@dataclasses.dataclass
class Patch:
    """One TILT problem: a canvas image and the window to rectify."""

    img: np.ndarray          # (H, W) float32 canvas, row-major
    m: int                   # window rows
    n: int                   # window columns
    ttype: int               # AFFINE (6) or PROJECTIVE (8)
    tau0: np.ndarray         # (p,) float64 initial transform
    tau_true: np.ndarray     # (p,) float64 transform used to render the canvas
    meta: dict

    @property
    def p(self) -> int:
        return self.ttype


# ----------------------------------------------------------------------------- textures
def _periodic_linear(knots: np.ndarray, cell: float, t: np.ndarray) -> np.ndarray:
    """Periodic piecewise-linear curve through ``knots`` spaced ``cell`` apart."""
    s = np.asarray(t, dtype=np.float64) / cell
    k0 = np.floor(s)
    f = s - k0
    L = knots.shape[-1]
    i0 = np.mod(k0.astype(np.int64), L)
    i1 = np.mod(i0 + 1, L)
    return (1.0 - f) * knots[..., i0] + f * knots[..., i1]


class LowRankTexture:
    def __init__(self, rng: np.random.Generator, rank: int, cell: float, nknots: int):
        self.rank = int(rank)
        self.cell = float(cell)
        self.a = rng.standard_normal((self.rank, nknots))
        self.b = rng.standard_normal((self.rank, nknots))
        # The texture is bilinear on every knot cell, so its extremes sit on the knot lattice.
        lattice = np.einsum("ki,kj->ij", self.a, self.b)
        self.lo = float(lattice.min())
        self.hi = float(lattice.max())

    def __call__(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(u, v).shape)
        for k in range(self.rank):
            out += _periodic_linear(self.a[k], self.cell, v) * _periodic_linear(self.b[k], self.cell, u)
        return (out - self.lo) / (self.hi - self.lo)


class CheckerTexture:
    def __init__(self, period: float, ramp: float = 1.0):
        self.period = float(period)
        self.ramp = float(ramp)

    def _sq(self, t: np.ndarray) -> np.ndarray:
        P = self.period
        tri = np.abs(np.mod(np.asarray(t, dtype=np.float64) / P, 1.0) - 0.5) * 4.0 - 1.0
        return np.clip(tri * (P / (2.0 * self.ramp)), -1.0, 1.0)

    def __call__(self, u: np.ndarray, v: np.ndarray) -> np.ndarray:
        return 0.5 + 0.5 * self._sq(u) * self._sq(v)


# ----------------------------------------------------------------------------- transforms
def linear_part(theta_deg: float, skew: float) -> np.ndarray:
    """L = R(theta) [[1, t], [0, 1]]."""
    th = math.radians(theta_deg)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    return R @ np.array([[1.0, skew], [0.0, 1.0]])


def tau_vector(L: np.ndarray, cx: float, cy: float, persp=(0.0, 0.0), ttype: int = AFFINE) -> np.ndarray:
    """Pack a transform as [L11, L12, cx, L21, L22, cy(, h7, h8)]."""
    t = [L[0, 0], L[0, 1], cx, L[1, 0], L[1, 1], cy]
    if ttype == PROJECTIVE:
        t += [persp[0], persp[1]]
    return np.asarray(t, dtype=np.float64)


def _render(texture, H: int, W: int, L: np.ndarray, cx: float, cy: float, persp) -> np.ndarray:
    Hm = np.array([[L[0, 0], L[0, 1], cx], [L[1, 0], L[1, 1], cy], [persp[0], persp[1], 1.0]])
    Hinv = np.linalg.inv(Hm)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    uw = Hinv[0, 0] * xs + Hinv[0, 1] * ys + Hinv[0, 2]
    vw = Hinv[1, 0] * xs + Hinv[1, 1] * ys + Hinv[1, 2]
    ww = Hinv[2, 0] * xs + Hinv[2, 1] * ys + Hinv[2, 2]
    return texture(uw / ww, vw / ww)


def make_patch(
    rng: np.random.Generator,
    m: int,
    n: int,
    *,
    kind: str = "lowrank",
    rank: int = 3,
    period: float = 8.0,
    cell: float | None = None,
    theta_deg: float = 0.0,
    skew: float = 0.0,
    persp=(0.0, 0.0),
    ttype: int = AFFINE,
    noise_sigma: float = 0.0,
    corruption: float = 0.0,
    canvas: tuple[int, int] | None = None,
    start_theta_deg: float = 0.0,
) -> Patch:
    """Render one patch.  The window starts centred on the canvas with linear part
    R(start_theta_deg) (identity by default)."""
    side = max(m, n)
    if canvas is None:
        canvas = (2 * side + 8, 2 * side + 8)
    H, W = canvas
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    if kind == "lowrank":
        if cell is None:
            cell = max(3.0, side / 10.0)
        nknots = int(math.ceil(4 * side / cell)) + 2
        tex = LowRankTexture(rng, rank, cell, nknots)
    elif kind == "checker":
        tex = CheckerTexture(period)
    else:
        raise ValueError(kind)
    L = linear_part(theta_deg, skew)
    if ttype == AFFINE:
        persp = (0.0, 0.0)
    img = _render(tex, H, W, L, cx, cy, persp)
    if noise_sigma > 0:
        img = img + noise_sigma * rng.standard_normal(img.shape)
    if corruption > 0:
        mask = rng.random(img.shape) < corruption
        img = np.where(mask, rng.random(img.shape), img)
    tau_true = tau_vector(L, cx, cy, persp, ttype)
    tau0 = tau_vector(linear_part(start_theta_deg, 0.0), cx, cy, (0.0, 0.0), ttype)
    meta = dict(kind=kind, rank=rank, period=period, cell=cell, theta_deg=theta_deg, skew=skew,
                persp=tuple(persp), noise_sigma=noise_sigma, corruption=corruption,
                start_theta_deg=start_theta_deg)
    return Patch(np.ascontiguousarray(img, dtype=np.float32), int(m), int(n), int(ttype),
                 tau0, tau_true, meta)


def seed_for(config_index: int, index: int) -> int:
    return config_index * 10**6 + index


# ----------------------------------------------------------------------------- workloads
def small_affine(index: int = 0) -> Patch:
    """One 50x50 affine patch: rank-3 texture, rotation 20 deg, skew 0.15, 5 % corruption."""
    rng = np.random.default_rng(seed_for(0, index))
    return make_patch(rng, 50, 50, kind="lowrank", rank=3, theta_deg=20.0, skew=0.15,
                      corruption=0.05, ttype=AFFINE)


def mixed_affine_batch(count: int = 1024, first: int = 0) -> list[Patch]:
    """Affine patches with sides uniform in 40..120 (independent m, n); half rank-1..5
    textures, half checkerboards of period 4..16; rotation +-30 deg, skew +-0.2,
    corruption 0..10 %."""
    out = []
    for i in range(first, first + count):
        rng = np.random.default_rng(seed_for(1, i))
        m = int(rng.integers(40, 121))
        n = int(rng.integers(40, 121))
        lowrank = rng.random() < 0.5
        rank = int(rng.integers(1, 6))
        period = float(rng.integers(4, 17))
        theta = float(rng.uniform(-30.0, 30.0))
        skew = float(rng.uniform(-0.2, 0.2))
        corr = float(rng.uniform(0.0, 0.10))
        out.append(make_patch(rng, m, n, kind="lowrank" if lowrank else "checker", rank=rank,
                              period=period, theta_deg=theta, skew=skew, corruption=corr,
                              ttype=AFFINE))
    return out


def projective_batch(count: int = 256, first: int = 0, side: int = 200) -> list[Patch]:
    """Projective 200x200 patches: rank-4 texture + N(0, 0.01^2) noise, rotation +-25 deg,
    skew +-0.2, perspective terms +-1e-3, 10 % corruption."""
    out = []
    for i in range(first, first + count):
        rng = np.random.default_rng(seed_for(2, i))
        theta = float(rng.uniform(-25.0, 25.0))
        skew = float(rng.uniform(-0.2, 0.2))
        persp = (float(rng.uniform(-1e-3, 1e-3)), float(rng.uniform(-1e-3, 1e-3)))
        out.append(make_patch(rng, side, side, kind="lowrank", rank=4, theta_deg=theta,
                              skew=skew, persp=persp, ttype=PROJECTIVE, noise_sigma=0.01,
                              corruption=0.10))
    return out


def served_stream(count: int, rate_hz: float = 2000.0, first: int = 0):
    """Poisson arrivals: returns (arrival_times_s, patches).  Sides uniform in 32..256,
    half affine / half projective, rank 1..6, corruption 0..15 %."""
    rng0 = np.random.default_rng(seed_for(3, 999_999))
    gaps = rng0.exponential(1.0 / rate_hz, size=first + count)
    times = np.cumsum(gaps)[first:]
    times = times - (times[0] if count else 0.0)
    patches = []
    for i in range(first, first + count):
        rng = np.random.default_rng(seed_for(3, i))
        m = int(rng.integers(32, 257))
        n = int(rng.integers(32, 257))
        ttype = AFFINE if rng.random() < 0.5 else PROJECTIVE
        rank = int(rng.integers(1, 7))
        theta = float(rng.uniform(-25.0, 25.0))
        skew = float(rng.uniform(-0.2, 0.2))
        persp = (float(rng.uniform(-1e-3, 1e-3)), float(rng.uniform(-1e-3, 1e-3)))
        corr = float(rng.uniform(0.0, 0.15))
        patches.append(make_patch(rng, m, n, kind="lowrank", rank=rank, theta_deg=theta, skew=skew,
                                  persp=persp, ttype=ttype, corruption=corr))
    return times, patches


MULTISTART_ANGLES = tuple(float(a) for a in range(-40, 41, 10))


def multistart_batch(count: int = 64, first: int = 0, side: int = 512) -> list[Patch]:
    """Large projective patches, rank-5 texture, 10 % corruption; each patch appears nine
    times with initial rotations -40..40 deg in 10 deg steps (``meta['group']`` names the
    source patch)."""
    out = []
    for i in range(first, first + count):
        rng = np.random.default_rng(seed_for(4, i))
        theta = float(rng.uniform(-25.0, 25.0))
        skew = float(rng.uniform(-0.2, 0.2))
        persp = (float(rng.uniform(-1e-3, 1e-3)), float(rng.uniform(-1e-3, 1e-3)))
        base = make_patch(rng, side, side, kind="lowrank", rank=5, theta_deg=theta, skew=skew,
                          persp=persp, ttype=PROJECTIVE, corruption=0.10)
        cx, cy = base.tau0[2], base.tau0[5]
        for a in MULTISTART_ANGLES:
            tau0 = tau_vector(linear_part(a, 0.0), cx, cy, (0.0, 0.0), PROJECTIVE)
            meta = dict(base.meta, start_theta_deg=a, group=i)
            out.append(Patch(base.img, side, side, PROJECTIVE, tau0, base.tau_true, meta))
    return out


# Range-of-convergence grid of Sec. 6.2: rotation 0 .. pi/6 in steps of pi/60, skew 0 .. 1 in
# steps of 0.05.
CONVERGENCE_THETAS = tuple(3.0 * i for i in range(11))
CONVERGENCE_SKEWS = tuple(round(0.05 * j, 2) for j in range(21))


def convergence_grid(count: int | None = None, first: int = 0, side: int = 60, period: float = 12.0) -> list[Patch]:
    """Checkerboards deformed by A(theta, t) = R(theta) [[1, t], [0, 1]] over the grid of
    CONVERGENCE_THETAS x CONVERGENCE_SKEWS (patch index = theta index * 21 + skew index), each
    to be rectified from the identity (the range-of-convergence experiment, Sec. 6.2)."""
    total = len(CONVERGENCE_THETAS) * len(CONVERGENCE_SKEWS)
    count = total - first if count is None else count
    out = []
    for idx in range(first, first + count):
        i, j = divmod(idx % total, len(CONVERGENCE_SKEWS))
        rng = np.random.default_rng(seed_for(5, idx))
        p = make_patch(rng, side, side, kind="checker", period=period, theta_deg=CONVERGENCE_THETAS[i],
                       skew=CONVERGENCE_SKEWS[j], ttype=AFFINE)
        p.meta["grid"] = (i, j)
        out.append(p)
    return out


# Corruption levels of the robustness experiment of Sec. 6.2: 0 .. 100 % in steps of 5 %.
CORRUPTION_LEVELS = tuple(round(0.05 * i, 2) for i in range(21))


def corruption_sweep(count: int | None = None, first: int = 0, textures: int = 10, side: int = 60) -> list[Patch]:
    """Rank-3 textures rotated by 10 degrees with a fraction of their pixels replaced by
    Uniform[0, 1] values, every level of CORRUPTION_LEVELS for each of ``textures`` textures
    (patch index = texture * 21 + level index; the robustness experiment, Sec. 6.2).  A
    texture draws the same random numbers at every level, so its corrupted pixel sets are
    nested as the level grows."""
    total = textures * len(CORRUPTION_LEVELS)
    count = total - first if count is None else count
    out = []
    for idx in range(first, first + count):
        k, lv = divmod(idx % total, len(CORRUPTION_LEVELS))
        rng = np.random.default_rng(seed_for(6, k))
        p = make_patch(rng, side, side, kind="lowrank", rank=3, theta_deg=10.0,
                       corruption=CORRUPTION_LEVELS[lv], ttype=AFFINE)
        p.meta["sweep"] = (k, lv)
        out.append(p)
    return out


def random_inner_problem(rng: np.random.Generator, m: int, n: int, p: int = 6):
    """Inputs of the inner-loop-only experiment (Sec. 6.1): D o tau with iid Uniform[0, 1]
    entries and a Jacobian with iid N(0, 1) entries (mn x p, rows in row-major pixel order)."""
    D = rng.random((m, n))
    J = rng.standard_normal((m * n, p))
    return D, J


# ----------------------------------------------------------------------------- RASL image sets
@dataclasses.dataclass
class RaslSet:
    """One RASL problem: ``nimg`` images of the same low-rank scene, each seen through its
    own transform, to be aligned jointly (one window of m x n pixels per image, the vectorised
    windows forming the columns of the data matrix)."""

    imgs: np.ndarray         # (nimg, H, W) float32 canvases, row-major
    m: int                   # window rows
    n: int                   # window columns
    ttype: int               # AFFINE (6) or PROJECTIVE (8)
    tau0: np.ndarray         # (nimg, p) float64 initial transforms
    tau_true: np.ndarray     # (nimg, p) float64 transforms used to render the canvases
    meta: dict

    @property
    def nimg(self) -> int:
        return int(self.imgs.shape[0])

    @property
    def p(self) -> int:
        return self.ttype


def rasl_set(rng: np.random.Generator, nimg: int, m: int, n: int, *, rank: int = 2,
             max_rot_deg: float = 3.0, max_scale: float = 0.03, max_shift: float = 1.5,
             corruption: float = 0.02, noise_sigma: float = 0.0, ttype: int = AFFINE,
             pad: int | None = None, cell: float | None = None) -> RaslSet:
    """Render ``nimg`` views of one rank-``rank`` texture.  View i shows
    g_i T + o_i (gain g_i ~ U[0.6, 1.4], offset o_i ~ U[0, 0.2]: the aligned windows form a
    matrix of rank <= 2) under the similarity s_i R(theta_i) with theta_i ~ U[-max_rot_deg,
    max_rot_deg], s_i ~ 1 + U[-max_scale, max_scale] and a centre shifted by U[-max_shift,
    max_shift] pixels on each axis, with a fraction ``corruption`` of its pixels replaced by
    Uniform[0, 1] values (occlusion / specularity).  Every view starts from the same window,
    centred on the canvas with the identity linear part."""
    side = max(m, n)
    pad = max(4, side // 2) if pad is None else int(pad)
    H, W = m + 2 * pad, n + 2 * pad
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    cell = max(3.0, side / 6.0) if cell is None else float(cell)
    nknots = int(math.ceil(4 * (side + 2 * pad) / cell)) + 2
    tex = LowRankTexture(rng, rank, cell, nknots)
    gains = rng.uniform(0.6, 1.4, nimg)
    offsets = rng.uniform(0.0, 0.2, nimg)
    imgs = np.empty((nimg, H, W), dtype=np.float32)
    p = ttype
    tau_true = np.empty((nimg, p))
    for i in range(nimg):
        th = float(rng.uniform(-max_rot_deg, max_rot_deg))
        s = 1.0 + float(rng.uniform(-max_scale, max_scale))
        dx, dy = rng.uniform(-max_shift, max_shift, 2)
        L = s * linear_part(th, 0.0)
        img = gains[i] * _render(tex, H, W, L, cx + dx, cy + dy, (0.0, 0.0)) + offsets[i]
        if noise_sigma > 0:
            img = img + noise_sigma * rng.standard_normal(img.shape)
        if corruption > 0:
            mask = rng.random(img.shape) < corruption
            img = np.where(mask, rng.random(img.shape), img)
        imgs[i] = img
        tau_true[i] = tau_vector(L, cx + dx, cy + dy, (0.0, 0.0), ttype)
    tau0 = np.tile(tau_vector(np.eye(2), cx, cy, (0.0, 0.0), ttype), (nimg, 1))
    meta = dict(rank=rank, max_rot_deg=max_rot_deg, max_scale=max_scale, max_shift=max_shift,
                corruption=corruption, noise_sigma=noise_sigma, gains=gains, offsets=offsets)
    return RaslSet(imgs, int(m), int(n), int(ttype), tau0, tau_true, meta)


def rasl_batch(count: int = 152, first: int = 0, nimg: int = 32, side: int = 32,
               ttype: int = AFFINE) -> list[RaslSet]:
    """Independent RASL problems: ``nimg`` views of a rank-2 texture in ``side`` x ``side``
    windows each (rotation +-3 deg, scale +-3 %, shift +-1.5 px, 2 % corrupted pixels)."""
    out = []
    for i in range(first, first + count):
        rng = np.random.default_rng(seed_for(9, i))
        out.append(rasl_set(rng, nimg, side, side, ttype=ttype))
    return out
