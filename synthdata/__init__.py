"""Seeded synthetic inputs shaped like the EFGP paper's workloads.

This module holds no part of the regression method.  It only draws points,
data values and targets from a counter-based generator so that any subset of
a data set (say points 10**8 .. 10**8+999 of a 10**9-point cloud) can be
regenerated exactly, on the host with numpy or on a CUDA device with torch
integer arithmetic.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Draw i of stream (seed, s) is the
SplitMix64 finaliser applied to ``key(seed, s) + (i + 1) * GAMMA`` (mod 2**64).
Uniform floats take the top 24 (float32) or 53 (float64) bits, so the
integer-derived coordinates are bit-identical on both backends.  Normal noise
uses Box-Muller, whose log/cos may differ by an ulp between backends; tests
that need identical data generate it on the host and copy it to the device.

Workload recipes (the paper's workloads are synthetic, Sec. 5 "synthetic data"):
points are iid uniform on [0,1]^d unless a recipe adds clusters, data are a
smooth trigonometric field plus N(0, sigma^2) noise, targets are a tensor grid
{0, 1/n_t, ..., (n_t-1)/n_t}^d or iid uniform points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# stream identifiers (fixed; each recipe draws from its own streams)
S_X = 1          # coordinates: stream S_X*8 + axis
S_NOISE_A = 40   # Box-Muller first uniform
S_NOISE_B = 41   # Box-Muller second uniform
S_FIELD = 50     # random wave vectors / phases of the data field
S_CLUSTER = 60   # cluster membership and centres
S_CLUSTER_N = 70  # cluster offsets (normal): 70 + 2*axis, 71 + 2*axis
S_TARGET = 90    # iid targets: 90*8 + axis


def _fmix_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of stream ``stream`` of seed ``seed`` (pure Python ints)."""
    return _fmix_int(_fmix_int((seed * GAMMA + 0x632BE59BD9B4E019) & MASK64) ^ (stream * M1 & MASK64))


def _u64_np(key: int, idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def uniform_np(seed: int, stream: int, start: int, count: int, dtype=np.float64) -> np.ndarray:
    """Draws start..start+count-1 of a stream as uniforms in [0, 1)."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    z = _u64_np(stream_key(seed, stream), idx)
    if np.dtype(dtype) == np.float32:
        return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal_np(seed: int, stream_a: int, stream_b: int, start: int, count: int) -> np.ndarray:
    """Box-Muller standard normals (float64)."""
    u1 = 1.0 - uniform_np(seed, stream_a, start, count)
    u2 = uniform_np(seed, stream_b, start, count)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------- torch twin
def _signed(v: int) -> int:
    return v - (1 << 64) if v >= (1 << 63) else v


def _u64_torch(key: int, start: int, count: int, device):
    import torch
    idx = torch.arange(start + 1, start + 1 + count, dtype=torch.int64, device=device)
    z = idx * _signed(GAMMA) + _signed(key)            # wraps mod 2**64
    def lsr(v, s):                                     # logical shift right
        return (v >> s) & ((1 << (64 - s)) - 1)
    z = (z ^ lsr(z, 30)) * _signed(M1)
    z = (z ^ lsr(z, 27)) * _signed(M2)
    z = z ^ lsr(z, 31)
    return z, lsr


def uniform_torch(seed: int, stream: int, start: int, count: int, dtype, device):
    """Same draws as :func:`uniform_np`, computed on ``device`` with torch."""
    import torch
    z, lsr = _u64_torch(stream_key(seed, stream), start, count, device)
    if dtype == torch.float32:
        return lsr(z, 40).to(torch.float64).mul_(2.0 ** -24).to(torch.float32)
    return lsr(z, 11).to(torch.float64).mul_(2.0 ** -53)


def normal_torch(seed: int, stream_a: int, stream_b: int, start: int, count: int, device):
    import torch
    u1 = 1.0 - uniform_torch(seed, stream_a, start, count, torch.float64, device)
    u2 = uniform_torch(seed, stream_b, start, count, torch.float64, device)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------- recipes
@dataclass
class Recipe:
    """A synthetic regression problem: where the points lie and what y is."""
    d: int
    n: int
    seed: int
    noise: float                       # standard deviation of the additive noise
    fn: str = "plane"                  # data field: "plane" | "cosines" | "c1"
    omega: tuple = ()                  # wave vector for "plane"
    n_cos: int = 5                     # number of random cosines for "cosines"
    kmax: float = 5.0                  # |k| <= kmax for "cosines"
    cluster_frac: float = 0.0          # fraction of points in Gaussian clusters
    n_clusters: int = 4
    cluster_std: float = 0.05
    coord_dtype: str = "float32"
    value_dtype: str = "float32"
    targets: str = "grid"              # "grid" | "iid"
    n_targets_1d: int = 60             # grid targets per dimension
    n_targets: int = 0                 # iid target count
    extra: dict = field(default_factory=dict)

    # field parameters drawn from the seed (wave vectors and phases)
    def cosines(self):
        r = self.n_cos
        a = uniform_np(self.seed, S_FIELD, 0, 3 * r)
        rad = self.kmax * np.sqrt(a[:r])
        th = 2 * np.pi * a[r:2 * r]
        phi = 2 * np.pi * a[2 * r:3 * r]
        if self.d == 1:
            ks = (rad * np.cos(th))[:, None]
        elif self.d == 2:
            ks = np.stack([rad * np.cos(th), rad * np.sin(th)], 1)
        else:
            b = uniform_np(self.seed, S_FIELD + 1, 0, r)
            cz = 2 * b - 1
            sz = np.sqrt(1 - cz * cz)
            ks = np.stack([rad * sz * np.cos(th), rad * sz * np.sin(th), rad * cz], 1)
        return ks, phi

    def cluster_centres(self):
        c = uniform_np(self.seed, S_CLUSTER + 1, 0, self.n_clusters * self.d)
        return 0.25 + 0.5 * c.reshape(self.n_clusters, self.d)


def _f_np(rec: Recipe, x: np.ndarray) -> np.ndarray:
    """Noise-free data field at points x (n, d), float64."""
    if rec.fn == "plane":
        om = np.asarray(rec.omega, float)
        return np.cos(2 * np.pi * (x @ om) + 1.3)
    if rec.fn == "c1":
        return np.cos(2 * np.pi * 3 * x[:, 0]) + 0.5 * np.sin(2 * np.pi * 7 * x[:, 0])
    ks, phi = rec.cosines()
    return np.cos(2 * np.pi * (x @ ks.T) + phi[None, :]).sum(1)


def points_np(rec: Recipe, start: int = 0, count: int | None = None) -> np.ndarray:
    """Coordinates of points start..start+count-1 as an (count, d) array."""
    count = rec.n - start if count is None else count
    dt = np.float32 if rec.coord_dtype == "float32" else np.float64
    x = np.stack([uniform_np(rec.seed, S_X * 8 + a, start, count, np.float64) for a in range(rec.d)], 1)
    if rec.cluster_frac > 0:
        sel = uniform_np(rec.seed, S_CLUSTER, start, count)
        inc = sel < rec.cluster_frac
        which = np.minimum((sel / rec.cluster_frac * rec.n_clusters).astype(np.int64), rec.n_clusters - 1)
        cen = rec.cluster_centres()
        for a in range(rec.d):
            g = normal_np(rec.seed, S_CLUSTER_N + 2 * a, S_CLUSTER_N + 2 * a + 1, start, count)
            v = cen[which, a] + rec.cluster_std * g
            v = np.abs(v)                   # mirror into [0, 1]
            v = 1.0 - np.abs(1.0 - v)
            v = np.clip(v, 0.0, 1.0)
            x[:, a] = np.where(inc, v, x[:, a])
    if dt == np.float32:
        xf = x.astype(np.float32)
        return np.minimum(xf, np.float32(1.0))
    return x


def values_np(rec: Recipe, x: np.ndarray, start: int = 0) -> np.ndarray:
    n = x.shape[0]
    y = _f_np(rec, x.astype(np.float64)) + rec.noise * normal_np(rec.seed, S_NOISE_A, S_NOISE_B, start, n)
    return y.astype(np.float32 if rec.value_dtype == "float32" else np.float64)


def targets_np(rec: Recipe) -> np.ndarray:
    dt = np.float32 if rec.coord_dtype == "float32" else np.float64
    if rec.targets == "grid":
        g = np.arange(rec.n_targets_1d, dtype=np.float64) / rec.n_targets_1d
        mesh = np.meshgrid(*([g] * rec.d), indexing="ij")
        return np.stack([m.ravel() for m in mesh], 1).astype(dt)
    t = np.stack([uniform_np(rec.seed, S_TARGET * 8 + a, 0, rec.n_targets) for a in range(rec.d)], 1)
    return t.astype(dt)


def make_np(rec: Recipe):
    """(x, y, targets) on the host, x and targets (n, d) row-major."""
    x = points_np(rec)
    y = values_np(rec, x)
    return x, y, targets_np(rec)


def make_torch(rec: Recipe, device, chunk: int = 1 << 26):
    """(x, y) generated on a CUDA device, chunk by chunk (for very large N).

    Coordinates are bit-identical to :func:`points_np` when there are no
    clusters; the data values agree with :func:`values_np` to float rounding.
    """
    import torch
    if rec.cluster_frac > 0:
        raise ValueError("device generation supports unclustered recipes only")
    tdt = torch.float32 if rec.coord_dtype == "float32" else torch.float64
    vdt = torch.float32 if rec.value_dtype == "float32" else torch.float64
    x = torch.empty((rec.n, rec.d), dtype=tdt, device=device)
    y = torch.empty((rec.n,), dtype=vdt, device=device)
    if rec.fn == "cosines":
        ks, phi = rec.cosines()
        ks_t = torch.tensor(ks, dtype=torch.float64, device=device)
        phi_t = torch.tensor(phi, dtype=torch.float64, device=device)
    for s in range(0, rec.n, chunk):
        c = min(chunk, rec.n - s)
        xs = torch.stack([uniform_torch(rec.seed, S_X * 8 + a, s, c, torch.float64, device)
                          for a in range(rec.d)], 1)
        if tdt == torch.float32:
            xs = torch.clamp(xs.to(torch.float32), max=1.0)
        x[s:s + c] = xs
        xd = xs.to(torch.float64)
        if rec.fn == "plane":
            om = torch.tensor(rec.omega, dtype=torch.float64, device=device)
            f = torch.cos(2 * math.pi * (xd @ om) + 1.3)
        elif rec.fn == "c1":
            f = torch.cos(2 * math.pi * 3 * xd[:, 0]) + 0.5 * torch.sin(2 * math.pi * 7 * xd[:, 0])
        else:
            f = torch.zeros(c, dtype=torch.float64, device=device)
            for r in range(ks_t.shape[0]):
                f += torch.cos(2 * math.pi * (xd @ ks_t[r]) + phi_t[r])
        f += rec.noise * normal_torch(rec.seed, S_NOISE_A, S_NOISE_B, s, c, device)
        y[s:s + c] = f.to(vdt)
        del xs, xd, f
    return x, y


# ------------------------------------------------- named workloads
def config(name: str, n: int | None = None) -> Recipe:
    """Named workloads.  ``n`` overrides the point count (N-reduced twins)."""
    if name == "se1d":          # 1D SE, l=0.1, sigma=0.3, eps=1e-6, N=1e4, float64
        r = Recipe(d=1, n=10_000, seed=1, noise=0.3, fn="c1", coord_dtype="float64",
                   value_dtype="float64", targets="grid", n_targets_1d=500)
    elif name == "matern2d":    # 2D Matern-3/2, l=0.1, sigma=0.3, eps=1e-4, N=1e6
        r = Recipe(d=2, n=1_000_000, seed=2, noise=0.3, fn="cosines", n_cos=5, kmax=5.0,
                   targets="iid", n_targets=100_000)
    elif name == "se3d":        # 3D SE, l=0.2, sigma=0.5, eps=1e-5, N=1e7, 30% clustered
        r = Recipe(d=3, n=10_000_000, seed=3, noise=0.5, fn="plane",
                   omega=(3 / math.sqrt(14), 9 / math.sqrt(14), 6 / math.sqrt(14)),
                   cluster_frac=0.3, n_clusters=4, cluster_std=0.05,
                   targets="grid", n_targets_1d=100)
    elif name == "matern2d_1e9":  # 2D Matern-3/2, l=0.05, sigma=0.5, eps=1e-3, N=1e9
        r = Recipe(d=2, n=1_000_000_000, seed=4, noise=0.5, fn="cosines", n_cos=8, kmax=5.0,
                   targets="grid", n_targets_1d=1000)
    elif name == "matern2d_table4":  # the paper's Table 4 shape: l=0.1, sigma=0.1, eps=1e-5
        r = Recipe(d=2, n=1_000_000_000, seed=5, noise=0.1, fn="plane", omega=(3.0, 4.0),
                   targets="grid", n_targets_1d=1000)
    elif name == "matern2d_table5":  # Table 5 regime: N / sigma^2 = 3e8 fixed, sigma = 1.83 at N = 1e9
        r = Recipe(d=2, n=1_000_000_000, seed=7, noise=TABLE5_SIGMA, fn="plane", omega=(3.0, 4.0),
                   targets="grid", n_targets_1d=1000)
    elif name == "batch_largest":  # the batch's largest FFT grid: Matern-1/2 l=0.0341, L = 2625
        r = Recipe(d=2, n=1_000_000, seed=77, noise=0.1115, fn="cosines", n_cos=5, kmax=5.0,
                   targets="iid", n_targets=10_000)
    else:
        raise KeyError(name)
    if n is not None:
        r.n = int(n)
    return r


# GP model of each named workload: (family, nu, lengthscale, sigma, eps)
# Sec. 5.4, Table 5: noise and regression sigma grow as sqrt(N / 3e8)
TABLE5_SIGMA = math.sqrt(1e9 / 3e8)

MODELS = {
    "se1d": ("se", 0.0, 0.1, 0.3, 1e-6),
    "matern2d": ("matern", 1.5, 0.1, 0.3, 1e-4),
    "se3d": ("se", 0.0, 0.2, 0.5, 1e-5),
    "matern2d_1e9": ("matern", 1.5, 0.05, 0.5, 1e-3),
    "matern2d_table4": ("matern", 1.5, 0.1, 0.1, 1e-5),
    "matern2d_table5": ("matern", 1.5, 0.1, TABLE5_SIGMA, 1e-5),
    "batch_largest": ("matern", 0.5, 0.0341, 0.1115, 1e-4),
}


def batch_problems(seed: int = 6, count: int = 64, n_lo: float = 1e4, n_hi: float = 1e7):
    """The heterogeneous batch: 2D Matern-1/2 and 3/2 problems of uneven size.

    Returns a list of (Recipe, (family, nu, lengthscale, sigma, eps)).
    N is log-uniform in [n_lo, n_hi], lengthscale U[0.03, 0.3], sigma U[0.1, 1].
    """
    u = uniform_np(seed, 100, 0, 3 * count).reshape(3, count)
    out = []
    for i in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[0, i] * (math.log(n_hi) - math.log(n_lo)))))
        ell = 0.03 + 0.27 * u[1, i]
        sig = 0.1 + 0.9 * u[2, i]
        nu = 0.5 if i % 2 == 0 else 1.5
        rec = Recipe(d=2, n=n, seed=1000 + i, noise=sig, fn="cosines", n_cos=5, kmax=5.0,
                     targets="iid", n_targets=10_000)
        out.append((rec, ("matern", nu, ell, sig, 1e-4)))
    return out
