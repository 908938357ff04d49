"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the discretisation: it only draws meshes,
fields and random vectors.  Connectivity, bases, quadrature and operators are
computed independently by the library and by the oracle.

Mesh family (stand-in for the paper's unstructured triangulations, Sec. 2.1):
an N x N periodic grid on the unit torus whose vertices are jittered by
U[-0.15h, 0.15h] in each coordinate and whose squares are split along a
seeded coin-flip diagonal.  Draw order: one (N, N, 2) uniform array indexed
[iy, ix, coord], then one (N, N) array of coin flips indexed [iy, ix].
Vertex (ix, iy) has id iy*N + ix.  Square (ix, iy) has corners
a=(ix,iy), b=(ix+1,iy), c=(ix+1,iy+1), d=(ix,iy+1) (indices mod N); coin 0
gives triangles (a,b,c), (a,c,d) and coin 1 gives (a,b,d), (b,c,d), all
counter-clockwise.  Triangle id = 2*(iy*N + ix) + t.
"""
from __future__ import annotations

import numpy as np

JITTER = 0.15


def jittered_periodic_mesh(N: int, seed: int, jitter: float = JITTER):
    """Return (xy f64[N*N, 2], tri i32[2*N*N, 3], period f64[2])."""
    if N < 1:
        raise ValueError("N must be positive")
    rng = np.random.default_rng(seed)
    u = rng.uniform(-jitter, jitter, size=(N, N, 2))
    coin = rng.integers(0, 2, size=(N, N))
    h = 1.0 / N
    iy, ix = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    xy = np.empty((N, N, 2), dtype=np.float64)
    xy[..., 0] = (ix + u[..., 0]) * h
    xy[..., 1] = (iy + u[..., 1]) * h
    xy = xy.reshape(N * N, 2)

    def vid(x, y):
        return (y % N) * N + (x % N)

    a = vid(ix, iy)
    b = vid(ix + 1, iy)
    c = vid(ix + 1, iy + 1)
    d = vid(ix, iy + 1)
    t0 = np.where(coin[..., None] == 0,
                  np.stack([a, b, c], -1), np.stack([a, b, d], -1))
    t1 = np.where(coin[..., None] == 0,
                  np.stack([a, c, d], -1), np.stack([b, c, d], -1))
    tri = np.stack([t0, t1], axis=2).reshape(2 * N * N, 3).astype(np.int32)
    return xy, tri, np.array([1.0, 1.0])


def standard_normal(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) array (f64)."""
    return np.random.default_rng(seed).standard_normal(shape) * scale


# ---------------------------------------------------------------- fields
# Plain point evaluations of analytic fields; callers decide where to sample.

def taylor_green_velocity(x, y):
    """Taylor-Green velocity of Sec. 4 rescaled to the unit square."""
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


def manufactured_pressure(x, y):
    """p = sin(2 pi x) cos(2 pi y) and f = -Laplace(p) = 8 pi^2 p."""
    tp = 2.0 * np.pi
    p = np.sin(tp * x) * np.cos(tp * y)
    return p, 2.0 * tp * tp * p


def fourier_modes(seed: int, n_modes: int = 32, kmax: int = 16):
    """Draw (k i64[m,2], amp f64[m], phase f64[m]) for f = sum a cos(2 pi k.x + phi).

    k is drawn uniformly without replacement from the integer vectors with
    1 <= |k| <= kmax; amplitudes are proportional to |k|^-2.
    """
    rng = np.random.default_rng(seed)
    r = np.arange(-kmax, kmax + 1)
    kx, ky = np.meshgrid(r, r, indexing="ij")
    kk = np.stack([kx.ravel(), ky.ravel()], 1)
    nrm = np.sqrt((kk ** 2).sum(1))
    cand = kk[(nrm >= 1) & (nrm <= kmax)]
    pick = rng.choice(len(cand), size=n_modes, replace=False)
    k = cand[pick]
    amp = 1.0 / (k ** 2).sum(1)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return k.astype(np.int64), amp, phase


def fourier_field(x, y, modes):
    k, amp, phase = modes
    tp = 2.0 * np.pi
    out = np.zeros(np.broadcast(x, y).shape)
    for (kx, ky), a, ph in zip(k, amp, phase):
        out = out + a * np.cos(tp * (kx * x + ky * y) + ph)
    return out
