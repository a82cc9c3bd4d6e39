"""Seeded synthetic inputs for the SN-like DLR workloads.

This module only prepares inputs (opacity fields, initial temperatures, edge
temperatures, sizes, request streams).  It holds none of the method's
arithmetic and is shared, as plain numpy arrays, by the oracle-side tests and
the GPU-side tests, benchmark and server.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15;
z = (s ^ s>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
out = z ^ z>>31.  Uniforms u = (out >> 11) * 2^-53; normals by Box-Muller
from consecutive uniform pairs (u1, u2): sqrt(-2 ln(1-u1)) (cos, sin)(2 pi u2).

Workloads (stand-ins for the paper's lattice and hohlraum problems, whose
meshes and material tables are not available; opacities span the paper's
1e-1 .. 1e4 range scaled down):
  lattice32     32x32, 4x4-cell blocks, sigma = 10^(2u) (log-uniform [1,100]),
                seed 0, r=6, 8x16 angles, 10 steps, left inflow at T=1
  checker256    256x256, 8x8 blocks thick (sigma=100) if u<1/2 else thin
                (0.1), seed 1, r=16, 16x32 angles, 100 steps, left inflow
  lognormal1024 1024x1024, sigma = exp(ln 5 + 1.5 z), z box-smoothed over 16
                cells (periodic window) and standardised, seed 2, central 128x128 hot square at
                T=1, vacuum edges, r=32, 32x64 angles, 200 steps
  batch64       64 instances from master seed 4 (sizes, ranks, angle sets
                uniform over the listed sets), opacity as lattice32 with
                seeds 100..163, 50 steps
  served2000    Poisson arrivals (mean gap 50 ms) from seed 5, side
                U{128..1024}, r in {8,16,32}, steps U{50..200}, 16x32
                angles, opacity as checker256 with seed = request id
Shared defaults: domain [0,1]^2, rho_cv = 1, T0 = 0.01, dt = 1e-3,
a = 0.01372, c = 299.792458.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

A_RAD = 0.01372
C_LIGHT = 299.792458
DT = 1e-3


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of SplitMix64 started at state `seed`."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def raw(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int = 1) -> np.ndarray:
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u = self.uniform(2 * m).reshape(m, 2)
        rad = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        z = np.stack([rad * np.cos(2 * math.pi * u[:, 1]),
                      rad * np.sin(2 * math.pi * u[:, 1])], 1).reshape(-1)
        return z[:n]


def _block_index(n: int, nblocks: int) -> np.ndarray:
    return (np.arange(n) * nblocks) // n


def block_loguniform_sigma(side: int, block: int, seed: int, lo: float = 1.0,
                           hi: float = 100.0) -> np.ndarray:
    """Piecewise-constant sigma on block x block cells, log-uniform [lo, hi];
    one draw per block in row-major (by, bx) order.  Returns (side, side)."""
    nb = max(1, side // block)
    u = Stream(seed).uniform(nb * nb).reshape(nb, nb)
    vals = lo * (hi / lo) ** u
    bi = _block_index(side, nb)
    return vals[bi[:, None], bi[None, :]]


def checkerboard_sigma(side: int, nblocks: int, seed: int, thick: float = 100.0,
                       thin: float = 0.1) -> np.ndarray:
    """nblocks x nblocks blocks, each thick if u < 1/2 else thin."""
    u = Stream(seed).uniform(nblocks * nblocks).reshape(nblocks, nblocks)
    vals = np.where(u < 0.5, thick, thin)
    bi = _block_index(side, nblocks)
    return vals[bi[:, None], bi[None, :]]


def _box_smooth(z: np.ndarray, width: int, axis: int) -> np.ndarray:
    """Periodic box filter: every cell averages `width` cells, so the
    smoothed field has the same variance everywhere (clamping the window at
    the edges would inflate the variance of edge and corner cells)."""
    return sum(np.roll(z, -d, axis=axis) for d in range(-(width // 2), width - width // 2)) / width


def lognormal_sigma(side: int, seed: int, mu: float = math.log(5.0), s: float = 1.5,
                    width: int = 16) -> np.ndarray:
    z = Stream(seed).normal(side * side).reshape(side, side)
    z = _box_smooth(_box_smooth(z, width, 1), width, 0)
    z = (z - z.mean()) / z.std()
    return np.exp(mu + s * z)


def _case(name, side, sigma, r, n_polar, n_azim, steps, T_edge, T0=None, precision="fp64"):
    return dict(name=name, nx=side, ny=side, lx=1.0, ly=1.0, n_polar=n_polar,
                n_azim=n_azim, r=r, steps=steps, dt=DT, c=C_LIGHT, a_rad=A_RAD,
                sigma=np.ascontiguousarray(sigma, dtype=np.float64),
                rho_cv=np.ones((side, side)),
                T0=np.full((side, side), 0.01) if T0 is None else T0,
                T_edge=tuple(T_edge), precision=precision)


LEFT_INFLOW = (1.0, -1.0, -1.0, -1.0)
VACUUM = (-1.0, -1.0, -1.0, -1.0)


def lattice32():
    return _case("lattice32", 32, block_loguniform_sigma(32, 4, 0), 6, 8, 16, 10,
                 LEFT_INFLOW)


def checker256(precision="mixed"):
    return _case("checker256", 256, checkerboard_sigma(256, 8, 1), 16, 16, 32, 100,
                 LEFT_INFLOW, precision=precision)


def lognormal1024():
    side = 1024
    T0 = np.full((side, side), 0.01)
    a = side // 2 - 64
    T0[a:a + 128, a:a + 128] = 1.0
    c = _case("lognormal1024", side, lognormal_sigma(side, 2), 32, 32, 64, 200,
              VACUUM, T0=T0, precision="mixed")
    # thick hot cells (sigma up to ~4e3 at T = 1) slow source iteration down
    c["si_max_iter"] = 20000
    return c


def lognormal_small(side: int = 64, seed: int = 2, r: int = 32, n_polar: int = 32,
                    n_azim: int = 64, ny: int = None):
    """lognormal1024's shape at a mesh the oracle steps in seconds: the same
    opacity law (smoothing window scaled with the side, at least 2 cells),
    a central hot square of 1/8 of the side at T = 1, vacuum edges, rank 32
    and 32 x 64 angles by default; ny != side gives a ragged mesh (the field
    is cut from a side x side draw)."""
    ny = side if ny is None else ny
    big = max(side, ny)
    sig = lognormal_sigma(big, seed, width=max(2, big // 64))[:ny, :side]
    T0 = np.full((ny, side), 0.01)
    hx, hy = max(1, side // 8), max(1, ny // 8)
    T0[ny // 2 - hy // 2:ny // 2 - hy // 2 + hy, side // 2 - hx // 2:side // 2 - hx // 2 + hx] = 1.0
    c = _case(f"lognormal{side}x{ny}", side, sig, r, n_polar, n_azim, 1, VACUUM, T0=T0,
              precision="mixed")
    c.update(ny=ny, rho_cv=np.ones((ny, side)))
    c["si_max_iter"] = 20000
    return c


ANGLE_SETS = [(8, 16), (8, 32), (16, 32), (16, 64)]


def batch64(n: int = 64, steps: int = 50):
    st = Stream(4)
    out = []
    for i in range(n):
        u = st.uniform(3)
        side = [64, 128, 256, 512][int(u[0] * 4)]
        r = [8, 16, 24, 32][int(u[1] * 4)]
        npol, naz = ANGLE_SETS[int(u[2] * 4)]
        out.append(_case(f"batch{i}", side, block_loguniform_sigma(side, 4, 100 + i), r,
                         npol, naz, steps, LEFT_INFLOW, precision="mixed"))
    return out


def served_requests(n: int = 2000, mean_gap: float = 0.05, seed: int = 5):
    """Request stream: list of (arrival_time_s, case dict).  The case's sigma
    is generated lazily by `materialize`."""
    st = Stream(seed)
    t = 0.0
    reqs = []
    for i in range(n):
        u = st.uniform(4)
        t += -math.log1p(-u[0]) * mean_gap
        side = 128 + int(u[1] * 897)
        r = [8, 16, 32][int(u[2] * 3)]
        steps = 50 + int(u[3] * 151)
        reqs.append((t, dict(id=i, side=side, r=r, steps=steps)))
    return reqs


def materialize(req: dict, n_polar: int = 16, n_azim: int = 32):
    side = req["side"]
    return _case(f"req{req['id']}", side, checkerboard_sigma(side, 8, req["id"]), req["r"],
                 n_polar, n_azim, req["steps"], LEFT_INFLOW, precision="mixed")


def small_case(nx: int, ny: int, r: int, n_polar: int, n_azim: int, seed: int = 7,
               T_edge=LEFT_INFLOW, block: int = 4, T0: float = 0.01):
    """A small lattice-style case with a ragged mesh for parity tests."""
    st = Stream(seed)
    nbx, nby = max(1, -(-nx // block)), max(1, -(-ny // block))
    u = st.uniform(nbx * nby).reshape(nby, nbx)
    vals = 10.0 ** (2.0 * u)
    sig = vals[(np.arange(ny) // block)[:, None], (np.arange(nx) // block)[None, :]]
    c = _case(f"small{nx}x{ny}", nx, sig, r, n_polar, n_azim, 1, T_edge)
    c.update(ny=ny, rho_cv=np.ones((ny, nx)), T0=np.full((ny, nx), T0))
    return c


CONFIGS = {"lattice32": lattice32, "checker256": checker256,
           "lognormal1024": lognormal1024}
