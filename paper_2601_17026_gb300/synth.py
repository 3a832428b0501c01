"""Seeded synthetic cost volumes shaped like the paper's seismic horizon workloads.

This module only draws inputs. It holds none of the min-cut method's arithmetic, so
both the CUDA path and the CPU oracle may consume what it produces.

The paper's seismic volumes (Section 3.4, Table 1: 551x426x426 and 1001x376x1375
images reduced to 10-100 M-node narrow-band graphs) are not available; these
layered-horizon volumes stand in for them. A cost volume is int32 [X, Y, Z] with z
fastest (C order), i.e. element (x, y, z) sits at ((x*Y + y)*Z + z).

Random numbers come from one counter-based generator: draw i of a stream is the
SplitMix64 output (Steele, Lea and Flood, OOPSLA 2014) for state key + (i+1)*gamma,
so any element can be drawn independently and the whole volume vectorises. Bounded
integers use the 32x32->64 multiply-shift map (Lemire 2019) on the high 32 bits;
normals use Box-Muller on two consecutive draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 17026

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, elementwise on uint64 (wrapping arithmetic)."""
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def _mix64_int(v: int) -> int:
    v &= _MASK64
    v ^= v >> 30
    v = (v * 0xBF58476D1CE4E5B9) & _MASK64
    v ^= v >> 27
    v = (v * 0x94D049BB133111EB) & _MASK64
    return v ^ (v >> 31)


def stream_key(seed: int, stream: int) -> int:
    """Key of an independent stream: a hash of (seed, stream)."""
    return _mix64_int(_mix64_int(seed) ^ ((stream * 0xD1B54A32D192ED03) & _MASK64))


def draws_u64(key: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the stream with this key (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(np.uint64(key) + i * _GAMMA)


def uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uint64 draws to integers in [lo, hi] inclusive (multiply-shift)."""
    span = np.uint64(hi - lo + 1)
    with np.errstate(over="ignore"):
        return (((u >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64) + lo


def _unit_open(u: np.ndarray) -> np.ndarray:
    """uint64 -> float64 in (0, 1): the top 53 bits, offset by half a step."""
    return ((u >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(key: int, start: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller; normal i uses draws 2i and 2i+1."""
    u = draws_u64(key, 2 * start, 2 * count)
    u1 = _unit_open(u[0::2])
    u2 = _unit_open(u[1::2])
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass(frozen=True)
class HorizonSpec:
    """Parameters of one layered-horizon cost volume.

    c(x,y,z) = min(cap, round_half_away(1000*(1 - exp(-d2/sigma2))) + U{0..umax}), with
    d2 = min_k (z - h(x,y) - off_k)^2 and h(x,y) = centre + amp*sin(2 pi x/px)*cos(2 pi y/py).
    """

    X: int
    Y: int
    Z: int
    sigma2: float
    centre: float
    amp: float
    px: float = 256.0
    py: float = 192.0
    offsets: tuple = (0.0,)
    umax: int = 200
    cap: int = 1200
    seed: int = BASE_SEED
    stream: int = 0

    @property
    def n(self) -> int:
        return self.X * self.Y * self.Z


def _horizon_d2(spec: HorizonSpec, x0: int, x1: int) -> np.ndarray:
    x = np.arange(x0, x1, dtype=np.float64)[:, None, None]
    y = np.arange(spec.Y, dtype=np.float64)[None, :, None]
    z = np.arange(spec.Z, dtype=np.float64)[None, None, :]
    h = spec.centre + spec.amp * np.sin(2.0 * math.pi * x / spec.px) * np.cos(2.0 * math.pi * y / spec.py)
    d2 = None
    for off in spec.offsets:
        d = (z - h - off) ** 2
        d2 = d if d2 is None else np.minimum(d2, d)
    return d2


def _smooth_part(spec: HorizonSpec, x0: int, x1: int) -> np.ndarray:
    """1000*(1 - exp(-d2/sigma2)) on the slab x0 <= x < x1, float64."""
    return 1000.0 * (1.0 - np.exp(-_horizon_d2(spec, x0, x1) / spec.sigma2))


def horizon_cost(spec: HorizonSpec, slab: int = 32) -> np.ndarray:
    """int32 [X, Y, Z] cost volume (generated in x-slabs to bound host memory)."""
    out = np.empty((spec.X, spec.Y, spec.Z), dtype=np.int32)
    key = stream_key(spec.seed, spec.stream)
    per_x = spec.Y * spec.Z
    for x0 in range(0, spec.X, slab):
        x1 = min(spec.X, x0 + slab)
        base = np.floor(_smooth_part(spec, x0, x1) + 0.5)  # half away from zero (values >= 0)
        u = uniform_int(draws_u64(key, x0 * per_x, (x1 - x0) * per_x), 0, spec.umax)
        c = np.minimum(base.reshape(-1) + u, spec.cap)
        out[x0:x1] = c.reshape(x1 - x0, spec.Y, spec.Z).astype(np.int32)
    return out


def float_horizon_cost(spec: HorizonSpec, slab: int = 32) -> np.ndarray:
    """float32 [X, Y, Z]: N(0,1) noise plus the noise-free horizon part (0..1000)."""
    out = np.empty((spec.X, spec.Y, spec.Z), dtype=np.float32)
    key = stream_key(spec.seed, spec.stream)
    per_x = spec.Y * spec.Z
    for x0 in range(0, spec.X, slab):
        x1 = min(spec.X, x0 + slab)
        g = _smooth_part(spec, x0, x1).reshape(-1)
        out[x0:x1] = (g + normal(key, x0 * per_x, (x1 - x0) * per_x)).reshape(x1 - x0, spec.Y, spec.Z)
    return out


def uniform_cost(X: int, Y: int, Z: int, lo: int, hi: int, seed: int = BASE_SEED, stream: int = 99) -> np.ndarray:
    """int32 [X, Y, Z] with i.i.d. U{lo..hi} entries (small random test volumes)."""
    key = stream_key(seed, stream)
    return uniform_int(draws_u64(key, 0, X * Y * Z), lo, hi).astype(np.int32).reshape(X, Y, Z)


# ---------------------------------------------------------------------------------------
# The five workloads. Each returns plain numpy arrays and the (delta, alpha) pair.
# ---------------------------------------------------------------------------------------

FIVE_HORIZONS = (0.0, 60.0, -60.0, 110.0, -110.0)


@dataclass
class Volume:
    cost: np.ndarray  # int32 [X,Y,Z]
    delta: int
    alpha: int
    name: str = ""
    fcost: np.ndarray | None = field(default=None, repr=False)  # float32 source (differentiable workload)

    @property
    def shape(self):
        return self.cost.shape

    @property
    def n(self) -> int:
        return int(self.cost.size)


def spec_small(seed: int = BASE_SEED) -> HorizonSpec:
    """16x16x32, one horizon at 16 + 6 sin(2 pi x/16) cos(2 pi y/16), sigma^2 = 8."""
    return HorizonSpec(16, 16, 32, sigma2=8.0, centre=16.0, amp=6.0, px=16.0, py=16.0,
                       offsets=(0.0,), umax=200, seed=seed, stream=0)


def spec_medium(seed: int = BASE_SEED) -> HorizonSpec:
    """256^3, five horizons around 128 + 40 sin(2 pi x/256) cos(2 pi y/192), sigma^2 = 32."""
    return HorizonSpec(256, 256, 256, sigma2=32.0, centre=128.0, amp=40.0, px=256.0, py=192.0,
                       offsets=FIVE_HORIZONS, umax=200, seed=seed, stream=1)


def spec_seismic(seed: int = BASE_SEED) -> HorizonSpec:
    """512x512x384, the medium formula with U{0..400} noise."""
    return HorizonSpec(512, 512, 384, sigma2=32.0, centre=128.0, amp=40.0, px=256.0, py=192.0,
                       offsets=FIVE_HORIZONS, umax=400, seed=seed, stream=2)


def scaled_spec(X: int, Y: int, Z: int, seed: int, stream: int, umax: int = 200) -> HorizonSpec:
    """The medium formula with centre Z/2 and amplitude/offsets scaled by Z/256."""
    s = Z / 256.0
    return HorizonSpec(X, Y, Z, sigma2=32.0, centre=Z / 2.0, amp=40.0 * s, px=256.0, py=192.0,
                       offsets=tuple(o * s for o in FIVE_HORIZONS), umax=umax, seed=seed, stream=stream)


def small_volume(seed: int = BASE_SEED) -> Volume:
    return Volume(horizon_cost(spec_small(seed)), delta=2, alpha=0, name="16x16x32 d2 a0")


def medium_volume(seed: int = BASE_SEED) -> Volume:
    return Volume(horizon_cost(spec_medium(seed)), delta=2, alpha=0, name="256x256x256 d2 a0")


def seismic_volume(seed: int = BASE_SEED) -> Volume:
    return Volume(horizon_cost(spec_seismic(seed)), delta=3, alpha=50, name="512x512x384 d3 a50")


def seismic_crop(n: int = 256, seed: int = BASE_SEED) -> Volume:
    """The n x n x 384 corner (x, y < n) of the 512 x 512 x 384 volume, same delta and alpha:
    a smaller case of the same kernels, for profiling."""
    v = seismic_volume(seed)
    return Volume(np.ascontiguousarray(v.cost[:n, :n]), delta=v.delta, alpha=v.alpha,
                  name=f"{n}x{n}x384 crop of 512x512x384 d3 a50")


def batch_shapes(seed: int = BASE_SEED, count: int = 64):
    """(X, Y, Z, delta, alpha) of the uneven batch: X,Y ~ U{32..256}, Z ~ U{64..256},
    delta ~ {1,2,4}, alpha = 0 for even and 25 for odd volume indices."""
    key = stream_key(seed, 3)
    u = draws_u64(key, 0, 4 * count)
    out = []
    for i in range(count):
        X = int(uniform_int(u[4 * i:4 * i + 1], 32, 256)[0])
        Y = int(uniform_int(u[4 * i + 1:4 * i + 2], 32, 256)[0])
        Z = int(uniform_int(u[4 * i + 2:4 * i + 3], 64, 256)[0])
        d = (1, 2, 4)[int(uniform_int(u[4 * i + 3:4 * i + 4], 0, 2)[0])]
        out.append((X, Y, Z, d, 0 if i % 2 == 0 else 25))
    return out


def batch_volumes(seed: int = BASE_SEED, count: int = 64, limit=None):
    """The uneven batch; volume i draws its costs from seed + i."""
    vols = []
    for i, (X, Y, Z, d, a) in enumerate(batch_shapes(seed, count)):
        if limit is not None and i >= limit:
            break
        spec = scaled_spec(X, Y, Z, seed + i, stream=1000 + i)
        vols.append(Volume(horizon_cost(spec), delta=d, alpha=a, name=f"batch[{i}] {X}x{Y}x{Z} d{d} a{a}"))
    return vols


def diff_specs(seed: int = BASE_SEED, count: int = 16, size: int = 128):
    return [scaled_spec(size, size, size, seed + i, stream=2000 + i) for i in range(count)]


def diff_volumes_f32(seed: int = BASE_SEED, count: int = 16, size: int = 128) -> np.ndarray:
    """float32 [B, S, S, S]: N(0,1) + the noise-free horizon pattern (delta 2, alpha 10)."""
    return np.stack([float_horizon_cost(s) for s in diff_specs(seed, count, size)])


DIFF_DELTA = 2
DIFF_ALPHA = 10.0  # soft penalty of the differentiable workload, in float cost units
DIFF_MARGIN = 1.0  # structured-hinge margin per mismatched column, in float cost units


def diff_target(count: int = 16, size: int = 128) -> np.ndarray:
    """int32 [B, S, S]: the hinge target surface of the differentiable workload, flat at
    height S/2 in every column (feasible for any delta)."""
    return np.full((count, size, size), size // 2, dtype=np.int32)


def horizon_landmarks(spec: HorizonSpec, grid: int = 8) -> np.ndarray:
    """int32 [grid*grid, 3]: landmark points (x, y, z) on the central horizon of a volume,
    z = round(centre + amp*sin(2 pi x/px)*cos(2 pi y/py)), at a grid x grid lattice of
    columns (cell centres), as a user would place them on a horizon of the image."""
    xs = ((np.arange(grid) + 0.5) * spec.X / grid).astype(np.int64)
    ys = ((np.arange(grid) + 0.5) * spec.Y / grid).astype(np.int64)
    pts = []
    for x in xs:
        for y in ys:
            h = spec.centre + spec.amp * math.sin(2.0 * math.pi * x / spec.px) * math.cos(2.0 * math.pi * y / spec.py)
            pts.append((int(x), int(y), min(max(int(math.floor(h + 0.5)), 0), spec.Z - 1)))
    return np.array(pts, dtype=np.int32)


BAND_STICK = 16       # rows above and below the center surface, before the band factor
BAND_FACTOR = 2       # narrow-band factor: half = 32, 65 rows per column
BAND_OUTSIDE = 1200   # cost of band rows outside the image (the costs' cap)


# ---------------------------------------------------------------------------------------
# Convex pairwise costs (the general proper-order graph): an edge interval of 10 vertices
# per adjacent column (height drops d = 0..9, delta = 9) with a quadratic cost f(t) = 4 t^2
# on the layered-horizon volumes (medium formula scaled to the volume's z extent).
# ---------------------------------------------------------------------------------------

CONVEX_DELTA = 9
CONVEX_QUAD = 4
CONVEX_SHAPE = (256, 256, 128)


def convex_profile(delta: int = CONVEX_DELTA, a: int = CONVEX_QUAD) -> np.ndarray:
    """int64 f(1..delta) of f(t) = a t^2."""
    t = np.arange(1, delta + 1, dtype=np.int64)
    return a * t * t


def convex_cost(X: int, Y: int, Z: int, seed: int = BASE_SEED) -> np.ndarray:
    """int32 [X, Y, Z] layered-horizon volume of the convex workload (stream 5)."""
    return horizon_cost(scaled_spec(X, Y, Z, seed, 5))
