"""Seeded synthetic high-speed video, the stand-in for the paper's facial HSDV clips.

The paper evaluates on high-speed video of faces with external markers (Sec. VII-A):
a mostly static textured scene with small, high-contrast features that move a few
pixels per frame. That data set is not available, so every workload here is drawn
from this generator instead.  It holds no arithmetic of the fused chain; it only
produces uint8 frames and the ground-truth motion of every object, and it serves
the oracle, the CUDA path, the tests and the benchmark alike.

Scene recipe (per frame, H rows x W columns, values in gray levels):
  * background: 110 + sum of 4 plane sinusoids, amplitude 10 each, random direction,
    period 64..256 px, random phase; static over time;
  * n_blobs isotropic Gaussian blobs, sigma in [3, 8] px, amplitude +-60;
  * n_patches 16x16 checker patches with 4-px cells of +-40;
  * every blob and patch moves at a constant velocity drawn uniformly from
    [-2, 2]^2 px/frame and wraps around the frame (toroidal);
  * patches are placed at sub-pixel positions by bilinear interpolation of the
    sprite (zero outside it); blobs are evaluated at their exact centre;
  * i.i.d. Gaussian noise of sigma 2, then round-half-to-even and clamp to [0, 255].

Randomness is counter based: every number is splitmix64 of (stream key + counter),
so a frame can be regenerated on its own and the result does not depend on numpy's
generator implementation.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) applied to x + golden gamma."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> int:
    """64-bit key of one random stream of one seed."""
    z = splitmix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1) & _MASK64],
                            dtype=np.uint64))
    return int(z[0])


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from stream `stream` of `seed`, counters offset..offset+n-1."""
    ctr = (np.uint64(_key(seed, stream)) + np.arange(offset, offset + n, dtype=np.uint64))
    bits = splitmix64(ctr) >> np.uint64(11)  # 53 random bits
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


_NORMAL_TABLE: np.ndarray | None = None


def _normal_table() -> np.ndarray:
    """Standard-normal quantiles at the 65536 mid-points (k + 1/2) / 65536."""
    global _NORMAL_TABLE
    if _NORMAL_TABLE is None:
        from scipy.special import ndtri
        _NORMAL_TABLE = ndtri((np.arange(65536, dtype=np.float64) + 0.5) / 65536.0)
    return _NORMAL_TABLE


def normals(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by inverse-CDF lookup of 16-bit uniforms.

    Each splitmix64 output gives four 16-bit uniforms; a uniform k maps to the normal
    quantile of (k + 1/2) / 65536. The tails are cut at |z| < 4.3, which is harmless
    for sensor-like noise and keeps the draw exact and fast on any platform.
    """
    m = (n + 3) // 4
    ctr = np.uint64(_key(seed, stream)) + np.arange(m, dtype=np.uint64)
    z = splitmix64(ctr)
    k = z.view(np.uint16)[: n]  # little-endian 16-bit lanes of each output
    return _normal_table()[k]


@dataclasses.dataclass(frozen=True)
class VideoSpec:
    """Shape and content of one synthetic clip. Frames are H rows x W columns."""
    T: int
    H: int
    W: int
    seed: int
    n_blobs: int = 32
    n_patches: int = 16
    noise_sigma: float = 2.0
    background: float = 110.0


# The workloads the benchmarks and tests use, named by what they are.
SMALL_192x432x60 = VideoSpec(T=60, H=192, W=432, seed=1)
PARTITIONS_192x432x600 = VideoSpec(T=600, H=192, W=432, seed=2)
HSDV_800x600x1000 = VideoSpec(T=1000, H=800, W=600, seed=3, n_blobs=64, n_patches=32)


@dataclasses.dataclass
class Scene:
    spec: VideoSpec
    bg: np.ndarray  # float64 H x W static background
    # objects: kind 0 = blob, 1 = checker patch
    kind: np.ndarray
    x0: np.ndarray  # float64 initial position (blob centre / patch top-left), columns
    y0: np.ndarray  # rows
    vx: np.ndarray  # px / frame, columns
    vy: np.ndarray  # px / frame, rows
    sigma: np.ndarray  # blobs only
    amp: np.ndarray  # blobs: signed amplitude; patches: cell contrast

    def position(self, t: int) -> tuple[np.ndarray, np.ndarray]:
        """Object reference positions at frame t, wrapped into [0, W) x [0, H)."""
        W, H = self.spec.W, self.spec.H
        return (np.mod(self.x0 + self.vx * t, W), np.mod(self.y0 + self.vy * t, H))


PATCH = 16
CELL = 4


def checker_sprite(contrast: float) -> np.ndarray:
    i = np.arange(PATCH)
    par = ((i[:, None] // CELL) + (i[None, :] // CELL)) % 2
    return np.where(par == 0, contrast, -contrast).astype(np.float64)


def make_scene(spec: VideoSpec) -> Scene:
    H, W = spec.H, spec.W
    # background sinusoids: stream 1
    u = uniforms(spec.seed, 1, 12)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    bg = np.full((H, W), spec.background)
    for k in range(4):
        theta = 2.0 * math.pi * u[3 * k]
        period = 64.0 + 192.0 * u[3 * k + 1]
        phase = 2.0 * math.pi * u[3 * k + 2]
        bg += 10.0 * np.sin(2.0 * math.pi * (xx * math.cos(theta) + yy * math.sin(theta))
                            / period + phase)
    n = spec.n_blobs + spec.n_patches
    # objects: stream 2, 8 numbers per object
    v = uniforms(spec.seed, 2, 8 * n).reshape(n, 8)
    kind = np.array([0] * spec.n_blobs + [1] * spec.n_patches, dtype=np.int32)
    x0 = v[:, 0] * W
    y0 = v[:, 1] * H
    vx = -2.0 + 4.0 * v[:, 2]
    vy = -2.0 + 4.0 * v[:, 3]
    sigma = 3.0 + 5.0 * v[:, 4]
    amp = np.where(v[:, 5] < 0.5, -60.0, 60.0)
    amp = np.where(kind == 1, 40.0, amp)
    return Scene(spec, bg, kind, x0, y0, vx, vy, sigma, amp)


def _add_wrapped(img: np.ndarray, r0: int, c0: int, patch: np.ndarray) -> None:
    H, W = img.shape
    rows = np.mod(np.arange(r0, r0 + patch.shape[0]), H)
    cols = np.mod(np.arange(c0, c0 + patch.shape[1]), W)
    if patch.shape[0] > H or patch.shape[1] > W:
        # object larger than a tiny frame: accumulate one element at a time
        np.add.at(img, (rows[:, None], cols[None, :]), patch)
    else:
        img[np.ix_(rows, cols)] += patch


def render_frame(scene: Scene, t: int) -> np.ndarray:
    """Frame t as uint8 H x W."""
    spec = scene.spec
    H, W = spec.H, spec.W
    img = scene.bg.copy()
    px, py = scene.position(t)
    for o in range(len(scene.kind)):
        if scene.kind[o] == 0:
            s = scene.sigma[o]
            rad = int(math.ceil(4.0 * s))
            cx, cy = px[o], py[o]
            ic, ir = int(math.floor(cx)), int(math.floor(cy))
            dc = np.arange(ic - rad, ic + rad + 2, dtype=np.float64) - cx
            dr = np.arange(ir - rad, ir + rad + 2, dtype=np.float64) - cy
            val = scene.amp[o] * np.exp(-(dr[:, None] ** 2 + dc[None, :] ** 2) / (2.0 * s * s))
            _add_wrapped(img, ir - rad, ic - rad, val)
        else:
            sp = np.zeros((PATCH + 2, PATCH + 2))
            sp[1:-1, 1:-1] = checker_sprite(scene.amp[o])
            ix, iy = int(math.floor(px[o])), int(math.floor(py[o]))
            fx, fy = px[o] - ix, py[o] - iy
            # pixel ix+i samples sprite coordinate i - fx: weights fx on cell i-1, 1-fx on cell i
            val = ((1 - fy) * (1 - fx) * sp[1:, 1:] + (1 - fy) * fx * sp[1:, :-1]
                   + fy * (1 - fx) * sp[:-1, 1:] + fy * fx * sp[:-1, :-1])
            _add_wrapped(img, iy, ix, val)
    if spec.noise_sigma > 0:
        img += spec.noise_sigma * normals(spec.seed, 1000 + t, H * W).reshape(H, W)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def generate(spec: VideoSpec, pitch: int | None = None, frames: range | None = None,
             out: np.ndarray | None = None) -> tuple[np.ndarray, Scene]:
    """Render frames (default all T) into a uint8 array [n, H, pitch] (pitch >= W).

    Columns W..pitch-1 of every row are zero. Returns (frames, scene).
    """
    scene = make_scene(spec)
    P = spec.W if pitch is None else pitch
    if P < spec.W:
        raise ValueError("pitch must be >= W")
    ts = range(spec.T) if frames is None else frames
    if out is None:
        out = np.zeros((len(ts), spec.H, P), dtype=np.uint8)
    for i, t in enumerate(ts):
        out[i, :, :spec.W] = render_frame(scene, t)
    return out, scene


def pitch_for(W: int, align: int = 16) -> int:
    """Row pitch in bytes: W rounded up to a multiple of `align`."""
    return (W + align - 1) // align * align


def rgba_of(gray: np.ndarray) -> np.ndarray:
    """Colour frames [..., 4] u8 from gray frames [...] u8, for the RGBA workloads: the
    channels are the gray value, a brightened copy and its negative (so no single channel
    carries the luma), alpha 255: R = v, G = min(255, (4 v) // 5 + 30), B = 255 - v."""
    v = gray.astype(np.int32)
    out = np.empty(gray.shape + (4,), dtype=np.uint8)
    out[..., 0] = v
    out[..., 1] = np.minimum(255, (4 * v) // 5 + 30)
    out[..., 2] = 255 - v
    out[..., 3] = 255
    return out
