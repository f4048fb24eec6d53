"""Seeded synthetic G-buffers, transparency buffers, scene vectors and weights.

The paper's inputs come from an OpenGL rasteriser (Sec. 3.2: one opaque
G-buffer plus one G-buffer per transparent object, ``(w, h, c*(t+1))``) and its
weights from training (Sec. 3.5).  Neither exists here, so this module draws
stand-ins with the shapes and value ranges of the paper's buffers (Fig. 4:
position, normal, albedo, material parameters, direct lighting).

Nothing in this module computes any part of the network.  Every array is a
draw from ``numpy.random.default_rng`` with a documented seed and draw order,
so the oracle and the CUDA path read bit-identical float32 inputs.

Layouts (structure of arrays, row-major pixels ``p = y*w + x``):
  gbuf    float32 [GBUF_CHANNELS][h][w]
  tbuf    float32 [K][TBUF_CHANNELS][h][w]; slots ``k >= counts[y, x]`` are
          invalid and hold garbage (NaN by default)
  counts  uint8   [h][w], each in ``0..K``
  scene   float32 [SCENE_DIM]
  weights dict name -> (W float32 [out][in], b float32 [out]); ``y = W x + b``
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Opaque G-buffer channels (Fig. 4 lists normal, position, albedo, roughness,
# view direction, depth and direct lighting; the synthetic layout keeps 14):
#   0-2 position U[-1,1]^3, 3-5 unit normal, 6-8 albedo U[0,1]^3,
#   9 roughness U[0,1], 10 metallic U[0,1], 11-13 direct RGB exp(N(0,1)).
GBUF_CHANNELS = 14
# Transparency-buffer channels, one layer per transparent object (Sec. 3.2):
#   0-2 position U[-1,1]^3, 3-5 unit normal, 6-8 tint U[0,1]^3,
#   9 opacity U[0,1], 10 IOR U[1.0,1.8], 11 direct luminance exp(N(0,1)).
TBUF_CHANNELS = 12
# Scene-parameter vector fed to the scene encoder F.
SCENE_DIM = 32
OUT_CHANNELS = 3


@dataclass(frozen=True)
class Widths:
    """Hidden width H and latent width Z of the per-pixel network, the
    frequency count L of the inputs' positional encoding (0: none), which
    widens every input block of n channels to n (1 + 2L), and the kernel size
    of R's first layer (1, or 3 over the frame: R1 is then [H][9 H])."""

    hidden: int
    latent: int
    pe_freqs: int = 0
    r_kernel: int = 1


BASE_WIDTHS = Widths(hidden=64, latent=128)
DOUBLED_WIDTHS = Widths(hidden=128, latent=256)
# Base widths with every input positionally encoded at 4 frequencies.
BASE_PE_WIDTHS = Widths(hidden=64, latent=128, pe_freqs=4)

# Linear layers in draw order: name, and (out, in) as a function of (H, Z).
WEIGHT_ORDER = ("F1", "F2", "phi1", "phi2", "rho", "B1", "B2", "R1", "R2")


def weight_shapes(widths: Widths) -> dict[str, tuple[int, int]]:
    """(out, in) of every linear layer, concat form (no folding)."""
    H, Z = widths.hidden, widths.latent
    e = 1 + 2 * widths.pe_freqs
    return {
        "F1": (Z, SCENE_DIM * e),
        "F2": (Z, Z),
        "phi1": (H, TBUF_CHANNELS * e + Z),
        "phi2": (H, H),
        "rho": (H, 2 * H),
        "B1": (H, GBUF_CHANNELS * e + H + Z),
        "B2": (H, H),
        "R1": (H, H * widths.r_kernel ** 2),
        "R2": (OUT_CHANNELS, H),
    }


def make_weights(widths: Widths, seed: int = 0, bias: str = "zero") -> dict:
    """Xavier-normal weights (std = sqrt(2 / (fan_in + fan_out)), gain 1).

    Draw order: one ``default_rng(seed)``; every W in ``WEIGHT_ORDER`` as a
    standard normal scaled by its std; then, if ``bias == "uniform"``, every b
    in the same order from U[-0.1, 0.1].  ``bias == "zero"`` gives zero biases.
    Values are drawn in float64 and stored as float32.  With positional
    encoding the dict also holds ``"pe_freqs": L``, with a 3x3 R
    ``"r_kernel": 3``.
    """
    if bias not in ("zero", "uniform"):
        raise ValueError(f"bias must be 'zero' or 'uniform', got {bias!r}")
    rng = np.random.default_rng(seed)
    shapes = weight_shapes(widths)
    out = {}
    for name in WEIGHT_ORDER:
        fo, fi = shapes[name]
        std = np.sqrt(2.0 / (fi + fo))
        out[name] = [(rng.standard_normal((fo, fi)) * std).astype(np.float32), None]
    for name in WEIGHT_ORDER:
        fo = shapes[name][0]
        if bias == "uniform":
            b = rng.uniform(-0.1, 0.1, size=fo)
        else:
            b = np.zeros(fo)
        out[name][1] = b.astype(np.float32)
    res = {k: (v[0], v[1]) for k, v in out.items()}
    if widths.pe_freqs:
        res["pe_freqs"] = widths.pe_freqs
    if widths.r_kernel != 1:
        res["r_kernel"] = widths.r_kernel
    return res


def make_scene(seed: int = 0) -> np.ndarray:
    """Scene-parameter vector: SCENE_DIM draws of N(0, 1), float32."""
    rng = np.random.default_rng([seed, 2])
    return rng.standard_normal(SCENE_DIM).astype(np.float32)


def make_counts(h: int, w: int, K: int, dist: str, rng: np.random.Generator) -> np.ndarray:
    """Valid-layer count per pixel.

    ``all``: every pixel has K layers.  ``uniform``: U{0..K}.
    ``poisson3``: min(Poisson(3), K).
    """
    if dist == "all":
        c = np.full((h, w), K)
    elif dist == "uniform":
        c = rng.integers(0, K + 1, size=(h, w))
    elif dist == "poisson3":
        c = np.minimum(rng.poisson(3.0, size=(h, w)), K)
    else:
        raise ValueError(f"unknown count distribution {dist!r}")
    return c.astype(np.uint8)


def _unit_normals(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((3, n))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


@dataclass
class Frame:
    gbuf: np.ndarray    # float32 [14][h][w]
    tbuf: np.ndarray    # float32 [K][12][h][w]
    counts: np.ndarray  # uint8 [h][w]

    @property
    def K(self) -> int:
        return int(self.tbuf.shape[0])

    @property
    def h(self) -> int:
        return int(self.gbuf.shape[1])

    @property
    def w(self) -> int:
        return int(self.gbuf.shape[2])


def make_frame(h: int, w: int, K: int, counts: str = "all", seed: int = 0,
               garbage: float = float("nan")) -> Frame:
    """One synthetic frame.

    Draw order with ``default_rng([seed, 3])``: counts, then the G-buffer
    channel groups in channel order, then for each slot k = 0..K-1 the
    transparency channel groups in channel order.  Valid layers of a pixel sit
    in slots ``0..c-1`` (draws are i.i.d., so their order is already random);
    slots ``>= c`` are overwritten with ``garbage``.
    """
    if not (0 <= K <= 8):
        raise ValueError("K must be in 0..8")
    rng = np.random.default_rng([seed, 3])
    P = h * w
    cnt = make_counts(h, w, K, counts, rng)
    g = np.empty((GBUF_CHANNELS, P), np.float64)
    g[0:3] = rng.uniform(-1.0, 1.0, (3, P))
    g[3:6] = _unit_normals(rng, P)
    g[6:9] = rng.uniform(0.0, 1.0, (3, P))
    g[9] = rng.uniform(0.0, 1.0, P)
    g[10] = rng.uniform(0.0, 1.0, P)
    g[11:14] = np.exp(rng.standard_normal((3, P)))
    t = np.empty((K, TBUF_CHANNELS, P), np.float32)
    for k in range(K):
        tk = np.empty((TBUF_CHANNELS, P), np.float64)
        tk[0:3] = rng.uniform(-1.0, 1.0, (3, P))
        tk[3:6] = _unit_normals(rng, P)
        tk[6:9] = rng.uniform(0.0, 1.0, (3, P))
        tk[9] = rng.uniform(0.0, 1.0, P)
        tk[10] = rng.uniform(1.0, 1.8, P)
        tk[11] = np.exp(rng.standard_normal(P))
        t[k] = tk.astype(np.float32)
        invalid = cnt.reshape(P) <= k
        t[k][:, invalid] = garbage
    return Frame(gbuf=g.astype(np.float32).reshape(GBUF_CHANNELS, h, w),
                 tbuf=t.reshape(K, TBUF_CHANNELS, h, w),
                 counts=cnt)


def permute_layers(frame: Frame, seed: int) -> Frame:
    """Shuffle each pixel's valid layers among its slots ``0..c-1``.

    Invalid slots keep their position and contents.  Uses
    ``default_rng([seed, 4])``: one uniform key per (slot, pixel); invalid
    slots get key +inf so a stable argsort keeps them last.
    """
    K, h, w = frame.K, frame.h, frame.w
    P = h * w
    rng = np.random.default_rng([seed, 4])
    keys = rng.random((K, P))
    c = frame.counts.reshape(P).astype(np.int64)
    slot = np.arange(K)[:, None]
    keys = np.where(slot < c[None, :], keys, np.inf)
    order = np.argsort(keys, axis=0, kind="stable")  # [K][P]
    t = frame.tbuf.reshape(K, TBUF_CHANNELS, P)
    idx = np.broadcast_to(order[:, None, :], t.shape)
    tp = np.take_along_axis(t, idx, axis=0)
    return Frame(gbuf=frame.gbuf.copy(), tbuf=tp.reshape(K, TBUF_CHANNELS, h, w),
                 counts=frame.counts.copy())


# Batched workload (16 frames of mixed size and layer count, a few scenes):
# per frame a square resolution drawn uniformly from `sizes`, K ~ U{2..8} and
# scene index i mod n_scenes; every slot of every pixel valid.
BATCH_SIZES_FULL = (128, 256, 512, 1024)


class BatchSpec:
    def __init__(self, h: int, w: int, K: int, scene: int):
        self.h, self.w, self.K, self.scene = h, w, K, scene

    def __repr__(self):
        return f"BatchSpec({self.h}x{self.w}, K={self.K}, scene={self.scene})"


def batch_specs(n: int = 16, sizes=BATCH_SIZES_FULL, n_scenes: int = 4,
                seed: int = 0) -> list[BatchSpec]:
    rng = np.random.default_rng([seed, 5])
    out = []
    for i in range(n):
        s = int(rng.choice(np.asarray(sizes)))
        K = int(rng.integers(2, 9))
        out.append(BatchSpec(s, s, K, i % n_scenes))
    return out
