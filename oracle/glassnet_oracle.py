"""FP64 CPU oracle of the GlassNet per-pixel forward pass (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
and reference arm may import this module.  It shares no code with the CUDA
library: it reads the float32 weights and buffers produced by ``gen.synth``,
upcasts them to float64 and evaluates the network as written, in concat form,
with no folding, fusion, blocking or reordering.

The network (paper Sec. 3.3-3.4, Fig. 2; widths of the per-pixel MLP form):
  sigma = F(s)                      scene encoder, run once per scene
  v_k   = h([b_k ; sigma])          shared per-layer network, Eq. 5
  pool  = [max_k v_k ; mean_k v_k]  symmetric function g over the valid layers
  r     = rho(pool), r = 0 when the pixel has no valid layer
  y     = B([g_p ; r ; sigma])      final blending network
  rgb   = R(y)                      rendering network, sigmoid output

Readings where the paper is silent (each is listed with its reason in the
design notes): ReLU after every linear layer except the last one of R, which
is a sigmoid; the mean divides by the number of valid layers; an empty layer
set gives r = 0; input concat orders are [b ; sigma] and [g ; r ; sigma];
pool order is [max ; mean].  The paper's own form of Eq. 5 is also given
(``pooling="sum"``): tau = sum_k h(b_k, sigma) enters B directly, no rho.

Positional encoding (Sec. 3.4: all inputs are encoded with the method of
Mildenhall et al.; the frequency count is not given): a weight set with
``weights["pe_freqs"] = L > 0`` feeds every network input x -- the scene
vector s, each layer b_k and the G-buffer g -- as
gamma_L(x) = [x ; sin(2^0 pi x) ; cos(2^0 pi x) ; ... ; sin(2^(L-1) pi x) ;
cos(2^(L-1) pi x)], each block over all channels of x.  L = 0 (or no key)
is the network above unchanged.

Spatial R (Sec. 3.4: larger kernels in R before 1x1 kernels at its end): a
weight set with ``weights["r_kernel"] = 3`` makes R's first layer a 3x3
convolution over the frame's neural buffer y (the output of B, H channels per
pixel): q(p) = ReLU(b + sum over (dy, dx) in {-1, 0, 1}^2 of
W[:, :, dy + 1, dx + 1] y(p + (dy, dx))), cross-correlation with zero padding
outside the frame; R1's weight is stored as [H][H * 9], the [out][in][3][3]
kernel flattened.  R2 stays 1x1.  Only the frame path evaluates it.

Every function below is pinned by ``tests/test_oracle_pins.py`` (hand-worked
closed forms, brute force, invariants and library routines).
"""
from __future__ import annotations

import numpy as np


def _f64(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64)


def linear(x, W, b) -> np.ndarray:
    """Affine layer ``y = W x + b`` on the last axis; W is [out][in]."""
    return _f64(x) @ _f64(W).T + _f64(b)


def relu(x) -> np.ndarray:
    return np.maximum(_f64(x), 0.0)


def sigmoid(x) -> np.ndarray:
    """Logistic function 1 / (1 + e^-x)."""
    x = _f64(x)
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-x))


def pe_freqs(weights) -> int:
    """Frequency count L of the weight set's positional encoding (0: none)."""
    return int(weights.get("pe_freqs", 0))


def positional_encoding(x, L: int) -> np.ndarray:
    """gamma_L(x) on the last axis (Sec. 3.4, after Mildenhall et al.):
    x itself, then for f = 0 .. L-1 the blocks sin(2^f pi x) and cos(2^f pi x).
    Width n (1 + 2L) for n channels; L = 0 returns x.
    """
    x = _f64(x)
    parts = [x]
    for f in range(L):
        a = (np.pi * 2.0 ** f) * x
        parts.append(np.sin(a))
        parts.append(np.cos(a))
    return np.concatenate(parts, axis=-1)


def scene_encoder(weights, s) -> np.ndarray:
    """Scene encoder F (Sec. 3.4): sigma = ReLU(F2 ReLU(F1 s + b1) + b2),
    on the encoded scene vector gamma_L(s)."""
    h1 = relu(linear(positional_encoding(s, pe_freqs(weights)), *weights["F1"]))
    return relu(linear(h1, *weights["F2"]))


def per_layer_h(weights, b_k, sigma) -> np.ndarray:
    """Shared per-layer network h(b_i, sigma) of Eq. 5.

    ``b_k`` is [..., n_t] (one transparency layer per row); sigma is
    broadcast to every row and appended after the layer's encoded channels
    gamma_L(b_k).
    """
    b_k = positional_encoding(b_k, pe_freqs(weights))
    sig = np.broadcast_to(_f64(sigma), b_k.shape[:-1] + (np.shape(sigma)[-1],))
    x = np.concatenate([b_k, sig], axis=-1)
    u = relu(linear(x, *weights["phi1"]))
    return relu(linear(u, *weights["phi2"]))


def set_pool(V) -> np.ndarray | None:
    """Symmetric function g over a set of per-layer vectors V [c][H].

    Returns [max ; mean] (length 2H), or None for the empty set.  The sum is
    taken over each channel's values sorted ascending, a canonical order that
    makes the result exactly independent of the order of the layers (Eq. 5,
    Table 4).
    """
    V = _f64(V)
    c = V.shape[0]
    if c == 0:
        return None
    mx = V.max(axis=0)
    srt = np.sort(V, axis=0)
    s = np.zeros(V.shape[1])
    for k in range(c):
        s = s + srt[k]
    return np.concatenate([mx, s / c])


def set_sum(V) -> np.ndarray:
    """Eq. 5's symmetric function as the paper writes it: tau = sum_k v_k over
    the set V [c][H], each channel's values summed in ascending order (a
    canonical order, so the result is exactly independent of the order of the
    layers).  The empty set sums to the zero vector.
    """
    V = _f64(V)
    s = np.zeros(V.shape[1])
    srt = np.sort(V, axis=0)
    for k in range(V.shape[0]):
        s = s + srt[k]
    return s


def post_pool_rho(weights, pool) -> np.ndarray:
    """Post-pooling network rho: r = ReLU(W_rho pool + b_rho)."""
    return relu(linear(pool, *weights["rho"]))


def final_blend_B(weights, g, r, sigma) -> np.ndarray:
    """Final blending network B (Sec. 3.4) on [gamma_L(g) ; r ; sigma]."""
    g, r = positional_encoding(g, pe_freqs(weights)), _f64(r)
    sig = np.broadcast_to(_f64(sigma), g.shape[:-1] + (np.shape(sigma)[-1],))
    x = np.concatenate([g, r, sig], axis=-1)
    y = relu(linear(x, *weights["B1"]))
    return relu(linear(y, *weights["B2"]))


def r_kernel(weights) -> int:
    """Kernel size of R's first layer: 1 (per pixel) or 3 (over the frame)."""
    return int(weights.get("r_kernel", 1))


def render_R_frame(weights, Y) -> np.ndarray:
    """R over a whole frame's neural buffer ``Y`` [h][w][H]; returns rgb [3][h][w].

    R1 with a 3x3 kernel: each of the 9 taps (dy, dx) multiplies the buffer
    shifted by (dy, dx), zero outside the frame; with a 1x1 kernel R is
    ``render_R`` pixel by pixel.
    """
    Y = _f64(Y)
    h, w, H = Y.shape
    if r_kernel(weights) == 1:
        return render_R(weights, Y).transpose(2, 0, 1)
    W, b = _f64(weights["R1"][0]).reshape(-1, H, 3, 3), _f64(weights["R1"][1])
    Yp = np.pad(Y, ((1, 1), (1, 1), (0, 0)))
    acc = np.broadcast_to(b, (h, w, W.shape[0])).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            acc = acc + Yp[1 + dy:1 + dy + h, 1 + dx:1 + dx + w, :] @ W[:, :, dy + 1, dx + 1].T
    q = relu(acc)
    return sigmoid(linear(q, *weights["R2"])).transpose(2, 0, 1)


def render_R(weights, y) -> np.ndarray:
    """Rendering network R (Sec. 3.4): rgb = sigmoid(R2 ReLU(R1 y + b) + b)."""
    q = relu(linear(y, *weights["R1"]))
    return sigmoid(linear(q, *weights["R2"]))


def _layer_width(weights, sigma) -> int:
    """Channels n_t of a raw transparency layer: phi1 reads n_t (1 + 2L) + Z."""
    enc = np.shape(weights["phi1"][0])[1] - np.shape(sigma)[-1]
    return enc // (1 + 2 * pe_freqs(weights))


def _per_pixel_R(weights) -> None:
    if r_kernel(weights) != 1:
        raise ValueError("a 3x3 R reads neighbouring pixels: use render_frame")


def render_pixel(weights, sigma, g, layers) -> np.ndarray:
    """One pixel: ``g`` [n_g] opaque G-buffer, ``layers`` [c][n_t] valid layers."""
    _per_pixel_R(weights)
    layers = _f64(layers).reshape(-1, _layer_width(weights, sigma))
    H = np.shape(weights["phi2"][0])[0]
    if layers.shape[0] == 0:
        r = np.zeros(H)
    else:
        V = np.stack([per_layer_h(weights, layers[k], sigma) for k in range(layers.shape[0])])
        r = post_pool_rho(weights, set_pool(V))
    y = final_blend_B(weights, g, r, sigma)
    return render_R(weights, y)


def render_pixel_sum(weights, sigma, g, layers) -> np.ndarray:
    """One pixel in the paper's form of Eq. 5: tau = sum_k h(b_k, sigma) enters
    B directly as [g ; tau ; sigma] (no rho; rho's weights are not used)."""
    _per_pixel_R(weights)
    layers = _f64(layers).reshape(-1, _layer_width(weights, sigma))
    H = np.shape(weights["phi2"][0])[0]
    V = np.stack([per_layer_h(weights, layers[k], sigma) for k in range(layers.shape[0])]) \
        if layers.shape[0] else np.zeros((0, H))
    y = final_blend_B(weights, g, set_sum(V), sigma)
    return render_R(weights, y)


def render_opaque_only(weights, sigma, gbuf_rows) -> np.ndarray:
    """Opaque-only path: B and R with the rho input removed.

    Written independently of ``render_pixel``: B1's columns that multiply r
    are dropped instead of multiplying a zero vector.  ``gbuf_rows`` is [P][n_g].
    """
    _per_pixel_R(weights)
    W1, b1 = weights["B1"]
    W1 = _f64(W1)
    G = positional_encoding(gbuf_rows, pe_freqs(weights))
    n_g = G.shape[-1]
    Z = np.shape(sigma)[-1]
    keep = np.r_[0:n_g, W1.shape[1] - Z:W1.shape[1]]
    x = np.concatenate([G,
                        np.broadcast_to(_f64(sigma), np.shape(gbuf_rows)[:-1] + (Z,))], axis=-1)
    y = relu(x @ W1[:, keep].T + _f64(b1))
    y = relu(linear(y, *weights["B2"]))
    return render_R(weights, y)


def render_frame(weights, scene, gbuf, tbuf, counts, chunk: int = 16384,
                 pooling: str = "max_mean") -> np.ndarray:
    """Whole frame, vectorised over pixels; returns rgb float64 [3][h][w].

    ``gbuf`` [n_g][h][w], ``tbuf`` [K][n_t][h][w], ``counts`` [h][w].  Slots
    ``k >= counts`` are never read into the result.  Pixels are processed in
    chunks only to bound memory; every pixel's arithmetic is the same as
    ``render_pixel`` (``pooling="max_mean"``) or ``render_pixel_sum``
    (``pooling="sum"``, the paper's Eq. 5 form), up to the neural buffer y;
    R then runs on the whole frame's y (``render_R_frame``).
    """
    if pooling not in ("max_mean", "sum"):
        raise ValueError(f"pooling must be 'max_mean' or 'sum', got {pooling!r}")
    sigma = scene_encoder(weights, scene)
    n_g, h, w = np.shape(gbuf)
    K, n_t = np.shape(tbuf)[0], np.shape(tbuf)[1]
    P = h * w
    G = np.asarray(gbuf).reshape(n_g, P)
    T = np.asarray(tbuf).reshape(K, n_t, P)
    C = np.asarray(counts).reshape(P).astype(np.int64)
    H = np.shape(weights["phi2"][0])[0]
    Y = np.empty((P, H))
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        n = p1 - p0
        c = C[p0:p1]
        if np.any(c > K) or np.any(c < 0):
            raise ValueError("layer count outside 0..K")
        V = np.zeros((K, n, H))
        for k in range(K):
            idx = np.nonzero(c > k)[0]
            if idx.size:
                V[k, idx] = per_layer_h(weights, _f64(T[k][:, p0 + idx]).T, sigma)
        mask = np.arange(K)[:, None] < c[None, :]
        mx = np.where(mask[:, :, None], V, -np.inf).max(axis=0) if K else np.zeros((n, H))
        srt = np.sort(np.where(mask[:, :, None], V, np.inf), axis=0)
        s = np.zeros((n, H))
        for k in range(K):
            s = s + np.where((k < c)[:, None], srt[k], 0.0)
        if pooling == "sum":
            r = s  # tau: the sum over the valid layers, 0 without any
        else:
            has = c > 0
            r = np.zeros((n, H))
            if np.any(has):
                pool = np.concatenate([mx[has], s[has] / c[has][:, None]], axis=1)
                r[has] = post_pool_rho(weights, pool)
        Y[p0:p1] = final_blend_B(weights, _f64(G[:, p0:p1]).T, r, sigma)
    return render_R_frame(weights, Y.reshape(h, w, H))


def alpha_blend(colors, alphas) -> np.ndarray:
    """Order-dependent alpha compositing of Eq. 3-4 (a negative control).

    ``colors`` [t][3], ``alphas`` [t]; T = sum_i alpha_i C_i z_i with
    z_t = 1 and z_i = prod_{j=1}^{t-i} (1 - alpha_j) otherwise.
    """
    C, a = _f64(colors), _f64(alphas)
    t = a.shape[0]
    out = np.zeros(C.shape[1])
    for i in range(1, t + 1):
        z = 1.0 if i == t else float(np.prod(1.0 - a[: t - i]))
        out += a[i - 1] * C[i - 1] * z
    return out
