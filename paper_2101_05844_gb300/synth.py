"""Seeded synthetic inputs for the bounding problems (networks, input boxes, properties, splits).

This module draws random numbers and lays out plain arrays. It holds none of the bounding
method's arithmetic (no interval propagation, no duals, no relaxation). Both the CUDA path and the
CPU oracle consume what it produces, so it is the only code the two sides share.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), written here from its published definition, used as a counter-based
generator: value k of a stream with seed s is mix(s + (k + 1) * 0x9E3779B97F4A7C15). Uniforms take
the top 53 bits; normals use the Box-Muller transform.

Stand-ins for the paper's workloads (Section 8.1 and Table 1 of the paper): CIFAR-shaped 3x32x32
inputs in [0, 1], MNIST-shaped 784 inputs, He-initialised weights, L-infinity boxes of the paper's
radii, and branch-and-bound style ReLU splits.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + k * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """n integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)


# --------------------------------------------------------------------------------------------
# Network descriptions. A layer is a dict:
#   {"kind": "linear", "n_in", "n_out", "W": f32[n_out, n_in], "b": f32[n_out]}
#   {"kind": "conv", "in_shape": (c, h, w), "out_c", "kh", "kw", "stride", "pad",
#    "out_shape": (out_c, oh, ow), "n_in", "n_out", "W": f32[out_c, c, kh, kw], "b": f32[out_c]}
# Hidden layers are followed by a ReLU; the last layer is linear with no ReLU.
# --------------------------------------------------------------------------------------------

def conv_out(h: int, k: int, stride: int, pad: int) -> int:
    return (h + 2 * pad - k) // stride + 1


def arch(name: str) -> list[dict]:
    """Layer shapes (no weights) of the named architecture."""
    if name == "mlp_8_16_16_1":
        return _mlp([8, 16, 16, 1])
    if name == "mlp_784_1024x3_10":
        return _mlp([784, 1024, 1024, 1024, 10])
    if name == "wide_conv":  # 3x32x32 -> conv16 4x4 s2 -> conv32 4x4 s2 -> FC100 -> FC10
        return _convnet((3, 32, 32), [(16, 4, 2, 1), (32, 4, 2, 1)], [100, 10])
    if name == "conv4":  # 3x32x32 -> 4 conv 3x3 (32,32,64,64; s1,s2,s1,s2) -> FC512 -> FC10
        return _convnet((3, 32, 32), [(32, 3, 1, 1), (32, 3, 2, 1), (64, 3, 1, 1), (64, 3, 2, 1)],
                        [512, 10])
    if name.startswith("mlp_"):
        return _mlp([int(t) for t in name[4:].split("_")])
    raise ValueError(f"unknown architecture {name!r}")


def _mlp(widths: list[int]) -> list[dict]:
    return [{"kind": "linear", "n_in": a, "n_out": b} for a, b in zip(widths[:-1], widths[1:])]


def _convnet(in_shape, convs, fcs) -> list[dict]:
    layers = []
    c, h, w = in_shape
    for out_c, k, s, p in convs:
        oh, ow = conv_out(h, k, s, p), conv_out(w, k, s, p)
        layers.append({"kind": "conv", "in_shape": (c, h, w), "out_c": out_c, "kh": k, "kw": k,
                       "stride": s, "pad": p, "out_shape": (out_c, oh, ow),
                       "n_in": c * h * w, "n_out": out_c * oh * ow})
        c, h, w = out_c, oh, ow
    n = c * h * w
    for m in fcs:
        layers.append({"kind": "linear", "n_in": n, "n_out": m})
        n = m
    return layers


def small_convnet(in_shape=(2, 6, 6), convs=((3, 3, 2, 1), (4, 3, 1, 1)), fcs=(7, 3)) -> list[dict]:
    """A small conv net for tests: every kind of layer, tiles that do not divide evenly."""
    return _convnet(tuple(in_shape), list(convs), list(fcs))


def make_net(layers: list[dict], seed: int) -> list[dict]:
    """He-normal weights N(0, 2/fan_in) and U(-0.1, 0.1) biases, rounded to float32."""
    rng = SplitMix64(seed)
    net = []
    for L in layers:
        L = dict(L)
        if L["kind"] == "linear":
            fan_in = L["n_in"]
            shape = (L["n_out"], L["n_in"])
            nb = L["n_out"]
        else:
            c = L["in_shape"][0]
            fan_in = c * L["kh"] * L["kw"]
            shape = (L["out_c"], c, L["kh"], L["kw"])
            nb = L["out_c"]
        W = rng.normal(int(np.prod(shape))) * np.sqrt(2.0 / fan_in)
        L["W"] = W.reshape(shape).astype(np.float32)
        L["b"] = (rng.uniform(nb) * 0.2 - 0.1).astype(np.float32)
        net.append(L)
    return net


def forward(net: list[dict], x: np.ndarray) -> np.ndarray:
    """Network outputs for a batch of inputs x [B, n_0] (float64). Used only to pick properties."""
    import torch
    import torch.nn.functional as F

    h = torch.from_numpy(np.asarray(x, dtype=np.float64))
    for idx, L in enumerate(net):
        W = torch.from_numpy(L["W"].astype(np.float64))
        b = torch.from_numpy(L["b"].astype(np.float64))
        if L["kind"] == "linear":
            h = h.reshape(h.shape[0], -1) @ W.T + b
        else:
            h = F.conv2d(h.reshape(h.shape[0], *L["in_shape"]), W, b, stride=L["stride"],
                         padding=L["pad"]).reshape(h.shape[0], -1)
        if idx + 1 < len(net):
            h = torch.relu(h)
    return h.numpy()


def make_boxes(n0: int, S: int, eps: float, seed: int):
    """S input boxes [c - eps, c + eps] with centres c ~ U[0, 1]^n0 (not clipped to [0, 1])."""
    rng = SplitMix64(seed)
    c = rng.uniform(S * n0).reshape(S, n0)
    lo = (c - eps).astype(np.float32)
    hi = (c + eps).astype(np.float32)
    return c, lo, hi


def properties_all_targets(logits: np.ndarray) -> np.ndarray:
    """For one input: the rows e_y - e_t for every t != y, y = argmax logit."""
    n_out = logits.shape[-1]
    y = int(np.argmax(logits))
    rows = []
    for t in range(n_out):
        if t != y:
            r = np.zeros(n_out, np.float32)
            r[y], r[t] = 1.0, -1.0
            rows.append(r)
    return np.stack(rows)


def properties_runner_up(logits: np.ndarray) -> np.ndarray:
    """One row per input: e_y - e_t2 with y the top logit and t2 the runner-up."""
    S, n_out = logits.shape
    C = np.zeros((S, n_out), np.float32)
    order = np.argsort(-logits, axis=1, kind="stable")
    C[np.arange(S), order[:, 0]] = 1.0
    C[np.arange(S), order[:, 1]] = -1.0
    return C


def hidden_preactivations(net: list[dict], x: np.ndarray) -> np.ndarray:
    """Pre-activations of every hidden neuron (hidden layers concatenated) for a batch of inputs
    x [B, n_0], float64: the network's own forward pass."""
    import torch
    import torch.nn.functional as F

    h = torch.from_numpy(np.asarray(x, dtype=np.float64))
    out = []
    for L in net[:-1]:
        W = torch.from_numpy(L["W"].astype(np.float64))
        b = torch.from_numpy(L["b"].astype(np.float64))
        if L["kind"] == "linear":
            z = h.reshape(h.shape[0], -1) @ W.T + b
        else:
            z = F.conv2d(h.reshape(h.shape[0], *L["in_shape"]), W, b, stride=L["stride"],
                         padding=L["pad"]).reshape(h.shape[0], -1)
        out.append(z)
        h = torch.relu(z)
    return torch.cat(out, 1).numpy()


def sign_changing_neurons(net: list[dict], lo: np.ndarray, hi: np.ndarray, n_samples: int, seed: int) -> np.ndarray:
    """Indices of the hidden neurons whose pre-activation takes both signs over sampled points of the
    box [lo, hi] (half of them uniform, half random vertices). The network reaches both signs inside
    the box, so every sound pair of bounds of such a neuron straddles zero: these are neurons that
    branch and bound may split."""
    rng = SplitMix64(seed)
    n0 = lo.size
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    half = n_samples // 2
    X = lo64 + rng.uniform(half * n0).reshape(half, n0) * (hi64 - lo64)
    V = np.where(rng.uniform((n_samples - half) * n0).reshape(-1, n0) < 0.5, lo64, hi64)
    Z = hidden_preactivations(net, np.vstack([X, V]))
    return np.flatnonzero((Z.min(axis=0) < 0) & (Z.max(axis=0) > 0))


def make_splits(candidates: np.ndarray, n_hidden: int, S: int, max_splits: int, seed: int) -> np.ndarray:
    """Branch-and-bound style ReLU splits: int8 [S, n_hidden].

    Each subdomain fixes k ~ U{0..max_splits} distinct neurons drawn from `candidates` (neurons that
    change sign inside the root box), each active (+1) or inactive (-1) with probability 1/2; 0
    means free. A split takes effect only where the neuron's bounds, with the splits of the layers
    before it applied, still straddle zero (the bounding code decides that).
    """
    rng = SplitMix64(seed)
    cand = np.asarray(candidates, np.int64)
    out = np.zeros((S, n_hidden), np.int8)
    for s in range(S):
        k = min(int(rng.integers(1, 0, max_splits)[0]), cand.size)
        # distinct candidates by a partial Fisher-Yates shuffle driven by the stream
        idx = cand.copy()
        for a in range(k):
            r = a + int(rng.integers(1, 0, cand.size - 1 - a)[0])
            idx[a], idx[r] = idx[r], idx[a]
        signs = np.where(rng.uniform(k) < 0.5, -1, 1).astype(np.int8)
        out[s, idx[:k]] = signs
    return out


def make_caps(S: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return SplitMix64(seed).integers(S, lo, hi).astype(np.int32)


# --------------------------------------------------------------------------------------------
# The workloads, by name and size.
# --------------------------------------------------------------------------------------------

def problem(name: str, S: int | None = None, seed: int = 0, part: tuple[int, int] | None = None) -> dict:
    """A complete synthetic bounding problem.

    Returns {"net", "lo", "hi", "C", "splits", "caps", "eps"}: C is the property matrix
    [S, n_out] (each subproblem lower-bounds C[s] . network(x) over its box). part = (a, b): only
    subproblems a .. b - 1 of the batch of S (the same values as in the whole batch; conv4 only).
    """
    base = 1000 * seed
    if name == "mlp_tiny":  # MLP 8-16-16-1, one box of half-width 0.1 around a U[0,1]^8 centre
        layers = arch("mlp_8_16_16_1")
        net = make_net(layers, base + 1)
        S = S or 1
        _, lo, hi = make_boxes(8, S, 0.1, base + 2)
        C = np.ones((S, 1), np.float32)
        return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=0.1)
    if name in ("wide_conv", "wide_conv_bab"):
        layers = arch("wide_conv")
        net = make_net(layers, base + 1)
        eps = 2.0 / 255.0
        if name == "wide_conv":  # one image, the 9 logit differences e_y - e_t
            c, lo1, hi1 = make_boxes(3072, 1, eps, base + 2)
            C = properties_all_targets(forward(net, c)[0])
            S2 = C.shape[0]
            lo = np.repeat(lo1, S2, axis=0)
            hi = np.repeat(hi1, S2, axis=0)
            return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=eps)
        S = S or 4096  # branch-and-bound batch: subdomains of one root box
        c, lo1, hi1 = make_boxes(3072, 1, eps, base + 2)
        C1 = properties_runner_up(forward(net, c))
        lo = np.repeat(lo1, S, axis=0)
        hi = np.repeat(hi1, S, axis=0)
        C = np.repeat(C1, S, axis=0)
        cand = sign_changing_neurons(net, lo1[0], hi1[0], 512, base + 5)
        splits = make_splits(cand, sum(L["n_out"] for L in layers[:-1]), S, 20, base + 3)
        caps = make_caps(S, 1, 5, base + 4)
        return dict(net=net, lo=lo, hi=hi, C=C, splits=splits, caps=caps, eps=eps)
    if name == "conv4":
        layers = arch("conv4")
        net = make_net(layers, base + 1)
        S = S or 1024
        eps = 8.0 / 255.0
        c, lo, hi = make_boxes(3072, S, eps, base + 2)
        if part is not None:
            c, lo, hi = c[part[0]:part[1]], lo[part[0]:part[1]], hi[part[0]:part[1]]
        C = properties_runner_up(forward(net, c))
        return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=eps)
    if name == "mlp_wide":
        layers = arch("mlp_784_1024x3_10")
        net = make_net(layers, base + 1)
        S = S or 256
        c, lo, hi = make_boxes(784, S, 0.1, base + 2)
        C = properties_runner_up(forward(net, c))
        return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=0.1)
    if name == "small_conv":  # small conv net with every layer kind, for parity tests
        layers = small_convnet()
        net = make_net(layers, base + 1)
        S = S or 3
        c, lo, hi = make_boxes(layers[0]["n_in"], S, 0.15, base + 2)
        C = properties_runner_up(forward(net, c))
        return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=0.15)
    if name.startswith("mlp_"):  # "mlp_<w0>_<w1>_..." random MLP, S boxes of half-width 0.1
        layers = arch(name)
        net = make_net(layers, base + 1)
        S = S or 2
        c, lo, hi = make_boxes(layers[0]["n_in"], S, 0.1, base + 2)
        n_out = layers[-1]["n_out"]
        C = properties_runner_up(forward(net, c)) if n_out > 1 else np.ones((S, 1), np.float32)
        return dict(net=net, lo=lo, hi=hi, C=C, splits=None, caps=None, eps=0.1)
    raise ValueError(f"unknown problem {name!r}")


def random_duals(rng: SplitMix64, widths: list[int], S: int, scale: float = 0.3,
                 p_zero: float = 0.3) -> np.ndarray:
    """Non-negative dual values with a share of exact zeros: float32 [S, sum(widths)]."""
    n = S * sum(widths)
    v = rng.uniform(n) * scale
    v[rng.uniform(n) < p_zero] = 0.0
    return v.astype(np.float32).reshape(S, -1)
