"""Seeded synthetic inputs for the Evoformer block.

This module draws random numbers and lays them out; it holds none of the
block's arithmetic. Both the CUDA path (tests, bench) and the FP64 oracle are
fed from it, so the two sides see the same bytes.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used counter-style: the i-th 64-bit word of a
stream with key ``k`` is ``mix(k + (i + 1) * GOLDEN)``. Pairs of words become
uniforms in (0, 1) (53-bit mantissa, offset by half an ulp so 0 never
occurs) and pairs of uniforms become standard normals by Box-Muller.

Each tensor gets its own stream key ``mix(seed * 1_000_003 + tag)``, tags in
the fixed order m, z, params, masks, cotangents, so that adding a tensor never
shifts the bytes of another.  The default seed is 32, the paper's fixed
random seed (Sec. "Hyperparameter setting").
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TAG_M, TAG_Z, TAG_PARAMS, TAG_MASK, TAG_COT_M, TAG_COT_Z = 1, 2, 3, 4, 5, 6
TAG_DROPOUT = 7  # + index of the dropout site


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> int:
    x = np.array([(seed * 1_000_003 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return int(_mix(x)[0])


def words(key: int, n: int, start: int = 0) -> np.ndarray:
    """n SplitMix64 outputs of stream ``key`` from counter ``start``."""
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + idx * GOLDEN)


def uniforms(key: int, n: int) -> np.ndarray:
    w = words(key, n)
    return ((w >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(key: int, n: int) -> np.ndarray:
    half = (n + 1) // 2
    u = uniforms(key, 2 * half)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * half, dtype=np.float64)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


@dataclass(frozen=True)
class Dims:
    """Channel and size settings of one Evoformer block (mirrors ``evo_dims``)."""

    n_seq: int
    n_res: int
    c_m: int = 256
    c_z: int = 128
    h_msa: int = 8
    c_msa: int = 32
    h_tri: int = 4
    c_tri: int = 32
    c_mul: int = 128
    c_opm: int = 32
    trans_n: int = 4
    msa_col_mode: int = 0  # 0 column attention, 1 global column attention
    pair_only: int = 0     # 1: a template pair stack block (pair half only, AF2 Alg. 16)

    def replace(self, **kw) -> "Dims":
        d = dict(self.__dict__)
        d.update(kw)
        return Dims(**d)


# Named workloads: the paper's initial-training crop (Table "model settings",
# N_res=256, N_seq=128, C_m=256, C_z=128, 8 heads) and the smaller shapes used
# for parity and finite differences.
DIMS_SMALL_FP32 = Dims(n_seq=16, n_res=64)
DIMS_TRAIN_CROP = Dims(n_seq=128, n_res=256)
DIMS_EXTRA_MSA = Dims(n_seq=1024, n_res=256, c_m=64, h_msa=8, c_msa=8, msa_col_mode=1)
DIMS_TINY = Dims(n_seq=3, n_res=5, c_m=8, c_z=4, h_msa=2, c_msa=4, h_tri=2, c_tri=4,
                 c_mul=4, c_opm=2, trans_n=2)
# Template pair stack block (AF2 Alg. 16, published template dims): c_t = 64,
# triangle multiplication 64 channels, triangle attention 4 heads of 16,
# pair transition factor 2.  The MSA fields are unused (n_seq = 1).
DIMS_TEMPLATE = Dims(n_seq=1, n_res=256, c_z=64, h_tri=4, c_tri=16, c_mul=64, trans_n=2, pair_only=1)


def param_entries(d: Dims):
    """(name, shape, kind) of each parameter tensor of one block, in buffer order.

    kind is 'gamma', 'beta', 'weight' or 'bias'; it decides the init rule.
    The layout is the library's flat parameter buffer (each tensor starts on a
    256-byte boundary, the alignment the paper uses for its fused tensors).
    """
    hm, cm, ht, ct = d.h_msa, d.c_msa, d.h_tri, d.c_tri
    e = []

    def ln(prefix, c):
        e.append((prefix + ".gamma", (c,), "gamma"))
        e.append((prefix + ".beta", (c,), "beta"))

    if d.pair_only:
        _pair_entries(d, e, ln)
        return e
    ln("row.ln_m", d.c_m)
    ln("row.ln_z", d.c_z)
    e.append(("row.w_b", (hm, d.c_z), "weight"))
    e.append(("row.w_qkvg", (4 * hm * cm, d.c_m), "weight"))
    e.append(("row.b_g", (hm * cm,), "bias"))
    e.append(("row.w_o", (d.c_m, hm * cm), "weight"))
    e.append(("row.b_o", (d.c_m,), "bias"))
    ln("col.ln", d.c_m)
    if d.msa_col_mode == 0:
        e.append(("col.w_qkvg", (4 * hm * cm, d.c_m), "weight"))
    else:
        e.append(("col.w_qkvg", (2 * hm * cm + 2 * cm, d.c_m), "weight"))
    e.append(("col.b_g", (hm * cm,), "bias"))
    e.append(("col.w_o", (d.c_m, hm * cm), "weight"))
    e.append(("col.b_o", (d.c_m,), "bias"))
    ln("msa_trans.ln", d.c_m)
    e.append(("msa_trans.w1", (d.trans_n * d.c_m, d.c_m), "weight"))
    e.append(("msa_trans.b1", (d.trans_n * d.c_m,), "bias"))
    e.append(("msa_trans.w2", (d.c_m, d.trans_n * d.c_m), "weight"))
    e.append(("msa_trans.b2", (d.c_m,), "bias"))
    ln("opm.ln", d.c_m)
    e.append(("opm.w_ab", (2 * d.c_opm, d.c_m), "weight"))
    e.append(("opm.b_ab", (2 * d.c_opm,), "bias"))
    e.append(("opm.w_o", (d.c_z, d.c_opm * d.c_opm), "weight"))
    e.append(("opm.b_o", (d.c_z,), "bias"))
    _pair_entries(d, e, ln)
    return e


def _pair_entries(d: Dims, e: list, ln):
    """The pair-stack tensors (triangle multiplications, triangle attentions,
    pair transition), shared by the Evoformer and the template pair block."""
    ht, ct = d.h_tri, d.c_tri
    for t in ("tri_out", "tri_in"):
        ln(t + ".ln_in", d.c_z)
        e.append((t + ".w_abg", (4 * d.c_mul + d.c_z, d.c_z), "weight"))
        e.append((t + ".b_abg", (4 * d.c_mul + d.c_z,), "bias"))
        ln(t + ".ln_out", d.c_mul)
        e.append((t + ".w_o", (d.c_z, d.c_mul), "weight"))
        e.append((t + ".b_o", (d.c_z,), "bias"))
    for t in ("att_start", "att_end"):
        ln(t + ".ln", d.c_z)
        e.append((t + ".w_b", (ht, d.c_z), "weight"))
        e.append((t + ".w_qkvg", (4 * ht * ct, d.c_z), "weight"))
        e.append((t + ".b_g", (ht * ct,), "bias"))
        e.append((t + ".w_o", (d.c_z, ht * ct), "weight"))
        e.append((t + ".b_o", (d.c_z,), "bias"))
    ln("pair_trans.ln", d.c_z)
    e.append(("pair_trans.w1", (d.trans_n * d.c_z, d.c_z), "weight"))
    e.append(("pair_trans.b1", (d.trans_n * d.c_z,), "bias"))
    e.append(("pair_trans.w2", (d.c_z, d.trans_n * d.c_z), "weight"))
    e.append(("pair_trans.b2", (d.c_z,), "bias"))


ALIGN_FLOATS = 64  # 256 bytes


def param_layout(d: Dims):
    """[(name, offset, shape, kind)] and the padded total count in floats."""
    out, off = [], 0
    for name, shape, kind in param_entries(d):
        out.append((name, off, shape, kind))
        n = int(np.prod(shape))
        off += (n + ALIGN_FLOATS - 1) // ALIGN_FLOATS * ALIGN_FLOATS
    return out, off


def make_params(d: Dims, seed: int = 32) -> np.ndarray:
    """Flat FP32 parameter buffer with the init rule below, zeros in padding.

    weights and biases ~ N(0, 1/fan_in); LayerNorm gamma = 1 + 0.1 N(0,1),
    beta = 0.1 N(0,1).  Zero-initialised gates/outputs (as in the published
    training recipe) would make the block an identity map with degenerate
    gradients, so every tensor is random here.
    """
    layout, total = param_layout(d)
    buf = np.zeros(total, dtype=np.float32)
    key = stream_key(seed, TAG_PARAMS)
    draws = normals(key, total)
    for name, off, shape, kind in layout:
        n = int(np.prod(shape))
        r = draws[off:off + n]
        if kind == "gamma":
            v = 1.0 + 0.1 * r
        elif kind == "beta":
            v = 0.1 * r
        else:
            # fan_in of a bias is that of the weight it follows
            fan_in = shape[-1] if kind == "weight" else _bias_fan_in(layout, name)
            v = r / math.sqrt(fan_in)
        buf[off:off + n] = v.astype(np.float32)
    return buf


def _bias_fan_in(layout, name):
    prefix = name.rsplit(".", 1)[0]
    leaf = name.rsplit(".", 1)[1]
    want = {"b_g": "w_qkvg", "b_o": "w_o", "b1": "w1", "b2": "w2", "b_ab": "w_ab",
            "b_abg": "w_abg"}[leaf]
    for n, _, shape, _ in layout:
        if n == prefix + "." + want:
            return shape[-1]
    raise KeyError(name)


def unpack_params(d: Dims, buf) -> dict:
    """name -> view of the flat buffer (numpy or torch), shaped."""
    layout, _ = param_layout(d)
    out = {}
    for name, off, shape, _ in layout:
        n = int(np.prod(shape))
        out[name] = buf[off:off + n].reshape(shape)
    return out


def make_activations(d: Dims, seed: int = 32):
    """m [S,R,c_m], z [R,R,c_z] ~ N(0,1), FP32."""
    S, R = d.n_seq, d.n_res
    m = normals(stream_key(seed, TAG_M), S * R * d.c_m).astype(np.float32).reshape(S, R, d.c_m)
    z = normals(stream_key(seed, TAG_Z), R * R * d.c_z).astype(np.float32).reshape(R, R, d.c_z)
    return m, z


def make_masks(d: Dims, seed: int = 32, pad_frac: float = 0.0, trailing: bool = False):
    """msa_mask [S,R], pair_mask [R,R] in {0,1} FP32 built from a residue mask.

    ceil(pad_frac * R) residues are padded: chosen at random (seeded) or, with
    ``trailing``, the last ones. msa_mask[s,i] = seq_mask[i] and
    pair_mask[i,j] = seq_mask[i] * seq_mask[j].
    """
    S, R = d.n_seq, d.n_res
    seq = np.ones(R, dtype=np.float32)
    k = int(math.ceil(pad_frac * R)) if pad_frac > 0 else 0
    if k:
        if trailing:
            seq[R - k:] = 0
        else:
            keys = uniforms(stream_key(seed, TAG_MASK), R)
            seq[np.argsort(keys, kind="stable")[:k]] = 0
    msa_mask = np.broadcast_to(seq[None, :], (S, R)).copy()
    pair_mask = (seq[:, None] * seq[None, :]).astype(np.float32)
    return msa_mask, pair_mask


def make_cotangents(d: Dims, seed: int = 32, msa_mask=None, pair_mask=None):
    """Seeded N(0,1) cotangents for m_out and z_out, zeroed at padded positions."""
    S, R = d.n_seq, d.n_res
    gm = normals(stream_key(seed, TAG_COT_M), S * R * d.c_m).astype(np.float32).reshape(S, R, d.c_m)
    gz = normals(stream_key(seed, TAG_COT_Z), R * R * d.c_z).astype(np.float32).reshape(R, R, d.c_z)
    if msa_mask is not None:
        gm = gm * msa_mask[:, :, None]
    if pair_mask is not None:
        gz = gz * pair_mask[:, :, None]
    return gm.astype(np.float32), gz.astype(np.float32)


def make_problem(d: Dims, seed: int = 32, pad_frac: float = 0.0, trailing: bool = False):
    """Everything one block call needs, as FP32 numpy arrays."""
    m, z = make_activations(d, seed)
    msa_mask, pair_mask = make_masks(d, seed, pad_frac, trailing)
    params = make_params(d, seed)
    gm, gz = make_cotangents(d, seed, msa_mask, pair_mask)
    return dict(m=m, z=z, msa_mask=msa_mask, pair_mask=pair_mask, params=params, gm=gm, gz=gz)


# Training-mode dropout sites of the Evoformer block (AF2 Alg. 6): the update
# each one scales, its rate, its shape and which axis of the updated tensor
# shares one draw ("row": the same scale for every row, i.e. every MSA
# sequence or every pair row i; "col": every pair column j).
DROPOUT_SITES = (
    ("msa_row", 0.15, "row"),    # MSA row attention with pair bias, [N_res, c_m]
    ("tri_out", 0.25, "row"),    # triangle multiplication outgoing, [N_res, c_z]
    ("tri_in", 0.25, "row"),     # triangle multiplication incoming
    ("att_start", 0.25, "row"),  # triangle attention starting node
    ("att_end", 0.25, "col"),    # triangle attention ending node, [N_res (i), c_z]
)


def make_dropout(d: Dims, seed: int = 32, scale_rates: float = 1.0) -> dict:
    """Seeded dropout scales: for each site an FP32 array of shape
    [N_res, channels] holding 0 (dropped, probability rate) or 1 / (1 - rate).
    The random draws are inputs of the block, so the CUDA path and the oracle
    apply the same scales.  ``scale_rates`` multiplies every rate (0 gives
    all-ones scales)."""
    out = {}
    for k, (name, rate, _) in enumerate(DROPOUT_SITES):
        rate = rate * scale_rates
        C = d.c_m if name == "msa_row" else d.c_z
        u = uniforms(stream_key(seed, TAG_DROPOUT + k), d.n_res * C).reshape(d.n_res, C)
        keep = (u >= rate).astype(np.float64)
        out[name] = (keep / (1.0 - rate)).astype(np.float32)
    return out


TAG_ADAM = 20  # + index of the tensor in ADAM_TENSORS
# Buffers of the fused training update and the scale of their values: weights
# about N(0, 0.05^2), gradients about N(0, 0.01^2), the moments of a run
# that has taken a few steps.
ADAM_TENSORS = ("params", "grad", "exp_avg", "exp_avg_sq", "ema")


def make_adam_state(n: int, seed: int = 32, fresh: bool = False, base: int = 1 << 20) -> dict:
    """Seeded FP32 buffers of n elements for the fused training update.

    Arrays longer than ``base`` repeat a ``base``-element draw, each repeat
    multiplied by its own factor in [0.5, 1.5), so that large buffers are
    cheap to make and still differ from tile to tile.  ``fresh``: the state
    before the first step (zero moments, EMA equal to the parameters)."""
    def draw(k, sd):
        m = min(n, base)
        x = normals(stream_key(seed, TAG_ADAM + k), m) * sd
        if n <= base:
            return x.astype(np.float32)
        reps = (n + base - 1) // base
        f = 0.5 + uniforms(stream_key(seed, TAG_ADAM + 10 + k), reps)
        return (f.astype(np.float32)[:, None] * x.astype(np.float32)[None, :]).reshape(-1)[:n]

    out = {"params": draw(0, 0.05), "grad": draw(1, 0.01)}
    if fresh:
        out["exp_avg"] = np.zeros(n, np.float32)
        out["exp_avg_sq"] = np.zeros(n, np.float32)
        out["ema"] = out["params"].copy()
    else:
        out["exp_avg"] = draw(2, 1e-3)
        out["exp_avg_sq"] = np.square(draw(3, 1e-2))
        out["ema"] = out["params"] + draw(4, 1e-3)
    return out
