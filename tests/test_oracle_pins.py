"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test states what fixes the expected value: a library routine the case
reduces to, a closed form, a symmetry of the AlphaFold2 Evoformer, or a
constructed input whose answer is known by inspection.
"""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import evoformer as O
from paper_2207_05477_gb300 import synth

DT = torch.float64
TINY = synth.DIMS_TINY


def _params(d, seed=7):
    buf = synth.make_params(d, seed)
    return {k: torch.tensor(np.array(v), dtype=DT) for k, v in synth.unpack_params(d, buf).items()}


def _acts(d, seed=7):
    m, z = synth.make_activations(d, seed)
    return torch.tensor(m, dtype=DT), torch.tensor(z, dtype=DT)


def _ones_masks(d):
    return torch.ones(d.n_seq, d.n_res, dtype=DT), torch.ones(d.n_res, d.n_res, dtype=DT)


# ---------------------------------------------------------------- LayerNorm

def test_layer_norm_matches_library_and_closed_form():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(7, 16, generator=g, dtype=DT) * 3 + 1
    gamma = torch.randn(16, generator=g, dtype=DT)
    beta = torch.randn(16, generator=g, dtype=DT)
    ref = F.layer_norm(x, (16,), gamma, beta, eps=1e-5)
    assert torch.allclose(O.layer_norm(x, gamma, beta), ref, atol=1e-12, rtol=0)
    # closed form on a worked input: x = [1,2,3,4]: mean 2.5, biased var 1.25
    y = O.layer_norm(torch.tensor([1.0, 2, 3, 4], dtype=DT), torch.ones(4, dtype=DT),
                     torch.zeros(4, dtype=DT))
    expect = torch.tensor([-1.5, -0.5, 0.5, 1.5], dtype=DT) / math.sqrt(1.25 + 1e-5)
    assert torch.allclose(y, expect, atol=1e-14, rtol=0)
    # normalised rows: mean 0 and variance var/(var+eps) before the affine map
    y = O.layer_norm(x, torch.ones(16, dtype=DT), torch.zeros(16, dtype=DT))
    v = x.var(dim=-1, unbiased=False)
    assert torch.allclose(y.mean(-1), torch.zeros(7, dtype=DT), atol=1e-13)
    assert torch.allclose(y.var(-1, unbiased=False), v / (v + 1e-5), atol=1e-12)


# --------------------------------------------------------------- softmax

def test_masked_softmax_against_library():
    g = torch.Generator().manual_seed(1)
    l = torch.randn(4, 9, generator=g, dtype=DT)
    full = torch.ones(4, 9, dtype=torch.bool)
    assert torch.allclose(O.masked_softmax(l, full), torch.softmax(l, -1), atol=1e-15)
    valid = torch.rand(4, 9, generator=g) > 0.4
    valid[:, 0] = True
    valid[3] = False  # a row with no valid key
    a = O.masked_softmax(l, valid)
    assert torch.all(a[~valid] == 0)
    assert torch.allclose(a[:3].sum(-1), torch.ones(3, dtype=DT), atol=1e-15)
    assert torch.all(a[3] == 0)
    # restricted to the valid keys it is the library softmax of those keys
    for r in range(3):
        idx = valid[r].nonzero().flatten()
        assert torch.allclose(a[r, idx], torch.softmax(l[r, idx], -1), atol=1e-15)


# ------------------------------------------------------------ row attention

def _attn_dims():
    # c_m = h*c so that W_o = I exposes the gated attention output directly
    return synth.Dims(n_seq=3, n_res=6, c_m=8, c_z=4, h_msa=2, c_msa=4, h_tri=2, c_tri=4,
                      c_mul=4, c_opm=2, trans_n=2)


def _expose_output(p, prefix, c_m):
    p[prefix + ".w_o"] = torch.eye(c_m, dtype=DT)
    p[prefix + ".b_o"] = torch.zeros(c_m, dtype=DT)


def test_row_attention_reduces_to_sdpa():
    """bias 0, saturated gate, all keys valid -> library scaled-dot-product attention."""
    d = _attn_dims()
    p = _params(d)
    m, z = _acts(d)
    msa_mask, _ = _ones_masks(d)
    _expose_output(p, "row", d.c_m)
    p["row.w_b"] = torch.zeros_like(p["row.w_b"])
    p["row.b_g"] = torch.full_like(p["row.b_g"], 60.0)  # sigmoid(60) = 1 - 9e-27
    out = O.msa_row_attention_with_pair_bias(m, z, msa_mask, p, d.h_msa, d.c_msa)
    x = F.layer_norm(m, (d.c_m,), p["row.ln_m.gamma"], p["row.ln_m.beta"], eps=1e-5)
    H, c = d.h_msa, d.c_msa
    w = p["row.w_qkvg"]
    q = (x @ w[:H * c].T).reshape(d.n_seq, d.n_res, H, c).permute(0, 2, 1, 3)
    k = (x @ w[H * c:2 * H * c].T).reshape(d.n_seq, d.n_res, H, c).permute(0, 2, 1, 3)
    v = (x @ w[2 * H * c:3 * H * c].T).reshape(d.n_seq, d.n_res, H, c).permute(0, 2, 1, 3)
    ref = F.scaled_dot_product_attention(q, k, v).permute(0, 2, 1, 3).reshape(d.n_seq, d.n_res, H * c)
    assert torch.allclose(out, ref, atol=1e-12)


def test_row_attention_weights_sum_to_one_and_respect_mask():
    d = _attn_dims()
    p = _params(d)
    m, z = _acts(d)
    msa_mask, _ = _ones_masks(d)
    msa_mask[1, 2] = 0
    msa_mask[2, 4] = 0
    _, a = O.msa_row_attention_with_pair_bias(m, z, msa_mask, p, d.h_msa, d.c_msa, return_weights=True)
    assert torch.allclose(a.sum(-1), torch.ones_like(a.sum(-1)), atol=1e-14)
    assert torch.all(a[1, :, :, 2] == 0) and torch.all(a[2, :, :, 4] == 0)


def test_row_attention_single_valid_key_and_zero_query():
    d = _attn_dims()
    p = _params(d)
    m, z = _acts(d)
    H, c, S, R = d.h_msa, d.c_msa, d.n_seq, d.n_res
    _expose_output(p, "row", d.c_m)
    x = F.layer_norm(m, (d.c_m,), p["row.ln_m.gamma"], p["row.ln_m.beta"], eps=1e-5)
    w = p["row.w_qkvg"]
    v = (x @ w[2 * H * c:3 * H * c].T)
    g = torch.sigmoid(x @ w[3 * H * c:].T + p["row.b_g"])
    # only key 3 valid in every row: every query returns g * v[key 3]
    mk = torch.zeros(S, R, dtype=DT)
    mk[:, 3] = 1
    out = O.msa_row_attention_with_pair_bias(m, z, mk, p, H, c)
    assert torch.allclose(out, g * v[:, 3:4, :], atol=1e-12)
    # q = 0 and no pair bias: uniform weights -> masked mean of v
    p["row.w_qkvg"] = w.clone()
    p["row.w_qkvg"][:H * c] = 0
    p["row.w_b"] = torch.zeros_like(p["row.w_b"])
    mk = torch.ones(S, R, dtype=DT)
    mk[0, 1] = 0
    mk[2, 5] = 0
    out = O.msa_row_attention_with_pair_bias(m, z, mk, p, H, c)
    mean_v = (v * mk[..., None]).sum(1, keepdim=True) / mk.sum(1)[:, None, None]
    assert torch.allclose(out, g * mean_v, atol=1e-12)


def _selector_pair(R, c_z, perm, big=10.0):
    """z with z[a, perm[a]] = big e_0 and every other position big e_1.

    After LayerNorm the two kinds of position differ only in which channel is
    high, so a bias projection W_b = [s, 0, ...] is large exactly at the
    (a, perm[a]) positions.
    """
    z = torch.zeros(R, R, c_z, dtype=DT)
    z[..., 1] = big
    for a in range(R):
        z[a, perm[a], 1] = 0
        z[a, perm[a], 0] = big
    return z


def test_row_attention_pair_bias_orientation():
    """bias b_ij (query i, key j): a large b at (i, perm[i]) selects key perm[i]."""
    d = _attn_dims()
    p = _params(d)
    m, _ = _acts(d)
    S, R, H, c = d.n_seq, d.n_res, d.h_msa, d.c_msa
    perm = [2, 0, 5, 1, 3, 4]  # not an involution: perm != perm^-1
    z = _selector_pair(R, d.c_z, perm)
    p["row.ln_z.gamma"] = torch.ones(d.c_z, dtype=DT)
    p["row.ln_z.beta"] = torch.zeros(d.c_z, dtype=DT)
    p["row.w_b"] = torch.zeros(H, d.c_z, dtype=DT)
    p["row.w_b"][:, 0] = 40.0
    _expose_output(p, "row", d.c_m)
    out = O.msa_row_attention_with_pair_bias(m, z, torch.ones(S, R, dtype=DT), p, H, c)
    x = F.layer_norm(m, (d.c_m,), p["row.ln_m.gamma"], p["row.ln_m.beta"], eps=1e-5)
    w = p["row.w_qkvg"]
    v = x @ w[2 * H * c:3 * H * c].T
    g = torch.sigmoid(x @ w[3 * H * c:].T + p["row.b_g"])
    expect = g * v[:, perm, :]
    assert torch.allclose(out, expect, atol=1e-6)


def test_row_attention_msa_row_permutation_and_independence():
    d = _attn_dims()
    p = _params(d)
    m, z = _acts(d)
    msa_mask, _ = _ones_masks(d)
    msa_mask[0, 1] = 0
    out = O.msa_row_attention_with_pair_bias(m, z, msa_mask, p, d.h_msa, d.c_msa)
    perm = torch.tensor([2, 0, 1])
    out_p = O.msa_row_attention_with_pair_bias(m[perm], z, msa_mask[perm], p, d.h_msa, d.c_msa)
    assert torch.allclose(out_p, out[perm], atol=1e-13)
    m2 = m.clone()
    m2[1] = m2[1] * 2.0 + torch.linspace(-1, 1, d.c_m, dtype=DT)  # LN is shift-invariant
    out2 = O.msa_row_attention_with_pair_bias(m2, z, msa_mask, p, d.h_msa, d.c_msa)
    assert torch.allclose(out2[0], out[0], atol=1e-14) and torch.allclose(out2[2], out[2], atol=1e-14)
    assert not torch.allclose(out2[1], out[1])


# ------------------------------------------------------------ column attention

def test_column_attention_reduces_to_sdpa_and_is_row_equivariant():
    d = _attn_dims()
    p = _params(d)
    m, _ = _acts(d)
    msa_mask, _ = _ones_masks(d)
    _expose_output(p, "col", d.c_m)
    p["col.b_g"] = torch.full_like(p["col.b_g"], 60.0)
    out = O.msa_column_attention(m, msa_mask, p, d.h_msa, d.c_msa)
    H, c, S, R = d.h_msa, d.c_msa, d.n_seq, d.n_res
    x = F.layer_norm(m, (d.c_m,), p["col.ln.gamma"], p["col.ln.beta"], eps=1e-5)
    w = p["col.w_qkvg"]
    sh = lambda t: t.reshape(S, R, H, c).permute(1, 2, 0, 3)  # [R,H,S,c]
    q, k, v = (sh(x @ w[i * H * c:(i + 1) * H * c].T) for i in range(3))
    ref = F.scaled_dot_product_attention(q, k, v).permute(2, 0, 1, 3).reshape(S, R, H * c)
    assert torch.allclose(out, ref, atol=1e-12)
    perm = torch.tensor([1, 2, 0])
    msa_mask[2, 3] = 0
    out = O.msa_column_attention(m, msa_mask, p, H, c)
    out_p = O.msa_column_attention(m[perm], msa_mask[perm], p, H, c)
    assert torch.allclose(out_p, out[perm], atol=1e-13)


def test_column_attention_masked_column_gives_zero_attention():
    d = _attn_dims()
    p = _params(d)
    m, _ = _acts(d)
    msa_mask, _ = _ones_masks(d)
    msa_mask[:, 4] = 0  # padded residue: no valid key in column 4
    _expose_output(p, "col", d.c_m)
    out = O.msa_column_attention(m, msa_mask, p, d.h_msa, d.c_msa)
    assert torch.all(out[:, 4] == 0)
    _, a = O.msa_column_attention(m, msa_mask, p, d.h_msa, d.c_msa, return_weights=True)
    s = a.sum(-1)
    assert torch.allclose(s[[0, 1, 2, 3, 5]], torch.ones_like(s[[0, 1, 2, 3, 5]]), atol=1e-14)


# ------------------------------------------------------------ global column

def test_global_column_attention_special_cases():
    d = synth.Dims(n_seq=5, n_res=4, c_m=8, c_z=4, h_msa=2, c_msa=4, msa_col_mode=1,
                   h_tri=2, c_tri=4, c_mul=4, c_opm=2, trans_n=2)
    p = _params(d)
    m, _ = _acts(d)
    S, R, H, c = d.n_seq, d.n_res, d.h_msa, d.c_msa
    _expose_output(p, "col", d.c_m)
    x = F.layer_norm(m, (d.c_m,), p["col.ln.gamma"], p["col.ln.beta"], eps=1e-5)
    w = p["col.w_qkvg"]
    v = x @ w[H * c + c:H * c + 2 * c].T                     # [S,R,c] single head
    g = torch.sigmoid(x @ w[H * c + 2 * c:].T + p["col.b_g"])  # [S,R,H*c]
    # W_q = 0: uniform weights over valid sequences -> masked mean of v
    p0 = dict(p)
    p0["col.w_qkvg"] = w.clone()
    p0["col.w_qkvg"][:H * c] = 0
    mk = torch.ones(S, R, dtype=DT)
    mk[1, 0] = 0
    mk[3, 2] = 0
    out = O.msa_global_column_attention(m, mk, p0, H, c)
    mean_v = (v * mk[..., None]).sum(0) / mk.sum(0)[:, None]     # [R,c]
    expect = g * mean_v.repeat(1, H)[None]
    assert torch.allclose(out, expect, atol=1e-12)
    # only sequence 2 valid in every column -> every row gets g * v[2]
    mk = torch.zeros(S, R, dtype=DT)
    mk[2] = 1
    out = O.msa_global_column_attention(m, mk, p, H, c)
    assert torch.allclose(out, g * v[2].repeat(1, H)[None], atol=1e-12)
    # weights sum to one per (column, head)
    _, a = O.msa_global_column_attention(m, torch.ones(S, R, dtype=DT), p, H, c, return_weights=True)
    assert torch.allclose(a.sum(-1), torch.ones(R, H, dtype=DT), atol=1e-14)


def test_global_column_attention_hand_computed():
    """Alg. 19 written out scalar by scalar on one residue column: three
    sequences with distinct query rows, sequence 1 masked, so the mean query
    is over sequences 0 and 2 only and the softmax has the two valid keys 0
    and 2.  Each head's output is g * (a_0 v_0 + a_2 v_2) with
    a_0 = 1 / (1 + exp((l_2 - l_0))) and l_t = qbar . k_t / sqrt(c).  An
    unmasked mean, a missing 1/sqrt(c) or a mask ignored on the keys each
    change the result (checked)."""
    d = synth.Dims(n_seq=3, n_res=1, c_m=8, c_z=4, h_msa=2, c_msa=4, msa_col_mode=1,
                   h_tri=2, c_tri=4, c_mul=4, c_opm=2, trans_n=2)
    p = _params(d, seed=11)
    m, _ = _acts(d, seed=11)
    S, H, c = d.n_seq, d.h_msa, d.c_msa
    _expose_output(p, "col", d.c_m)
    mk = torch.ones(S, 1, dtype=DT)
    mk[1, 0] = 0
    out = O.msa_global_column_attention(m, mk, p, H, c)

    x = F.layer_norm(m, (d.c_m,), p["col.ln.gamma"], p["col.ln.beta"], eps=1e-5)[:, 0].tolist()  # [S][c_m]
    w = p["col.w_qkvg"].tolist()
    bg = p["col.b_g"].tolist()

    def proj(row, s):  # one output column of the fused projection for sequence s
        return sum(w[row][t] * x[s][t] for t in range(d.c_m))

    def sig(u):
        return 1.0 / (1.0 + math.exp(-u))

    q = [[[proj(h * c + e, s) for e in range(c)] for h in range(H)] for s in range(S)]
    kk = [[proj(H * c + e, s) for e in range(c)] for s in range(S)]
    vv = [[proj(H * c + c + e, s) for e in range(c)] for s in range(S)]
    g = [[[sig(proj(H * c + 2 * c + h * c + e, s) + bg[h * c + e]) for e in range(c)] for h in range(H)]
         for s in range(S)]

    def expected(valid_q, valid_k, scale):
        res = [[0.0] * (H * c) for _ in range(S)]
        for h in range(H):
            qbar = [sum(q[s][h][e] for s in valid_q) / (len(valid_q) + 1e-10) for e in range(c)]
            logit = {t: scale * sum(qbar[e] * kk[t][e] for e in range(c)) for t in valid_k}
            mx = max(logit.values())
            den = sum(math.exp(logit[t] - mx) for t in valid_k)
            att = {t: math.exp(logit[t] - mx) / den for t in valid_k}
            for s in range(S):
                for e in range(c):
                    res[s][h * c + e] = g[s][h][e] * sum(att[t] * vv[t][e] for t in valid_k)
        return torch.tensor(res, dtype=DT)[:, None, :]

    ref = expected([0, 2], [0, 2], 1.0 / math.sqrt(c))
    assert torch.allclose(out, ref, atol=1e-12)
    for wrong in (expected([0, 1, 2], [0, 2], 1.0 / math.sqrt(c)),   # unmasked mean of q
                  expected([0, 2], [0, 2], 1.0),                       # no 1/sqrt(c)
                  expected([0, 2], [0, 1, 2], 1.0 / math.sqrt(c))):    # masked key kept
        assert (wrong - ref).abs().max() > 1e-4


# --------------------------------------------------------------- triangle ops

def _tri_dims():
    return synth.Dims(n_seq=3, n_res=6, c_m=8, c_z=8, h_msa=2, c_msa=4, h_tri=2, c_tri=4,
                      c_mul=4, c_opm=2, trans_n=2)


def test_triangle_attention_end_is_start_on_transpose():
    d = _tri_dims()
    p = _params(d)
    _, z = _acts(d)
    _, pm = _ones_masks(d)
    pm[1, 4] = 0
    pm[3, 0] = 0
    pe = dict(p)
    for k in list(p):
        if k.startswith("att_start."):
            pe["att_end." + k[len("att_start."):]] = p[k]
    end = O.triangle_attention_ending_node(z, pm, pe, d.h_tri, d.c_tri)
    start_t = O.triangle_attention_starting_node(z.transpose(0, 1), pm.transpose(0, 1), p,
                                                 d.h_tri, d.c_tri)
    assert torch.allclose(end, start_t.transpose(0, 1), atol=1e-13)


def test_triangle_attention_bias_orientation():
    """start: bias b_jk for query (i,j), key (i,k); end: bias b_ki for query (i,j), key (k,j)."""
    d = _tri_dims()
    R, H, c = d.n_res, d.h_tri, d.c_tri
    perm = [2, 0, 5, 1, 3, 4]
    inv = [perm.index(a) for a in range(R)]
    z = _selector_pair(R, d.c_z, perm)
    for prefix, fn in (("att_start", O.triangle_attention_starting_node),
                       ("att_end", O.triangle_attention_ending_node)):
        p = _params(d)
        p[prefix + ".ln.gamma"] = torch.ones(d.c_z, dtype=DT)
        p[prefix + ".ln.beta"] = torch.zeros(d.c_z, dtype=DT)
        w2 = p[prefix + ".w_qkvg"].clone()
        w2[:2 * H * c] = 0  # q = k = 0: the logits are the bias alone
        w2[2 * H * c:3 * H * c] = 0
        w2[2 * H * c:3 * H * c, 2] = 1.0  # v reads channel 2, a per-position ramp
        p[prefix + ".w_qkvg"] = w2
        p[prefix + ".w_b"] = torch.zeros(H, d.c_z, dtype=DT)
        p[prefix + ".w_b"][:, 0] = 40.0
        _expose_output(p, prefix, d.c_z)
        zz = z.clone()
        zz[..., 2] = torch.arange(R * R, dtype=DT).reshape(R, R) * 1e-3
        out = fn(zz, torch.ones(R, R, dtype=DT), p, H, c)
        x = F.layer_norm(zz, (d.c_z,), p[prefix + ".ln.gamma"], p[prefix + ".ln.beta"], eps=1e-5)
        v = x @ w2[2 * H * c:3 * H * c].T
        g = torch.sigmoid(x @ w2[3 * H * c:].T + p[prefix + ".b_g"])
        if prefix == "att_start":
            # query (i,j) picks key (i, perm[j])
            expect = torch.stack([torch.stack([v[i, perm[j]] for j in range(R)]) for i in range(R)])
        else:
            # query (i,j) picks key (k,j) with b_ki large: i = perm[k] -> k = inv[i]
            expect = torch.stack([torch.stack([v[inv[i], j] for j in range(R)]) for i in range(R)])
        # selector z changes LN(z) rows, so compare with the bias-selected key
        assert torch.allclose(out, g * expect, atol=1e-5), prefix


def _tri_att_sdpa_case(prefix):
    """Triangle attention with W_b = 0, a saturated gate and W_o = I, with a
    pair mask that leaves every key row at least one valid key."""
    d = _tri_dims()
    p = _params(d)
    _, z = _acts(d)
    p[prefix + ".w_b"] = torch.zeros_like(p[prefix + ".w_b"])
    p[prefix + ".b_g"] = torch.full_like(p[prefix + ".b_g"], 60.0)  # sigmoid(60) = 1 - 9e-27
    _expose_output(p, prefix, d.c_z)
    _, pm = _ones_masks(d)
    pm[0, 3] = 0
    pm[2, 1] = 0
    pm[2, 5] = 0
    pm[4, 0] = 0
    R, H, c = d.n_res, d.h_tri, d.c_tri
    x = F.layer_norm(z, (d.c_z,), p[prefix + ".ln.gamma"], p[prefix + ".ln.beta"], eps=1e-5)
    w = p[prefix + ".w_qkvg"]
    q, k, v = ((x @ w[t * H * c:(t + 1) * H * c].T).reshape(R, R, H, c) for t in range(3))
    return d, p, z, pm, q, k, v


def test_triangle_attention_starting_node_reduces_to_sdpa_per_row():
    """Starting node, bias 0 and gate 1: for each pair row i, the queries
    (i, j) attend over the keys (i, k) of the same row with the library's
    scaled-dot-product attention, key k excluded where pair_mask[i, k] = 0.
    This fixes the q.k term: which key a query meets and the 1/sqrt(c) scale."""
    d, p, z, pm, q, k, v = _tri_att_sdpa_case("att_start")
    R, H, c = d.n_res, d.h_tri, d.c_tri
    out = O.triangle_attention_starting_node(z, pm, p, H, c)
    ref = torch.empty(R, R, H * c, dtype=DT)
    for i in range(R):
        qi, ki, vi = (t[i].permute(1, 0, 2) for t in (q, k, v))  # [H, R, c]
        allowed = (pm[i] > 0)[None, None, :].expand(H, R, R)
        o = F.scaled_dot_product_attention(qi, ki, vi, attn_mask=allowed)
        ref[i] = o.permute(1, 0, 2).reshape(R, H * c)
    assert torch.allclose(out, ref, atol=1e-12)


def test_triangle_attention_ending_node_reduces_to_sdpa_per_column():
    """Ending node, bias 0 and gate 1: for each pair column j, the queries
    (i, j) attend over the keys (k, j) of the same column, key k excluded
    where pair_mask[k, j] = 0."""
    d, p, z, pm, q, k, v = _tri_att_sdpa_case("att_end")
    R, H, c = d.n_res, d.h_tri, d.c_tri
    out = O.triangle_attention_ending_node(z, pm, p, H, c)
    ref = torch.empty(R, R, H * c, dtype=DT)
    for j in range(R):
        qj, kj, vj = (t[:, j].permute(1, 0, 2) for t in (q, k, v))  # [H, R, c]
        allowed = (pm[:, j] > 0)[None, None, :].expand(H, R, R)
        o = F.scaled_dot_product_attention(qj, kj, vj, attn_mask=allowed)
        ref[:, j] = o.permute(1, 0, 2).reshape(R, H * c)
    assert torch.allclose(out, ref, atol=1e-12)
    # the same inputs through the starting node give a different result (the
    # two orientations are not interchangeable on this input)
    pe = {("att_start." + key[len("att_end."):]): val for key, val in p.items() if key.startswith("att_end.")}
    other = O.triangle_attention_starting_node(z, pm, {**p, **pe}, H, c)
    assert (other - ref).abs().max() > 1e-3


def _swap_ab(p, prefix, c_mul):
    q = dict(p)
    w, b = p[prefix + ".w_abg"], p[prefix + ".b_abg"]
    idx = torch.cat([torch.arange(2 * c_mul, 4 * c_mul), torch.arange(0, 2 * c_mul),
                     torch.arange(4 * c_mul, w.shape[0])])
    q[prefix + ".w_abg"] = w[idx]
    q[prefix + ".b_abg"] = b[idx]
    return q


def test_triangle_multiplication_incoming_is_outgoing_on_transpose_with_swapped_ab():
    d = _tri_dims()
    p = _params(d)
    _, z = _acts(d)
    _, pm = _ones_masks(d)
    pm[2, 5] = 0
    pm[0, 3] = 0
    inc = O.triangle_multiplication_incoming(z, pm, p, d.c_mul)
    po = dict(p)
    for k in list(p):
        if k.startswith("tri_in."):
            po["tri_out." + k[len("tri_in."):]] = p[k]
    po = _swap_ab(po, "tri_out", d.c_mul)
    out_t = O.triangle_multiplication_outgoing(z.transpose(0, 1), pm.transpose(0, 1), po, d.c_mul)
    assert torch.allclose(inc, out_t.transpose(0, 1), atol=1e-13)


def test_triangle_multiplication_core_is_per_channel_matrix_product():
    """X_c = A_c B_c^T (outgoing) and A_c^T B_c (incoming) as plain matrix products."""
    d = _tri_dims()
    p = _params(d)
    _, z = _acts(d)
    _, pm = _ones_masks(d)
    a, b, g = O._tri_mul_projections(z, pm, p, "tri_out", d.c_mul)
    X_out = torch.einsum("ikc,jkc->ijc", a, b)
    X_in = torch.einsum("kic,kjc->ijc", a, b)
    for ch in range(d.c_mul):
        A, B = a[..., ch], b[..., ch]
        assert torch.allclose(X_out[..., ch], A @ B.T, atol=1e-13)
        assert torch.allclose(X_in[..., ch], A.T @ B, atol=1e-13)
    # and the module applies the gated output to that product
    ref = g * (F.layer_norm(X_out, (d.c_mul,), p["tri_out.ln_out.gamma"], p["tri_out.ln_out.beta"],
                            eps=1e-5) @ p["tri_out.w_o"].T + p["tri_out.b_o"])
    assert torch.allclose(O.triangle_multiplication_outgoing(z, pm, p, d.c_mul), ref, atol=1e-13)


def test_triangle_multiplication_mask_excludes_k():
    """A masked pair (i,k) contributes nothing: perturbing z there leaves X unchanged
    for every (i', j') that would read it only through the masked a/b entries."""
    d = _tri_dims()
    p = _params(d)
    _, z = _acts(d)
    R = d.n_res
    seq = torch.ones(R, dtype=DT)
    seq[4] = 0
    pm = seq[:, None] * seq[None, :]
    out = O.triangle_multiplication_outgoing(z, pm, p, d.c_mul)
    z2 = z.clone()
    z2[4, :] = z2[4, :] * 3.0 + torch.linspace(-1, 1, d.c_z, dtype=DT)
    z2[:, 4] = -z2[:, 4]
    out2 = O.triangle_multiplication_outgoing(z2, pm, p, d.c_mul)
    valid = pm > 0
    assert torch.allclose(out[valid], out2[valid], atol=1e-13)


# ----------------------------------------------------------------------- OPM

def test_outer_product_mean_closed_form():
    """b_o = 0, all-ones mask, c_z = c_opm^2, W_o = I: update_ij[c,d] = (A_c^T B_d)_ij / (S + 1e-3)."""
    for S in (1, 4):
        d = synth.Dims(n_seq=S, n_res=5, c_m=8, c_z=9, c_opm=3, h_msa=2, c_msa=4, h_tri=2,
                       c_tri=4, c_mul=4, trans_n=2)
        p = _params(d)
        m, _ = _acts(d)
        p["opm.w_o"] = torch.eye(9, dtype=DT)
        p["opm.b_o"] = torch.zeros(9, dtype=DT)
        mk = torch.ones(S, d.n_res, dtype=DT)
        upd = O.outer_product_mean(m, mk, p, 3)
        x = F.layer_norm(m, (8,), p["opm.ln.gamma"], p["opm.ln.beta"], eps=1e-5)
        ab = x @ p["opm.w_ab"].T + p["opm.b_ab"]
        a, b = ab[..., :3], ab[..., 3:]
        for c in range(3):
            for dd in range(3):
                ref = a[..., c].T @ b[..., dd] / (S + 1e-3)
                assert torch.allclose(upd[..., c * 3 + dd], ref, atol=1e-13)
        if S == 1:
            assert torch.allclose(upd[..., 4] * (1 + 1e-3), torch.outer(a[0, :, 1], b[0, :, 1]), atol=1e-13)


def test_outer_product_mean_normaliser_and_bias_inside():
    """a = b = mask (W_ab = 0, b_ab = 1), W_o = [1]: update = (n_ij + b_o)/(1e-3 + n_ij)."""
    d = synth.Dims(n_seq=6, n_res=4, c_m=8, c_z=1, c_opm=1, h_msa=2, c_msa=4, h_tri=1,
                   c_tri=4, c_mul=4, trans_n=2)
    p = _params(d)
    m, _ = _acts(d)
    p["opm.w_ab"] = torch.zeros(2, 8, dtype=DT)
    p["opm.b_ab"] = torch.ones(2, dtype=DT)
    p["opm.w_o"] = torch.ones(1, 1, dtype=DT)
    p["opm.b_o"] = torch.tensor([0.25], dtype=DT)
    mk = torch.ones(6, 4, dtype=DT)
    mk[0, 1] = 0
    mk[3, 1] = 0
    mk[5, 2] = 0
    upd = O.outer_product_mean(m, mk, p, 1)[..., 0]
    n = torch.tensor([[sum(mk[s, i] * mk[s, j] for s in range(6)) for j in range(4)] for i in range(4)],
                     dtype=DT)
    assert torch.allclose(upd, (n + 0.25) / (1e-3 + n), atol=1e-13)
    upd_out = O.outer_product_mean(m, mk, p, 1, bias_inside=False)[..., 0]
    assert torch.allclose(upd_out, n / (1e-3 + n) + 0.25, atol=1e-13)


# --------------------------------------------------------------- transition

def test_transition_is_two_layer_mlp():
    d = TINY
    p = _params(d)
    m, _ = _acts(d)
    y = O.transition(m, p, "msa_trans")
    x = F.layer_norm(m, (d.c_m,), p["msa_trans.ln.gamma"], p["msa_trans.ln.beta"], eps=1e-5)
    ref = F.linear(F.relu(F.linear(x, p["msa_trans.w1"], p["msa_trans.b1"])), p["msa_trans.w2"],
                   p["msa_trans.b2"])
    assert torch.allclose(y, ref, atol=1e-13)


# ------------------------------------------------------------------- block

def _block_dims():
    return synth.Dims(n_seq=4, n_res=6, c_m=8, c_z=8, h_msa=2, c_msa=4, h_tri=2, c_tri=4,
                      c_mul=4, c_opm=2, trans_n=2)


def test_param_table_matches_oracle_statement():
    for d in (synth.DIMS_TRAIN_CROP, synth.DIMS_EXTRA_MSA, TINY):
        lay, total = synth.param_layout(d)
        exp = O.expected_param_shapes(d)
        assert {n: tuple(s) for n, _, s, _ in lay} == exp
    _, total = synth.param_layout(synth.DIMS_TRAIN_CROP)
    assert total == 1829952  # every tensor at the training crop is a multiple of 64 floats


def test_block_residue_permutation_equivariance():
    d = _block_dims()
    p = _params(d)
    m, z = _acts(d)
    seq = torch.ones(d.n_res, dtype=DT)
    seq[2] = 0
    mm = seq[None].repeat(d.n_seq, 1)
    pm = seq[:, None] * seq[None]
    mo, zo = O.evoformer_block(m, z, mm, pm, p, d)
    P = torch.tensor([3, 5, 0, 1, 4, 2])
    mo2, zo2 = O.evoformer_block(m[:, P], z[P][:, P], mm[:, P], pm[P][:, P], p, d)
    assert torch.allclose(mo2, mo[:, P], atol=1e-11)
    assert torch.allclose(zo2, zo[P][:, P], atol=1e-11)


def test_block_msa_row_permutation():
    d = _block_dims()
    p = _params(d)
    m, z = _acts(d)
    mm, pm = _ones_masks(d)
    mo, zo = O.evoformer_block(m, z, mm, pm, p, d)
    P = torch.tensor([2, 0, 3, 1])
    mo2, zo2 = O.evoformer_block(m[P], z, mm[P], pm, p, d)
    assert torch.allclose(mo2, mo[P], atol=1e-11)
    assert torch.allclose(zo2, zo, atol=1e-11)


def test_block_padded_entries_do_not_leak():
    d = _block_dims()
    p = _params(d)
    m, z = _acts(d)
    seq = torch.ones(d.n_res, dtype=DT)
    seq[1] = 0
    seq[4] = 0
    mm = seq[None].repeat(d.n_seq, 1)
    pm = seq[:, None] * seq[None]
    mo, zo = O.evoformer_block(m, z, mm, pm, p, d)
    m2, z2 = m.clone(), z.clone()
    m2[:, 1] = m2[:, 1] * 3.0 + torch.linspace(-2, 2, d.c_m, dtype=DT)
    z2[4, :] = z2[4, :] * -1.5 + torch.linspace(-1, 1, d.c_z, dtype=DT)
    z2[:, 1] *= -2.0
    mo2, zo2 = O.evoformer_block(m2, z2, mm, pm, p, d)
    vm = mm > 0
    vz = pm > 0
    assert torch.allclose(mo2[vm], mo[vm], atol=1e-11)
    assert torch.allclose(zo2[vz], zo[vz], atol=1e-11)


def test_block_row_chunking_is_exact():
    """Splitting the MSA rows of row attention into chunks changes nothing (the
    Subbatch exactness along a batch-like axis, Sec. 3.4.4)."""
    d = _attn_dims()
    p = _params(d)
    m, z = _acts(d)
    mm, _ = _ones_masks(d)
    full = O.msa_row_attention_with_pair_bias(m, z, mm, p, d.h_msa, d.c_msa)
    parts = [O.msa_row_attention_with_pair_bias(m[s:s + 1], z, mm[s:s + 1], p, d.h_msa, d.c_msa)
             for s in range(d.n_seq)]
    assert torch.allclose(torch.cat(parts, 0), full, atol=1e-14)
