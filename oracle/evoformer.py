"""FP64 CPU oracle of the AlphaFold2 Evoformer block (test infrastructure).

This file is test infrastructure: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path
never calls it, and it imports nothing from the product package.

What it computes.  HelixFold (arXiv 2207.05477) reimplements AlphaFold2 and
states that its fused operators and parallel schemes keep the exact
semantics of the original model (Sec. 3.3.4 on Branch Parallelism, and the
Subbatch discussion of Sec. 3.4.4); it names the modules of the Evoformer
block -- MSARowAttentionWithPairBias, MSAColumnAttention, the MSA stack and
pair stack, Outer Product Mean (Sec. 3.1, Fig. 2; Sec. 3.3.3; Table
"communication") -- but prints no formula for them.  The formulas below are
the AlphaFold2 Evoformer as published by Jumper et al. 2021 (supplementary
Algorithms 6-15 and 19), restated from the published method, one function per
module, in plain tensor algebra: no blocking, no fusion, no reordering.

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository):
  * sub-module order is the sequential Algorithm 6 order;
  * dropout is off (evaluation semantics) unless its scales are given
    (training mode: the random draw is an input, AF2 row-wise / column-wise
    sharing);
  * a masked key is excluded from the softmax exactly; a query with no valid
    key gets an attention output of 0;
  * LayerNorm: biased variance, eps = 1e-5;
  * outer-product-mean: the output bias sits inside the division by
    (1e-3 + number of valid sequence pairs);
  * triangle multiplication: the gate multiplies after the output Linear;
  * softmax scale 1/sqrt(head dim) on the logits;
  * a template pair stack block (AF2 Alg. 16) is the pair half of Alg. 6 with
    the same dropout sites; the LayerNorm applied after the whole template
    stack is not part of a block.

Gradients: the backward of the block is the exact gradient of this forward,
taken by reverse-mode differentiation of the FP64 graph (``torch.autograd``);
the tests pin it independently with central finite differences.

Parity pins (tests/test_oracle_*.py): closed forms, special cases that reduce
to a library routine, permutation equivariances, the start/end and in/out
transposition identities, mask invariances and finite differences.
"""
from __future__ import annotations

import math

import torch

LN_EPS = 1e-5
OPM_EPS = 1e-3
DT = torch.float64


# ---------------------------------------------------------------- primitives

def layer_norm(x, gamma, beta, eps=LN_EPS):
    """LayerNorm over the last (channel) axis with biased variance."""
    mu = x.mean(dim=-1, keepdim=True)
    var = ((x - mu) ** 2).mean(dim=-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + eps) * gamma + beta


def linear(x, w, b=None):
    """y = x W^T (+ b), W stored [out, in]."""
    y = torch.matmul(x, w.transpose(0, 1))
    return y if b is None else y + b


def masked_softmax(logits, key_valid):
    """Softmax over the last axis restricted to keys with key_valid True.

    Masked keys get weight exactly 0.  A row with no valid key gets all-zero
    weights (so its attention output is 0).
    """
    neg = torch.full_like(logits, -math.inf)
    l = torch.where(key_valid, logits, neg)
    mx = l.amax(dim=-1, keepdim=True)
    mx = torch.where(torch.isinf(mx), torch.zeros_like(mx), mx).detach()
    e = torch.where(key_valid, torch.exp(l - mx), torch.zeros_like(l))
    s = e.sum(dim=-1, keepdim=True)
    s = torch.where(s > 0, s, torch.ones_like(s))
    return e / s


def _split_qkvg(y, h, c):
    """Columns of the fused projection: [q | k | v | g], each h*c, head-major."""
    q, k, v, g = torch.split(y, h * c, dim=-1)
    shp = y.shape[:-1] + (h, c)
    return q.reshape(shp), k.reshape(shp), v.reshape(shp), g.reshape(shp)


# ------------------------------------------------------------------- modules

def msa_row_attention_with_pair_bias(m, z, msa_mask, p, h, c, return_weights=False):
    """MSA row-wise gated self-attention with pair bias (AF2 Alg. 7).

    m [S,R,c_m], z [R,R,c_z], msa_mask [S,R].  Per MSA row s and head h:
    logits_ij = q_si.k_sj / sqrt(c) + b_ij^h with b^h = LN(z) W_b^h, key j
    excluded where msa_mask[s,j] = 0; o_si = g_si * sum_j a_sij v_sj;
    output = concat_h(o) W_o + b_o.  This is the gated self-attention with
    ``nonbatched_bias`` that the paper fuses (Sec. 3.1, Fig. 2).
    """
    x = layer_norm(m, p["row.ln_m.gamma"], p["row.ln_m.beta"])
    q, k, v, g = _split_qkvg(linear(x, p["row.w_qkvg"]), h, c)
    g = torch.sigmoid(g + p["row.b_g"].reshape(h, c))
    zb = layer_norm(z, p["row.ln_z.gamma"], p["row.ln_z.beta"])
    bias = torch.einsum("ijc,hc->hij", zb, p["row.w_b"])
    logits = torch.einsum("sihd,sjhd->shij", q, k) / math.sqrt(c) + bias[None]
    valid = (msa_mask > 0)[:, None, None, :]
    a = masked_softmax(logits, valid)
    o = torch.einsum("shij,sjhd->sihd", a, v) * g
    out = linear(o.reshape(o.shape[0], o.shape[1], h * c), p["row.w_o"], p["row.b_o"])
    return (out, a) if return_weights else out


def msa_column_attention(m, msa_mask, p, h, c, return_weights=False):
    """MSA column-wise gated self-attention (AF2 Alg. 8).

    Per residue column i and head h: logits_st = q_si.k_ti / sqrt(c), key t
    excluded where msa_mask[t,i] = 0; o_si = g_si * sum_t a_ist v_ti.
    """
    x = layer_norm(m, p["col.ln.gamma"], p["col.ln.beta"])
    q, k, v, g = _split_qkvg(linear(x, p["col.w_qkvg"]), h, c)
    g = torch.sigmoid(g + p["col.b_g"].reshape(h, c))
    logits = torch.einsum("sihd,tihd->ihst", q, k) / math.sqrt(c)
    valid = (msa_mask.transpose(0, 1) > 0)[:, None, None, :]
    a = masked_softmax(logits, valid)
    o = torch.einsum("ihst,tihd->sihd", a, v) * g
    out = linear(o.reshape(o.shape[0], o.shape[1], h * c), p["col.w_o"], p["col.b_o"])
    return (out, a) if return_weights else out


def msa_global_column_attention(m, msa_mask, p, h, c, return_weights=False):
    """MSA global column attention of the extra-MSA stack (AF2 Alg. 19).

    q has h heads, k and v a single head of width c.  Per column i:
    qbar_i^h = sum_s mask_si q_si^h / (sum_s mask_si + 1e-10);
    a_it^h = softmax_t(qbar_i^h . k_ti / sqrt(c)), key t excluded where
    msa_mask[t,i] = 0; o_si^h = g_si^h * sum_t a_it^h v_ti.
    Fused projection columns: [q (h*c) | k (c) | v (c) | g (h*c)].
    """
    x = layer_norm(m, p["col.ln.gamma"], p["col.ln.beta"])
    y = linear(x, p["col.w_qkvg"])
    q, k, v, g = torch.split(y, [h * c, c, c, h * c], dim=-1)
    S, R = m.shape[0], m.shape[1]
    q = q.reshape(S, R, h, c)
    g = torch.sigmoid(g + p["col.b_g"]).reshape(S, R, h, c)
    mk = msa_mask
    qbar = torch.einsum("si,sihd->ihd", mk, q) / (mk.sum(dim=0)[:, None, None] + 1e-10)
    logits = torch.einsum("ihd,tid->iht", qbar, k) / math.sqrt(c)
    valid = (mk.transpose(0, 1) > 0)[:, None, :]
    a = masked_softmax(logits, valid)
    o = torch.einsum("iht,tid->ihd", a, v)[None] * g
    out = linear(o.reshape(S, R, h * c), p["col.w_o"], p["col.b_o"])
    return (out, a) if return_weights else out


def transition(x, p, prefix):
    """LayerNorm, Linear(c -> n c), ReLU, Linear(n c -> c) (AF2 Alg. 9 / 15)."""
    y = layer_norm(x, p[prefix + ".ln.gamma"], p[prefix + ".ln.beta"])
    hdn = torch.relu(linear(y, p[prefix + ".w1"], p[prefix + ".b1"]))
    return linear(hdn, p[prefix + ".w2"], p[prefix + ".b2"])


def outer_product_mean(m, msa_mask, p, c_opm, bias_inside=True):
    """Outer product mean, the MSA -> pair update (AF2 Alg. 10).

    a_si = mask_si (LN(m_si) W_a + b_a), b_sj likewise (c_opm wide each);
    O_ij[c*c_opm + d] = sum_s a_si[c] b_sj[d];
    update_ij = (O_ij W_o + b_o) / (1e-3 + sum_s mask_si mask_sj).
    With ``bias_inside=False`` the bias is added after the division (the
    "mean then Linear" reading).
    """
    x = layer_norm(m, p["opm.ln.gamma"], p["opm.ln.beta"])
    ab = linear(x, p["opm.w_ab"], p["opm.b_ab"]) * msa_mask[..., None]
    a, b = ab[..., :c_opm], ab[..., c_opm:]
    O = torch.einsum("sic,sjd->ijcd", a, b)
    R = m.shape[1]
    O = O.reshape(R, R, c_opm * c_opm)
    norm = torch.einsum("si,sj->ij", msa_mask, msa_mask)[..., None]
    if bias_inside:
        return linear(O, p["opm.w_o"], p["opm.b_o"]) / (OPM_EPS + norm)
    return linear(O, p["opm.w_o"]) / (OPM_EPS + norm) + p["opm.b_o"]


def _tri_mul_projections(z, pair_mask, p, prefix, c_mul):
    x = layer_norm(z, p[prefix + ".ln_in.gamma"], p[prefix + ".ln_in.beta"])
    y = linear(x, p[prefix + ".w_abg"], p[prefix + ".b_abg"])
    ap, ag, bp, bg, g = torch.split(y, [c_mul, c_mul, c_mul, c_mul, z.shape[-1]], dim=-1)
    mk = pair_mask[..., None]
    a = mk * torch.sigmoid(ag) * ap
    b = mk * torch.sigmoid(bg) * bp
    return a, b, torch.sigmoid(g)


def _tri_mul_output(X, g, p, prefix):
    y = layer_norm(X, p[prefix + ".ln_out.gamma"], p[prefix + ".ln_out.beta"])
    return g * linear(y, p[prefix + ".w_o"], p[prefix + ".b_o"])


def triangle_multiplication_outgoing(z, pair_mask, p, c_mul, prefix="tri_out"):
    """Triangular multiplicative update, outgoing edges (AF2 Alg. 11).

    a_ik = mask_ik sigmoid(LN(z)W_ag + b) * (LN(z)W_ap + b), b_jk likewise,
    g = sigmoid(LN(z)W_g + b_g); X_ij = sum_k a_ik * b_jk (per channel);
    update = g * (LN(X) W_o + b_o).  Fused projection columns:
    [a_proj | a_gate | b_proj | b_gate | g].
    """
    a, b, g = _tri_mul_projections(z, pair_mask, p, prefix, c_mul)
    X = torch.einsum("ikc,jkc->ijc", a, b)
    return _tri_mul_output(X, g, p, prefix)


def triangle_multiplication_incoming(z, pair_mask, p, c_mul, prefix="tri_in"):
    """Triangular multiplicative update, incoming edges (AF2 Alg. 12).

    As the outgoing update but X_ij = sum_k a_ki * b_kj.
    """
    a, b, g = _tri_mul_projections(z, pair_mask, p, prefix, c_mul)
    X = torch.einsum("kic,kjc->ijc", a, b)
    return _tri_mul_output(X, g, p, prefix)


def _tri_att_projections(z, p, prefix, h, c):
    x = layer_norm(z, p[prefix + ".ln.gamma"], p[prefix + ".ln.beta"])
    q, k, v, g = _split_qkvg(linear(x, p[prefix + ".w_qkvg"]), h, c)
    g = torch.sigmoid(g + p[prefix + ".b_g"].reshape(h, c))
    bias = torch.einsum("jkc,hc->hjk", x, p[prefix + ".w_b"])
    return q, k, v, g, bias


def triangle_attention_starting_node(z, pair_mask, p, h, c, prefix="att_start",
                                     return_weights=False):
    """Triangle self-attention around the starting node (AF2 Alg. 13).

    logits_ijk^h = q_ij.k_ik / sqrt(c) + b_jk^h, key k excluded where
    pair_mask[i,k] = 0; o_ij = g_ij * sum_k a_ijk v_ik.
    """
    q, k, v, g, bias = _tri_att_projections(z, p, prefix, h, c)
    logits = torch.einsum("ijhd,ikhd->ihjk", q, k) / math.sqrt(c) + bias[None]
    valid = (pair_mask > 0)[:, None, None, :]
    a = masked_softmax(logits, valid)
    o = torch.einsum("ihjk,ikhd->ijhd", a, v) * g
    R = z.shape[0]
    out = linear(o.reshape(R, R, h * c), p[prefix + ".w_o"], p[prefix + ".b_o"])
    return (out, a) if return_weights else out


def triangle_attention_ending_node(z, pair_mask, p, h, c, prefix="att_end",
                                   return_weights=False):
    """Triangle self-attention around the ending node (AF2 Alg. 14).

    logits_ijk^h = q_ij.k_kj / sqrt(c) + b_ki^h, key k excluded where
    pair_mask[k,j] = 0; o_ij = g_ij * sum_k a_ijk v_kj.
    """
    q, k, v, g, bias = _tri_att_projections(z, p, prefix, h, c)
    logits = torch.einsum("ijhd,kjhd->jhik", q, k) / math.sqrt(c) \
        + bias.permute(0, 2, 1)[None]
    valid = (pair_mask.transpose(0, 1) > 0)[:, None, None, :]
    a = masked_softmax(logits, valid)
    o = torch.einsum("jhik,kjhd->ijhd", a, v) * g
    R = z.shape[0]
    out = linear(o.reshape(R, R, h * c), p[prefix + ".w_o"], p[prefix + ".b_o"])
    return (out, a) if return_weights else out


# --------------------------------------------------------------------- block

def dropout_rowwise(update, scale):
    """AF2 DropoutRowwise with the random draw given: one scale per (column,
    channel), shared by every row of the [rows, columns, channels] update."""
    return update * scale[None, :, :]


def dropout_columnwise(update, scale):
    """AF2 DropoutColumnwise: one scale per (row, channel), shared by every
    column."""
    return update * scale[:, None, :]


def evoformer_block(m, z, msa_mask, pair_mask, p, dims, dropout=None):
    """One Evoformer block in AF2 Algorithm 6 order, each step seeing the last.

    ``dims`` carries h_msa, c_msa, h_tri, c_tri, c_mul, c_opm, msa_col_mode.
    With msa_col_mode = 1 the column step is global column attention (the
    extra-MSA block of AF2 Alg. 18).  ``dropout`` (training mode) maps the
    sites msa_row, tri_out, tri_in, att_start (row-wise) and att_end
    (column-wise) to their scales (0 or 1/(1-rate), the random draw being an
    input); a missing site is not dropped.
    """
    hm, cm, ht, ct = dims.h_msa, dims.c_msa, dims.h_tri, dims.c_tri
    dr = dropout or {}

    def rowwise(name, u):
        return dropout_rowwise(u, dr[name]) if name in dr else u

    def colwise(name, u):
        return dropout_columnwise(u, dr[name]) if name in dr else u

    m = m + rowwise("msa_row", msa_row_attention_with_pair_bias(m, z, msa_mask, p, hm, cm))
    if dims.msa_col_mode == 0:
        m = m + msa_column_attention(m, msa_mask, p, hm, cm)
    else:
        m = m + msa_global_column_attention(m, msa_mask, p, hm, cm)
    m = m + transition(m, p, "msa_trans")
    z = z + outer_product_mean(m, msa_mask, p, dims.c_opm)
    z = z + rowwise("tri_out", triangle_multiplication_outgoing(z, pair_mask, p, dims.c_mul))
    z = z + rowwise("tri_in", triangle_multiplication_incoming(z, pair_mask, p, dims.c_mul))
    z = z + rowwise("att_start", triangle_attention_starting_node(z, pair_mask, p, ht, ct))
    z = z + colwise("att_end", triangle_attention_ending_node(z, pair_mask, p, ht, ct))
    z = z + transition(z, p, "pair_trans")
    return m, z


def pair_stack_block(z, pair_mask, p, dims, dropout=None):
    """One template pair stack block (AF2 Alg. 16): the pair half of the
    Evoformer block -- triangle multiplications, triangle attentions, pair
    transition, with the same dropout sites -- on the template pair
    representation alone (no MSA, no outer product mean)."""
    ht, ct = dims.h_tri, dims.c_tri
    dr = dropout or {}

    def rowwise(name, u):
        return dropout_rowwise(u, dr[name]) if name in dr else u

    def colwise(name, u):
        return dropout_columnwise(u, dr[name]) if name in dr else u

    z = z + rowwise("tri_out", triangle_multiplication_outgoing(z, pair_mask, p, dims.c_mul))
    z = z + rowwise("tri_in", triangle_multiplication_incoming(z, pair_mask, p, dims.c_mul))
    z = z + rowwise("att_start", triangle_attention_starting_node(z, pair_mask, p, ht, ct))
    z = z + colwise("att_end", triangle_attention_ending_node(z, pair_mask, p, ht, ct))
    z = z + transition(z, p, "pair_trans")
    return z


def pair_block_forward(z, pair_mask, params: dict, dims, dropout=None):
    """FP64 template pair block forward; returns z_out."""
    with torch.no_grad():
        return pair_stack_block(torch.as_tensor(z).to(DT), torch.as_tensor(pair_mask).to(DT), to_f64(params), dims,
                                _dropout_f64(dropout))


def pair_block_forward_backward(z, pair_mask, params: dict, dims, gz, dropout=None):
    """FP64 template pair block forward and the gradient of <z_out, gz>.

    Returns (z_out, dz_in, dparams: dict name -> tensor)."""
    p = to_f64(params, requires_grad=True)
    z0 = torch.as_tensor(z).to(DT).clone().requires_grad_(True)
    zo = pair_stack_block(z0, torch.as_tensor(pair_mask).to(DT), p, dims, _dropout_f64(dropout))
    loss = (zo * torch.as_tensor(gz).to(DT)).sum()
    names = list(p.keys())
    grads = torch.autograd.grad(loss, [z0] + [p[n] for n in names])
    return zo.detach(), grads[0], {n: g for n, g in zip(names, grads[1:])}


# -------------------------------------------------------------- param table

def expected_param_shapes(dims):
    """The oracle's own statement of each parameter tensor's shape.

    Written here independently of the library's table; a test checks that
    the two agree name for name and shape for shape.
    """
    hm, cm, ht, ct = dims.h_msa, dims.c_msa, dims.h_tri, dims.c_tri
    C, Z = dims.c_m, dims.c_z
    s = {
        "row.ln_m.gamma": (C,), "row.ln_m.beta": (C,),
        "row.ln_z.gamma": (Z,), "row.ln_z.beta": (Z,),
        "row.w_b": (hm, Z), "row.w_qkvg": (4 * hm * cm, C), "row.b_g": (hm * cm,),
        "row.w_o": (C, hm * cm), "row.b_o": (C,),
        "col.ln.gamma": (C,), "col.ln.beta": (C,),
        "col.w_qkvg": ((4 * hm * cm, C) if dims.msa_col_mode == 0
                       else (2 * hm * cm + 2 * cm, C)),
        "col.b_g": (hm * cm,), "col.w_o": (C, hm * cm), "col.b_o": (C,),
        "msa_trans.ln.gamma": (C,), "msa_trans.ln.beta": (C,),
        "msa_trans.w1": (dims.trans_n * C, C), "msa_trans.b1": (dims.trans_n * C,),
        "msa_trans.w2": (C, dims.trans_n * C), "msa_trans.b2": (C,),
        "opm.ln.gamma": (C,), "opm.ln.beta": (C,),
        "opm.w_ab": (2 * dims.c_opm, C), "opm.b_ab": (2 * dims.c_opm,),
        "opm.w_o": (Z, dims.c_opm ** 2), "opm.b_o": (Z,),
        "pair_trans.ln.gamma": (Z,), "pair_trans.ln.beta": (Z,),
        "pair_trans.w1": (dims.trans_n * Z, Z), "pair_trans.b1": (dims.trans_n * Z,),
        "pair_trans.w2": (Z, dims.trans_n * Z), "pair_trans.b2": (Z,),
    }
    if getattr(dims, "pair_only", 0):
        s = {k: v for k, v in s.items() if k.startswith("pair_trans.")}
    for t in ("tri_out", "tri_in"):
        s.update({
            t + ".ln_in.gamma": (Z,), t + ".ln_in.beta": (Z,),
            t + ".w_abg": (4 * dims.c_mul + Z, Z), t + ".b_abg": (4 * dims.c_mul + Z,),
            t + ".ln_out.gamma": (dims.c_mul,), t + ".ln_out.beta": (dims.c_mul,),
            t + ".w_o": (Z, dims.c_mul), t + ".b_o": (Z,),
        })
    for t in ("att_start", "att_end"):
        s.update({
            t + ".ln.gamma": (Z,), t + ".ln.beta": (Z,),
            t + ".w_b": (ht, Z), t + ".w_qkvg": (4 * ht * ct, Z), t + ".b_g": (ht * ct,),
            t + ".w_o": (Z, ht * ct), t + ".b_o": (Z,),
        })
    return s


def to_f64(params: dict, requires_grad=False):
    out = {}
    for k, v in params.items():
        t = torch.as_tensor(v).to(DT).clone()
        if requires_grad:
            t.requires_grad_(True)
        out[k] = t
    return out


# ---------------------------------------------------------- fwd / bwd entry

def _dropout_f64(dropout):
    return None if dropout is None else {k: torch.as_tensor(v).to(DT) for k, v in dropout.items()}


def block_forward(m, z, msa_mask, pair_mask, params: dict, dims, dropout=None):
    """FP64 forward. Inputs may be numpy or torch; returns (m_out, z_out)."""
    with torch.no_grad():
        p = to_f64(params)
        return evoformer_block(torch.as_tensor(m).to(DT), torch.as_tensor(z).to(DT),
                               torch.as_tensor(msa_mask).to(DT),
                               torch.as_tensor(pair_mask).to(DT), p, dims, _dropout_f64(dropout))


def block_forward_backward(m, z, msa_mask, pair_mask, params: dict, dims, gm, gz, dropout=None):
    """FP64 forward and the gradient of <m_out, gm> + <z_out, gz>.

    Returns (m_out, z_out, dm_in, dz_in, dparams: dict name -> tensor).
    """
    p = to_f64(params, requires_grad=True)
    m0 = torch.as_tensor(m).to(DT).clone().requires_grad_(True)
    z0 = torch.as_tensor(z).to(DT).clone().requires_grad_(True)
    mo, zo = evoformer_block(m0, z0, torch.as_tensor(msa_mask).to(DT),
                             torch.as_tensor(pair_mask).to(DT), p, dims, _dropout_f64(dropout))
    loss = (mo * torch.as_tensor(gm).to(DT)).sum() + (zo * torch.as_tensor(gz).to(DT)).sum()
    names = list(p.keys())
    grads = torch.autograd.grad(loss, [m0, z0] + [p[n] for n in names])
    dparams = {n: g for n, g in zip(names, grads[2:])}
    return mo.detach(), zo.detach(), grads[0], grads[1], dparams
