"""Pins of the oracle's training-mode dropout (AF2 Alg. 6: row-wise dropout
after MSA row attention, triangle multiplications and starting-node
attention; column-wise after ending-node attention), independent of how the
oracle applies the scales:

  * scales of 1 everywhere give the evaluation-mode block exactly;
  * a scale of 0 on a site gives the block whose module there has zero output
    weights and bias (the update vanishes by a different route);
  * a row-wise scale is one draw per (column, channel): an MSA whose
    sequences are all equal stays row-symmetric through the block, which a
    draw per element would break;
  * the gradients with dropout match central finite differences.
"""
import numpy as np
import pytest
import torch

from oracle import evoformer as O
from paper_2207_05477_gb300 import synth

DT = torch.float64
SITES = [name for name, _, _ in synth.DROPOUT_SITES]
# the output weight and bias of the module at each dropout site
ZERO_OUT = {"msa_row": ("row.w_o", "row.b_o"), "tri_out": ("tri_out.w_o", "tri_out.b_o"),
            "tri_in": ("tri_in.w_o", "tri_in.b_o"), "att_start": ("att_start.w_o", "att_start.b_o"),
            "att_end": ("att_end.w_o", "att_end.b_o")}


def _setup(d, seed=13, pad=0.0):
    prob = synth.make_problem(d, seed, pad_frac=pad)
    params = synth.unpack_params(d, prob["params"])
    return prob, params


def test_unit_scales_are_evaluation_mode():
    d = synth.DIMS_TINY
    prob, params = _setup(d, pad=0.2)
    ones = synth.make_dropout(d, 13, scale_rates=0.0)
    assert all(np.all(v == 1.0) for v in ones.values())
    a = O.block_forward_backward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], params, d,
                                 prob["gm"], prob["gz"])
    b = O.block_forward_backward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], params, d,
                                 prob["gm"], prob["gz"], dropout=ones)
    for x, y in zip(a[:4], b[:4]):
        assert torch.equal(x, y)
    for k in a[4]:
        assert torch.equal(a[4][k], b[4][k]), k


@pytest.mark.parametrize("site", SITES)
def test_zero_scale_removes_the_update(site):
    d = synth.DIMS_TINY
    prob, params = _setup(d, pad=0.2)
    dr = synth.make_dropout(d, 13)
    dr[site] = np.zeros_like(dr[site])
    mo, zo = O.block_forward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], params, d, dropout=dr)
    zeroed = dict(params)
    for n in ZERO_OUT[site]:
        zeroed[n] = np.zeros_like(params[n])
    rest = {k: v for k, v in dr.items() if k != site}
    mo2, zo2 = O.block_forward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], zeroed, d, dropout=rest)
    assert torch.allclose(mo, mo2, rtol=0, atol=1e-12)
    assert torch.allclose(zo, zo2, rtol=0, atol=1e-12)


def test_rowwise_draw_is_shared_by_every_msa_row():
    d = synth.DIMS_TINY
    prob, params = _setup(d)
    m = np.broadcast_to(prob["m"][:1], prob["m"].shape).copy()  # every sequence the same
    dr = synth.make_dropout(d, 13)
    mo, _ = O.block_forward(m, prob["z"], prob["msa_mask"], prob["pair_mask"], params, d, dropout=dr)
    assert float((mo - mo[:1]).abs().max()) < 1e-12
    # a scale drawn per element instead breaks the symmetry
    rng = np.random.default_rng(3)
    per_elem = (rng.random(prob["m"].shape) >= 0.15) / 0.85
    upd = O.msa_row_attention_with_pair_bias(torch.tensor(m, dtype=DT), torch.tensor(prob["z"], dtype=DT),
                                             torch.tensor(prob["msa_mask"], dtype=DT), O.to_f64(params),
                                             d.h_msa, d.c_msa)
    m1 = torch.tensor(m, dtype=DT) + upd * torch.tensor(per_elem, dtype=DT)
    assert float((m1 - m1[:1]).abs().max()) > 1e-3


def test_dropout_gradients_match_central_differences():
    d = synth.DIMS_TINY
    prob, params = _setup(d, pad=0.2)
    dr = synth.make_dropout(d, 13)
    _, _, dm, dz, dp = O.block_forward_backward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], params,
                                                d, prob["gm"], prob["gz"], dropout=dr)
    p = O.to_f64(params)
    drT = {k: torch.tensor(v, dtype=DT) for k, v in dr.items()}
    mmT, pmT = torch.tensor(prob["msa_mask"], dtype=DT), torch.tensor(prob["pair_mask"], dtype=DT)
    gmT, gzT = torch.tensor(prob["gm"], dtype=DT), torch.tensor(prob["gz"], dtype=DT)
    m = torch.tensor(prob["m"], dtype=DT)
    z = torch.tensor(prob["z"], dtype=DT)
    gen = torch.Generator().manual_seed(7)

    def loss(mm_, zz_, pp):
        mo, zo = O.evoformer_block(mm_, zz_, mmT, pmT, pp, d, drT)
        return float((mo * gmT).sum() + (zo * gzT).sum())

    def fd_check(grad, f):
        u = torch.randn(grad.shape, generator=gen, dtype=DT)
        h = 1e-5
        fd = (f(h * u) - f(-h * u)) / (2 * h)
        an = float((grad * u).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)

    fd_check(dm, lambda e: loss(m + e, z, p))
    fd_check(dz, lambda e: loss(m, z + e, p))
    for name in ("row.w_o", "tri_out.w_o", "att_end.w_o", "att_start.b_o", "tri_in.b_o"):
        fd_check(dp[name], lambda e, n=name: loss(m, z, {**p, n: p[n] + e}))


def test_generator_draws_are_seeded_and_have_the_rates():
    d = synth.Dims(n_seq=2, n_res=256)
    a, b = synth.make_dropout(d, 5), synth.make_dropout(d, 5)
    c = synth.make_dropout(d, 6)
    for name, rate, _ in synth.DROPOUT_SITES:
        assert np.array_equal(a[name], b[name])
        assert not np.array_equal(a[name], c[name])
        keep = 1.0 / (1.0 - rate)
        vals = np.unique(a[name])
        assert set(vals.tolist()) <= {0.0, np.float32(keep)}
        frac = float((a[name] == 0).mean())
        n = a[name].size
        # within five standard deviations of the rate
        assert abs(frac - rate) <= 5 * np.sqrt(rate * (1 - rate) / n), (name, frac)
