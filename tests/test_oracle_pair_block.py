"""Pins of the oracle's template pair stack block (AF2 Alg. 16).

  * The Evoformer block touches the pair representation through the outer
    product mean and then runs exactly the template block's steps, so with
    the outer product mean's output weights and bias zeroed its z_out equals
    the pair block's (with and without dropout).
  * The pair block's gradients match central finite differences.
  * Its parameter table (the pair-stack tensors only) agrees with the
    oracle's own shape list.
"""
import numpy as np
import torch

from oracle import evoformer as O
from paper_2207_05477_gb300 import synth

DT = torch.float64
TINY_PAIR = synth.DIMS_TINY.replace(pair_only=1)


def test_evoformer_with_silent_opm_is_the_pair_block():
    d = synth.DIMS_TINY
    prob = synth.make_problem(d, 17, pad_frac=0.2)
    params = synth.unpack_params(d, prob["params"])
    params = dict(params)
    params["opm.w_o"] = np.zeros_like(params["opm.w_o"])
    params["opm.b_o"] = np.zeros_like(params["opm.b_o"])
    for dr in (None, synth.make_dropout(d, 17)):
        _, zo = O.block_forward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], params, d, dropout=dr)
        pair = {k: v for k, v in params.items() if k.split(".")[0] in
                ("tri_out", "tri_in", "att_start", "att_end", "pair_trans")}
        zp = O.pair_block_forward(prob["z"], prob["pair_mask"], pair, TINY_PAIR, dropout=dr)
        assert torch.allclose(zo, zp, rtol=0, atol=1e-12)


def test_pair_block_gradients_match_central_differences():
    d = TINY_PAIR
    prob = synth.make_problem(d, 19, pad_frac=0.2)
    params = synth.unpack_params(d, prob["params"])
    dr = synth.make_dropout(d, 19)
    _, dz, dp = O.pair_block_forward_backward(prob["z"], prob["pair_mask"], params, d, prob["gz"], dropout=dr)
    p = O.to_f64(params)
    z = torch.tensor(prob["z"], dtype=DT)
    pm = torch.tensor(prob["pair_mask"], dtype=DT)
    gz = torch.tensor(prob["gz"], dtype=DT)
    drT = {k: torch.tensor(v, dtype=DT) for k, v in dr.items()}
    gen = torch.Generator().manual_seed(9)

    def loss(zz, pp):
        return float((O.pair_stack_block(zz, pm, pp, d, drT) * gz).sum())

    def check(grad, f):
        u = torch.randn(grad.shape, generator=gen, dtype=DT)
        h = 1e-5
        fd = (f(h * u) - f(-h * u)) / (2 * h)
        an = float((grad * u).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)

    check(dz, lambda e: loss(z + e, p))
    for name in p:
        check(dp[name], lambda e, n=name: loss(z, {**p, n: p[n] + e}))


def test_pair_param_table_matches_oracle_shapes():
    d = synth.DIMS_TEMPLATE
    lay, _ = synth.param_layout(d)
    exp = O.expected_param_shapes(d)
    assert {n for n, _, _, _ in lay} == set(exp)
    for n, _, shape, _ in lay:
        assert tuple(shape) == tuple(exp[n]), n
