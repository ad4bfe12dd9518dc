"""Central finite differences pin the oracle's gradients.

The oracle's backward is reverse-mode differentiation of its FP64 forward;
these tests check it against (L(x + h u) - L(x - h u)) / 2h, which needs only
forward evaluations, for every parameter tensor and both inputs, along random
directions u, on tiny shapes with a padded residue.
"""
import numpy as np
import pytest
import torch

from oracle import evoformer as O
from paper_2207_05477_gb300 import synth

DT = torch.float64


def _problem(d, pad_res=(2,)):
    prob = synth.make_problem(d, seed=11)
    seq = np.ones(d.n_res, dtype=np.float32)
    for r in pad_res:
        seq[r] = 0
    mm = np.broadcast_to(seq[None], (d.n_seq, d.n_res)).copy()
    pm = seq[:, None] * seq[None]
    gm, gz = synth.make_cotangents(d, 11, mm, pm)
    return prob, mm, pm, gm, gz


def _loss(d, m, z, mm, pm, p, gm, gz):
    mo, zo = O.evoformer_block(m, z, mm, pm, p, d)
    return float((mo * gm).sum() + (zo * gz).sum())


@pytest.mark.parametrize("mode", [0, 1])
def test_block_gradients_match_central_differences(mode):
    d = synth.DIMS_TINY.replace(msa_col_mode=mode)
    prob, mm, pm, gm, gz = _problem(d)
    params = synth.unpack_params(d, prob["params"])
    _, _, dm, dz, dp = O.block_forward_backward(prob["m"], prob["z"], mm, pm, params, d, gm, gz)

    p = O.to_f64(params)
    m = torch.tensor(prob["m"], dtype=DT)
    z = torch.tensor(prob["z"], dtype=DT)
    mmT, pmT = torch.tensor(mm, dtype=DT), torch.tensor(pm, dtype=DT)
    gmT, gzT = torch.tensor(gm, dtype=DT), torch.tensor(gz, dtype=DT)
    gen = torch.Generator().manual_seed(5)

    def check(name, x, grad, setter):
        for _ in range(2):
            u = torch.randn(x.shape, generator=gen, dtype=DT)
            h = 1e-5
            setter(x + h * u)
            lp = _loss(d, *cur())
            setter(x - h * u)
            lm = _loss(d, *cur())
            setter(x)
            fd = (lp - lm) / (2 * h)
            an = float((grad * u).sum())
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)

    state = {"m": m, "z": z}

    def cur():
        return state["m"], state["z"], mmT, pmT, p, gmT, gzT

    check("m", m, dm, lambda v: state.__setitem__("m", v))
    check("z", z, dz, lambda v: state.__setitem__("z", v))
    for name in p:
        base = p[name].clone()
        check(name, base, dp[name], lambda v, n=name: p.__setitem__(n, v))


def test_elementwise_fd_on_a_small_tensor():
    """Full element-by-element differences for one weight and one input slice."""
    d = synth.DIMS_TINY
    prob, mm, pm, gm, gz = _problem(d, pad_res=())
    params = synth.unpack_params(d, prob["params"])
    _, _, dm, dz, dp = O.block_forward_backward(prob["m"], prob["z"], mm, pm, params, d, gm, gz)
    p = O.to_f64(params)
    m = torch.tensor(prob["m"], dtype=DT)
    z = torch.tensor(prob["z"], dtype=DT)
    args = lambda mm_, zz_: (mm_, zz_, torch.tensor(mm, dtype=DT), torch.tensor(pm, dtype=DT), p,
                              torch.tensor(gm, dtype=DT), torch.tensor(gz, dtype=DT))
    w = p["att_end.w_b"]
    for idx in np.ndindex(*w.shape):
        h = 1e-6 * max(1.0, abs(float(w[idx])))
        orig = float(w[idx])
        w[idx] = orig + h
        lp = _loss(d, *args(m, z))
        w[idx] = orig - h
        lm = _loss(d, *args(m, z))
        w[idx] = orig
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(dp["att_end.w_b"][idx])) <= 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (1, 3, 5), (2, 4, 7)]:
        h = 1e-6 * max(1.0, abs(float(m[idx])))
        mp, mn = m.clone(), m.clone()
        mp[idx] += h
        mn[idx] -= h
        fd = (_loss(d, *args(mp, z)) - _loss(d, *args(mn, z))) / (2 * h)
        assert abs(fd - float(dm[idx])) <= 1e-6 * max(1.0, abs(fd))


def test_pair_bias_layernorm_shift_has_zero_gradient():
    """beta of the pair-bias LayerNorm adds beta.W_b^h to every logit of head h;
    softmax is shift-invariant, so its gradient vanishes while gamma's does not."""
    d = synth.DIMS_TINY
    prob, mm, pm, gm, gz = _problem(d)
    params = synth.unpack_params(d, prob["params"])
    _, _, _, _, dp = O.block_forward_backward(prob["m"], prob["z"], mm, pm, params, d, gm, gz)
    assert dp["row.ln_z.beta"].abs().max().item() < 1e-12
    assert dp["row.ln_z.gamma"].abs().max().item() > 1e-3
