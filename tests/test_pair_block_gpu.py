"""Parity of the template pair stack block (AF2 Alg. 16) through the C ABI
with the FP64 oracle, at the published template dims (c_t 64, 4 heads of 16,
c_mul 64, transition factor 2), with training-mode dropout; bounds as for the
Evoformer block (BF16 with the oracle's own BF16 floor rule at the ragged
size, where the pair transition's ReLU mask makes the same few tensors
noisy)."""
import numpy as np
import pytest
import torch

from helpers import _to_bf16_grid, param_grad_errors, rel_l2
from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth
from test_block_gpu import BF16_FLOOR_FACTOR, BF16_GRAD_TOL, BF16_TOL, FP32_GRAD_TOL, FP32_TOL, RELU_MASKED_TOL

pytestmark = pytest.mark.gpu

RELU_MASKED = {"pair_trans." + t for t in ("ln.gamma", "ln.beta", "w1", "b1")}
RAGGED = synth.DIMS_TEMPLATE.replace(n_res=37)


def _problem(d, seed=41, pad=0.1):
    prob = synth.make_problem(d, seed, pad_frac=pad)
    return prob, synth.make_dropout(d, seed)


def _oracle(d, prob, dr, bf16_inputs=False):
    cast = _to_bf16_grid if bf16_inputs else (lambda x: x)
    p = synth.unpack_params(d, cast(prob["params"]))
    return O.pair_block_forward_backward(cast(prob["z"]), prob["pair_mask"], p, d, cast(prob["gz"]), dropout=dr)


def _gpu(d, prob, dr, act):
    dev = torch.device("cuda:0")
    dt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
    cd = evo.cdims(d, act)
    params = torch.tensor(prob["params"], device=dev)
    p16 = evo.pair_bf16_params(cd, params)
    z = torch.tensor(prob["z"], device=dev).to(dt)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    drd = {k: torch.tensor(v, device=dev) for k, v in dr.items()}
    z_out = torch.empty_like(z)
    evo.pair_block_fwd(cd, params, p16, z, z_out, pm, evo.pair_workspace(cd, evo.EVO_MODE_FWD, dev), drd)
    gz = torch.tensor(prob["gz"], device=dev).to(dt)
    dz = torch.empty_like(z)
    dp = torch.zeros_like(params)
    evo.pair_block_bwd(cd, params, p16, z, pm, gz, dz, dp, evo.pair_workspace(cd, evo.EVO_MODE_BWD, dev), drd)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    return z_out.double().cpu(), dz.double().cpu(), dp.double().cpu()


def _errors(d, out, ref):
    zo, dz, dp = out
    errs = {"z": rel_l2(zo, ref[0]), "dz": rel_l2(dz, ref[1])}
    errs.update(param_grad_errors(d, dp, ref[2]))
    return errs


def _bounds(errs, tol, gtol, relu_tol, floor=None):
    lim = {k: (tol if k == "z" else relu_tol if k in RELU_MASKED else gtol) for k in errs}
    if floor is not None:
        lim = {k: max(v, BF16_FLOOR_FACTOR * floor[k]) for k, v in lim.items()}
    return {k: v for k, v in errs.items() if not v <= lim[k]}


def test_fp32_pair_block_ragged_dropout(built_lib):
    prob, dr = _problem(RAGGED)
    ref = _oracle(RAGGED, prob, dr)
    bad = _bounds(_errors(RAGGED, _gpu(RAGGED, prob, dr, evo.EVO_F32), ref), FP32_TOL, FP32_GRAD_TOL, FP32_GRAD_TOL)
    assert not bad, bad


def _packed(d, dp):
    """The flat (padded) buffer layout of a name -> gradient dict."""
    lay, total = synth.param_layout(d)
    out = torch.zeros(total, dtype=torch.float64)
    for name, off, shape, _ in lay:
        out[off:off + int(np.prod(shape))] = torch.as_tensor(dp[name]).double().flatten()
    return out


def test_bf16_pair_block_ragged_dropout(built_lib):
    prob, dr = _problem(RAGGED)
    ref = _oracle(RAGGED, prob, dr)
    zo_f, dz_f, dp_f = _oracle(RAGGED, prob, dr, bf16_inputs=True)
    floor = _errors(RAGGED, (zo_f, dz_f, _packed(RAGGED, dp_f)), ref)
    bad = _bounds(_errors(RAGGED, _gpu(RAGGED, prob, dr, evo.EVO_BF16), ref), BF16_TOL, BF16_GRAD_TOL,
                  RELU_MASKED_TOL, floor)
    assert not bad, bad


@pytest.mark.slow
def test_bf16_pair_block_template_crop_dropout(built_lib):
    d = synth.DIMS_TEMPLATE
    prob, dr = _problem(d, pad=0.05)
    ref = _oracle(d, prob, dr)
    bad = _bounds(_errors(d, _gpu(d, prob, dr, evo.EVO_BF16), ref), BF16_TOL, BF16_GRAD_TOL, RELU_MASKED_TOL)
    assert not bad, bad
