"""Parity of the template pair stack block (AF2 Alg. 16) through the C ABI
with the FP64 oracle, at the published template dims (c_t 64, 4 heads of 16,
c_mul 64, transition factor 2), with training-mode dropout; bounds and slice
check as for the Evoformer block (``tolerances.py``)."""
import numpy as np
import pytest
import torch

from helpers import param_grad_errors, rel_l2, to_bf16_grid
from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth
from tolerances import BF16_GRAD_TOL, BF16_TOL, FP32_GRAD_TOL, FP32_TOL, check, slice_errors

pytestmark = pytest.mark.gpu

RAGGED = synth.DIMS_TEMPLATE.replace(n_res=37)


def _problem(d, seed=41, pad=0.1):
    prob = synth.make_problem(d, seed, pad_frac=pad)
    return prob, synth.make_dropout(d, seed)


def _oracle(d, prob, dr, bf16_inputs=False):
    cast = to_bf16_grid if bf16_inputs else (lambda x: x)
    p = synth.unpack_params(d, prob["params"])
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


def _check(case, d, out, ref, tol, gtol):
    zo, dz, dp = out
    errs = {"z": rel_l2(zo, ref[0]), "dz": rel_l2(dz, ref[1])}
    errs.update(param_grad_errors(d, dp, ref[2]))
    check(case, errs, tol, gtol, slice_errors({"z": zo, "dz": dz}, {"z": ref[0], "dz": ref[1]}))


def test_fp32_pair_block_ragged_dropout(built_lib):
    prob, dr = _problem(RAGGED)
    _check("pair_fp32_ragged_dropout", RAGGED, _gpu(RAGGED, prob, dr, evo.EVO_F32), _oracle(RAGGED, prob, dr),
           FP32_TOL, FP32_GRAD_TOL)


def test_bf16_pair_block_ragged_dropout(built_lib):
    prob, dr = _problem(RAGGED)
    _check("pair_bf16_ragged_dropout", RAGGED, _gpu(RAGGED, prob, dr, evo.EVO_BF16),
           _oracle(RAGGED, prob, dr, bf16_inputs=True), BF16_TOL, BF16_GRAD_TOL)


@pytest.mark.slow
def test_bf16_pair_block_template_crop_dropout(built_lib):
    d = synth.DIMS_TEMPLATE
    prob, dr = _problem(d, pad=0.05)
    _check("pair_bf16_crop_dropout", d, _gpu(d, prob, dr, evo.EVO_BF16), _oracle(d, prob, dr, bf16_inputs=True),
           BF16_TOL, BF16_GRAD_TOL)
