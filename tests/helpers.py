"""Shared helpers of the parity tests: run the library and the oracle on the same seeded inputs."""
import functools
import math

import numpy as np
import torch

from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth


def rel_l2(x, ref, mask=None):
    x = torch.as_tensor(x).double().cpu()
    ref = torch.as_tensor(ref).double().cpu()
    if mask is not None:
        m = torch.as_tensor(mask).bool().cpu()
        while m.dim() < x.dim():
            m = m[..., None]
        m = m.expand_as(x)
        x, ref = x[m], ref[m]
    den = ref.norm().item()
    return (x - ref).norm().item() / (den if den > 0 else 1.0)


@functools.lru_cache(maxsize=4)
def problem(d, seed=32, pad_frac=0.0, trailing=False):
    return synth.make_problem(d, seed, pad_frac, trailing)


def to_bf16_grid(x):
    """x rounded to the nearest BF16 value (round-to-nearest-even), back in fp64.

    A BF16 run hands the library m, z and the cotangents as BF16 bytes, so
    the oracle of a BF16 run reads these same values (parameters, masks and
    dropout scales reach the library as FP32 and stay as they are)."""
    return torch.as_tensor(np.asarray(x)).float().bfloat16().double().numpy()


@functools.lru_cache(maxsize=3)
def oracle_fwd_bwd(d, seed=32, pad_frac=0.0, trailing=False, dropout=False, bf16_inputs=False):
    """dropout: apply the seeded training-mode dropout scales (synth.make_dropout).
    bf16_inputs: the oracle reads m, z, gm, gz rounded to BF16 (the bytes a BF16 run receives)."""
    prob = problem(d, seed, pad_frac, trailing)
    cast = to_bf16_grid if bf16_inputs else (lambda x: x)
    p = synth.unpack_params(d, prob["params"])
    dr = synth.make_dropout(d, seed) if dropout else None
    mo, zo, dm, dz, dp = O.block_forward_backward(cast(prob["m"]), cast(prob["z"]), prob["msa_mask"],
                                                  prob["pair_mask"], p, d, cast(prob["gm"]), cast(prob["gz"]),
                                                  dropout=dr)
    return mo, zo, dm, dz, dp


@functools.lru_cache(maxsize=3)
def oracle_fwd(d, seed=32, pad_frac=0.0, trailing=False, bf16_inputs=False):
    prob = problem(d, seed, pad_frac, trailing)
    cast = to_bf16_grid if bf16_inputs else (lambda x: x)
    p = synth.unpack_params(d, prob["params"])
    return O.block_forward(cast(prob["m"]), cast(prob["z"]), prob["msa_mask"], prob["pair_mask"], p, d)


def slice_rel_l2_max(x, ref, axes, min_nonzero=32):
    """Largest relative L2 error over the slices of x along each of ``axes``
    (e.g. per MSA row, per residue, per channel).  A wrong head, row or
    column that a whole-tensor norm averages away shows here.

    A slice whose reference norm is below a quarter of the typical (RMS)
    slice norm is measured against that quarter, so a slice that is nearly
    zero in the reference (a padded row, a channel with a tiny gradient)
    neither divides by zero nor turns rounding into a large ratio.  An axis
    whose median slice holds fewer than ``min_nonzero`` nonzero reference
    elements is not reported (too few elements for a relative error to mean
    anything: the degenerate and mostly-padded problems)."""
    x = torch.as_tensor(x).double().cpu()
    ref = torch.as_tensor(ref).double().cpu()
    worst = {}
    for ax in axes:
        dims = [i for i in range(x.dim()) if i != ax]
        if (ref != 0).sum(dim=dims).double().median().item() < min_nonzero:
            continue
        num = (x - ref).pow(2).sum(dim=dims).sqrt()
        den = ref.pow(2).sum(dim=dims).sqrt()
        floor = 0.25 * ref.norm().item() / math.sqrt(ref.shape[ax])
        worst[ax] = float((num / torch.clamp(den, min=max(floor, 1e-300))).max().item())
    return worst


def gpu_run(d, act_dtype, seed=32, pad_frac=0.0, trailing=False, backward=True, dropout=False):
    """Block forward (and backward) through the C ABI on cuda:0; results on the CPU in fp64.
    dropout: training mode with the seeded scales of synth.make_dropout."""
    prob = problem(d, seed, pad_frac, trailing)
    dev = torch.device("cuda:0")
    dt = torch.bfloat16 if act_dtype == evo.EVO_BF16 else torch.float32
    cd = evo.cdims(d, act_dtype)
    params = torch.tensor(prob["params"], device=dev)
    p16 = evo.bf16_params(cd, params)
    m = torch.tensor(prob["m"], device=dev).to(dt)
    z = torch.tensor(prob["z"], device=dev).to(dt)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    m_out, z_out = torch.empty_like(m), torch.empty_like(z)
    ws = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
    dr = {k: torch.tensor(v, device=dev) for k, v in synth.make_dropout(d, seed).items()} if dropout else None
    if dropout:
        evo.block_fwd_dropout(cd, params, p16, m, z, m_out, z_out, mm, pm, dr, ws)
    else:
        evo.block_fwd(cd, params, p16, m, z, m_out, z_out, mm, pm, ws)
    out = {"m": m_out.double().cpu(), "z": z_out.double().cpu()}
    if backward:
        gm = torch.tensor(prob["gm"], device=dev).to(dt)
        gz = torch.tensor(prob["gz"], device=dev).to(dt)
        dm, dz = torch.empty_like(m), torch.empty_like(z)
        dp = torch.zeros_like(params)
        wsb = evo.workspace(cd, evo.EVO_MODE_BWD, dev)
        if dropout:
            evo.block_bwd_dropout(cd, params, p16, m, z, mm, pm, dr, gm, gz, dm, dz, dp, wsb)
        else:
            evo.block_bwd(cd, params, p16, m, z, mm, pm, gm, gz, dm, dz, dp, wsb)
        out.update(dm=dm.double().cpu(), dz=dz.double().cpu(), dparams=dp.double().cpu())
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    return out


def param_grad_errors(d, gpu_dparams, oracle_dp):
    """Relative L2 error of each parameter tensor's gradient.

    A tensor whose exact gradient vanishes (e.g. the shift of the pair-bias
    LayerNorm, row.ln_z.beta: it adds one constant to every logit of a head,
    which the softmax cancels; or, at N_res = 1, every weight feeding a
    one-key softmax) has no relative error; its error is measured against the
    norm of the whole parameter gradient instead.
    """
    lay, _ = synth.param_layout(d)
    total = float(np.sqrt(sum(torch.as_tensor(v).double().norm().item() ** 2 for v in oracle_dp.values())))
    errs = {}
    for name, off, shape, _ in lay:
        n = int(np.prod(shape))
        g = torch.as_tensor(gpu_dparams[off:off + n]).double().reshape(shape)
        ref = torch.as_tensor(oracle_dp[name]).double()
        if ref.norm().item() <= 1e-9 * total:
            errs[name] = (g - ref).norm().item() / total
        else:
            errs[name] = rel_l2(g, ref)
    return errs
