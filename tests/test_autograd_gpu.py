"""The torch.autograd path (EvoBlockFn, evoformer_stack) against the FP64 oracle:
one block and a two-block stack with per-block recompute, evaluation mode and
training-mode dropout (the backward must replay the forward's draw)."""
import pytest
import torch

from helpers import rel_l2
from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

D = synth.Dims(n_seq=6, n_res=40)


def _inputs(d, seed, dev):
    prob = synth.make_problem(d, seed, pad_frac=0.1)
    params = torch.tensor(prob["params"], device=dev, requires_grad=True)
    m = torch.tensor(prob["m"], device=dev, dtype=torch.bfloat16).requires_grad_(True)
    z = torch.tensor(prob["z"], device=dev, dtype=torch.bfloat16).requires_grad_(True)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    return prob, params, m, z, mm, pm


@pytest.mark.parametrize("dropout", [False, True])
def test_autograd_block_matches_oracle(built_lib, dropout):
    dev = torch.device("cuda:0")
    prob, params, m, z, mm, pm = _inputs(D, 21, dev)
    cd = evo.cdims(D, evo.EVO_BF16)
    dr_np = synth.make_dropout(D, 21) if dropout else None
    dr = {k: torch.tensor(v, device=dev) for k, v in dr_np.items()} if dropout else None
    mo, zo = evo.evoformer_block(m, z, params, mm, pm, cd, dr)
    gm, gz = torch.tensor(prob["gm"], device=dev), torch.tensor(prob["gz"], device=dev)
    ((mo.float() * gm).sum() + (zo.float() * gz).sum()).backward()
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    p = synth.unpack_params(D, prob["params"])
    rmo, rzo, rdm, rdz, _ = O.block_forward_backward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"], p, D,
                                                     prob["gm"], prob["gz"], dropout=dr_np)
    errs = {"m": rel_l2(mo.detach().double().cpu(), rmo), "z": rel_l2(zo.detach().double().cpu(), rzo),
            "dm": rel_l2(m.grad.double().cpu(), rdm), "dz": rel_l2(z.grad.double().cpu(), rdz)}
    assert errs["m"] <= 2e-2 and errs["z"] <= 2e-2 and errs["dm"] <= 5e-2 and errs["dz"] <= 5e-2, errs


def test_autograd_two_block_stack_matches_oracle(built_lib):
    dev = torch.device("cuda:0")
    prob, p0, m, z, mm, pm = _inputs(D, 22, dev)
    p1_np = synth.make_params(D, 1022)
    p1 = torch.tensor(p1_np, device=dev, requires_grad=True)
    cd = evo.cdims(D, evo.EVO_BF16)
    drs_np = [synth.make_dropout(D, 22), synth.make_dropout(D, 23)]
    drs = [{k: torch.tensor(v, device=dev) for k, v in x.items()} for x in drs_np]
    mo, zo = evo.evoformer_stack(m, z, [p0, p1], mm, pm, cd, drs)
    gm, gz = torch.tensor(prob["gm"], device=dev), torch.tensor(prob["gz"], device=dev)
    ((mo.float() * gm).sum() + (zo.float() * gz).sum()).backward()
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK

    P0 = O.to_f64(synth.unpack_params(D, prob["params"]), requires_grad=True)
    P1 = O.to_f64(synth.unpack_params(D, p1_np), requires_grad=True)
    m0 = torch.tensor(prob["m"], dtype=torch.float64, requires_grad=True)
    z0 = torch.tensor(prob["z"], dtype=torch.float64, requires_grad=True)
    mmT = torch.tensor(prob["msa_mask"], dtype=torch.float64)
    pmT = torch.tensor(prob["pair_mask"], dtype=torch.float64)
    dr64 = [{k: torch.tensor(v, dtype=torch.float64) for k, v in x.items()} for x in drs_np]
    m1, z1 = O.evoformer_block(m0, z0, mmT, pmT, P0, D, dr64[0])
    m2, z2 = O.evoformer_block(m1, z1, mmT, pmT, P1, D, dr64[1])
    loss = (m2 * torch.tensor(prob["gm"], dtype=torch.float64)).sum() + \
        (z2 * torch.tensor(prob["gz"], dtype=torch.float64)).sum()
    dm, dz = torch.autograd.grad(loss, [m0, z0])
    errs = {"m": rel_l2(mo.detach().double().cpu(), m2.detach()), "z": rel_l2(zo.detach().double().cpu(), z2.detach()),
            "dm": rel_l2(m.grad.double().cpu(), dm), "dz": rel_l2(z.grad.double().cpu(), dz)}
    # two blocks of BF16 rounding: twice the one-block bounds
    assert errs["m"] <= 4e-2 and errs["z"] <= 4e-2 and errs["dm"] <= 1e-1 and errs["dz"] <= 1e-1, errs
