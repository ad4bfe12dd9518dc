"""evo_stack_fwd (the EvoformerStack forward, Fig. 1: blocks applied in turn,
m and z updated in place) against two FP64 oracle blocks chained, on both
tiers, with the two blocks' parameters packed at a padded stride."""
import numpy as np
import pytest
import torch

from helpers import rel_l2
from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

D = synth.Dims(n_seq=6, n_res=40)


@pytest.mark.parametrize("act_dtype,tol", [(evo.EVO_F32, 2e-4), (evo.EVO_BF16, 4e-2)])
def test_two_block_stack_matches_chained_oracle(built_lib, act_dtype, tol):
    dev = torch.device("cuda:0")
    prob = synth.make_problem(D, 41, pad_frac=0.1)
    p1_np = synth.make_params(D, 1041)
    cd = evo.cdims(D, act_dtype)
    n = evo.param_count(cd)
    stride = (n + 127) // 128 * 128 + 128  # padded beyond the minimum on purpose
    packed = torch.zeros(2 * stride, device=dev)
    packed[:n] = torch.tensor(prob["params"], device=dev)
    packed[stride:stride + n] = torch.tensor(p1_np, device=dev)
    p16 = None
    if act_dtype == evo.EVO_BF16:
        p16 = torch.zeros(2 * stride, dtype=torch.bfloat16, device=dev)
        for b in range(2):
            p16[b * stride:b * stride + n] = evo.bf16_params(cd, packed[b * stride:b * stride + n].contiguous())
    dt = torch.bfloat16 if act_dtype == evo.EVO_BF16 else torch.float32
    m = torch.tensor(prob["m"], device=dev).to(dt)
    z = torch.tensor(prob["z"], device=dev).to(dt)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    ws = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
    evo.stack_fwd(cd, 2, packed, p16, stride, m, z, mm, pm, ws)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK

    m1, z1 = O.block_forward(prob["m"], prob["z"], prob["msa_mask"], prob["pair_mask"],
                             synth.unpack_params(D, prob["params"]), D)
    m2, z2 = O.block_forward(m1, z1, prob["msa_mask"], prob["pair_mask"], synth.unpack_params(D, p1_np), D)
    errs = {"m": rel_l2(m.double().cpu(), m2), "z": rel_l2(z.double().cpu(), z2)}
    # two blocks of rounding: twice the one-block bound of the tier
    assert errs["m"] <= tol and errs["z"] <= tol, errs
    assert np.isfinite(m.float().cpu().numpy()).all() and np.isfinite(z.float().cpu().numpy()).all()
