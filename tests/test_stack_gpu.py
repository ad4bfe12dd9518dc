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


@pytest.mark.parametrize("act_dtype", [evo.EVO_BF16, evo.EVO_F32])
def test_padded_batch_equals_each_protein_alone(built_lib, act_dtype):
    """A padded batch of proteins of uneven sizes through one evo_stack_fwd
    call equals, bit for bit, each protein through its own call at its own
    sizes; the padding of every slot is neither read nor written (NaN there
    stays NaN and leaks nowhere)."""
    dev = torch.device("cuda:0")
    Smax, Rmax, nb = 12, 40, 2
    sizes = [(12, 40), (5, 23), (8, 33)]
    dt = torch.bfloat16 if act_dtype == evo.EVO_BF16 else torch.float32
    dmax = synth.Dims(n_seq=Smax, n_res=Rmax)
    cd = evo.cdims(dmax, act_dtype)
    n = evo.param_count(cd)
    stride = (n + 127) // 128 * 128
    packed = torch.zeros(nb * stride, device=dev)
    for k in range(nb):
        packed[k * stride:k * stride + n] = torch.tensor(synth.make_params(dmax, 500 + k), device=dev)
    p16 = None
    if act_dtype == evo.EVO_BF16:
        p16 = torch.zeros(nb * stride, dtype=torch.bfloat16, device=dev)
        for k in range(nb):
            p16[k * stride:k * stride + n] = evo.bf16_params(cd, packed[k * stride:k * stride + n].contiguous())
    B = len(sizes)
    nan = float("nan")
    m = torch.full((B, Smax, Rmax, dmax.c_m), nan, dtype=dt, device=dev)
    z = torch.full((B, Rmax, Rmax, dmax.c_z), nan, dtype=dt, device=dev)
    mm = torch.full((B, Smax, Rmax), nan, device=dev)
    pm = torch.full((B, Rmax, Rmax), nan, device=dev)
    singles = []
    for i, (S, R) in enumerate(sizes):
        d = synth.Dims(n_seq=S, n_res=R)
        prob = synth.make_problem(d, 60 + i, pad_frac=0.1)
        mi = torch.tensor(prob["m"], device=dev).to(dt)
        zi = torch.tensor(prob["z"], device=dev).to(dt)
        mmi = torch.tensor(prob["msa_mask"], device=dev)
        pmi = torch.tensor(prob["pair_mask"], device=dev)
        m[i, :S, :R], z[i, :R, :R], mm[i, :S, :R], pm[i, :R, :R] = mi, zi, mmi, pmi
        cdi = evo.cdims(d, act_dtype)
        evo.stack_fwd(cdi, nb, packed, p16, stride, mi, zi, mmi, pmi, evo.workspace(cdi, evo.EVO_MODE_FWD, dev))
        singles.append((mi, zi))
    ws = evo.workspace(cd, evo.EVO_MODE_FWD, dev, batch=B)
    evo.stack_fwd(cd, nb, packed, p16, stride, m, z, mm, pm, ws,
                  n_seq_b=[s for s, _ in sizes], n_res_b=[r for _, r in sizes])
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    for i, (S, R) in enumerate(sizes):
        mi, zi = singles[i]
        assert torch.equal(m[i, :S, :R], mi), i
        assert torch.equal(z[i, :R, :R], zi), i
        pad_m = torch.ones(Smax, Rmax, dtype=torch.bool, device=dev)
        pad_m[:S, :R] = False
        pad_z = torch.ones(Rmax, Rmax, dtype=torch.bool, device=dev)
        pad_z[:R, :R] = False
        assert torch.isnan(m[i][pad_m].float()).all() and torch.isnan(z[i][pad_z].float()).all(), i
