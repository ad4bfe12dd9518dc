"""evo_block_fwd_noalloc against evo_block_fwd.

The no-allocation entry point serves callers that cannot allocate device
memory when they call (memory divided up at start-up, or a context where
cudaMalloc's possible synchronisation is not allowed): it runs the same
forward with scratch held inside the library.  Its outputs must match the
workspace entry point's on two calls in a row (the second call reuses the
scratch the first one left behind).  This file is collected last on purpose.
"""
import pytest
import torch

from helpers import rel_l2
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("act", [evo.EVO_BF16, evo.EVO_F32])
def test_noalloc_forward_matches_workspace_forward(built_lib, act):
    tol = 2e-2 if act == evo.EVO_BF16 else 1e-4
    dev = torch.device("cuda:0")
    dt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
    for d, seed in ((synth.Dims(n_seq=8, n_res=24), 7), (synth.Dims(n_seq=5, n_res=37), 8)):
        cd = evo.cdims(d, act)
        prob = synth.make_problem(d, seed, pad_frac=0.1)
        params = torch.tensor(prob["params"], device=dev)
        p16 = evo.bf16_params(cd, params)
        m = torch.tensor(prob["m"], device=dev).to(dt)
        z = torch.tensor(prob["z"], device=dev).to(dt)
        mm = torch.tensor(prob["msa_mask"], device=dev)
        pm = torch.tensor(prob["pair_mask"], device=dev)
        ref_m, ref_z = torch.empty_like(m), torch.empty_like(z)
        ws = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
        evo.block_fwd(cd, params, p16, m, z, ref_m, ref_z, mm, pm, ws)
        for _ in range(2):
            out_m, out_z = torch.full_like(m, float("nan")), torch.full_like(z, float("nan"))
            evo.block_fwd_noalloc(cd, params, p16, m, z, out_m, out_z, mm, pm)
            torch.cuda.synchronize()
            assert torch.isfinite(out_m.float()).all() and torch.isfinite(out_z.float()).all()
            assert rel_l2(out_m, ref_m) <= tol
            assert rel_l2(out_z, ref_z) <= tol
        assert evo.get_error() == evo.EVO_OK


def test_noalloc_rejects_problems_beyond_its_scratch(built_lib):
    d = synth.DIMS_TRAIN_CROP  # needs ~1.3 GiB of forward scratch
    cd = evo.cdims(d, evo.EVO_BF16)
    dev = torch.device("cuda:0")
    params = torch.zeros(evo.param_count(cd), device=dev)
    p16 = torch.zeros(evo.param_count(cd), dtype=torch.bfloat16, device=dev)
    m = torch.zeros(d.n_seq, d.n_res, d.c_m, dtype=torch.bfloat16, device=dev)
    z = torch.zeros(d.n_res, d.n_res, d.c_z, dtype=torch.bfloat16, device=dev)
    mm = torch.ones(d.n_seq, d.n_res, device=dev)
    pm = torch.ones(d.n_res, d.n_res, device=dev)
    with pytest.raises(evo.EvoError) as e:
        evo.block_fwd_noalloc(cd, params, p16, m, z, m, z, mm, pm)
    assert e.value.code == evo.EVO_ERR_WORKSPACE
