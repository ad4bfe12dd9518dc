"""The block forward + backward can be captured into one CUDA graph and replayed.

The library makes no allocation and no host synchronisation inside a block
call, so a captured step replays the same kernels on the same buffers; the
replay must reproduce the eager results (up to the order of the FP32
atomics in the attention backward)."""
import pytest
import torch

from helpers import rel_l2
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu


def test_captured_step_matches_eager(built_lib):
    d = synth.Dims(n_seq=16, n_res=48)
    cd = evo.cdims(d, evo.EVO_BF16)
    dev = torch.device("cuda:0")
    prob = synth.make_problem(d, 21, pad_frac=0.1)
    params = torch.tensor(prob["params"], device=dev)
    p16 = torch.empty(evo.param_count(cd), dtype=torch.bfloat16, device=dev)
    m = torch.tensor(prob["m"], device=dev).to(torch.bfloat16)
    z = torch.tensor(prob["z"], device=dev).to(torch.bfloat16)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    gm = torch.tensor(prob["gm"], device=dev).to(torch.bfloat16)
    gz = torch.tensor(prob["gz"], device=dev).to(torch.bfloat16)
    mo, zo, dm, dz = (torch.empty_like(t) for t in (m, z, m, z))
    dp = torch.zeros_like(params)
    wsf = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
    wsb = evo.workspace(cd, evo.EVO_MODE_BWD, dev)

    def step():
        dp.zero_()
        evo.params_to_bf16(cd, params, p16)
        evo.block_fwd(cd, params, p16, m, z, mo, zo, mm, pm, wsf)
        evo.block_bwd(cd, params, p16, m, z, mm, pm, gm, gz, dm, dz, dp, wsb)

    step()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (mo, zo, dm, dz, dp)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    for t in (mo, zo, dm, dz, dp):
        t.fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    for got, want in zip((mo, zo, dm, dz, dp), ref):
        assert torch.isfinite(got.float()).all()
        assert rel_l2(got, want) <= 1e-2
    assert torch.equal(mo, ref[0]) and torch.equal(zo, ref[1])  # the forward has no atomics: bitwise equal
