"""i-slab subbatching of the pair stack (Sec. 3.4.4) in the inference plan
against the unsliced forward.

With evo_dims.pair_slab set, evo_block_fwd_infer runs steps 5-9 (and the
pair-side parts of steps 1 and 4) a slab of rows at a time, incoming
multiplication and ending attention as their outgoing / starting forms on
the transposed grid.  Every output element is computed by the same kernels
with the same operands in the same order as in the unsliced forward, so the
result must be the same bit for bit: ragged last slabs (down to one row),
n_res off the multiple of 8, more keys than the one-pass attention kernel
takes (the streaming kernel on both sides), and the global column attention
variant of the MSA stack.
"""
import pytest
import torch

from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

CASES = [
    (synth.Dims(n_seq=8, n_res=40), 16, 3),
    (synth.Dims(n_seq=5, n_res=37), 12, 4),
    (synth.Dims(n_seq=4, n_res=300), 128, 5),
    (synth.DIMS_EXTRA_MSA.replace(n_seq=16, n_res=48), 20, 6),
    (synth.Dims(n_seq=4, n_res=1024), 256, 7),  # 16 key blocks: the long-stream attention kernel
]


@pytest.mark.parametrize("d,slab,seed", CASES, ids=[f"R{c[0].n_res}_slab{c[1]}" for c in CASES])
def test_slabbed_inference_equals_unsliced_forward(built_lib, d, slab, seed):
    dev = torch.device("cuda:0")
    cd = evo.cdims(d, evo.EVO_BF16)
    cds = evo.cdims(d, evo.EVO_BF16, pair_slab=slab)
    prob = synth.make_problem(d, seed, pad_frac=0.1)
    params = torch.tensor(prob["params"], device=dev)
    p16 = evo.bf16_params(cd, params)
    m = torch.tensor(prob["m"], device=dev).to(torch.bfloat16)
    z = torch.tensor(prob["z"], device=dev).to(torch.bfloat16)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    ref_m, ref_z = torch.empty_like(m), torch.empty_like(z)
    evo.block_fwd(cd, params, p16, m, z, ref_m, ref_z, mm, pm, evo.workspace(cd, evo.EVO_MODE_FWD, dev))
    ws = evo.workspace(cds, evo.EVO_MODE_INFER, dev)
    assert ws.numel() < evo.workspace_size(cd, evo.EVO_MODE_INFER)
    ws.fill_(0xFF)  # NaN in every BF16 / FP32 slot: a byte read before written shows
    out_m, out_z = torch.full_like(m, float("nan")), torch.full_like(z, float("nan"))
    evo.block_fwd_infer(cds, params, p16, m, z, out_m, out_z, mm, pm, ws)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    dz = (out_z.float() - ref_z.float()).abs()
    assert torch.equal(out_m, ref_m)
    assert torch.equal(out_z, ref_z), (int((dz > 0).sum()), float(dz.max()))
