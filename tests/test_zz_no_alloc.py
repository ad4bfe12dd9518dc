"""evo_block_fwd_noalloc against evo_block_fwd.

The no-allocation entry point serves callers that cannot allocate device
memory when they call (memory divided up at start-up, or a context where
cudaMalloc's possible synchronisation is not allowed): it runs the same
forward with scratch held inside the library, in the inference workspace
plan, whose outputs equal the workspace entry point's bit for bit.

The library's scratch array starts zeroed, so a read of a byte that no call
wrote would go unnoticed on a fresh array.  The first call here therefore
fills the array with NaN (a forward on NaN inputs at the largest shape of the
file); every later call must still match evo_block_fwd exactly, twice in a
row (the second call reuses the scratch the first one left behind).

Collected last (the file name sorts after every other test file): the first
call reserves the library's 128 MiB array on the GPU for the rest of the
process, which the memory-sized tests before it should not see, and a
failure here leaves every other test already run under ``-x``.
"""
import pytest
import torch

from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

# (dims, seed, pair_slab): the last case also runs the i-slab plan on the
# BF16 path (rows 12 at a time, a last slab of one row)
CASES = [(synth.DIMS_SMALL_FP32, 32, 0), (synth.Dims(n_seq=8, n_res=24), 7, 0), (synth.Dims(n_seq=5, n_res=37), 8, 12)]


def _inputs(d, act, seed, dev, slab=0):
    dt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
    cd = evo.cdims(d, act, pair_slab=slab if act == evo.EVO_BF16 else 0)
    prob = synth.make_problem(d, seed, pad_frac=0.1)
    params = torch.tensor(prob["params"], device=dev)
    p16 = evo.bf16_params(cd, params)
    m = torch.tensor(prob["m"], device=dev).to(dt)
    z = torch.tensor(prob["z"], device=dev).to(dt)
    mm = torch.tensor(prob["msa_mask"], device=dev)
    pm = torch.tensor(prob["pair_mask"], device=dev)
    return cd, params, p16, m, z, mm, pm


def _poison_scratch(act, dev):
    """One forward on NaN inputs at the largest shape of the file: its
    intermediates leave NaN all over the shared scratch array."""
    d = max((c[0] for c in CASES), key=lambda d: evo.workspace_size(evo.cdims(d, act), evo.EVO_MODE_INFER))
    cd, params, p16, m, z, mm, pm = _inputs(d, act, 1, dev)
    m.fill_(float("nan"))
    z.fill_(float("nan"))
    params.fill_(float("nan"))
    if p16 is not None:
        p16.fill_(float("nan"))
    evo.block_fwd_noalloc(cd, params, p16, m, z, torch.empty_like(m), torch.empty_like(z), mm, pm)
    torch.cuda.synchronize()


@pytest.mark.parametrize("act", [evo.EVO_BF16, evo.EVO_F32])
def test_noalloc_forward_matches_workspace_forward(built_lib, act):
    dev = torch.device("cuda:0")
    _poison_scratch(act, dev)
    for d, seed, slab in CASES:
        cd, params, p16, m, z, mm, pm = _inputs(d, act, seed, dev, slab)
        ref_m, ref_z = torch.empty_like(m), torch.empty_like(z)
        ws = evo.workspace(cd, evo.EVO_MODE_FWD, dev)
        evo.block_fwd(cd, params, p16, m, z, ref_m, ref_z, mm, pm, ws)
        for _ in range(2):
            out_m, out_z = torch.full_like(m, float("nan")), torch.full_like(z, float("nan"))
            evo.block_fwd_noalloc(cd, params, p16, m, z, out_m, out_z, mm, pm)
            torch.cuda.synchronize()
            assert torch.equal(out_m, ref_m), d
            assert torch.equal(out_z, ref_z), d
        assert evo.get_error() == evo.EVO_OK


def test_noalloc_rejects_problems_beyond_its_scratch(built_lib):
    d = synth.DIMS_TRAIN_CROP.replace(n_res=208)  # the inference plan needs ~135 MiB here
    cd = evo.cdims(d, evo.EVO_BF16)
    assert evo.workspace_size(cd, evo.EVO_MODE_INFER) > 128 << 20
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
