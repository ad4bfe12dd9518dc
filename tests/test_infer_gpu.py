"""evo_block_fwd_infer (the block forward in the inference workspace, where
the sub-modules share one scratch region) against evo_block_fwd and the FP64
oracle.  Both entries launch the same kernels on the same inputs, only at
other workspace offsets, so their outputs must agree bit for bit; the
inference workspace is filled with a NaN pattern first, so that a buffer read
after another sub-module reused its memory would show."""
import pytest
import torch

from helpers import rel_l2
from oracle import evoformer as O
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

RAGGED = synth.Dims(n_seq=5, n_res=37)
EXTRA = synth.Dims(n_seq=64, n_res=40, c_m=64, h_msa=8, c_msa=8, msa_col_mode=1)
CASES = [(RAGGED, evo.EVO_BF16), (RAGGED, evo.EVO_F32), (EXTRA, evo.EVO_BF16),
         (synth.DIMS_TRAIN_CROP, evo.EVO_BF16), (synth.Dims(n_seq=32, n_res=512), evo.EVO_BF16)]


def _inputs(d, act, seed, dev):
    dt = torch.bfloat16 if act == evo.EVO_BF16 else torch.float32
    cd = evo.cdims(d, act)
    params = torch.tensor(synth.make_params(d, seed), device=dev)
    m, z = synth.make_activations(d, seed)
    mm, pm = synth.make_masks(d, seed, pad_frac=0.1)
    return dict(cd=cd, params=params, p16=evo.bf16_params(cd, params), m=torch.tensor(m, device=dev).to(dt),
                z=torch.tensor(z, device=dev).to(dt), mm=torch.tensor(mm, device=dev),
                pm=torch.tensor(pm, device=dev), np=(m, z, mm, pm))


@pytest.mark.parametrize("d,act", CASES)
def test_infer_equals_forward_bit_for_bit(built_lib, d, act):
    dev = torch.device("cuda:0")
    X = _inputs(d, act, 45, dev)
    cd = X["cd"]
    mo, zo = torch.empty_like(X["m"]), torch.empty_like(X["z"])
    evo.block_fwd(cd, X["params"], X["p16"], X["m"], X["z"], mo, zo, X["mm"], X["pm"],
                  evo.workspace(cd, evo.EVO_MODE_FWD, dev))
    wsi = evo.workspace(cd, evo.EVO_MODE_INFER, dev)
    wsi.fill_(0xFF)  # NaN in both float types
    mi, zi = torch.empty_like(X["m"]), torch.empty_like(X["z"])
    evo.block_fwd_infer(cd, X["params"], X["p16"], X["m"], X["z"], mi, zi, X["mm"], X["pm"], wsi)
    # in place, in the same workspace
    m2, z2 = X["m"].clone(), X["z"].clone()
    evo.block_fwd_infer(cd, X["params"], X["p16"], m2, z2, m2, z2, X["mm"], X["pm"], wsi)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    assert torch.equal(mi, mo) and torch.equal(zi, zo)
    assert torch.equal(m2, mo) and torch.equal(z2, zo)
    assert wsi.numel() < 0.3 * evo.workspace_size(cd, evo.EVO_MODE_FWD)


@pytest.mark.parametrize("d,act,tol", [(RAGGED, evo.EVO_BF16, 2e-2), (RAGGED, evo.EVO_F32, 1e-4)])
def test_infer_matches_oracle(built_lib, d, act, tol):
    dev = torch.device("cuda:0")
    X = _inputs(d, act, 46, dev)
    cd = X["cd"]
    ws = evo.workspace(cd, evo.EVO_MODE_INFER, dev)
    mo, zo = torch.empty_like(X["m"]), torch.empty_like(X["z"])
    evo.block_fwd_infer(cd, X["params"], X["p16"], X["m"], X["z"], mo, zo, X["mm"], X["pm"], ws)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    m, z, mm, pm = X["np"]
    rm, rz = O.block_forward(m, z, mm, pm, synth.unpack_params(d, X["params"].cpu().numpy()), d)
    assert rel_l2(mo.double().cpu(), rm) <= tol and rel_l2(zo.double().cpu(), rz) <= tol
