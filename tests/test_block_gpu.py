"""Parity of the CUDA Evoformer block (through the C ABI) with the FP64 oracle.

The bounds (stated, and measured where the ReLU mask of the transitions
makes a tensor miss them) and the slice check are in ``tolerances.py``.  The
oracle of a BF16 case reads the BF16 bytes the library receives.
"""
import pytest

from helpers import gpu_run, oracle_fwd, oracle_fwd_bwd, param_grad_errors, rel_l2
from paper_2207_05477_gb300 import evo, synth
from tolerances import BF16_GRAD_TOL, BF16_TOL, FP32_GRAD_TOL, FP32_TOL, check, slice_errors

pytestmark = pytest.mark.gpu

RAGGED = synth.Dims(n_seq=5, n_res=37)  # ragged against every 64/128-wide tile


def _errors(out, ref, d):
    mo, zo, dm, dz, dp = ref
    errs = {"m": rel_l2(out["m"], mo), "z": rel_l2(out["z"], zo)}
    refs = {"m": mo, "z": zo}
    if "dm" in out:
        errs.update(dm=rel_l2(out["dm"], dm), dz=rel_l2(out["dz"], dz))
        errs.update(param_grad_errors(d, out["dparams"], dp))
        refs.update(dm=dm, dz=dz)
    return errs, slice_errors(out, refs)


def _run(case, d, act, pad_frac=0.0, trailing=False, dropout=False, seed=32):
    bf = act == evo.EVO_BF16
    out = gpu_run(d, act, seed=seed, pad_frac=pad_frac, trailing=trailing, dropout=dropout)
    ref = oracle_fwd_bwd(d, seed, pad_frac, trailing, dropout, bf16_inputs=bf)
    errs, sl = _errors(out, ref, d)
    check(case, errs, BF16_TOL if bf else FP32_TOL, BF16_GRAD_TOL if bf else FP32_GRAD_TOL, sl)
    return out, ref


def _run_fwd(case, d, act, seed=32, pad_frac=0.0):
    bf = act == evo.EVO_BF16
    out = gpu_run(d, act, seed=seed, pad_frac=pad_frac, backward=False)
    mo, zo = oracle_fwd(d, seed, pad_frac, bf16_inputs=bf)
    errs = {"m": rel_l2(out["m"], mo), "z": rel_l2(out["z"], zo)}
    check(case, errs, BF16_TOL if bf else FP32_TOL, None, slice_errors(out, {"m": mo, "z": zo}))


def test_fp32_forward_small_config(built_lib):
    _run_fwd("block_fp32_fwd_config1", synth.DIMS_SMALL_FP32, evo.EVO_F32)


def test_bf16_forward_small_config(built_lib):
    _run_fwd("block_bf16_fwd_config1", synth.DIMS_SMALL_FP32, evo.EVO_BF16)


def test_fp32_fwd_bwd_ragged_padded(built_lib):
    _run("block_fp32_ragged", RAGGED, evo.EVO_F32, pad_frac=0.1)


def test_bf16_fwd_bwd_ragged_padded(built_lib):
    _run("block_bf16_ragged", RAGGED, evo.EVO_BF16, pad_frac=0.1)


@pytest.mark.parametrize("d", [synth.Dims(n_seq=1, n_res=8), synth.Dims(n_seq=3, n_res=1)])
def test_bf16_degenerate_sizes(built_lib, d):
    """One MSA row; one residue.  At N_res = 1 every pair-stack gradient is a
    single-position quantity with no averaging over positions."""
    import numpy as np
    import torch
    out, ref = _run(f"block_bf16_degenerate_S{d.n_seq}_R{d.n_res}", d, evo.EVO_BF16)
    lay, _ = synth.param_layout(d)
    flat_ref = torch.cat([torch.as_tensor(ref[4][n]).double().flatten() for n, _, _, _ in lay])
    flat_gpu = torch.cat([out["dparams"][o:o + int(np.prod(s))].double() for _, o, s, _ in lay])
    assert rel_l2(flat_gpu, flat_ref) <= BF16_GRAD_TOL


def test_bf16_trailing_padding_and_single_valid_residue(built_lib):
    _run("block_bf16_trailing", synth.Dims(n_seq=4, n_res=20), evo.EVO_BF16, pad_frac=0.95, trailing=True)


@pytest.mark.slow
def test_bf16_fwd_bwd_training_crop(built_lib):
    """The paper's initial-training crop: N_seq=128, N_res=256, 5% padded residues."""
    _run("block_bf16_crop", synth.DIMS_TRAIN_CROP, evo.EVO_BF16, pad_frac=0.05)


@pytest.mark.slow
def test_fp32_fwd_bwd_training_crop(built_lib):
    _run("block_fp32_crop", synth.DIMS_TRAIN_CROP, evo.EVO_F32, pad_frac=0.05)


# ------------------------------------------------- keys beyond 256 (fine-tune crop)
@pytest.mark.slow
def test_bf16_fwd_bwd_finetune_crop(built_lib):
    """The paper's fine-tune crop, one block: N_seq=512, N_res=384 (model
    settings table).  Row and triangle attention run over 384 keys, column
    attention over 512: every attention kind beyond the 256-key tile."""
    _run("block_bf16_finetune", synth.Dims(n_seq=512, n_res=384), evo.EVO_BF16, pad_frac=0.05)


@pytest.mark.slow
def test_bf16_forward_long_sequence(built_lib):
    """A forward at N_res = 768 with four sequences: row and triangle
    attention with pair bias over 768 keys (twelve 64-key blocks: the
    long-stream forward kernel), the pair stack at three times the crop."""
    _run_fwd("block_bf16_fwd_R768", synth.Dims(n_seq=4, n_res=768), evo.EVO_BF16)


@pytest.mark.slow
def test_bf16_fwd_bwd_deep_msa_column_attention(built_lib):
    """Column attention over 1100 sequences (18 key blocks of 64, the last
    ragged): the long-stream forward kernel (one softmax warp per TMEM lane
    quarter) and the streaming backward, fwd+bwd against the oracle at a
    small N_res so that the FP64 oracle stays quick."""
    _run("block_bf16_deep_msa_S1100_R16", synth.Dims(n_seq=1100, n_res=16), evo.EVO_BF16, pad_frac=0.05)


# The two smallest proteins of the seeded 16-protein batch (N_res ~ U[64, 1024],
# N_seq ~ U[32, 512], the batched-inference workload), one block forward each
# at its own sizes, 5 % padded residues.
def _batch16_smallest(k=2):
    import numpy as np
    rng = np.random.default_rng(32)
    prot = [(int(rng.integers(32, 513)), int(rng.integers(64, 1025))) for _ in range(16)]
    return sorted(prot, key=lambda p: p[1])[:k]


@pytest.mark.slow
@pytest.mark.parametrize("S,R", _batch16_smallest())
def test_bf16_forward_batch16_smallest_proteins(built_lib, S, R):
    _run_fwd(f"block_bf16_fwd_S{S}_R{R}", synth.Dims(n_seq=S, n_res=R), evo.EVO_BF16, pad_frac=0.05)


# ------------------------------------------------- extra-MSA block (global column attention)
EXTRA_SMALL = synth.DIMS_EXTRA_MSA.replace(n_seq=64, n_res=40)
EXTRA_MID = synth.DIMS_EXTRA_MSA.replace(n_seq=512, n_res=96)


def test_extra_msa_fp32_fwd_bwd(built_lib):
    _run("extra_fp32_small", EXTRA_SMALL, evo.EVO_F32, pad_frac=0.1)


def test_extra_msa_bf16_fwd_bwd(built_lib):
    _run("extra_bf16_mid", EXTRA_MID, evo.EVO_BF16, pad_frac=0.05)


@pytest.mark.slow
def test_extra_msa_bf16_full_size(built_lib):
    """The paper's initial-training extra-MSA block: N_extra_seq=1024, N_res=256, c_e=64."""
    _run("extra_bf16_full", synth.DIMS_EXTRA_MSA, evo.EVO_BF16, pad_frac=0.05)


# ------------------------------------------------------- training-mode dropout
# The seeded scales of synth.make_dropout (rates 0.15 / 0.25, AF2 row-wise and
# column-wise sharing) go to the oracle and, through evo_block_*_dropout, to
# the kernels; the bounds are those of evaluation mode.

def test_fp32_fwd_bwd_dropout_ragged_padded(built_lib):
    _run("block_fp32_ragged_dropout", RAGGED, evo.EVO_F32, pad_frac=0.1, dropout=True)


def test_bf16_fwd_bwd_dropout_ragged_padded(built_lib):
    _run("block_bf16_ragged_dropout", RAGGED, evo.EVO_BF16, pad_frac=0.1, dropout=True)


@pytest.mark.slow
def test_bf16_fwd_bwd_dropout_training_crop(built_lib):
    _run("block_bf16_crop_dropout", synth.DIMS_TRAIN_CROP, evo.EVO_BF16, pad_frac=0.05, dropout=True)
