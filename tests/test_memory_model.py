"""The paper's worked memory example (Sec. 3.4.4, tests/golden/
paper_extra_msa_logits.json) and the library's workspace plans against it.

The paper sizes the row-attention logits of the extra-MSA stack in
fine-tuning (5120 sequences, 384 residues, 8 heads, BF16) at 11.25 GiB,
against about 0.2 GiB for the stack's input and output.  The library never
stores logits (the attention kernels keep them on chip), so its workspace
grows with N_seq by a per-(sequence, residue) amount that does not depend on
N_res, and its whole-block backward workspace at that shape stays below the
paper's single logits tensor."""
import json
import os

from paper_2207_05477_gb300 import evo, synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_extra_msa_logits.json")))


def _extra(S, R):
    return evo.cdims(synth.Dims(n_seq=S, n_res=R, c_m=64, h_msa=8, c_msa=8, msa_col_mode=1), evo.EVO_BF16)


def test_paper_logits_example():
    B, S, R, C = GOLD["input_shape_B_Nseq_Nres_Cm"]
    logits = B * S * GOLD["heads"] * R * R * GOLD["bytes_per_element"]
    assert logits / 2 ** 30 == GOLD["logits_gib"]
    io = B * S * R * C * GOLD["bytes_per_element"] / 2 ** 30
    assert abs(io - GOLD["input_output_gib_each"]) < 0.05


def test_no_logits_in_any_workspace_plan(built_lib):
    _, S, R, _ = GOLD["input_shape_B_Nseq_Nres_Cm"]
    for mode in (evo.EVO_MODE_FWD, evo.EVO_MODE_BWD, evo.EVO_MODE_INFER):
        per = []
        for r in (R, 2 * R):
            grow = evo.workspace_size(_extra(S, r), mode) - evo.workspace_size(_extra(S // 2, r), mode)
            per.append(grow / ((S - S // 2) * r))
        # bytes per (sequence, residue): independent of N_res, and below what
        # one logits row of 8 heads x N_res keys in BF16 would add
        assert per[0] == per[1], (mode, per)
        assert per[0] < GOLD["heads"] * R * GOLD["bytes_per_element"], (mode, per)


def test_whole_block_backward_fits_below_the_paper_logits(built_lib):
    _, S, R, _ = GOLD["input_shape_B_Nseq_Nres_Cm"]
    bwd = evo.workspace_size(_extra(S, R), evo.EVO_MODE_BWD)
    assert bwd / 2 ** 30 < GOLD["logits_gib"]
