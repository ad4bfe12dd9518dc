"""Writes bf16_floor_extra_msa.json: the FP64 oracle's own change under BF16
rounding of the block's inputs (m, z, parameters, cotangents) for the
extra-MSA block at its full size (N_extra_seq = 1024, N_res = 256, c_e = 64,
5 % padded residues, seed 32), per output gradient.  Only the oracle and the
seeded input generator run here.

    python tests/golden/make_bf16_floor.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from helpers import oracle_bf16_floor  # noqa: E402
from paper_2207_05477_gb300 import synth  # noqa: E402

if __name__ == "__main__":
    floor = oracle_bf16_floor(synth.DIMS_EXTRA_MSA, pad_frac=0.05)
    with open(os.path.join(HERE, "bf16_floor_extra_msa.json"), "w") as f:
        json.dump({k: round(float(v), 6) for k, v in sorted(floor.items())}, f, indent=1)
