"""GEMM tile autotuning: every candidate launch configuration the tuner tries
computes the same block, and the tuned table is used afterwards.

During a tuning session the k-th GEMM launch of each shape runs the k-th
candidate (tile width BN in {64, 128, 256}; for the atomic weight-gradient
products also the split count), so twelve block fwd+bwd passes cover every
candidate of every shape at least once.  Each pass is checked against the FP64
oracle with the same bounds as the untuned BF16 path.
"""
import pytest

from helpers import gpu_run, oracle_fwd_bwd
from paper_2207_05477_gb300 import evo, synth
from test_block_gpu import _errors
from tolerances import BF16_GRAD_TOL, BF16_TOL, check

pytestmark = pytest.mark.gpu

# N_seq * N_res = 1024 rows in the MSA weight gradients: four 256-deep K ranges
# at most, so the split-count candidates are exercised too; N_res = 48 is
# ragged against every tile width
TUNE_DIMS = synth.Dims(n_seq=16, n_res=48)


def test_bf16_every_tuning_candidate_matches_oracle(built_lib):
    d = TUNE_DIMS
    ref = oracle_fwd_bwd(d, pad_frac=0.1, bf16_inputs=True)

    def _check(out):
        errs, slices = _errors(out, ref, d)
        check("tune_bf16_16x48", errs, BF16_TOL, BF16_GRAD_TOL, slices)

    evo.tune_clear()
    evo.tune_begin()
    try:
        for _ in range(12):
            out = gpu_run(d, evo.EVO_BF16, pad_frac=0.1)
            _check(out)
        n = evo.tune_end()
        entries = evo.tune_entries()
        assert n == len(entries) > 0
        assert all(e["bn"] in (64, 128, 256) and e["splits"] >= 1 for e in entries), entries
        assert max(e["candidates"] for e in entries) >= 4, entries
        assert any(e["splits"] != 1 or e["default_splits"] != 1 for e in entries), entries
        # the tuned table is what later launches use
        out = gpu_run(d, evo.EVO_BF16, pad_frac=0.1)
        _check(out)
    finally:
        evo.tune_clear()
    assert evo.tune_entries() == []
