"""Failure detection without a GPU fault: a bounded in-kernel wait that nothing
satisfies gives up, records EVO_ERR_TIMEOUT in the device error word, and the
context stays usable for the next launch."""
import pytest
import torch

from helpers import gpu_run
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("unit", [evo.EVO_UNIT_GEMM, evo.EVO_UNIT_ATTENTION, evo.EVO_UNIT_TRIMUL, evo.EVO_UNIT_MLP])
def test_bounded_wait_reports_timeout_and_context_survives(built_lib, unit):
    """Each unit's own bounded wait (GEMM, attention, triangle multiplication)
    runs out, its error word reports the timeout, and a block runs afterwards."""
    torch.cuda.init()
    assert evo.get_error() == evo.EVO_OK
    evo.debug_wait_timeout(200_000_000, unit)  # 0.2 s
    assert evo.get_error() == evo.EVO_ERR_TIMEOUT
    assert evo.get_error() == evo.EVO_OK  # reading clears the word
    out = gpu_run(synth.Dims(n_seq=2, n_res=16), evo.EVO_BF16, backward=False)
    assert torch.isfinite(out["m"]).all() and torch.isfinite(out["z"]).all()


def test_debug_wait_rejects_unknown_unit(built_lib):
    with pytest.raises(evo.EvoError) as e:
        evo.debug_wait_timeout(1000, 7)
    assert e.value.code == evo.EVO_ERR_INVALID_ARG


def test_workspace_too_small_is_an_error_not_a_fault(built_lib):
    d = synth.Dims(n_seq=2, n_res=16)
    cd = evo.cdims(d, evo.EVO_F32)
    dev = torch.device("cuda:0")
    params = torch.zeros(evo.param_count(cd), device=dev)
    m = torch.zeros(2, 16, 256, device=dev)
    z = torch.zeros(16, 16, 128, device=dev)
    mm = torch.ones(2, 16, device=dev)
    pm = torch.ones(16, 16, device=dev)
    ws = torch.empty(1024, dtype=torch.uint8, device=dev)
    with pytest.raises(evo.EvoError) as e:
        evo.block_fwd(cd, params, None, m, z, m, z, mm, pm, ws)
    assert e.value.code == evo.EVO_ERR_WORKSPACE
