"""Host logic of the GEMM tile table (no GPU): file load, save and rejection."""
import pytest

from paper_2207_05477_gb300 import evo

HEADER = "# libevo GEMM tile table v1\n"
# key: M N K batch a_mn b_mn splits flags plain s_m0 ndiv mdiv; then the
# built-in (bn, splits) and the chosen (bn, splits)
PLAIN = "32768 512 128 1 0 0 1 0 1 512 2147483648 2147483648 256 1 128 1\n"
ATOMIC = "128 256 32768 1 1 1 4 6 1 256 2147483648 2147483648 256 4 128 8\n"


@pytest.fixture(autouse=True)
def _clean_table(built_lib):
    evo.tune_clear()
    yield
    evo.tune_clear()


def test_load_save_round_trip(tmp_path):
    f = tmp_path / "tiles.txt"
    f.write_text(HEADER + PLAIN + ATOMIC)
    evo.tune_load(f)
    ents = sorted(evo.tune_entries(), key=lambda e: e["M"])
    assert [(e["M"], e["N"], e["K"], e["batch"]) for e in ents] == [(128, 256, 32768, 1), (32768, 512, 128, 1)]
    assert (ents[0]["default_bn"], ents[0]["default_splits"], ents[0]["bn"], ents[0]["splits"]) == (256, 4, 128, 8)
    assert (ents[1]["default_bn"], ents[1]["bn"], ents[1]["splits"]) == (256, 128, 1)
    g = tmp_path / "again.txt"
    evo.tune_save(g)
    evo.tune_clear()
    assert evo.tune_entries() == []
    evo.tune_load(g)
    assert sorted(evo.tune_entries(), key=lambda e: e["M"]) == ents


@pytest.mark.parametrize("bad", [
    "32768 512 128 1 0 0 1 0 1 512 2147483648 2147483648 256 1 96 1\n",   # tile width not 64/128/256
    "32768 512 128 1 0 0 1 0 1 512 2147483648 2147483648 256 1 128 2\n",  # split of a non-atomic product
    "32768 512 128 1 0 0 1 0 1 512 2147483648 2147483648 256 1 128\n",    # a field short
    "32768 512 128 1 0 0 1 0 1 512 2147483648 2147483648 256 1 128 0\n",  # zero splits
])
def test_malformed_file_rejected_and_table_kept(tmp_path, bad):
    good = tmp_path / "good.txt"
    good.write_text(HEADER + PLAIN)
    evo.tune_load(good)
    before = evo.tune_entries()
    f = tmp_path / "bad.txt"
    f.write_text(HEADER + ATOMIC + bad)
    with pytest.raises(evo.EvoError):
        evo.tune_load(f)
    assert evo.tune_entries() == before


def test_missing_file_rejected(tmp_path):
    with pytest.raises(evo.EvoError):
        evo.tune_load(tmp_path / "absent.txt")
