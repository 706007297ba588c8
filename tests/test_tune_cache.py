"""The tuner's cache file (host code, no GPU): lines "device<TAB>kind<TAB>class<TAB>value"
are loaded, saved back unchanged, and a malformed file is rejected without adding anything."""
import pytest

from paper_2207_07488_gb300 import spnet

LINES = ["NVIDIA GB300 sm152 cc103\t0\t4,22,17,31\t8",
         "NVIDIA GB300 sm152 cc103\t1\t34,2,1,0\t2",
         "Other GPU sm100 cc100\t2\t288,23,18,1\t4"]


def test_cache_file_round_trip(tmp_path):
    spnet.tune_cache_clear()
    src = tmp_path / "in.tsv"
    src.write_text("\n".join(LINES) + "\n")
    spnet.tune_cache_load(str(src))
    out = tmp_path / "out.tsv"
    spnet.tune_cache_save(str(out))
    assert sorted(out.read_text().splitlines()) == sorted(LINES)
    assert spnet.tune_counts() == (0, 0)
    spnet.tune_cache_clear()
    spnet.tune_cache_save(str(out))
    assert out.read_text() == ""


@pytest.mark.parametrize("bad", ["dev\t0\t1,2,3\t4", "dev\t0\t1,2,3,4\t0", "dev\t9\t1,2,3,4\t4",
                                 "dev\t0\t1,2,3,4", "dev\tx\t1,2,3,4\t4", "dev\t0\t1,2,3,4\t4\textra"])
def test_malformed_lines_are_rejected(tmp_path, bad):
    spnet.tune_cache_clear()
    src = tmp_path / "bad.tsv"
    src.write_text(LINES[0] + "\n" + bad + "\n")
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.tune_cache_load(str(src))
    assert ei.value.code == spnet.ERR_BAD_INPUT and "line 2" in str(ei.value)
    out = tmp_path / "out.tsv"
    spnet.tune_cache_save(str(out))
    assert out.read_text() == ""  # nothing of the file was added
    with pytest.raises(spnet.SpnetError):
        spnet.tune_cache_load(str(tmp_path / "missing.tsv"))
