"""Host-side entry points that need no GPU: the autotuner's shapes as text
(tmotif_tuner_export / tmotif_tuner_import) and the checked build's
forced-timeout switch, which the normal build refuses."""
import pytest

tm = pytest.importorskip("paper_2001_07158_gb300")


def lines(text):
    return sorted(l for l in text.splitlines() if l.strip())


def test_round_trip_and_replacement():
    tm.tmotif_tuner_import("7 64 21 64 0\n7 128 25 256 4\n\n7 32 24 1024 3\n")
    got = lines(tm.tmotif_tuner_export())
    for want in ("7 64 21 64 0", "7 128 25 256 4", "7 32 24 1024 3"):
        assert want in got
    # a second import of the same key replaces the shape
    tm.tmotif_tuner_import("7 64 21 512 2\n")
    got = lines(tm.tmotif_tuner_export())
    assert "7 64 21 512 2" in got and "7 64 21 64 0" not in got
    # exporting and importing again changes nothing
    before = tm.tmotif_tuner_export()
    tm.tmotif_tuner_import(before)
    assert tm.tmotif_tuner_export() == before


@pytest.mark.parametrize("bad", ["8 64 21 100 0", "8 48 21 64 0", "8 32 21 64 1", "8 16 21 64 4", "x",
                                 "8 64 21 64 0 9", "-1 64 21 64 0", "8 64 64 64 0", "300 64 21 64 0"])
def test_malformed_lines_are_refused_and_add_nothing(bad):
    before = tm.tmotif_tuner_export()
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_tuner_import("8 64 20 128 1\n" + bad + "\n")
    assert e.value.code == 1
    assert tm.tmotif_tuner_export() == before


def test_forced_timeout_switch_is_checked_build_only():
    if tm.tmotif_checked_build():
        pytest.skip("the checked build accepts the switch")
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_debug_stage_timeout(True)
    assert e.value.code == 5
