"""The autotuner's candidate set (host only): the paper's fusion with fused
block widths k_max = 2..5 and the Pauli-gadget rotations, at the three largest
tile sizes; one block per state (tile = n) for states that fit one block."""
from paper_2310_17739_gb300 import autotune


def test_candidates_cover_block_widths_and_tiles():
    c = autotune.candidates(21, "c64")
    assert {x["k_max"] for x in c if x["fusion"] == 1} == {2, 3, 4, 5}
    assert {x["tile_bits"] for x in c} == {12, 13, 14}
    assert any(x["fusion"] == 2 for x in c) and any(x.get("threads") == 512 for x in c)
    assert any(x["fusion"] == 1 and x.get("threads") == 512 for x in c)
    assert {x["tile_bits"] for x in autotune.candidates(21, "c128")} == {11, 12, 13}
    assert not any(x.get("threads") for x in autotune.candidates(21, "c128"))
    small = autotune.candidates(12, "c64")
    assert {x["tile_bits"] for x in small} == {12}
    assert {x["k_max"] for x in small if x["fusion"] == 1} == {2, 3, 4, 5}
    assert autotune.candidates(12, "c64", allow_rotations=False) == [x for x in small if x["fusion"] == 1]
