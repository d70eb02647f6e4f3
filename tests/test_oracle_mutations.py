"""Planted mistakes in the oracle's climb must fail its pins.

Each case edits one line of a copy of the oracle's C source (the copy is
compiled into a temporary directory; the oracle itself is untouched), loads
the copy in place of the oracle and runs the exact climb pins of
test_oracle_climb.py against it: the corner cap dropped from either climb,
the offset |s_a - s_A| of Eq. rmax_2 added twice, and the moonlets' spread
taken about the wrong centre.
"""
import pytest

import test_oracle_climb as climb
from paper_2310_20374_gb300 import diskgen

MUTATIONS = {
    "gravity corner cap dropped": ("if (cap < x->rmax) x->rmax = cap;", ";"),
    "collision corner cap dropped": ("if (cap < x->rmax_c) x->rmax_c = cap;", ";"),
    "offset added twice (gravity)": ("double r = y->rmax + norm3(d);", "double r = y->rmax + 2.0 * norm3(d);"),
    "offset added twice (collisions)": ("double r = y->rmax_c + norm3(d);",
                                        "double r = y->rmax_c + 2.0 * norm3(d);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_climb_mistake_fails_the_pins(oracle_lib, tmp_path, name):
    old, new = MUTATIONS[name]
    src = oracle_lib.source()
    assert src.count(old) == 1, f"mutation target not found once: {old}"
    path = oracle_lib.build_variant(src.replace(old, new), str(tmp_path))
    cases = [(climb.crafted_cell(), 2, 0.5), (diskgen.make_disk(2500, 22), 4, 0.6),
             (diskgen.make_disk(3000, 21), 16, 0.5)]
    with oracle_lib.use_library(path):
        failed = 0
        for d, leaf, theta in cases:
            try:
                climb.check_geometry(oracle_lib, d, leaf, theta, 1e-3)
            except AssertionError:
                failed += 1
    assert failed > 0, f"planted mistake '{name}' passed every climb pin"
