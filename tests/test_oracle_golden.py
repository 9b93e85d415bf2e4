"""The oracle reproduces its committed reference values (tests/golden/tiny_oracle.json)."""
import json
import os

import pytest

from tests.golden.make_golden import compute


def test_oracle_matches_golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_oracle.json")) as f:
        ref = json.load(f)
    got = compute()
    for key in ("mu", "zeta", "chi0_trace", "chi0_fro", "w_trace", "w_fro"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15)
    for group in ("chi0_entries", "w_entries"):
        for k, v in ref[group].items():
            assert got[group][k] == pytest.approx(v, rel=1e-11, abs=1e-15)
