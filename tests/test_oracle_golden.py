"""The oracle against its stored regression values (tests/golden/).

The stored values were written by ``tests/golden/make_golden.py``, which calls
only the oracle and the seeded input generators.  They are not a pin of the
oracle (the pins are the closed forms, brute force and finite differences of
the other ``test_oracle_*`` files): they freeze the pinned oracle, so that a
change to its arithmetic cannot pass unnoticed.  Integers and digests of the
discrete results (keys, values, ranges, n_contrib, insertion and merging
decisions, scheduler draws) must match exactly; floating-point values to
1e-9 relative, the room left for the summation order of the oracle's
parallel gradient partials.
"""
import importlib.util
import math
import os

import pytest

pytestmark = pytest.mark.usefixtures("oracle_lib")

_HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(_HERE, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def values():
    g = _golden()
    return g.read(), g.compute()


def test_inputs_unchanged(values):
    stored, now = values
    for k in stored:
        if k.endswith("inputs_sha256"):
            assert now[k] == stored[k], f"{k}: the seeded generator changed, not the oracle"


def test_same_keys(values):
    stored, now = values
    assert sorted(stored) == sorted(now)


@pytest.mark.parametrize("section", ["small_box", "multi_view", "insertion", "merging", "frequency"])
def test_section_matches(values, section):
    stored, now = values
    keys = [k for k in stored if k.split(".", 1)[0] == section]
    assert keys
    bad = []
    for k in keys:
        s, v = stored[k], now[k]
        if isinstance(v, float):
            ref = float(s)
            if not math.isclose(v, ref, rel_tol=1e-9, abs_tol=1e-15):
                bad.append(f"{k}: stored {s}, now {v!r}")
        elif str(v) != s:
            bad.append(f"{k}: stored {s}, now {v}")
    assert not bad, "\n".join(bad)
