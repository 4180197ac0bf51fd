"""The fixtures under tests/golden/ against the oracle (CPU only).

paper_facts.txt holds the numbers the paper states about its generators
(Sec. 4.1 and 4.2); each is checked here against what the oracle computes,
with the matrix powers redone in Python integers (not the oracle's code).
oracle_fixtures.json holds first draws written by
tests/golden/make_oracle_fixtures.py from the oracle alone; the oracle must
still reproduce them (a regression guard, not an independent pin)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _facts():
    facts = {}
    with open(os.path.join(GOLDEN, "paper_facts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, *where = line.split()
            assert where and where[0] == "Sec.", line  # every fact names its section
            facts[name] = int(value)
    return facts


FACTS = _facts()

# MRG32k3a component matrices for the state (x[n-3], x[n-2], x[n-1]), L'Ecuyer 1999
_A = {1: ([[0, 1, 0], [0, 0, 1], [-810728, 1403580, 0]], O.M1),
      2: ([[0, 1, 0], [0, 0, 1], [-1370589, 0, 527612]], O.M2)}


def _matmul(a, b, m):
    return [[sum(a[i][k] * b[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]


def _matpow(comp, e):
    a, m = _A[comp]
    r = [[int(i == j) for j in range(3)] for i in range(3)]
    b = [[x % m for x in row] for row in a]
    while e:
        if e & 1:
            r = _matmul(r, b, m)
        b = _matmul(b, b, m)
        e >>= 1
    return r


def _jump(state, e):
    out = []
    for comp, part in ((1, state[:3]), (2, state[3:])):
        p = _matpow(comp, e)
        m = _A[comp][1]
        out += [sum(p[i][k] * int(part[k]) for k in range(3)) % m for i in range(3)]
    return out


def test_every_fact_is_checked():
    assert set(FACTS) == {"mrg32k3a_state_words", "mrg32k3a_log2_period", "mrg32k3a_log2_streams",
                          "mrg32k3a_log2_stream_length", "mrg32k3a_log2_substream_length",
                          "tinymt32_log2_period", "tinymt32_log2_statuses"}


def test_mrg_state_is_six_words():
    assert O.seed_expand(1).shape == (FACTS["mrg32k3a_state_words"],)
    assert O.mrg_stream_starts([12345] * 6, 127, 0, 3).shape == (3, FACTS["mrg32k3a_state_words"])


def test_mrg_period():
    """The combined period lcm(m1^3 - 1, m2^3 - 1) is about 2^191, and the
    oracle's matrices have orders dividing m^3 - 1 (their exact order is
    pinned in test_oracle_pins.py)."""
    period = math.lcm(O.M1 ** 3 - 1, O.M2 ** 3 - 1)
    assert round(math.log2(period)) == FACTS["mrg32k3a_log2_period"]
    for comp, m in ((0, O.M1), (1, O.M2)):  # the oracle numbers its components 0 and 1
        assert np.array_equal(O.mrg_matpow(comp, m ** 3 - 1), np.eye(3, dtype=np.uint64))
        assert O.mrg_matrix(comp).tolist() == [[x % m for x in row] for row in _A[comp + 1][0]]


def test_mrg_streams_tile_the_period():
    assert FACTS["mrg32k3a_log2_streams"] + FACTS["mrg32k3a_log2_stream_length"] == FACTS["mrg32k3a_log2_period"]
    seed = [int(x) for x in O.seed_expand(0x5EED5EED5EED5EED)]
    e = FACTS["mrg32k3a_log2_stream_length"]
    last = (1 << FACTS["mrg32k3a_log2_streams"]) - 1
    assert O.mrg_stream_starts(seed, e, last, 1)[0].tolist() == _jump(seed, last << e)


@pytest.mark.parametrize("key", ["mrg32k3a_log2_stream_length", "mrg32k3a_log2_substream_length"])
def test_mrg_stream_and_substream_spacing(key):
    e = FACTS[key]
    seed = [12345] * 6
    starts = O.mrg_stream_starts(seed, e, 0, 3)
    for i in range(3):
        assert starts[i].tolist() == _jump(seed, i << e)


def test_substreams_divide_a_stream():
    seed = [12345] * 6
    es, ess = FACTS["mrg32k3a_log2_stream_length"], FACTS["mrg32k3a_log2_substream_length"]
    assert np.array_equal(O.mrg_stream_starts(seed, ess, 1 << (es - ess), 1), O.mrg_stream_starts(seed, es, 1, 1))


def test_tinymt_period():
    mat1, mat2, tmat = (int(x) for x in O.tinymt32_find_params(0x5EED, 1)[0])
    s = O.tinymt32_init(1234, [mat1, mat2, tmat])
    e = FACTS["tinymt32_log2_period"]
    assert np.array_equal(O.tinymt32_jump(s, mat1, mat2, (1 << e) - 1), s)
    assert not np.array_equal(O.tinymt32_jump(s, mat1, mat2, 1 << (e - 1)), s)


def test_tinymt_parameter_space_holds_the_stated_statuses():
    """(mat1, mat2) range over 2^64 pairs; the fraction with period 2^127 - 1,
    estimated from seeded candidates, times 2^64 exceeds the 2^48 statuses the
    paper counts."""
    rng = np.random.default_rng(7)
    cand = rng.integers(0, 1 << 32, size=(1024, 2), dtype=np.uint64)
    good = sum(O.tinymt32_max_period(int(a), int(b)) for a, b in cand)
    assert good > 0
    assert 64 + math.log2(good / len(cand)) > FACTS["tinymt32_log2_statuses"]


def _fixtures():
    with open(os.path.join(GOLDEN, "oracle_fixtures.json")) as f:
        return json.load(f)


def test_oracle_reproduces_its_fixtures():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_fixtures",
                                                  os.path.join(GOLDEN, "make_oracle_fixtures.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert mod.cases() == _fixtures()["cases"]
