"""Stored expected values (tests/golden/): the published SplitMix64 outputs and
regression values written by tests/golden/make_oracle_golden.py (oracle only)."""
import json
import os

import numpy as np
import pytest

import gen

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_splitmix64_published_outputs():
    ref = [int(l, 16) for l in open(os.path.join(HERE, "splitmix64_seed0.txt"))
           if l.strip() and not l.startswith("#")]
    got = [int(v) for v in gen.splitmix64(0, len(ref))]
    assert got == ref


def test_oracle_reproduces_stored_values():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "make_oracle_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored = json.load(open(os.path.join(HERE, "oracle_small_problems.json")))
    now = mk.values()
    assert stored.keys() == now.keys()
    for k in stored:
        for q, v in stored[k].items():
            if isinstance(v, int):
                assert now[k][q] == v, (k, q)
            else:
                assert now[k][q] == pytest.approx(v, rel=1e-9), (k, q)
