"""Pins for the canonical FP64 reduction order (CRO) that every FP64 sum of the path uses
(moments for the 6D metric's sigma_x, sigma_v; bulk velocity; FP64 potential; halo properties).
Checked against hand-derived order-sensitive sums, exact integer sums and the exactly rounded
sum (math.fsum) within the error bound of the CRO's summation depth."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _val(tok):
    if tok.startswith("2^53"):
        return float(2 ** 53 + (int(tok[4:]) if len(tok) > 4 else 0))
    return float(tok)


def _cases():
    for line in open(os.path.join(GOLDEN, "cro_order_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        m, terms, expect, _ = [p.strip() for p in line.split("|")]
        a = np.zeros(int(m))
        for t in terms.split():
            i, v = t.split(":")
            a[int(i)] = _val(v)
        yield a, _val(expect)


@pytest.mark.parametrize("a,expect", list(_cases()))
def test_golden_order_cases(a, expect):
    assert oracle.cro_sum(a) == expect


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 1023, 1024, 1025, 3000, 70001])
def test_error_bound_vs_exact(m):
    rng = np.random.default_rng(m)
    a = rng.normal(0, 1, m) * np.exp(rng.uniform(-20, 20, m))
    exact = math.fsum(a)
    depth = 32 + 5 + max(1, math.ceil(math.log2(max(1, (m + 1023) // 1024)))) + 1
    u = 2.0 ** -53
    bound = depth * u / (1 - depth * u) * np.abs(a).sum()
    assert abs(oracle.cro_sum(a) - exact) <= bound


def test_exact_integer_sums():
    rng = np.random.default_rng(5)
    a = rng.integers(-1000, 1000, 123457).astype(np.float64)
    assert oracle.cro_sum(a) == float(int(a.astype(np.int64).sum()))


def test_sum_of_ones_and_empty():
    assert oracle.cro_sum(np.ones(100000)) == 100000.0
    assert oracle.cro_sum(np.zeros(0)) == 0.0
