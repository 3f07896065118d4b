"""Host logic of the probe-window autotuner (paper_1601_04017_gb300/tune.py) and
the rule it generated (csrc/cht_tuned.inc).  No GPU: the selection functions
are pure, and the rule file is checked for the shape the runtime's lookup
assumes -- every (operation, size, load) covered exactly once by a window the
kernels have.
"""
import os
import re

import pytest

from paper_1601_04017_gb300 import tune

INC = os.path.join(os.path.dirname(tune.__file__), "csrc", "cht_tuned.inc")
LINE = re.compile(r"^\{cht::(k\w+), (\d+), (\d+), ([\d.]+)f, ([\d.]+)f, (-?\d+), (\d+), (\d+)\},  // [\d.]+ ms for \d+ ops$")
# windows the operation kernels exist for (group width, cells per lane)
KERNEL_WINDOWS = {(-1, 2), (-1, 4), (1, 2), (1, 4), (2, 1), (2, 2), (2, 4), (4, 1), (4, 2), (4, 4),
                  (8, 1), (8, 2), (8, 4), (16, 1), (16, 2), (32, 1)}


def test_rank_by_sum():
    a = {(1, 2, 0): 1.0, (2, 4, 0): 2.0, (4, 4, 4): 0.5}
    b = {(1, 2, 0): 3.0, (2, 4, 0): 1.0, (4, 4, 4): 4.0}
    assert tune.rank_by_sum(a, b) == [(2, 4, 0, 3.0), (1, 2, 0, 4.0), (4, 4, 4, 4.5)]
    # a window timed on one batch only is not ranked
    assert tune.rank_by_sum(a, {(1, 2, 0): 1.0}) == [(1, 2, 0, 2.0)]


def test_choose_keeps_the_builtin_window_within_the_margin():
    res = [(-1, 4, 0, 0.98), (2, 4, 0, 1.00)]
    assert tune.choose(res, (2, 4, 0), margin=0.03) == (2, 4, 0, 1.00)  # 2 % faster: noise
    res = [(-1, 4, 0, 0.90), (2, 4, 0, 1.00)]
    assert tune.choose(res, (2, 4, 0), margin=0.03) == (-1, 4, 0, 0.90)  # 10 % faster
    res = [(2, 4, 0, 1.00), (1, 2, 0, 1.20)]
    assert tune.choose(res, (2, 4, 0)) == (2, 4, 0, 1.00)  # the built-in one is the fastest


def test_builtin_window():
    assert tune.builtin_window(0, 0.5) == (2, 4, 0)
    assert tune.builtin_window(1, 0.5) == (1, 2, 0)
    assert tune.builtin_window(0, 0.9) == (4, 4, 0)
    assert tune.builtin_window(1, 0.9) == (4, 4, 0)
    assert tune.builtin_window(4, 0.9) == (4, 2, 0)


def test_rule_line_round_trips():
    line = tune.rule_line("cht::kFind", 0, 22, 0.0, 0.375, -1, 2, 0, 0.0123, 524288)
    m = LINE.match(line.rstrip("\n"))
    assert m and m.group(1) == "kFind" and m.group(6) == "-1"


def _rules():
    rows = []
    with open(INC) as f:
        for ln in f:
            if ln.startswith("//") or not ln.strip():
                continue
            m = LINE.match(ln.rstrip("\n"))
            assert m, ln
            op, lo, hi, blo, bhi, g, v, ct = m.groups()
            rows.append((op, int(lo), int(hi), float(blo), float(bhi), int(g), int(v), int(ct)))
    return rows


def test_generated_rule_covers_every_size_and_load_once():
    rows = _rules()
    ops = {r[0] for r in rows}
    assert ops == {"kFind", "kInsert", "kErase", "kUpdAdd"}
    sizes = sorted({(r[1], r[2]) for r in rows})
    assert sizes[0][0] == 0 and sizes[-1][1] == 40
    for (lo_a, hi_a), (lo_b, hi_b) in zip(sizes, sizes[1:]):
        assert lo_b == hi_a + 1  # contiguous, no overlap
    bands = sorted({(r[3], r[4]) for r in rows})
    assert bands[0][0] == 0.0 and bands[-1][1] > 1.0
    for (a0, a1), (b0, b1) in zip(bands, bands[1:]):
        assert b0 == pytest.approx(a1)
    assert len(rows) == len(ops) * len(sizes) * len(bands)
    assert len({r[:5] for r in rows}) == len(rows)


def test_generated_rule_names_existing_windows():
    for op, lo, hi, blo, bhi, g, v, ct in _rules():
        assert (g, v) in KERNEL_WINDOWS, (op, lo, blo, g, v)
        assert ct in (0, 4)
