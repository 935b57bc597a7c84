"""Pins of the oracle against values the paper and the generator's authors print
(fixtures under tests/golden/, each with its citation in its header).

* Table 5 (posterior moments and numerical accuracy, Sec. 5.2): every SPS entry prints a
  posterior SD, an NSE and an RNE. For each entry the test builds J groups of N values whose
  pooled SD and RNE are the printed ones and runs them through the oracle's group moments
  (Eqs. 3-10). With the reading NSE = (v-hat / (J N))^(1/2) the oracle reproduces the printed NSE
  within the table's rounding for 48 of the 52 entries; the four others are printed
  inconsistently in the table itself (the Germany SPS/GPU columns, whose means are misprinted
  too, and two more SPS/GPU entries) and are listed here. The formula as typeset, (v-hat / J)^(1/2),
  matches none of the 52.
* Philox4x32-10: the published known-answer vectors.
"""
import math
import os

import numpy as np

from oracle.philox import philox4x32_10
from oracle.smc import group_moments

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# entries of Table 5 printed inconsistently with the table's own SD and RNE under either reading
INCONSISTENT = {("Germany", 1, "gpu", 10), ("Germany", 1, "gpu", 40), ("Cars", 1, "gpu", 10),
                ("Caesarean_2", 1, "gpu", 10)}


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def _groups_with(sd, rne, J, N):
    """J x N values (group-major) with pooled SD `sd` and RNE `rne`: group means +-a around 0 and
    offsets +-b within each group (J and N even), so that v-hat = N J a^2 / (J - 1) = sd^2 / rne
    and the pooled variance is a^2 + b^2 = sd^2."""
    a = sd * math.sqrt((J - 1) / (rne * J * N))
    b = math.sqrt(sd * sd - a * a)
    sj = np.where(np.arange(J) % 2 == 0, 1.0, -1.0)
    tn = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    return (sj[:, None] * a + tn[None, :] * b).reshape(-1)


def test_table5_nse_reading_against_the_printed_entries():
    rows = _rows("table5_moments.txt")
    assert len(rows) == 52
    consistent, typeset = set(), 0
    for name, k, impl, J, N, sd, nse, rne in rows:
        k, J, N, sd, nse, rne = int(k), int(J), int(N), float(sd), float(nse), float(rne)
        m = group_moments(_groups_with(sd, rne, J, N), J, N)
        # the construction reproduces the printed SD and RNE
        assert abs(m.sd[0] - sd) <= 1e-12 and abs(m.rne[0] - rne) <= 1e-9
        # rounding of the printed figures: NSE to 4 decimals, SD to 3, RNE to 2
        tol = 0.5e-4 + m.nse[0] * (0.5e-3 / sd + 0.5e-2 / (2 * rne))
        if abs(m.nse[0] - nse) <= tol:
            consistent.add((name, k, impl, J))
        if abs(math.sqrt(m.vhat[0] / J) - nse) <= tol:
            typeset += 1
    every = {(r[0], int(r[1]), r[2], int(r[3])) for r in rows}
    assert every - consistent == INCONSISTENT
    assert typeset == 0


def test_philox_known_answer_vectors():
    rows = _rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox4x32_10(v[0:4], v[4:6]) == v[6:10]
