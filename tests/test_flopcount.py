"""The FLOP counts behind the roofline of the fused RHS kernel
(oracle/flop_counts.json) are those of the oracle as it stands: a fresh
instrumented count gives the committed numbers (no GPU)."""
import json
import os

from oracle import flopcount

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_committed_counts_match_a_fresh_count():
    stored = json.load(open(os.path.join(ROOT, 'oracle', 'flop_counts.json')))
    for d in (1, 2, 3):
        assert flopcount.count(d) == stored[str(d)], d


def test_counts_grow_with_the_dimension():
    # every extra dimension adds a tangential velocity to each face state and
    # a variable to each cell: more work per face and per cell
    c = {d: flopcount.count(d) for d in (1, 2, 3)}
    for key in ('face', 'cell', 'face_central'):
        assert c[1][key] < c[2][key] < c[3][key], key
    for d in (1, 2, 3):
        nv = d + 2
        assert c[d]['divergence'] == 3 * d * nv and c[d]['update'] == 5 * nv
        assert c[d]['cell'] == c[d]['primitives'] + c[d]['divergence'] + c[d]['update']
        assert c[d]['face_central'] < c[d]['face'] / 5           # no characteristic WENO, no Riemann solver
