"""The executors' phase table (internal.h) against the data flow of the elastic loop chain.

Within a phase one thread takes a cell through all of the phase's loops, so no loop of a phase may
read a neighbour's value of a field that any loop of the same phase writes (that neighbour's thread
may not have written it yet, or may overwrite it meanwhile).  The table must obey this and be the
coarsest such split: merging any two adjacent phases would break it, and no legal split has fewer."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the chain of one time step (velocity sub-chain 0-8, stress sub-chain 9-16): fields read at the
# cell itself, fields read at the neighbours across the loop's faces, fields written at the cell
R, N, W = "own", "nbr", "write"
CHAIN = [
    {R: {"S"}, N: set(), W: {"U1"}},                 # 0 volume part of A(sigma)
    {R: {"S", "U1"}, N: {"S"}, W: {"U1"}},           # 1 interior faces of A(sigma)
    {R: {"S", "U1"}, N: set(), W: {"U1"}},           # 2 free-surface faces of A(sigma)
    {R: {"U1"}, N: set(), W: {"E"}},                 # 3 volume part of E(U1)
    {R: {"U1", "E"}, N: {"U1"}, W: {"E"}},           # 4 interior faces of E(U1)
    {R: {"E"}, N: set(), W: {"S1", "U2"}},           # 5 Hooke, volume part of A(S1)
    {R: {"S1", "U2"}, N: {"S1"}, W: {"U2"}},         # 6 interior faces of A(S1)
    {R: {"S1", "U2"}, N: set(), W: {"U2"}},          # 7 free-surface faces of A(S1)
    {R: {"U1", "U2", "V"}, N: set(), W: {"V"}},      # 8 velocity update
    {R: {"V"}, N: set(), W: {"E"}},                  # 9 volume part of E(v)
    {R: {"V", "E"}, N: {"V"}, W: {"E"}},             # 10 interior faces of E(v)
    {R: {"E"}, N: set(), W: {"S1", "U1"}},           # 11 Hooke, volume part of A(S1)
    {R: {"S1", "U1"}, N: {"S1"}, W: {"U1"}},         # 12 interior faces of A(S1)
    {R: {"S1", "U1"}, N: set(), W: {"U1"}},          # 13 free-surface faces of A(S1)
    {R: {"U1"}, N: set(), W: {"E"}},                 # 14 volume part of E(U1)
    {R: {"U1", "E"}, N: {"U1"}, W: {"E"}},           # 15 interior faces of E(U1)
    {R: {"E", "S1", "S"}, N: set(), W: {"S"}},       # 16 stress update and source
]


def legal(first, last):
    written = set().union(*(CHAIN[j][W] for j in range(first, last)))
    return all(not (CHAIN[j][N] & written) for j in range(first, last))


def phase_starts():
    with open(os.path.join(ROOT, "paper_1708_03183_gb300", "csrc", "internal.h")) as f:
        src = f.read()
    body = re.search(r"constexpr int phase_first\(int h\)\s*\{(.*?)\}", src, re.S).group(1)
    pairs = [(int(h), int(v)) for h, v in re.findall(r"h == (\d+) \? (\d+)", body)]
    tail = int(re.search(r":\s*(\d+);", body).group(1))
    starts = [v for _, v in sorted(pairs)] + [tail]
    nphases = int(re.search(r"constexpr int kPhases = (\d+);", src).group(1))
    assert [h for h, _ in sorted(pairs)] == list(range(len(pairs)))
    assert len(starts) == nphases + 1
    return starts


def test_the_phase_table_covers_the_chain_in_order():
    starts = phase_starts()
    assert starts[0] == 0 and starts[-1] == 17 and all(a < b for a, b in zip(starts, starts[1:]))


def test_no_phase_reads_a_neighbour_value_it_writes():
    starts = phase_starts()
    for a, b in zip(starts, starts[1:]):
        assert legal(a, b), (a, b)


def test_the_phases_are_the_coarsest_legal_split():
    starts = phase_starts()
    for a, b, c in zip(starts, starts[1:], starts[2:]):
        assert not legal(a, c), (a, b, c)
    # as few phases as any legal split: greedy (each phase as long as it stays legal) is optimal for
    # a property that holds for every part of a legal run.  The table ends its phases after each
    # operator's faces instead, so that an operator's volume part and faces share a pass.
    greedy, a = 0, 0
    while a < 17:
        b = a + 1
        while b < 17 and legal(a, b + 1):
            b += 1
        greedy, a = greedy + 1, b
    assert len(starts) - 1 == greedy


@pytest.mark.parametrize("split", [(9,), (3, 9, 12), (1, 5, 9, 13)])
def test_segments_of_any_split_are_legal(split):
    # a tiled executor runs the part of each phase inside a sub-chain; a part of a legal phase is legal
    starts = phase_starts()
    bounds = sorted(set(starts) | set(split))
    for a, b in zip(bounds, bounds[1:]):
        assert legal(a, b)
