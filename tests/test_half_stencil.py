"""Host checks of the half-stencil list build's rules (paper Sec. II.C: the
3^d linked subcells of a home subcell), replayed on the CPU.

The device builder (`nbr_cell<D, true>` in csrc/dev_nbr.cuh) walks, for each home
subcell, the stencil rows (offsets on axes 0..d-2) whose first non-zero
offset is positive, all three pieces along the last axis; of the row of zero
offsets only the pieces at last-axis offset 0 (pairs i < j) and +1.  Each
pair it finds goes into both lists, the candidate's entry with the opposite
offset code, written as (0b10 in every 2-bit field) - code.  These tests
check that the rule visits every unordered pair of atoms in neighbouring
subcells exactly once, and the code negation for every code.
"""
import itertools

import numpy as np
import pytest


def visits(off):
    """True where the half-stencil rule takes subcell offset `off` (tuple of
    d offsets in {-1, 0, 1}; the last entry is the last axis)."""
    head, last = off[:-1], off[-1]
    sgn = next((o for o in head if o != 0), 0)
    if sgn > 0:
        return True
    if sgn < 0:
        return False
    return last >= 0          # zero row: last-axis pieces 0 (i < j) and +1


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_each_offset_or_its_mirror_exactly_once(d):
    for off in itertools.product((-1, 0, 1), repeat=d):
        mirror = tuple(-o for o in off)
        if all(o == 0 for o in off):
            assert visits(off)   # the home piece itself (pairs i < j)
            continue
        assert visits(off) != visits(mirror), off


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3), (3, 4), (4, 3), (6, 3)])
def test_every_pair_of_atoms_found_once(d, n):
    """Atoms on a periodic n^d subcell grid (n >= 3, one to three atoms per
    subcell): every unordered pair of atoms in the same or neighbouring
    subcells is found exactly once by the rule, from the home subcell of one
    of its two atoms."""
    rng = np.random.default_rng(d * 10 + n)
    cells = list(itertools.product(range(n), repeat=d))
    atoms = []   # (atom index, subcell)
    for c in cells:
        for _ in range(int(rng.integers(1, 4))):
            atoms.append((len(atoms), c))
    by_cell = {}
    for i, c in atoms:
        by_cell.setdefault(c, []).append(i)
    found = {}
    for c in cells:
        for off in itertools.product((-1, 0, 1), repeat=d):
            if not visits(off):
                continue
            c2 = tuple((ck + ok) % n for ck, ok in zip(c, off))
            same = all(o == 0 for o in off)
            for i in by_cell[c]:
                for j in by_cell[c2]:
                    if same and not i < j:
                        continue
                    key = (min(i, j), max(i, j))
                    found[key] = found.get(key, 0) + 1
    want = set()
    for i, c in atoms:
        for j, c2 in atoms:
            if i < j and all(((a - b) % n) in (0, 1, n - 1) for a, b in zip(c, c2)):
                want.add((i, j))
    assert set(found) == want
    assert all(v == 1 for v in found.values())


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
def test_opposite_offset_code(d):
    """(0b10 in each of the d 2-bit fields) - code is the code of -o for every
    offset vector o (field value o + 1); no field borrows from its neighbour."""
    mask = (1 << (2 * d)) - 1
    twos = 0xAAAAAAAA & mask
    for off in itertools.product((-1, 0, 1), repeat=d):
        code = sum((o + 1) << (2 * k) for k, o in enumerate(off))
        neg = sum((-o + 1) << (2 * k) for k, o in enumerate(off))
        assert twos - code == neg
