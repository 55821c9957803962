"""The library's symmetry table (§2.2), host only, against the oracle's coupling blocks.

The symmetry-compressed store keeps G_c for c = sorted |d| only and applies
G_d[U(u)][U(v)] = sign(u) sign(v) G_c[u][v] through a 48 x 192 table of the signed axis
permutations Q (d = Q c).  The oracle generates G_d and G_c independently (FP64 sums
over the dipole pairs), so a wrong site map, component map, sign or permutation index in
the library's table fails the block relation below.
"""
import itertools

import numpy as np
import pytest

import oracle
import paper_2501_04684_gb300 as ie
import workloads as W

PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _apply(q, c):
    """Q c for the index q = 8 p + s as ie.h defines it."""
    p, s = divmod(q, 8)
    return np.array([(-1) ** ((s >> i) & 1) * c[PERMS[p][i]] for i in range(3)])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2501_04684_gb300 import build
    return build.build()


@pytest.fixture(scope="module")
def table(built):
    return ie.ie_sym_map()


def test_canonical_displacement_and_index_reconstruct_d():
    for d in itertools.product(range(-4, 5), repeat=3):
        d = np.array(d)
        c, q = ie.ie_sym_canon(d)
        assert list(c) == sorted(np.abs(d)) and 0 <= q < 48
        assert np.array_equal(_apply(q, c), d), (d, c, q)


def test_every_map_row_is_a_signed_permutation_of_the_unknowns(table):
    U = table & 0xFF
    assert np.all(table >> 9 == 0)
    for q in range(48):
        assert sorted(U[q]) == list(range(192)), q
    assert np.array_equal(U[0], np.arange(192)) and np.all(table[0] < 0x100)   # q = 0 is the identity


def test_map_relates_the_oracle_blocks_for_all_48_permutations(table):
    """c with three distinct nonzero components: its 48 images d are distinct, the library
    returns the q that made each, and G_d = S_q G_c S_q^T with S_q[U(u), u] = sign(u)."""
    p = W.tiny()
    c = np.array([1, 2, 3])
    Gc = oracle.coupling_block(p, c)
    tol = 1e-12 * np.abs(Gc).max()
    for q in range(48):
        d = _apply(q, c)
        c2, q2 = ie.ie_sym_canon(d)
        assert list(c2) == [1, 2, 3] and q2 == q
        S = np.zeros((192, 192))
        S[table[q] & 0xFF, np.arange(192)] = np.where(table[q] & 0x100, -1.0, 1.0)
        assert np.abs(oracle.coupling_block(p, d) - S @ Gc @ S.T).max() <= tol, q


@pytest.mark.parametrize("d", [(0, 0, 2), (2, -2, 0), (-2, -2, -2), (0, -3, 3), (3, -1, 3), (-4, 2, 2)])
def test_map_relates_the_oracle_blocks_with_equal_or_zero_components(d, table):
    """With ties or zeros several Q give the same d; the one returned must still map G_c."""
    p = W.tiny()
    c, q = ie.ie_sym_canon(d)
    Gc = oracle.coupling_block(p, c)
    S = np.zeros((192, 192))
    S[table[q] & 0xFF, np.arange(192)] = np.where(table[q] & 0x100, -1.0, 1.0)
    assert np.abs(oracle.coupling_block(p, np.array(d)) - S @ Gc @ S.T).max() <= 1e-12 * np.abs(Gc).max()
