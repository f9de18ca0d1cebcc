"""The merged outer updates of the split-BF16 LU, checked on the CPU.

A numpy model of the right-looking blocked LU with LINPACK-order row
exchanges (rows left of a panel are never exchanged again) in two forms:
one trailing update per 256-column panel, and the merged form of
csrc/lu.cu (factor_pairs) that updates only the second panel's columns by
the first, corrects the second panel's block rows with the first panel's
multipliers of the rows they came from, and applies one update of depth 512
to the rows below the pair, with those multipliers gathered through the
second panel's exchanges.  In FP64 both forms give the same pivots and the
same factors up to rounding.  The bench's accounting of the outer updates
is checked to cover the same method flops in both forms."""
import importlib.util
import os

import numpy as np
import pytest

NB = 256


def _panel(S, c0, piv):
    """partial-pivoting LU of columns [c0, c0+NB), exchanges applied to those columns only"""
    for j in range(c0, c0 + NB):
        p = j + int(np.argmax(np.abs(S[j:, j])))
        piv[j] = p
        if p != j:
            S[[j, p], c0:c0 + NB] = S[[p, j], c0:c0 + NB]
        S[j + 1:, j] /= S[j, j]
        S[j + 1:, j + 1:c0 + NB] -= np.outer(S[j + 1:, j], S[j, j + 1:c0 + NB])


def _source(piv, c0, n):
    """src[r]: the old row that row r holds after the exchanges of panel c0"""
    idx = np.arange(n)
    for j in range(c0, c0 + NB):
        idx[[j, piv[j]]] = idx[[piv[j], j]]
    return idx


def _unit_lower(S, a, b):
    return np.tril(S[a:b, a:b], -1) + np.eye(b - a)


def one_panel(A):
    S, n = A.copy(), A.shape[0]
    piv = np.zeros(n, int)
    for c0 in range(0, n, NB):
        _panel(S, c0, piv)
        j0 = c0 + NB
        if j0 >= n:
            break
        S[:, j0:] = S[_source(piv, c0, n), j0:]
        S[c0:j0, j0:] = np.linalg.solve(_unit_lower(S, c0, j0), S[c0:j0, j0:])
        S[j0:, j0:] -= S[j0:, c0:j0] @ S[c0:j0, j0:]
    return S, piv


def merged_pairs(A):
    S, n = A.copy(), A.shape[0]
    piv = np.zeros(n, int)
    for ca in range(0, n, 2 * NB):
        cb, jr = ca + NB, ca + 2 * NB
        _panel(S, ca, piv)
        if cb >= n:
            break
        S[:, cb:] = S[_source(piv, ca, n), cb:]
        S[ca:cb, cb:] = np.linalg.solve(_unit_lower(S, ca, cb), S[ca:cb, cb:])
        Ua = S[ca:cb, cb:].copy()
        S[cb:, cb:jr] -= S[cb:, ca:cb] @ S[ca:cb, cb:jr]           # b's columns only
        _panel(S, cb, piv)
        if jr >= n:
            break
        src = _source(piv, cb, n)
        S[:, jr:] = S[src, jr:]                                   # b's exchanges on R
        S[cb:jr, jr:] -= S[src[cb:jr], ca:cb] @ Ua[:, NB:]        # block-row correction
        S[cb:jr, jr:] = np.linalg.solve(_unit_lower(S, cb, jr), S[cb:jr, jr:])
        La = S[src[jr:], ca:cb]                                   # a's multipliers, gathered
        S[jr:, jr:] -= np.hstack([La, S[jr:, cb:jr]]) @ np.vstack([Ua[:, NB:], S[cb:jr, jr:]])
    return S, piv


@pytest.mark.parametrize("n", [768, 1024, 1280])
def test_merged_pairs_equal_one_panel_factors(n):
    """3, 4 and 5 panels: a pair with a single panel after it, two pairs,
    two pairs and a single panel"""
    A = np.random.default_rng(n).standard_normal((n, n))
    S1, p1 = one_panel(A)
    S2, p2 = merged_pairs(A)
    assert (p1 == p2).all()
    assert np.abs(S1 - S2).max() < 1e-11 * np.abs(S1).max()
    # and the factors solve the system: the one-panel form's solve replays
    # each panel's exchanges before its block column (LINPACK order)
    b = np.random.default_rng(n + 1).standard_normal(n)
    y = b.copy()
    for c0 in range(0, n, NB):
        y[c0:] = y[_source(p2, c0, n)[c0:]]
        y[c0:c0 + NB] = np.linalg.solve(_unit_lower(S2, c0, c0 + NB), y[c0:c0 + NB])
        y[c0 + NB:] -= S2[c0 + NB:, c0:c0 + NB] @ y[c0:c0 + NB]
    x = np.linalg.solve(np.triu(S2), y)
    assert np.linalg.norm(A @ x - b) < 1e-10 * np.linalg.norm(b)


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("ld", [256, 768, 1792, 5120, 11008])
def test_outer_update_accounting_covers_the_same_flops(ld):
    """the merged form's updates carry the one-panel form's method flops
    (each trailing entry gets every outer panel's depth once), with fewer
    algorithmic bytes from four panels on (at three, the operand panels of
    the extra narrow updates outweigh the C traffic saved)"""
    B = _bench()
    one, pairs = B.outer_updates(ld, False), B.outer_updates(ld, True)
    fl = lambda ups: sum(2 * M * N * Kd for _, M, N, Kd in ups)
    assert fl(one) == fl(pairs)
    if ld >= 4 * NB:
        assert B.trailing_bytes(ld, 1, True) < B.trailing_bytes(ld, 1, False)
    assert {k for k, *_ in pairs} <= {"cols", "rows", "merged"}
