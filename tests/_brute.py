"""Brute-force dynamic programming used to pin the oracle.

Everything here follows textbook definitions, independently of Algorithm 1:
Levenshtein distance by the classic O(nm) table, and the free-text-end
("semi-global") distance as the minimum of Levenshtein distances over text
prefixes.
"""
import numpy as np


def lev(a, b) -> int:
    """Classic Levenshtein distance (unit cost substitution/insertion/deletion)."""
    a, b = list(a), list(b)
    prev = list(range(len(b) + 1))
    for x in range(1, len(a) + 1):
        cur = [x] + [0] * len(b)
        for y in range(1, len(b) + 1):
            cur[y] = min(prev[y] + 1, cur[y - 1] + 1, prev[y - 1] + (a[x - 1] != b[y - 1]))
        prev = cur
    return prev[-1]


def suffix_lev_table(a, b) -> np.ndarray:
    """D[x][y] = lev(a[x:], b[y:]) for all suffix pairs."""
    n, m = len(a), len(b)
    D = np.zeros((n + 1, m + 1), dtype=np.int64)
    D[n, :] = m - np.arange(m + 1)
    D[:, m] = n - np.arange(n + 1)
    for x in range(n - 1, -1, -1):
        for y in range(m - 1, -1, -1):
            D[x, y] = min(D[x + 1, y] + 1, D[x, y + 1] + 1, D[x + 1, y + 1] + (a[x] != b[y]))
    return D


def free_end_table_literal(text, pattern) -> np.ndarray:
    """dist[i][j] = min over t of lev(text[i:i+t], pattern[j:]) -- the definition, literally."""
    n, m = len(text), len(pattern)
    out = np.full((n + 1, m + 1), 1 << 30, dtype=np.int64)
    for i in range(n + 1):
        for t in range(0, n - i + 1):
            D = suffix_lev_table(text[i:i + t], pattern)
            out[i, :] = np.minimum(out[i, :], D[0, :])
    return out


def free_end_table(text, pattern) -> np.ndarray:
    """Same table by the O(nm) recurrence with a free text end (E[i][m] = 0)."""
    n, m = len(text), len(pattern)
    E = np.zeros((n + 1, m + 1), dtype=np.int64)
    E[n, :] = m - np.arange(m + 1)
    E[:, m] = 0
    for i in range(n - 1, -1, -1):
        for j in range(m - 1, -1, -1):
            E[i, j] = min(E[i + 1, j + 1] + (text[i] != pattern[j]), E[i, j + 1] + 1, E[i + 1, j] + 1)
    return E


def free_end_distance(text, pattern) -> int:
    """Semi-global distance of a whole pair: pattern fully, text prefix free."""
    n, m = len(text), len(pattern)
    prev = np.arange(m + 1, dtype=np.int64)  # row for text prefix of length 0 vs pattern prefixes
    best = prev[m]
    t = np.asarray(text)
    p = np.asarray(pattern)
    for x in range(1, n + 1):
        cur = np.empty(m + 1, dtype=np.int64)
        cur[0] = x
        sub = prev[:-1] + (p != t[x - 1])
        dele = prev[1:] + 1
        best_row = np.minimum(sub, dele)
        # insertion chain along the row
        for y in range(1, m + 1):
            cur[y] = min(best_row[y - 1], cur[y - 1] + 1)
        prev = cur
        best = min(best, prev[m])
    return int(best)


def free_end_distance_rows(text, pattern) -> int:
    """free_end_distance with the insertion chain of a row as a running minimum:
    cur[y] = y + min(x, min over y' <= y of (best_row[y'-1] - y'))."""
    n, m = len(text), len(pattern)
    prev = np.arange(m + 1, dtype=np.int64)
    best = prev[m]
    t = np.asarray(text)
    p = np.asarray(pattern)
    ys = np.arange(1, m + 1, dtype=np.int64)
    for x in range(1, n + 1):
        best_row = np.minimum(prev[:-1] + (p != t[x - 1]), prev[1:] + 1)
        cur = np.empty(m + 1, dtype=np.int64)
        cur[0] = x
        cur[1:] = ys + np.minimum(x, np.minimum.accumulate(best_row - ys))
        prev = cur
        best = min(best, prev[m])
    return int(best)


def cigar_ops(runs):
    """uint32 runs -> list of (op, len)."""
    return [(int(r) & 15, int(r) >> 4) for r in runs]


def check_cigar(text, pattern, runs, text_consumed, edit_count):
    """The invariants every windowed alignment must satisfy; returns an error string or ''."""
    i = j = 0
    edits = 0
    for op, ln in cigar_ops(runs):
        if ln <= 0:
            return "empty run"
        for _ in range(ln):
            if op == 7:
                if i >= len(text) or j >= len(pattern) or text[i] != pattern[j]:
                    return f"bad '=' at {i},{j}"
                i += 1
                j += 1
            elif op == 8:
                if i >= len(text) or j >= len(pattern) or text[i] == pattern[j]:
                    return f"bad 'X' at {i},{j}"
                i += 1
                j += 1
                edits += 1
            elif op == 1:
                if j >= len(pattern):
                    return "I past pattern end"
                j += 1
                edits += 1
            elif op == 2:
                if i >= len(text):
                    return "D past text end"
                i += 1
                edits += 1
            else:
                return f"unknown op {op}"
    if j != len(pattern):
        return f"pattern consumed {j} != {len(pattern)}"
    if i != text_consumed:
        return f"text consumed {i} != reported {text_consumed}"
    if edits != edit_count:
        return f"edits {edits} != reported {edit_count}"
    return ""
