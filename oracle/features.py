"""Independent numpy statement of the tuner's 16 matrix features -- TEST INFRASTRUCTURE ONLY.

Written from the feature definitions (not from the library's code) to pin ``ehyb_features``; every output is
pinned to closed forms in tests/test_oracle_features.py:
0 log2(n+1); 1 log2(nnz+1); 2 mean, 3 population std, 4 log2(max+1), 5 min, 6 p50, 7 p90, 8 p99 of the
row lengths (percentile q = element floor(q (n-1)) of the ascending lengths); 9 share of rows longer
than 32; 10 Gini coefficient sum_i (2i - n - 1) l_(i) / (n sum l) over ascending lengths, ranks from 1;
11 mean |i - j| / n over entries; 12 share of entries with |i - j| <= ceil(n / P); 13 share of rows with
|a_ii| >= sum_{j != i} |a_ij| among non-empty rows (divided by n); 14 share of the entries (i, j) of rows
0, s, 2s, ... (s = max(1, n // 1000)) that have an entry (j, i); 15 share of entries whose row and column
lie in the same block of ceil(n / P) consecutive rows.  P = 152 by default.
"""
import math

import numpy as np


def features(A, P: int = 152) -> np.ndarray:
    n = A.n
    rp = np.asarray(A.row_ptr, np.int64)
    col = np.asarray(A.col, np.int64)
    val = np.asarray(A.val, np.float64)
    nnz = int(rp[-1]) if n else 0
    f = np.zeros(16, np.float64)
    f[0] = math.log2(n + 1)
    f[1] = math.log2(nnz + 1)
    if n == 0:
        return f
    lens = np.diff(rp)
    s = np.sort(lens)
    f[2] = lens.mean()
    f[3] = lens.std()
    f[4] = math.log2(s[-1] + 1)
    f[5] = s[0]
    for k, q in ((6, 0.5), (7, 0.9), (8, 0.99)):
        f[k] = s[int(math.floor(q * (n - 1)))]
    f[9] = np.mean(lens > 32)
    ranks = np.arange(1, n + 1)
    f[10] = np.sum((2 * ranks - n - 1) * s) / (n * s.sum()) if s.sum() else 0.0
    rows = np.repeat(np.arange(n), lens)
    d = np.abs(col - rows)
    band = -(-n // P)
    f[11] = d.mean() / n if nnz else 0.0
    f[12] = np.mean(d <= band) if nnz else 0.0
    dom = 0
    for i in range(n):
        seg = slice(rp[i], rp[i + 1])
        c, v = col[seg], np.abs(val[seg])
        if c.size and v[c == i].sum() >= v[c != i].sum():
            dom += 1
    f[13] = dom / n
    step = max(1, n // 1000)
    checked = mirrored = 0
    for i in range(0, n, step):
        for j in col[rp[i]:rp[i + 1]]:
            checked += 1
            mirrored += bool(np.any(col[rp[j]:rp[j + 1]] == i))
    f[14] = mirrored / checked if checked else 1.0
    f[15] = np.mean(rows // band == col // band) if nnz else 0.0
    return f
