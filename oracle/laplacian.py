"""Graph Laplacians in CSR form (test infrastructure; see package header).

Sec. 2 of the paper defines, for an undirected graph with positive weights
A_ij (1 if unweighted) and degrees D_ii = sum_j A_ij,

* the combinatorial Laplacian  L = D - A, spectrum in [0, 2 max D];
* the normalized Laplacian     I - D^{-1/2} A D^{-1/2}, spectrum in [0, 2];

and Sec. 2.1 the density matrix P = L / tr(L).

Readings where the paper is silent:
* Input cleaning: each listed pair is an undirected edge; self-loops are
  dropped and duplicate pairs (in either orientation) are merged, keeping the
  largest weight.
* Isolated nodes (D_ii = 0): D^{-1/2} is undefined there; they get scale
  s_i = 0 and a zero row (eigenvalue 0), Chung's convention.  With
  ``drop_isolated`` they are removed and the remaining ids are compacted in
  increasing order.
* Weighted degrees are summed left to right in increasing column order.
* Off-diagonal values: normalized  -(A_ij * s_i) * s_j with s_i = 1/sqrt(D_ii);
  combinatorial -A_ij.  Diagonal: 1 (normalized, D_ii > 0), D_ii
  (combinatorial).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

NORMALIZED = "normalized"
COMBINATORIAL = "combinatorial"


@dataclass
class Laplacian:
    n: int                 # nodes kept (n')
    kind: str
    rowptr: np.ndarray     # int64[n+1]
    colidx: np.ndarray     # int32[nnz], ascending within each row
    vals: np.ndarray       # float64[nnz] off-diagonal values
    diag: np.ndarray       # float64[n]
    scale: np.ndarray      # float64[n]   s_i = D_ii^{-1/2} (normalized) or 1
    degree: np.ndarray     # float64[n]   D_ii
    old_id: np.ndarray     # int64[n]     original node id of each kept node
    trace: float           # tr(L)

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    def matrix(self) -> sp.csr_matrix:
        """Sparse L including its diagonal (for matvecs)."""
        off = sp.csr_matrix((self.vals, self.colidx.astype(np.int64), self.rowptr),
                            shape=(self.n, self.n))
        return (off + sp.diags(self.diag)).tocsr()

    def dense(self) -> np.ndarray:
        return self.matrix().toarray()

    def norm_bound(self) -> float:
        """Gershgorin bound on the spectrum (Sec. 2): 2, or 2 max D."""
        if self.kind == NORMALIZED:
            return 2.0
        return 2.0 * float(self.degree.max()) if self.n else 0.0


def build_laplacian(src, dst, n_nodes: int, weights=None, kind: str = NORMALIZED,
                    drop_isolated: bool = False) -> Laplacian:
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if n_nodes < 0:
        raise ValueError("negative node count")
    if src.size and (min(src.min(), dst.min()) < 0 or max(src.max(), dst.max()) >= n_nodes):
        raise ValueError("node id out of range")
    if kind not in (NORMALIZED, COMBINATORIAL):
        raise ValueError("unknown Laplacian kind")
    w = None
    if weights is not None:
        w = np.asarray(weights, dtype=np.float64)
        if w.shape != src.shape:
            raise ValueError("weights differ in length")
        if not np.all(w > 0):
            raise ValueError("weights must be positive")

    # undirected: both orientations, self-loops dropped
    keep = src != dst
    rows = np.concatenate([src[keep], dst[keep]])
    cols = np.concatenate([dst[keep], src[keep]])
    wts = None if w is None else np.concatenate([w[keep], w[keep]])

    # sort by (row, col) and merge duplicates (largest weight kept)
    key = rows * max(n_nodes, 1) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    starts = np.flatnonzero(first)
    ukey = key[starts]
    urow = ukey // max(n_nodes, 1)
    ucol = ukey % max(n_nodes, 1)
    if wts is None:
        uw = np.ones(ukey.size)
    else:
        uw = np.maximum.reduceat(wts[order], starts) if starts.size else np.zeros(0)

    counts = np.bincount(urow, minlength=n_nodes).astype(np.int64)
    rowptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])

    if wts is None:
        degree = counts.astype(np.float64)
    else:
        degree = np.zeros(n_nodes)
        for i in range(n_nodes):              # left to right, ascending column
            acc = 0.0
            for e in range(rowptr[i], rowptr[i + 1]):
                acc += uw[e]
            degree[i] = acc

    old_id = np.arange(n_nodes, dtype=np.int64)
    if drop_isolated:
        kept = counts > 0
        new_id = np.cumsum(kept) - 1
        old_id = old_id[kept]
        ucol = new_id[ucol]
        degree = degree[kept]
        counts = counts[kept]
        rowptr = np.zeros(old_id.size + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
    n = int(old_id.size)
    colidx = ucol.astype(np.int32)
    row_of = np.repeat(np.arange(n), np.diff(rowptr))

    if kind == NORMALIZED:
        scale = np.zeros(n)
        pos = degree > 0
        scale[pos] = 1.0 / np.sqrt(degree[pos])
        vals = -((uw * scale[row_of]) * scale[colidx])
        diag = pos.astype(np.float64)
        trace = float(np.count_nonzero(pos))
    else:
        scale = np.ones(n)
        vals = -uw
        diag = degree.copy()
        trace = math.fsum(degree)
    return Laplacian(n=n, kind=kind, rowptr=rowptr, colidx=colidx, vals=vals,
                     diag=diag, scale=scale, degree=degree, old_id=old_id, trace=trace)


def density_matrix_scale(lap: Laplacian) -> float:
    """c = tr(L): P = L / c (Sec. 2.1)."""
    return lap.trace
