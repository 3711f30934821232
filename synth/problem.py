"""Container for one conic program in the standard form of the paper (Sec. 2.1).

Cone codes follow the C-ABI header (``include/cosmo_du.h``): they are an
interface, not arithmetic.

PSD blocks are stored in ``svec`` form: the upper triangle of the symmetric
p x p matrix, column by column, with off-diagonal entries multiplied by
sqrt(2) so that svec(X)'svec(Y) = <X, Y> (the paper leaves the layout open;
this is the isometric convention).
"""
from dataclasses import dataclass, field
from typing import List, Tuple, Optional

import numpy as np
import scipy.sparse as sp

ZERO, NONNEG, BOX, SOC, PSD = 0, 1, 2, 3, 4
CONE_NAMES = {ZERO: "zero", NONNEG: "nonneg", BOX: "box", SOC: "soc", PSD: "psd"}


def svec_len(p: int) -> int:
    """Number of svec rows of a p x p PSD block."""
    return p * (p + 1) // 2


def svec_index(i: int, j: int) -> int:
    """Row of entry (i, j) (i <= j) inside a block's svec: column-major upper triangle."""
    if i > j:
        i, j = j, i
    return j * (j + 1) // 2 + i


def cone_rows(ctype: int, dim: int) -> int:
    """Rows a cone occupies: dim for every type except PSD, whose dim is p."""
    return svec_len(dim) if ctype == PSD else dim


@dataclass
class ConicProblem:
    P: sp.csr_matrix            # n x n, symmetric, both triangles stored
    q: np.ndarray               # n
    A: sp.csr_matrix            # m x n
    b: np.ndarray               # m
    cones: List[Tuple[int, int]]  # (type, dim) in row order; PSD dim = p
    box_l: Optional[np.ndarray] = None   # m (used on BOX rows only)
    box_u: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    def cone_offsets(self):
        """Yield (type, dim, row_begin, row_end) for each cone."""
        r = 0
        for t, d in self.cones:
            k = cone_rows(t, d)
            yield t, d, r, r + k
            r += k

    def row_types(self) -> np.ndarray:
        out = np.empty(self.m, dtype=np.int32)
        for t, d, r0, r1 in self.cone_offsets():
            out[r0:r1] = t
        return out

    def check(self):
        """Structural sanity: shapes, cone rows summing to m, symmetric P."""
        n, m = self.n, self.m
        assert self.P.shape == (n, n)
        assert self.q.shape == (n,) and self.b.shape == (m,)
        tot = sum(cone_rows(t, d) for t, d in self.cones)
        assert tot == m, (tot, m)
        d = abs(self.P - self.P.T)
        assert d.nnz == 0 or d.max() < 1e-12
        if any(t == BOX for t, _ in self.cones):
            assert self.box_l is not None and self.box_u is not None
        return self
