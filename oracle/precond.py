"""Preconditioners of Appendix A ("Preconditioning"), on the explicitly assembled system.

TEST INFRASTRUCTURE ONLY (see the package header).

Both are written exactly as the appendix defines them, on the oracle's assembled sparse
velocity matrix A (one block row per element, block size d * N_phi * N_gamma):

  pre1(A, ne)   Eq. pre1: P_1 = diag(D_1^{-1}, ..., D_N^{-1}), D_i the diagonal block of
                element i.
  pre2(A, ne, nbr)
                Eqs. APPRE1 / APPRE2: for element i, the local system A_i = A restricted
                to the stencil S_i (i first, then its face neighbours) is inverted
                densely and the first block row of A_i^{-1} is kept; block row i of P_2
                maps the stencil's values to element i.

Pins (tests/test_oracle_precond.py): both are checked against what the definition fixes
independently of how the inverse is formed -- (P_1 A x)_i = x_i for x supported on
element i, (P_2 A x)_i = x_i for x supported on the stencil S_i (A x restricted to S_i
is A_i x_{S_i}), P_2 = A^{-1} rows on a mesh that one stencil covers, and P_2 = P_1 when
the off-diagonal blocks vanish.
"""
import numpy as np
import scipy.sparse as sp


def _nb(A, ne):
    n = A.shape[0]
    if n % ne:
        raise ValueError("matrix size is not a multiple of the element count")
    return n // ne


def stencil(e, nbr):
    """S_i of Appendix A: element e first, then its face neighbours (boundary faces have none)."""
    out = [int(e)]
    for g in nbr[e]:
        g = int(g)
        if g >= 0 and g not in out:
            out.append(g)
    return out


def pre1(A, ne):
    """Eq. pre1: block-diagonal inverse of the element blocks."""
    A = sp.csr_matrix(A)
    nb = _nb(A, ne)
    blocks = []
    for e in range(ne):
        sl = slice(e * nb, (e + 1) * nb)
        blocks.append(sp.csr_matrix(np.linalg.inv(A[sl, sl].toarray())))
    return sp.block_diag(blocks, format="csr")


def pre2(A, ne, nbr):
    """Eqs. APPRE1 / APPRE2: first block row of the inverse of the stencil system, per element."""
    A = sp.csr_matrix(A)
    nb = _nb(A, ne)
    rows, cols, vals = [], [], []
    for e in range(ne):
        st = stencil(e, nbr)
        idx = np.concatenate([np.arange(g * nb, (g + 1) * nb) for g in st])
        Ai = A[idx][:, idx].toarray()                  # Eq. APPRE1
        first = np.linalg.inv(Ai)[:nb]                 # A_i^{-1}(0, e') for every e' in S_i
        r, c = np.meshgrid(np.arange(e * nb, (e + 1) * nb), idx, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(first.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=A.shape)
