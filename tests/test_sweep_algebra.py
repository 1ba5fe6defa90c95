"""The algebra of the single-sweep Arnoldi form (arnoldi_form KX_ARN_SWEEP),
checked on the CPU in FP64 against the oracle's Arnoldi process (Sect. 3.2,
eqs. (Arn), (Arn1)).

The GPU form builds column j from the explicit t1 = A v_{j-1}, removes the
basis from x = t1 and from y = t2 - h_{j-1,j-1} t1 (t2 = A t1, y = A x by
the Arnoldi relation A v_i = sum_k h_{k,i} v_k) in the order i = 0..j-1,
and takes the dots b'_i = v_i . x^(i), a'_i = v_i . y^(i) just before
removing column i; the next Hessenberg column and the Gram column then
follow from
    G_{i,j} = (b'_i - sum_{l>=i} G_{i,l} h_{l,j-1}) / beta,
    h_{i,j} = (a'_i - sum_{k>=i} G_{i,k} c_k) / beta,   h_{j,j} = x.y / x.x,
with c = H(0:j, 0:j-1) h(0:j-1, j-1) and beta = ||x||.  Written out here in
numpy on small Yee operators (2D, 3D and the PML model), the process must
equal classical Gram-Schmidt, i.e. the oracle's V and H to rounding, and
the same formulas with each dot taken after column i is removed (a slip of
one line in the sweep's loop) must not.  (In FP64 the Gram matrix is the
identity to rounding, so whether the correction sums the whole row or its
upper part is invisible here; it matters in FP32, where the GPU tests cover
it.)"""
import numpy as np
import pytest

import scenario as S
from oracle import krylov, pml, yee


def single_sweep(A, g, m, dot_first=True):
    n = g.size
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    G = np.eye(m + 1)
    V[:, 0] = g / np.linalg.norm(g)
    t1 = A @ V[:, 0]
    H[0, 0] = V[:, 0] @ t1
    for j in range(1, m + 1):
        t1 = A @ V[:, j - 1]
        t2 = A @ t1
        hc = H[:j, j - 1]
        c = H[:j, :j - 1] @ hc[:j - 1]
        x = t1.copy()
        y = t2 - hc[j - 1] * t1
        a = np.zeros(j)
        b = np.zeros(j)
        for i in range(j):
            if dot_first:
                b[i] = V[:, i] @ x
                a[i] = V[:, i] @ y
            x -= hc[i] * V[:, i]
            y -= c[i] * V[:, i]
            if not dot_first:   # the slip: dots after column i is removed
                b[i] = V[:, i] @ x
                a[i] = V[:, i] @ y
        beta = np.linalg.norm(x)
        H[j, j - 1] = beta
        V[:, j] = x / beta
        if j == m:
            break
        gcol = np.array([(b[i] - G[i, i:j] @ hc[i:]) / beta for i in range(j)])
        h = np.array([(a[i] - G[i, i:j] @ c[i:]) / beta for i in range(j)])
        G[:j, j] = gcol
        G[j, :j] = gcol
        H[:j, j] = h
        H[j, j] = (x @ y) / (x @ x)
    return V, H


def operators():
    g2 = S.Grid(2, (13, 11), (S.PEC, S.PEC), 0, 3, 1.0)
    g3 = S.Grid(3, (6, 5, 7), (S.PERIODIC, S.PERIODIC, S.PEC), 2, 2, 1.0)
    gp = S.Grid(2, (12, 9), (S.PEC, S.PERIODIC), 0, 3, 3.0, pml=1)
    rng = np.random.default_rng(3)
    out = []
    for grid in (g2, g3, gp):
        eps = 1.0 + 3.0 * rng.random(grid.shape)
        op = pml.PmlOperator(grid, eps) if getattr(grid, "pml", 0) else yee.Operator(grid, eps)
        out.append((grid, op.matrix().toarray()))
    return out


@pytest.mark.parametrize("k", [0, 1, 2])
def test_single_sweep_equals_gram_schmidt(k):
    grid, A = operators()[k]
    g = S.masked_random_vector(grid, 7)
    m = 24
    V, H = single_sweep(A, g, m)
    Vo, Ho, beta, md = krylov.arnoldi(lambda v: A @ v, g, m)
    assert md == m
    assert np.abs(H - Ho).max() < 1e-10 * np.abs(Ho).max()
    assert np.abs(V - Vo).max() < 1e-9
    assert np.abs(V.T @ V - np.eye(m + 1)).max() < 1e-11
    assert np.linalg.norm(A @ V[:, :m] - V @ H) < 1e-11 * np.linalg.norm(H)


def test_dots_after_the_removal_break_it():
    grid, A = operators()[1]
    g = S.masked_random_vector(grid, 7)
    V, H = single_sweep(A, g, 16, dot_first=False)
    Vo, Ho, _, _ = krylov.arnoldi(lambda v: A @ v, g, 16)
    assert np.abs(H - Ho).max() > 1e-3 * np.abs(Ho).max()
