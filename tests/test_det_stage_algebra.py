"""Host check of the algebra of the pair-of-FP32 determinant stage.

The FP32X2 determinant stage keeps one row of a spin block per lane and
eliminates in place with implicit pivoting: at step k the unused row p_k with
the largest |a[p_k][k]| becomes the pivot, and every row is updated from it
without moving rows.  Afterwards row i holds Z[i][k] = (A^-1)[m_i][p_k], m_i
being the step at which row i was the pivot, and the tables of the table
method (App. F, App. H) follow from Z and the pivot order:

    t[m_i]   = sum_k Z[i][k] Phi_p[p_k]          = (A^-1 Phi_p)[m_i]
    y[r]     = B_p[r] - sum_m B_0[r][m] t[m]
    Top[m_i] = sum_k Z[i][k] y[p_k]              = (A^-1 (B_p - B_0 A^-1 Phi_p))[m_i]
    tr0      = sum_i sum_k Z[i][k] B_0[p_k][m_i] = Tr(A^-1 B_0)
    det A    = (-1)^inv(p) prod_k pivot_k

Rows scaled by powers of two (A = D A^, B = D B^) leave t, Top and tr0
unchanged and multiply det A by 2^(sum e_r).  This file restates that
elimination in float64 numpy, in the kernel's order of operations, and checks
the identities against numpy's inverse and determinant on random matrices of
every block size the stage supports (1 to 8 rows).  It pins the algorithm,
not the GPU code (whose results the GPU parity tests compare with the oracle).
"""
import numpy as np
import pytest


def eliminate_in_place(a):
    """In-place Gauss-Jordan with implicit pivoting, every row updated from the
    pivot row as it stands (the pivot row as 0 - (-1/pivot) a_p, the others as
    a - g a_p with g = a[k] / pivot).  Returns (Z, pivot rows p_k, steps m_i,
    det)."""
    a = np.array(a, dtype=np.float64)
    n = a.shape[0]
    used = np.zeros(n, bool)
    pk = np.zeros(n, int)
    mi = np.zeros(n, int)
    det = 1.0
    for k in range(n):
        key = np.where(used, -1.0, np.abs(a[:, k]))
        p = int(np.argmax(key))  # lowest index on ties
        pk[k] = p
        inv = 1.0 / a[p, k]
        prw = a[p].copy()
        det *= a[p, k]
        used[p] = True
        mi[p] = k
        for r in range(n):
            piv = r == p
            g = a[r, k] * inv
            gg = -inv if piv else g
            for c in range(n):
                if c == k:
                    a[r, c] = inv if piv else -g
                else:
                    a[r, c] = (0.0 if piv else a[r, c]) - gg * prw[c]
    inversions = sum(1 for k in range(n) for l in range(k + 1, n) if pk[k] > pk[l])
    return a, pk, mi, det * (-1.0) ** inversions


def tables(Z, pk, mi, phi, bp, b0):
    n = Z.shape[0]
    t = np.zeros(n)
    for i in range(n):
        t[mi[i]] = sum(Z[i, k] * phi[pk[k]] for k in range(n))
    y = np.array([bp[r] - sum(b0[r, m] * t[m] for m in range(n)) for r in range(n)])
    top = np.zeros(n)
    for i in range(n):
        top[mi[i]] = sum(Z[i, k] * y[pk[k]] for k in range(n))
    tr0 = sum(Z[i, k] * b0[pk[k], mi[i]] for i in range(n) for k in range(n))
    return t, top, tr0


@pytest.mark.parametrize("n", range(1, 9))
def test_in_place_elimination_gives_the_permuted_inverse(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(20):
        A = rng.standard_normal((n, n))
        Z, pk, mi, det = eliminate_in_place(A)
        Ainv = np.linalg.inv(A)
        for i in range(n):
            for k in range(n):
                assert Z[i, k] == pytest.approx(Ainv[mi[i], pk[k]], rel=1e-9, abs=1e-9 * np.abs(Ainv).max())
        assert det == pytest.approx(np.linalg.det(A), rel=1e-9)
        # the pivot order is a permutation and m is its inverse
        assert sorted(pk) == list(range(n))
        assert all(pk[mi[i]] == i for i in range(n))


@pytest.mark.parametrize("n", range(1, 9))
def test_tables_and_trace_from_the_in_place_result(n):
    rng = np.random.default_rng(200 + n)
    for _ in range(20):
        A = rng.standard_normal((n, n))
        B0 = rng.standard_normal((n, n))
        phi, bp = rng.standard_normal(n), rng.standard_normal(n)
        Z, pk, mi, _ = eliminate_in_place(A)
        t, top, tr0 = tables(Z, pk, mi, phi, bp, B0)
        Ainv = np.linalg.inv(A)
        scale = 1.0 + np.abs(Ainv).max() ** 2 * (1.0 + np.abs(B0).max())
        np.testing.assert_allclose(t, Ainv @ phi, rtol=0, atol=1e-9 * scale)
        np.testing.assert_allclose(top, Ainv @ (bp - B0 @ (Ainv @ phi)), rtol=0, atol=1e-9 * scale ** 2)
        assert tr0 == pytest.approx(np.trace(Ainv @ B0), abs=1e-9 * scale)


@pytest.mark.parametrize("n", [1, 3, 7, 8])
def test_power_of_two_row_scaling(n):
    rng = np.random.default_rng(300 + n)
    A = rng.standard_normal((n, n))
    B0 = rng.standard_normal((n, n))
    phi, bp = rng.standard_normal(n), rng.standard_normal(n)
    e = rng.integers(-40, 40, size=n)
    D = np.diag(2.0 ** e)
    # A^ = A and the caller's rows D A^ (the pivot order may differ)
    Z, pk, mi, det_hat = eliminate_in_place(A)
    Zs, pks, mis, det_s = eliminate_in_place(D @ A)
    t, top, tr0 = tables(Z, pk, mi, phi, bp, B0)
    ts, tops, tr0s = tables(Zs, pks, mis, D @ phi, D @ bp, D @ B0)
    np.testing.assert_allclose(ts, t, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(tops, top, rtol=1e-9, atol=1e-12)
    assert tr0s == pytest.approx(tr0, rel=1e-9, abs=1e-12)
    assert det_s == pytest.approx(det_hat * 2.0 ** e.sum(), rel=1e-9)


def test_pivot_ties_take_the_lowest_row():
    # equal magnitudes in column 0: the lowest unused row is the pivot, as in
    # the lane reduction (the kernel breaks ties by lane index)
    A = np.array([[1.0, 2.0, 0.0], [-1.0, 0.0, 1.0], [1.0, 1.0, 3.0]])
    _, pk, _, det = eliminate_in_place(A)
    assert pk[0] == 0
    assert det == pytest.approx(np.linalg.det(A))
