"""Pins for the CPU oracle: each test ties it to something other than itself.

Closed forms (hand-derived TPFA matrices, exact Cholesky on a tridiagonal
matrix), dense linear algebra built independently from the paper's formulas
(Eq. barB, Eq. tildeB1, the block form of Section 2.1.2, the V-cycle recursion
of Section 3.3, the Galerkin product of Section 3.2), dense solves and
eigenvalues (Theorems 2.1 and 2.2), and invariants of the splitting rules.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1205_6113_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_op(apply, n):
    """Materialise a linear operator column by column from unit vectors."""
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = apply(e)
        e[j] = 0.0
    return M


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def a_norm(E, A):
    """||E||_A = ||A^{1/2} E A^{-1/2}||_2."""
    w, V = np.linalg.eigh(A)
    Ah = V @ np.diag(np.sqrt(w)) @ V.T
    Aih = V @ np.diag(1.0 / np.sqrt(w)) @ V.T
    return np.linalg.norm(Ah @ E @ Aih, 2)


@pytest.fixture(scope="module")
def small3d():
    """A 9 x 8 x 6 correlated problem with a 4-level hierarchy (coarse_max 20)."""
    p = inputs.small_3d(9, 8, 6, seed=11)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=20)
    assert orc.nlevels >= 3
    return p, A, orc, A.to_dense()


# --------------------------------------------------------------------------------------------
# Mixed-hybrid system (Section 4; Section 5, Eq. alge_sys), unit bricks
# --------------------------------------------------------------------------------------------
def test_mhfem_one_cell_matches_hand_derivation():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "mhfem_cell.txt")) if l.strip() and l[0] != "#"]
    expect = np.zeros((6, 6))
    for r, c, v in rows:
        expect[int(r), int(c)] = float(v)
    A = O.mhfem(1, 1, 1, np.zeros(1), 1.0, inputs.FACE_X0)
    assert A.n == 6 and np.array_equal(A.to_dense(), expect)


def test_mhfem_patch_test_1d():
    """A column of unit cells, k = 1, p = 0 at x = 0, unit source in the last cell: the exact
    pressure is p = x up to the last cell and a parabola inside it (p'(8) = 0).  The lowest-order
    mixed method is exact here: face multipliers equal p at the x-faces, cell pressures equal the
    cell averages of p (7 + 1/2 - 1/6 in the source cell), and the no-flow y/z faces of each cell
    carry its pressure."""
    nx = 8
    p = inputs.Problem("column", nx, 1, 1, np.zeros(nx), 1.0, inputs.FACE_X0)
    p.wells = [(nx - 1, 1.0)]
    A, b = O.mhfem_problem(p)
    x = np.linalg.solve(A.to_dense(), b)
    cells, xf = x[:nx], x[nx:2 * nx]
    assert np.allclose(cells, np.r_[np.arange(nx - 1) + 0.5, nx - 1 + 0.5 - 1.0 / 6.0], atol=1e-12)
    assert np.allclose(xf, np.r_[np.arange(1, nx), nx - 0.5], atol=1e-12)
    yz = x[2 * nx:].reshape(-1, nx)                       # y0, y1, z0, z1 faces, one per cell each
    assert np.allclose(yz, cells[None, :], atol=1e-12)


def test_mhfem_is_spd_with_positive_couplings():
    p = inputs.small_3d(5, 4, 3, seed=31)
    A = O.mhfem(p.nx, p.ny, p.nz, p.logk, p.kz_ratio, p.dirichlet)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    off = D - np.diag(np.diag(D))
    assert (off > 0).any()                                # opposite faces: not an M-matrix


# --------------------------------------------------------------------------------------------
# TPFA assembly (Section 4, Eq. model with c = 0)
# --------------------------------------------------------------------------------------------
def test_tpfa_matches_hand_derived_2x2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tpfa_2x2.txt")) if l.strip() and l[0] != "#"]
    expect = np.zeros((4, 4))
    for r, c, num, den in rows:
        expect[int(r), int(c)] = float(num) / float(den)
    A = O.tpfa(2, 2, 1, np.log([1.0, 3.0, 2.0, 4.0]), 1.0, inputs.FACE_X0)
    assert A.nnz == 12
    assert rel(A.to_dense(), expect) < 1e-14


def test_tpfa_homogeneous_is_kronecker_laplacian():
    nx, ny, nz, r = 5, 4, 3, 0.1

    def lap1(m):      # 1-D Neumann Laplacian with unit transmissibility
        L = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
        L[0, 0] = L[-1, -1] = 1.0
        return L if m > 1 else np.zeros((1, 1))

    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    expect = (np.kron(Iz, np.kron(Iy, lap1(nx))) + np.kron(Iz, np.kron(lap1(ny), Ix))
              + r * np.kron(lap1(nz), np.kron(Iy, Ix)))
    for c in range(nx * ny * nz):
        if c % nx == 0:
            expect[c, c] += 2.0
    A = O.tpfa(nx, ny, nz, np.zeros(nx * ny * nz), r, inputs.FACE_X0)
    assert A.nnz == O.lib().orc_tpfa_nnz(nx, ny, nz)
    assert rel(A.to_dense(), expect) < 1e-15


def test_tpfa_properties_random_field(small3d):
    p, A, _, D = small3d
    assert np.array_equal(D, D.T)
    off = D - np.diag(np.diag(D))
    assert np.all(off <= 0)
    # A 1 = Dirichlet half-cell transmissibility on x = 0 cells, zero elsewhere
    k = np.exp(p.logk)
    bnd = np.where(np.arange(A.n) % p.nx == 0, 2.0 * k, 0.0)
    assert np.max(np.abs(D.sum(axis=1) - bnd)) < 1e-12 * np.max(np.abs(D))
    assert np.linalg.eigvalsh(D)[0] > 0


# --------------------------------------------------------------------------------------------
# IC(0) = Algorithm 3.1 with k = 0 (Section 3.1, Section 3.3)
# --------------------------------------------------------------------------------------------
def ic_factors(A, lu):
    n = A.n
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for p in range(A.rowptr[i], A.rowptr[i + 1]):
            j = A.col[p]
            if j < i:
                L[i, j] = lu[p]
            else:
                U[i, j] = lu[p]
    return L, U


def test_ic0_on_tridiagonal_is_exact_cholesky():
    logk = inputs.random_vector(40, seed=3)
    A = O.tpfa(40, 1, 1, logk, 1.0, inputs.FACE_X0)
    orc = O.Oracle(A, coarse_max=8)
    L, U = ic_factors(A, orc.ic0_values())
    D = A.to_dense()
    assert rel(L @ U, D) < 1e-14               # no fill is dropped: LU = A exactly
    assert rel(U, np.diag(np.diag(U)) @ L.T) < 1e-14
    b = inputs.random_vector(40, seed=4)
    r = orc.pcg(b, op=O.B, tol=1e-12, maxit=10)
    assert r["status"] == 0 and r["iters"] == 1
    # B = A^{-1} => B_co = A^{-1} (Eq. tildeB1 with (I - S^T A) A^{-1} (I - A S) = A^{-1} - S~)
    r = orc.pcg(b, op=O.BCO, tol=1e-12, maxit=10)
    assert r["status"] == 0 and r["iters"] == 1


def test_ic0_matches_a_on_its_pattern(small3d):
    _, A, orc, D = small3d
    L, U = ic_factors(A, orc.ic0_values())
    LU = L @ U
    pat = D != 0
    assert rel(LU[pat], D[pat]) < 1e-13        # residual R = A - LU vanishes on the pattern
    assert np.all(np.diag(U) > 0)
    assert rel(U, np.diag(np.diag(U)) @ L.T) < 1e-13    # SPD => U = D L^T (IC(0))
    B = np.linalg.inv(LU)
    Bm = dense_op(lambda v: orc.apply(O.B, v), A.n)
    assert rel(Bm, B) < 1e-11


def test_ic0_breakdown_is_reported():
    # [[1, 2], [2, 1]] has a negative second pivot
    A = O.Csr(2, [0, 2, 4], [0, 1, 0, 1], [1.0, 2.0, 2.0, 1.0])
    with pytest.raises(O.OracleError) as e:
        O.Oracle(A)
    assert e.value.status == 2


def test_invalid_csr_is_rejected():
    A = O.Csr(2, [0, 2, 3], [1, 0, 1], [1.0, 2.0, 1.0])     # unsorted row, missing diagonal
    with pytest.raises(O.OracleError) as e:
        O.Oracle(A)
    assert e.value.status == 1


# --------------------------------------------------------------------------------------------
# AMG hierarchy (Section 3.2) and the V-cycle (Algorithm 3.2, Section 3.3)
# --------------------------------------------------------------------------------------------
def strength_dense(D, theta):
    n = D.shape[0]
    S = np.zeros((n, n), dtype=bool)
    for i in range(n):
        neg = -D[i].copy()
        neg[i] = -np.inf
        mx = neg.max()
        if mx > 0:
            S[i] = neg >= theta * mx
            S[i, i] = False
    return S


def test_galerkin_products(small3d):
    _, _, orc, _ = small3d
    for l in range(orc.nlevels - 1):
        Al = orc.level_A(l).to_dense()
        P = orc.level_P(l).to_dense()
        Ac = orc.level_A(l + 1).to_dense()
        assert rel(Ac, P.T @ Al @ P) < 1e-13
        assert rel(Ac, Ac.T) < 1e-14


def test_splitting_and_interpolation_invariants(small3d):
    _, _, orc, _ = small3d
    for l in range(orc.nlevels - 1):
        D = orc.level_A(l).to_dense()
        S = strength_dense(D, 0.12)
        cf, _ = orc.level_cf_colour(l)
        P = orc.level_P(l).to_dense()
        C = cf == 1
        cnt_t = S.sum(axis=0)                          # |S^T_i|
        assert set(np.unique(cf)) <= {0, 1}
        assert np.all(cnt_t[C] > 0)                    # no C point without dependants
        for i in np.where(~C)[0]:
            if cnt_t[i] > 0:                           # F by a C point it strongly depends on
                assert np.any(S[i] & C)
        mutual = S & S.T
        assert not np.any(mutual[np.ix_(C, C)])        # no two C points strongly coupled both ways
        # C rows are identity rows; F rows interpolate only from strong C neighbours
        cidx = np.cumsum(C) - 1
        for i in range(D.shape[0]):
            nzc = np.nonzero(P[i])[0]
            if C[i]:
                assert list(nzc) == [cidx[i]] and P[i, cidx[i]] == 1.0
            else:
                allowed = set(cidx[np.where(S[i] & C)[0]])
                assert set(nzc) <= allowed
                # zero row sum and no positive couplings => constants are interpolated exactly
                if len(nzc) and abs(D[i].sum()) < 1e-12 * D[i, i] and np.all(np.delete(D[i], i) <= 0):
                    assert abs(P[i].sum() - 1.0) < 1e-13
        # every F point with strong C neighbours has a nonempty interpolation row
        for i in np.where(~C)[0]:
            if np.any(S[i] & C):
                assert np.count_nonzero(P[i]) > 0


@pytest.mark.parametrize("shape,seed", [((4, 3, 2), 61), ((5, 4, 3), 62)])
def test_direct_interpolation_with_positive_couplings(shape, seed):
    """The positive-coupling branch of direct interpolation (Section 3.2 reading: positive
    off-diagonals lumped into the diagonal), pinned on the mixed-hybrid matrix, whose face rows
    couple positively to the opposite faces of each cell.  Two facts fix the weights of an F row
    i with interpolation set C_i, whatever formula produced them:
    (a) they are proportional to the couplings: P_ij / P_ik = a_ij / a_ik for j, k in C_i;
    (b) smooth error satisfies (A e)_i ~ 0 with positive neighbours taken at e_i and the negative
        ones averaged over C_i, so where A annihilates constants (zero row sum, no Dirichlet face)
        constants are interpolated exactly: sum_j P_ij = 1.  (Rows next to a Dirichlet face have
        lost a coupling and a nonzero row sum; (a) still holds there.)
    A sign slip in the lumped diagonal, a dropped positive term, or positive entries counted
    among the negative ones breaks (b) on rows that have positive couplings; this test checks
    that such rows exist and are F rows with nonempty interpolation."""
    p = inputs.small_3d(*shape, seed=seed)
    A = O.mhfem(p.nx, p.ny, p.nz, p.logk, p.kz_ratio, p.dirichlet)
    orc = O.Oracle(A, coarse_max=8)
    assert orc.nlevels >= 2
    D = A.to_dense()
    S = strength_dense(D, 0.12)
    cf, _ = orc.level_cf_colour(0)
    P = orc.level_P(0).to_dense()
    cidx = np.cumsum(cf == 1) - 1
    checked = 0
    for i in np.where(cf == 0)[0]:
        off = np.delete(D[i], i)
        if not (off > 0).any():
            continue
        interp = np.where(S[i] & (cf == 1))[0]
        w = P[i, cidx[interp]]
        if len(interp) == 0:
            assert not P[i].any()
            continue
        assert np.count_nonzero(P[i]) == len(interp)
        # (a) proportional to the couplings (all negative: strength is on -a_ij)
        assert np.all(D[i, interp] < 0) and np.all(w > 0)
        assert np.allclose(w / w.sum(), D[i, interp] / D[i, interp].sum(), rtol=1e-13, atol=0)
        # (b) constants on rows that annihilate them
        if abs(D[i].sum()) <= 1e-13 * D[i, i]:
            assert abs(w.sum() - 1.0) < 1e-13, i
            checked += 1
    assert checked >= 10


def test_colouring_is_proper(small3d):
    _, _, orc, _ = small3d
    for l in range(orc.nlevels - 1):
        D = orc.level_A(l).to_dense()
        _, colour = orc.level_cf_colour(l)
        ii, jj = np.nonzero(D)
        off = ii != jj
        assert np.all(colour[ii[off]] != colour[jj[off]])
        assert colour.min() == 0 and orc.level_sizes(l)["ncolours"] == colour.max() + 1


def test_colouring_is_a_greedy_colouring(small3d):
    """Every point of colour c has a neighbour of each colour c' < c (true of any greedy colouring,
    whatever its order), so no colour class can be merged into a smaller one point by point."""
    _, _, orc, _ = small3d
    for l in range(orc.nlevels - 1):
        A = orc.level_A(l)
        _, colour = orc.level_cf_colour(l)
        for i in range(A.n):
            nb = {int(colour[j]) for j in A.col[A.rowptr[i]:A.rowptr[i + 1]] if j != i}
            assert set(range(colour[i])) <= nb, (l, i)


def fan_matrix(m):
    """Hub 0 joined to the path 1 - 2 - ... - m: max degree m, degeneracy 2 (odd triangles, so
    not bipartite).  Unit off-diagonal couplings, diagonal degree + 1 (SPD)."""
    n = m + 1
    D = np.zeros((n, n))
    for j in range(1, n):
        D[0, j] = D[j, 0] = -1.0
    for j in range(1, m):
        D[j, j + 1] = D[j + 1, j] = -1.0
    D += np.diag(1.0 - D.sum(axis=1))
    return D


def dense_to_csr(D):
    n = D.shape[0]
    rowptr, col, val = [0], [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        col += nz.tolist()
        val += D[i, nz].tolist()
        rowptr.append(len(col))
    return O.Csr(n, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(val))


def test_colouring_bounded_by_degeneracy():
    """Peel rounds take points of degree <= 2 d_min, and d_min of any subgraph is at most the
    degeneracy k, so a point sees at most 2k neighbours of higher priority: <= 2k + 1 colours.
    The fan graph has k = 2 but a hub of degree 40, so a colouring that ignores the peel order
    would be allowed up to 41 colours by the plain greedy bound."""
    A = dense_to_csr(fan_matrix(40))
    orc = O.Oracle(A, coarse_max=4)
    assert orc.nlevels >= 2
    _, colour = orc.level_cf_colour(0)
    D = A.to_dense()
    ii, jj = np.nonzero(D)
    off = ii != jj
    assert np.all(colour[ii[off]] != colour[jj[off]])
    assert 3 <= colour.max() + 1 <= 5


def test_colouring_bound_on_amg_levels(small3d):
    nx = pytest.importorskip("networkx")
    _, _, orc, _ = small3d
    for l in range(1, orc.nlevels - 1):
        A = orc.level_A(l)
        G = nx.Graph()
        G.add_nodes_from(range(A.n))
        for i in range(A.n):
            G.add_edges_from((i, int(j)) for j in A.col[A.rowptr[i]:A.rowptr[i + 1]] if j != i)
        k = max(nx.core_number(G).values())
        assert orc.level_sizes(l)["ncolours"] <= 2 * k + 1, l


def gs_dense(D, colour, backward):
    n = D.shape[0]
    M = np.diag(np.diag(D)).copy()
    for i in range(n):
        for j in range(n):
            if i != j and D[i, j] != 0:
                if (colour[j] < colour[i]) != backward and colour[j] != colour[i]:
                    M[i, j] = D[i, j]
    return np.linalg.inv(M)


def test_gauss_seidel_smoother_is_multicolour_gs(small3d):
    _, _, orc, _ = small3d
    for l in range(orc.nlevels - 1):
        D = orc.level_A(l).to_dense()
        _, colour = orc.level_cf_colour(l)
        n = D.shape[0]
        Sf = dense_op(lambda v: orc.level_apply(l, 1, v), n)
        Sb = dense_op(lambda v: orc.level_apply(l, 2, v), n)
        assert rel(Sf, gs_dense(D, colour, False)) < 1e-12
        assert rel(Sb, gs_dense(D, colour, True)) < 1e-12
        assert rel(Sb, Sf.T) < 1e-12                   # backward sweep = adjoint of forward sweep
        assert a_norm(np.eye(n) - Sf @ D, D) < 1.0      # GS is norm-convergent


def test_vcycle_matches_recursion(small3d):
    """I - B_l A_l = (I - S_l^T A_l)(I - P B_{l-1} P^T A_l)(I - S_l A_l), B_0 = A_0^{-1} (Section 3.3)."""
    _, _, orc, _ = small3d
    L = orc.nlevels
    Dc = orc.level_A(L - 1).to_dense()
    Bc = np.linalg.inv(Dc)
    assert rel(dense_op(lambda v: orc.level_apply(L - 1, 3, v), Dc.shape[0]), Bc) < 1e-12
    Bnext = Bc
    for l in range(L - 2, -1, -1):
        D = orc.level_A(l).to_dense()
        n = D.shape[0]
        _, colour = orc.level_cf_colour(l)
        P = orc.level_P(l).to_dense()
        I = np.eye(n)
        Sf, Sb = gs_dense(D, colour, False), gs_dense(D, colour, True)
        E = (I - Sb @ D) @ (I - P @ Bnext @ P.T @ D) @ (I - Sf @ D)
        B = (I - E) @ np.linalg.inv(D)
        V = dense_op(lambda v: orc.level_apply(l, 4, v), n)
        assert rel(V, B) < 1e-11
        assert a_norm(E, D) < 1.0                      # the cycle is norm-convergent
        Bnext = B


def test_amg_ilu_cycle_matches_error_propagation(small3d):
    """AMG(ILU(0)) of Section 5: the V-cycle with the IC(0) preconditioner B as the finest smoother,
    I - S A = (I - B A)(I - P B_1 P^T A)(I - B A) with B_1 the GS V-cycle of level 1 (pinned by the
    recursion test) and B the IC(0) solve (pinned by the IC tests), applied as two cycles:
    I - S~ A = (I - S A)^2 (S is symmetric since B is)."""
    _, A, orc, D = small3d
    n = D.shape[0]
    I = np.eye(n)
    B = dense_op(lambda v: orc.apply(O.B, v), n)
    P = orc.level_P(0).to_dense()
    B1 = dense_op(lambda v: orc.level_apply(1, 4, v), P.shape[1])
    E = (I - B @ D) @ (I - P @ B1 @ P.T @ D) @ (I - B @ D)
    Ainv = np.linalg.inv(D)
    S = dense_op(lambda v: orc.apply(O.S_ILU, v), n)
    assert rel(S, (I - E) @ Ainv) < 1e-11
    St = dense_op(lambda v: orc.apply(O.AMG_ILU, v), n)
    assert rel(St, (I - E @ E) @ Ainv) < 1e-11
    assert rel(St, St.T) < 1e-11


def test_vcycle_symmetric_and_adjoint(small3d):
    _, A, orc, D = small3d
    n = A.n
    S = dense_op(lambda v: orc.apply(O.S, v), n)
    ST = dense_op(lambda v: orc.apply(O.ST, v), n)
    assert rel(S, S.T) < 1e-12
    assert rel(ST, S.T) < 1e-12
    rho = a_norm(np.eye(n) - S @ D, D) ** 2
    assert rho < 1.0


def test_natural_order_gauss_seidel_is_triangular_solve():
    """Natural-order ("standard") GS of Section 3.3: the forward sweep is S_l = (D + L)^{-1} and the
    backward sweep S_l^T = (D + U)^{-1} with the natural row order, i.e. the lower and upper
    triangles of A_l including the diagonal; the V-cycle built on them obeys the recursion of
    Algorithm 3.2 and B_co built on it is symmetric."""
    p = inputs.small_3d(9, 8, 6, seed=11)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=20, gs_natural=True)
    L = orc.nlevels
    assert L >= 3
    Bnext = np.linalg.inv(orc.level_A(L - 1).to_dense())
    for l in range(L - 2, -1, -1):
        D = orc.level_A(l).to_dense()
        n = D.shape[0]
        I = np.eye(n)
        Sf = dense_op(lambda v: orc.level_apply(l, 1, v), n)
        Sb = dense_op(lambda v: orc.level_apply(l, 2, v), n)
        assert rel(Sf, np.linalg.inv(np.tril(D))) < 1e-12
        assert rel(Sb, np.linalg.inv(np.triu(D))) < 1e-12
        P = orc.level_P(l).to_dense()
        E = (I - Sb @ D) @ (I - P @ Bnext @ P.T @ D) @ (I - Sf @ D)
        Bl = (I - E) @ np.linalg.inv(D)
        assert rel(dense_op(lambda v: orc.level_apply(l, 4, v), n), Bl) < 1e-11
        Bnext = Bl
    D = A.to_dense()
    Bco = dense_op(lambda v: orc.apply(O.BCO, v), A.n)
    assert rel(Bco, Bco.T) < 1e-11
    assert np.min(np.linalg.eigvalsh(0.5 * (Bco + Bco.T))) > 0.0
    # the multicolour cycle is a different operator (the orderings differ)
    mc = O.Oracle(A, coarse_max=20)
    assert rel(dense_op(lambda v: mc.level_apply(0, 1, v), A.n), Sf) > 1e-3
    b = np.zeros(A.n)
    b[A.n // 2] = 1.0
    res = orc.pcg(b, op=O.BCO, tol=1e-12, maxit=200)
    x = np.linalg.solve(D, b)
    assert np.linalg.norm(res["x"] - x) <= 1e-8 * np.linalg.norm(x)


def test_block_pcg_reduces_to_pcg_for_one_column(small3d):
    """Block CG with K = 1 is textbook PCG: same iterates, same residual history."""
    p, A, orc, D = small3d
    b = inputs.random_vector(A.n, seed=17)
    ref = orc.pcg(b, op=O.BCO, tol=1e-10, maxit=200)
    blk = O.block_pcg(orc, b[:, None], op=O.BCO, tol=1e-10, maxit=200)
    assert blk["status"] == 0 and blk["iters"] == ref["iters"]
    assert np.linalg.norm(blk["X"][:, 0] - ref["x"]) <= 1e-12 * np.linalg.norm(ref["x"])
    assert np.allclose(blk["res_hist"][:, 0], ref["res_hist"], rtol=1e-7, atol=0.0)


def test_block_cg_finite_termination_and_solution():
    """Unpreconditioned block CG on n = 60 with K = 6 columns spans the whole space after n / K = 10
    block iterations (exact arithmetic; two more allowed for rounding), and the solution is the
    dense solve.  With B_co, every column is solved to the dense solution at tol 1e-12."""
    p = inputs.small_3d(5, 4, 3, seed=3)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=20)
    D = A.to_dense()
    Bm = np.stack([inputs.random_vector(A.n, seed=40 + j) for j in range(6)], axis=1)
    plain = O.block_pcg(orc, Bm, op=O.I, tol=1e-10, maxit=60)
    assert plain["status"] == 0 and plain["iters"] <= A.n // 6 + 2
    Xd = np.linalg.solve(D, Bm)
    assert np.linalg.norm(plain["X"] - Xd) <= 1e-8 * np.linalg.norm(Xd)
    pre = O.block_pcg(orc, Bm, op=O.BCO, tol=1e-12, maxit=60)
    assert pre["status"] == 0
    assert np.linalg.norm(pre["X"] - Xd) <= 1e-9 * np.linalg.norm(Xd)


def test_block_cg_needs_no_more_iterations_than_its_columns(small3d):
    """The block Krylov space contains each column's own Krylov space, so block CG minimises each
    column's error over a larger space: it stops no later than the slowest single solve."""
    p, A, orc, D = small3d
    Bm = np.ascontiguousarray(inputs.batch_rhs(A.n, 8, cells_per_rhs=4, seed=6).T)
    blk = O.block_pcg(orc, Bm, op=O.BCO, tol=1e-8, maxit=200)
    single = [orc.pcg(Bm[:, j], op=O.BCO, tol=1e-8, maxit=200)["iters"] for j in range(8)]
    assert blk["status"] == 0 and blk["iters"] <= max(single)
    for j in range(8):
        assert np.linalg.norm(Bm[:, j] - A.matvec(blk["X"][:, j])) <= 1.0001e-8 * np.linalg.norm(Bm[:, j])


def test_block_cg_rank_deficient_block_is_a_breakdown(small3d):
    p, A, orc, D = small3d
    b = inputs.random_vector(A.n, seed=5)
    blk = O.block_pcg(orc, np.stack([b, b], axis=1), op=O.BCO, tol=1e-8, maxit=50)
    assert blk["status"] == 4


def test_single_level_hierarchy_is_exact():
    p = inputs.small_3d(5, 4, 3, seed=2)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=1000)
    assert orc.nlevels == 1
    D = A.to_dense()
    S = dense_op(lambda v: orc.apply(O.S, v), A.n)
    assert rel(S, np.linalg.inv(D)) < 1e-12            # S = A^{-1}
    Bco = dense_op(lambda v: orc.apply(O.BCO, v), A.n)
    assert rel(Bco, np.linalg.inv(D)) < 1e-11          # S = A^{-1} => B_co = A^{-1}
    r = orc.pcg(p.rhs(), op=O.BCO, tol=1e-12, maxit=10)
    assert r["status"] == 0 and r["iters"] == 1


# --------------------------------------------------------------------------------------------
# The combined preconditioner (Algorithm 2.1, Eqs. barB and tildeB1, Section 2.1)
# --------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def materialised(small3d):
    _, A, orc, D = small3d
    n = A.n
    ops = {k: dense_op(lambda v, op=op: orc.apply(op, v), n)
           for k, op in dict(S=O.S, ST=O.ST, B=O.B, Bco=O.BCO, St=O.STILDE, Bh=O.BHAT).items()}
    return D, ops


def test_error_propagation_eq_barB(materialised):
    D, M = materialised
    I = np.eye(D.shape[0])
    lhs = I - M["Bco"] @ D
    rhs = (I - M["ST"] @ D) @ (I - M["B"] @ D) @ (I - M["S"] @ D)
    assert rel(lhs, rhs) < 1e-11


def test_closed_form_eq_tildeB1(materialised):
    D, M = materialised
    I = np.eye(D.shape[0])
    S, ST, B = M["S"], M["ST"], M["B"]
    St = S + ST - ST @ D @ S
    assert rel(M["St"], St) < 1e-11                   # two cycles give S~
    assert rel(M["Bco"], St + (I - ST @ D) @ B @ (I - D @ S)) < 1e-11
    assert rel(M["Bco"], St + B - ST @ D @ B - B @ D @ S + ST @ D @ B @ D @ S) < 1e-11
    assert rel(M["Bh"], St + B) < 1e-11                # additive variant, Eq. Ba


def test_block_factorisation_form(materialised):
    """(I, I) [[I, -S^T A], [0, I]] diag(S~, B) [[I, 0], [-A S, I]] (I; I) = B_co (Section 2.1.2)."""
    D, M = materialised
    n = D.shape[0]
    I, Z = np.eye(n), np.zeros((n, n))
    St = M["St"]
    left = np.block([[I, -M["ST"] @ D], [Z, I]])
    mid = np.block([[St, Z], [Z, M["B"]]])
    right = np.block([[I, Z], [-D @ M["S"], I]])
    II = np.vstack([I, I])
    assert rel(II.T @ left @ mid @ right @ II, M["Bco"]) < 1e-11


def test_bco_is_spd_theorem_2_1(materialised):
    _, M = materialised
    Bco = M["Bco"]
    assert rel(Bco, Bco.T) < 1e-11
    assert np.linalg.eigvalsh(0.5 * (Bco + Bco.T))[0] > 0


def test_theorem_2_2_condition_bound(materialised):
    D, M = materialised
    Lh = np.linalg.cholesky(D)                         # similarity to symmetric forms
    def eig(Bm):
        return np.linalg.eigvalsh(Lh.T @ (0.5 * (Bm + Bm.T)) @ Lh)
    ev_b = eig(M["B"])
    m0, m1 = ev_b[0], ev_b[-1]
    rho = 1.0 - eig(M["St"])[0]                        # ||I - S A||_A^2 = 1 - lambda_min(S~ A)
    assert 0 < rho < 1
    ev = eig(M["Bco"])
    kappa = ev[-1] / ev[0]
    lo, hi, bound = O.thm22_bound(m0, m1, rho)
    assert ev[0] >= lo * (1 - 1e-10) and ev[-1] <= hi * (1 + 1e-10)
    assert kappa <= bound * (1 + 1e-10)
    assert kappa < m1 / m0                             # Eq. ine:better_B
    if m1 > 1 >= m0 and rho >= 1 - m0 / (m1 - 1):     # Eq. ine:better_S
        assert kappa <= 1.0 / (1.0 - rho) * (1 + 1e-10)


def test_lanczos_estimate_matches_dense_extremes(small3d, materialised):
    p, A, orc, D = small3d
    _, M = materialised
    r = orc.pcg(inputs.random_vector(A.n, seed=9), op=O.BCO, tol=1e-13, maxit=500)
    assert r["status"] == 0
    lo, hi = O.lanczos_extremes(r["alpha"], r["beta"])
    Lh = np.linalg.cholesky(D)
    ev = np.linalg.eigvalsh(Lh.T @ M["Bco"] @ Lh)
    # Ritz values lie inside the spectrum; the small end (which sets kappa here) has converged
    assert ev[0] * (1 - 1e-10) <= lo and hi <= ev[-1] * (1 + 1e-10)
    assert abs(lo - ev[0]) < 1e-6 * ev[-1]
    assert hi > 0.99 * ev[-1]


# --------------------------------------------------------------------------------------------
# PCG against dense Cholesky solves, SPD probes, status codes
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(6, 6, 1), (4, 4, 3), (7, 5, 4)])
@pytest.mark.parametrize("opname", ["bco", "amg", "ilu", "bhat", "none"])
def test_pcg_matches_dense_cholesky(shape, opname):
    nx, ny, nz = shape
    p = inputs.small_3d(nx, ny, nz, seed=5) if nz > 1 else inputs.lognormal_2d(nx, ny, seed=5)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=12)
    b = inputs.random_vector(A.n, seed=6)
    D = A.to_dense()
    c = np.linalg.cholesky(D)
    xs = np.linalg.solve(c.T, np.linalg.solve(c, b))
    r = orc.pcg(b, op=O.OPS[opname], tol=1e-12, maxit=2000)
    assert r["status"] == 0
    assert np.linalg.norm(r["x"] - xs) / np.linalg.norm(xs) <= 1e-8
    assert r["true_res"] < 1e-11
    assert r["res_hist"][0] == 1.0 and r["res_hist"][-1] < 1e-12


def test_pcg_on_64x64_lognormal_matches_dense():
    p = inputs.lognormal_2d()
    A = O.tpfa_problem(p)
    orc = O.Oracle(A)
    b = p.rhs()
    xs = np.linalg.solve(A.to_dense(), b)
    for opname in ("bco", "amg", "ilu"):
        r = orc.pcg(b, op=O.OPS[opname], tol=1e-12, maxit=3000)
        assert r["status"] == 0
        assert np.linalg.norm(r["x"] - xs) / np.linalg.norm(xs) <= 1e-8


def test_bco_symmetric_positive_on_random_vectors():
    p = inputs.lognormal_2d()
    A = O.tpfa_problem(p)
    orc = O.Oracle(A)
    rng = np.random.Generator(np.random.PCG64(12))
    for _ in range(100):
        x, y = rng.standard_normal(A.n), rng.standard_normal(A.n)
        Bx, By = orc.apply(O.BCO, x), orc.apply(O.BCO, y)
        assert abs(x @ By - y @ Bx) <= 1e-12 * abs(x @ By) + 1e-14 * np.linalg.norm(x) * np.linalg.norm(By)
        assert x @ Bx > 0


def test_status_codes():
    p = inputs.small_3d(6, 5, 4, seed=1)
    A = O.tpfa_problem(p)
    orc = O.Oracle(A, coarse_max=12)
    b = p.rhs()
    r = orc.pcg(b, op=O.I, tol=1e-14, maxit=3)
    assert r["status"] == 3 and r["iters"] == 3
    r = orc.pcg(np.zeros(A.n), op=O.BCO, tol=1e-6, maxit=10)
    assert r["status"] == 0 and r["iters"] == 0 and not r["x"].any()
    bad = b.copy()
    bad[3] = np.nan
    r = orc.pcg(bad, op=O.BCO, tol=1e-6, maxit=10)
    assert r["status"] == 4


def test_colour_ordered_ic0_is_ic0_of_permuted_matrix(small3d):
    p, A, _, D = small3d
    orc = O.Oracle(A, coarse_max=20, ic_colour_order=True)
    _, colour = orc.level_cf_colour(0)
    order = np.concatenate([np.where(colour == c)[0] for c in range(colour.max() + 1)])
    Dp = D[np.ix_(order, order)]
    B = dense_op(lambda v: orc.apply(O.B, v), A.n)
    Bp = B[np.ix_(order, order)]
    # (L U) of the permuted matrix equals it on its pattern and L U is lower x upper
    LU = np.linalg.inv(Bp)
    pat = Dp != 0
    assert rel(LU[pat], Dp[pat]) < 1e-11
    r = orc.pcg(p.rhs(), op=O.BCO, tol=1e-10, maxit=200)
    assert r["status"] == 0


def test_fine_grid_colouring_is_red_black(small3d):
    """The pattern graph of a structured grid is bipartite: colour = (i + j + k) mod 2."""
    p, _, orc, _ = small3d
    _, colour = orc.level_cf_colour(0)
    idx = np.arange(p.n)
    i, j, k = idx % p.nx, (idx // p.nx) % p.ny, idx // (p.nx * p.ny)
    assert np.array_equal(colour, (i + j + k) % 2)
    assert orc.level_sizes(0)["ncolours"] == 2


# --------------------------------------------------------------------------------------------
# Adjoint gradient through the assembly: dJ/dlog k = -lambda^T (dA/dlog k) p
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dirichlet", [inputs.FACE_X0, inputs.FACE_X0 | inputs.FACE_Z1])
def test_adjoint_gradient_matches_central_differences(dirichlet):
    p = inputs.small_3d(6, 5, 4, seed=31, dirichlet=dirichlet)
    wells = [[p.idx(1, 1, k) for k in range(p.nz)], [p.idx(4, 3, k) for k in range(p.nz)]]
    p.wells = [(c, 1.0 / p.nz) for c in wells[0]] + [(c, -1.0 / p.nz) for c in wells[1]]
    d = np.array([0.3, -0.2])
    q = p.rhs()

    def J(logk):   # independent of the oracle's solver: dense solve of the oracle's assembly
        A = O.tpfa(p.nx, p.ny, p.nz, logk, p.kz_ratio, p.dirichlet).to_dense()
        x = np.linalg.solve(A, q)
        r = O.well_means(x, wells) - d
        return 0.5 * r @ r

    A = O.tpfa_problem(p)
    j0, g = O.misfit_gradient(A, p, p.logk, wells, d, orc=O.Oracle(A, coarse_max=8))
    assert abs(j0 - J(p.logk)) <= 1e-10 * abs(j0)
    h = 1e-5
    fd = np.zeros(p.n)
    for c in range(p.n):
        e = np.zeros(p.n)
        e[c] = h
        fd[c] = (J(p.logk + e) - J(p.logk - e)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * np.max(np.abs(g))


def test_gradient_contraction_is_bilinear_form_of_dA():
    """g_c = -lambda^T (dA/dtheta_c) p with dA/dtheta_c taken by differencing the dense assembly."""
    p = inputs.small_3d(4, 3, 3, seed=5)
    lam = inputs.random_vector(p.n, seed=1)
    x = inputs.random_vector(p.n, seed=2)
    g = O.tpfa_gradient(p.nx, p.ny, p.nz, p.logk, p.kz_ratio, p.dirichlet, lam, x)
    h = 1e-6
    for c in range(p.n):
        e = np.zeros(p.n)
        e[c] = h
        dA = (O.tpfa(p.nx, p.ny, p.nz, p.logk + e, p.kz_ratio, p.dirichlet).to_dense()
              - O.tpfa(p.nx, p.ny, p.nz, p.logk - e, p.kz_ratio, p.dirichlet).to_dense()) / (2 * h)
        assert abs(g[c] + lam @ dA @ x) <= 1e-7 * (1 + abs(g[c]))
