"""Pins of the oracle's two-level multigrid preconditioner (an extension: the
paper runs CG unpreconditioned).  Each ingredient is checked against what
fixes it independently of the code:
 - the P1 prolongation interpolates every linear function exactly on every
   triangle (nodal interpolation) and reproduces constants;
 - the vertex numbering is a first-appearance permutation;
 - the Galerkin coarse operator keeps the pressure operator's nullspace
   span{1}, is symmetric positive semidefinite with exactly one zero
   eigenvalue, and its pattern holds every structural nonzero;
 - the greedy aggregation gives hand-computed aggregates on small graphs,
   and the vertex graph joins exactly the vertices that share a triangle;
 - the smoothed prolongation reproduces constants on the pressure levels;
 - the V-cycle contracts the coarse problem by a mesh-independent factor;
 - the preconditioner is symmetric and positive definite;
 - PCG with it reaches the direct solution, in an iteration count that stays
   flat as the mesh is refined (where block-Jacobi PCG doubles)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as OA
from oracle import basis as B
from oracle import mesh as OM
from oracle import multigrid as MG
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def _setup(N, p, seed=2):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    conn = OM.connectivity(xy, tri, per)
    ops = OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))
    return conn, tri, ops


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_p1_prolongation_interpolates_linear_functions(p):
    conn, tri, ops = _setup(5, p)
    cvid, nv = MG.vertex_numbering(conn, tri)
    Pc = MG.p1_prolongation(cvid, nv, p)
    np.testing.assert_allclose(Pc @ np.ones(nv), 1.0, rtol=0, atol=1e-15)
    f = lambda x, y: 0.3 - 1.7 * x + 2.9 * y
    X = B.triangle_points(conn.tri_xy, B.nodes(p))          # nodes in each triangle's frame
    nphi = B.n_phi(p)
    for t in range(conn.n_tri):
        v = np.zeros(nv)
        v[cvid[t]] = f(conn.tri_xy[t, :, 0], conn.tri_xy[t, :, 1])
        got = (Pc @ v)[t * nphi:(t + 1) * nphi]
        np.testing.assert_allclose(got, f(X[t, :, 0], X[t, :, 1]), rtol=0, atol=1e-13)


def test_vertex_numbering_is_first_appearance():
    conn, tri, _ = _setup(6, 1)
    cvid, nv = MG.vertex_numbering(conn, tri)
    assert nv == 36 and sorted(set(cvid.ravel().tolist())) == list(range(36))
    perm = OM.rcm_order(conn)
    seen = []
    for t in perm:
        for m in range(3):
            if cvid[t, m] not in seen:
                assert cvid[t, m] == len(seen)
                seen.append(cvid[t, m])


@pytest.mark.parametrize("p", [1, 3])
def test_coarse_operator_nullspace_and_pattern(p):
    conn, tri, ops = _setup(4, p)
    S = ops.schur_matrix(1e-2)
    cvid, nv = MG.vertex_numbering(conn, tri)
    Pc = MG.p1_prolongation(cvid, nv, p)
    pat = MG.coarse_pattern(conn, cvid, nv)
    struct = (abs(Pc).T @ (abs(S) > 0).astype(float) @ abs(Pc)) != 0
    assert (struct.astype(int) - struct.multiply(pat).astype(int)).nnz == 0     # pattern holds every nonzero
    assert (pat != pat.T).nnz == 0
    A0 = MG.on_pattern(Pc.T @ S @ Pc, pat).toarray()
    np.testing.assert_allclose(A0, A0.T, rtol=0, atol=1e-14 * np.abs(A0).max())
    assert np.abs(A0 @ np.ones(nv)).max() <= 1e-13 * np.abs(A0).max()
    ev = np.linalg.eigvalsh(A0)
    assert abs(ev[0]) <= 1e-12 * ev[-1] < ev[1]


def test_aggregation_hand_examples():
    # chain 0-1-...-9 (closed neighbourhoods): roots 0, 3, 6, 9
    n = 10
    rows = [i for i in range(n) for j in (i - 1, i, i + 1) if 0 <= j < n]
    cols = [j for i in range(n) for j in (i - 1, i, i + 1) if 0 <= j < n]
    chain = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    agg, na = MG.aggregate(chain)
    assert na == 4 and agg.tolist() == [0, 0, 1, 1, 1, 2, 2, 2, 3, 3]
    # edges 0-1, 1-2, 2-3, 3-4, 1-3: roots 0 and 4, node 2 joins its first
    # aggregated neighbour (1, aggregate 0) in pass 2
    E = [(0, 1), (1, 2), (2, 3), (3, 4), (1, 3)]
    rows = list(range(5)) + [a for a, b in E] + [b for a, b in E]
    cols = list(range(5)) + [b for a, b in E] + [a for a, b in E]
    g = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(5, 5))
    agg, na = MG.aggregate(g)
    assert na == 2 and agg.tolist() == [0, 0, 0, 1, 1]
    # an isolated node becomes its own aggregate
    g = sp.identity(3, format="csr")
    agg, na = MG.aggregate(g)
    assert na == 3 and agg.tolist() == [0, 1, 2]


def test_vertex_graph_is_the_mesh_edges():
    conn, tri, ops = _setup(6, 1)
    cvid, nv = MG.vertex_numbering(conn, tri)
    G = MG.vertex_graph(cvid, nv)
    edges = {tuple(sorted((cvid[t, a], cvid[t, b]))) for t in range(conn.n_tri) for a in range(3) for b in range(3)}
    got = {tuple(sorted((i, j))) for i, j in zip(*G.nonzero())}
    assert got == edges
    # a periodic triangulation: every vertex has 6 neighbours on average
    assert (G.nnz - nv) == 2 * 3 * nv


def test_hierarchy_keeps_constants_and_coarsens():
    conn, tri, ops = _setup(32, 1)
    M = MG.TwoLevel(ops.schur_matrix(1e-3), conn, tri, 1, singular=True)
    sizes = [L.A.shape[0] for L in M.levels]
    assert sizes[0] == 32 * 32 and sizes[-1] <= MG.COARSEST and len(sizes) >= 2
    for L in M.levels[:-1]:
        assert L.agg.min() == 0 and len(set(L.agg.tolist())) == L.P.shape[1]
        np.testing.assert_allclose(L.P @ np.ones(L.P.shape[1]), 1.0, rtol=0, atol=1e-13)
        assert np.abs(L.A @ np.ones(L.A.shape[0])).max() <= 1e-12 * np.abs(L.A).max()


def test_vcycle_preconditions_the_coarse_problem_independently_of_the_mesh():
    """CG on A_0 preconditioned by one V-cycle: a mesh-independent iteration
    count (and a real multilevel cycle at every size)."""
    its = []
    for N in (32, 64, 128):
        conn, tri, ops = _setup(N, 1)
        M = MG.TwoLevel(ops.schur_matrix(1e-3), conn, tri, 1, singular=True)
        assert len(M.levels) >= 2
        A0 = M.levels[0].A
        b = synth.standard_normal(A0.shape[0], 3)
        _, it, _ = OP.pcg(lambda v: A0 @ v, b, lambda r: MG.vcycle(M.levels, r), tol=1e-10, mean_zero=True)
        its.append(it)
    assert max(its) <= 1.25 * min(its) and max(its) < 35, its


@pytest.mark.parametrize("kind", [0, 1])
def test_preconditioner_is_symmetric_positive_definite(kind):
    conn, tri, ops = _setup(8, 3)
    A = ops.schur_matrix(1e-3) if kind == 0 else ops.helmholtz_matrix(1e-3)
    M = MG.TwoLevel(A, conn, tri, 3, singular=kind == 0)
    u, v = synth.standard_normal(ops.n, 1), synth.standard_normal(ops.n, 2)
    if kind == 0:
        u, v = u - u.mean(), v - v.mean()
    a, b = u @ M(v), v @ M(u)
    assert abs(a - b) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(M(v))
    for s in range(5):
        w = synth.standard_normal(ops.n, 10 + s)
        if kind == 0:
            w -= w.mean()
        assert w @ M(w) > 0


@pytest.mark.parametrize("p", [1, 3])
def test_pcg_iterations_flat_under_refinement_and_direct_solution(p):
    its, bj = [], []
    for N in (16, 32, 64):
        conn, tri, ops = _setup(N, p)
        S = ops.schur_matrix(1e-3)
        M = MG.TwoLevel(S, conn, tri, p, singular=True)
        b = synth.standard_normal(ops.n, 1)
        x, it, _ = OP.pcg(lambda v: S @ v, b, M, tol=1e-10, mean_zero=True)
        its.append(it)
        if N == 32:
            assert np.linalg.norm(x - OP.schur_solve_direct(S, b)) <= 1e-8 * np.linalg.norm(x)
        if N in (16, 32):
            D = OP.block_jacobi_blocks(S, ops.nphi)
            bj.append(OP.pcg(lambda v: S @ v, b, lambda r: OP.apply_blocks(D, r), tol=1e-10, mean_zero=True)[1])
    # nearly mesh-independent: at most 15% more per doubling of N (block-Jacobi: 1.9x)
    assert all(b <= 1.15 * a for a, b in zip(its, its[1:])), its
    assert bj[1] >= 1.7 * bj[0] and its[-1] < bj[0] / 4, (its, bj)


def test_helmholtz_pcg_matches_direct():
    conn, tri, ops = _setup(24, 2)
    H = ops.helmholtz_matrix(1e-3)
    M = MG.TwoLevel(H, conn, tri, 2, singular=False)
    b = synth.standard_normal(ops.n, 5)
    x, it, _ = OP.pcg(lambda v: H @ v, b, M, tol=1e-11)
    assert it < 60
    xd = OP.direct_solve(H, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
