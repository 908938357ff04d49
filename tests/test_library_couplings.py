"""Host-side parity of the assembled couplings (no GPU): the FP64 values the
device copies are made from equal, entry by entry, the oracle's separately
assembled K = G^T Mhat^-1 G (eq. pressure_final), and they are exactly
symmetric (every pair of transposed entries bit for bit, as CG assumes)."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def host_op(N, p, seed):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return dgsl.Operator(xy, tri, per, p, host_only=True), (xy, tri, per)


@pytest.mark.parametrize("N,p,seed", [(4, 1, 0), (5, 2, 1), (6, 3, 2), (5, 4, 3)])
def test_couplings_match_the_oracle(dgsl_lib, N, p, seed):
    op, (xy, tri, per) = host_op(N, p, seed)
    Kd, Ko, nbr = op.couplings()
    perm = op.maps()["perm"]
    K = OP.Operators(OA.assemble(xy, tri, per, p)).schur_matrix(1.0).toarray()
    n = op.n_phi
    L = np.zeros_like(K)
    for i in range(op.n_tri):
        rows = slice(perm[i] * n, perm[i] * n + n)
        L[rows, rows] += Kd[i]
        for e in range(3):
            j = nbr[i, e]
            L[rows, perm[j] * n:perm[j] * n + n] += Ko[i, e]
    scale = np.abs(K).max()
    assert np.abs(L - K).max() <= 1e-13 * scale, np.abs(L - K).max() / scale
    # the stored operator annihilates constants to rounding (S 1 = 0)
    assert np.abs(L.sum(axis=1)).max() <= 1e-13 * scale * n


@pytest.mark.parametrize("N,p,seed", [(3, 2, 0), (7, 3, 5), (6, 4, 1)])
def test_couplings_exactly_symmetric(dgsl_lib, N, p, seed):
    op, _ = host_op(N, p, seed)
    Kd, Ko, nbr = op.couplings()
    for i in range(op.n_tri):
        assert np.array_equal(Kd[i], Kd[i].T)
        for e in range(3):
            j = nbr[i, e]
            back = [f for f in range(3) if nbr[j, f] == i]
            assert len(back) == 1  # one shared edge per neighbour pair on these meshes
            assert np.array_equal(Ko[i, e], Ko[j, back[0]].T), (i, e, j)


def test_couplings_need_the_blocks(dgsl_lib):
    import ctypes as C
    from paper_2401_17806_gb300 import dgsl
    assert dgsl.load().dgsl_query_couplings(None, None, None, None) == dgsl.EINVAL
    op, _ = host_op(3, 1, 0)
    kd = np.zeros((op.n_tri, 3, 3))
    assert dgsl.load().dgsl_query_couplings(op.h, C.c_void_p(kd.ctypes.data), None, None) == dgsl.OK
