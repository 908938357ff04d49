"""Host-side parity of the library (no GPU): connectivity, RCM, colouring and
edge order bit-exact against the oracle; node positions and the FP64 block
precompute (reference-operator form of Sec. 2.4) against the oracle's
physical-coordinate quadrature."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import basis as OB
from oracle import fields as OF
from oracle import mesh as OM
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def host_op(N, p, seed=0):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return dgsl.Operator(xy, tri, per, p, host_only=True), (xy, tri, per)


@pytest.mark.parametrize("N,seed", [(3, 0), (5, 1), (16, 2), (33, 3)])
def test_maps_bit_exact(dgsl_lib, N, seed):
    op, (xy, tri, per) = host_op(N, 1, seed)
    m = op.maps()
    c = OM.connectivity(xy, tri, per)
    perm = OM.rcm_order(c)
    colour, eperm, offs = OM.colouring(c, perm)
    np.testing.assert_array_equal(m["edge_vtx"], c.edge_vtx)
    np.testing.assert_array_equal(m["lr"], c.lr)
    np.testing.assert_array_equal(m["loc"], c.loc)
    np.testing.assert_array_equal(m["shift"], c.shift)
    np.testing.assert_array_equal(m["tri_edge"], c.tri_edge)
    np.testing.assert_array_equal(m["perm"], perm)
    np.testing.assert_array_equal(m["colour"], colour)
    np.testing.assert_array_equal(m["edge_perm"], eperm)
    np.testing.assert_array_equal(m["colour_offsets"], offs)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_node_coordinates(dgsl_lib, p):
    op, (xy, tri, per) = host_op(6, p, 4)
    m = op.maps()
    c = OM.connectivity(xy, tri, per)
    main = op.node_coords(0).reshape(op.n_tri, op.n_phi, 2)
    np.testing.assert_allclose(main, OF.main_nodes(c, p)[m["perm"]], rtol=0, atol=1e-15)
    dual = op.node_coords(1).reshape(op.n_edge, op.n_psi, 2)
    np.testing.assert_allclose(dual, OF.dual_nodes(c, p)[m["edge_perm"]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_blocks_match_oracle(dgsl_lib, p):
    op, (xy, tri, per) = host_op(5, p, 6)
    m = op.maps()
    G, Minv, Mref, area = op.blocks()
    bl = OA.assemble(xy, tri, per, p)
    L, R = OB.dual_maps(p)
    ep = m["edge_perm"]
    scale = np.abs(bl.Q).max()
    for s, mp in enumerate([L, R]):
        # library G[e][s][c][m][k] = Q_{s,j}[map_s(m), k, c], j = edge_perm[e]
        want = np.moveaxis(bl.Q[ep, s][:, mp, :, :], -1, 1)
        np.testing.assert_allclose(G[:, s], want, rtol=0, atol=1e-13 * scale)
    mi = OP.dual_mass_inverse(bl)[ep]
    np.testing.assert_allclose(Minv, mi, rtol=1e-11, atol=1e-11 * np.abs(mi).max())
    np.testing.assert_allclose(area, bl.area2[m["perm"]], rtol=1e-15)
    mb = bl.Mbar[m["perm"][0]]
    np.testing.assert_allclose(Mref * area[0], mb, rtol=1e-13, atol=1e-14 * np.abs(mb).max())


def test_bad_inputs_rejected(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(4, 0)
    with pytest.raises(dgsl.DgslError) as e:
        dgsl.Operator(xy, tri, per, 5, host_only=True)
    assert e.value.code == dgsl.EINVAL
    bad = tri.copy()
    bad[3] = bad[3][::-1]
    with pytest.raises(dgsl.DgslError) as e:
        dgsl.Operator(xy, bad, per, 2, host_only=True)
    assert e.value.code == dgsl.EMESH
    xy2, tri2, per2 = synth.jittered_periodic_mesh(2, 0)
    with pytest.raises(dgsl.DgslError) as e:
        dgsl.Operator(xy2, tri2, per2, 1, host_only=True)
    assert e.value.code == dgsl.EMESH
    with pytest.raises(dgsl.DgslError) as e:
        dgsl.Operator(xy, tri, [0.0, 1.0], 1, host_only=True)
    assert e.value.code == dgsl.EINVAL
    op = dgsl.Operator(xy, tri, per, 1, host_only=True)
    with pytest.raises(dgsl.DgslError) as e:
        import torch
        x = torch.zeros(op.n_dof, dtype=torch.float64)
        dgsl.load().dgsl_apply_schur(op.h, 0, 1.0, x.data_ptr() or 8, x.data_ptr() or 8, 1, None)
        dgsl._check(dgsl.load().dgsl_apply_schur(op.h, 0, 1.0, 8, 8, 1, None))
    assert e.value.code == dgsl.ENODEVICE


def test_sl_quadrature_matches_the_oracle_rule(dgsl_lib):
    """dgsl_sl_quadrature (host call): the collapsed Gauss-Legendre rule of
    the semi-Lagrangian projection, point for point the oracle's."""
    from oracle import sl as SL
    from paper_2401_17806_gb300 import dgsl
    for p in (1, 2, 3, 4):
        pts, w = dgsl.sl_quadrature(p)
        po, wo = SL.quadrature(p)
        assert pts.shape == ((p + 1) ** 2, 2)
        np.testing.assert_allclose(pts, po, rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, wo, rtol=0, atol=1e-15)
    with pytest.raises(dgsl.DgslError):
        dgsl.sl_quadrature(5)


@pytest.mark.parametrize("N,seed", [(3, 0), (7, 1), (20, 2)])
def test_sl_tables_bit_exact(dgsl_lib, N, seed):
    """The walk's neighbour table, packed back indices and frame translations
    (Sec. 2.5) equal the oracle's, bit for bit, after the RCM renumbering."""
    from oracle import sl as SL
    op, (xy, tri, per) = host_op(N, 2, seed)
    nbr, trans = op.sl_tables()
    perm = op.maps()["perm"]
    c = OM.connectivity(xy, tri, per)
    nbr_o, trans_o, back_o = SL.frames(c, per)
    for ti in range(op.n_tri):
        t = perm[ti]
        for k in range(3):
            assert perm[nbr[ti, k]] == nbr_o[t, k]
            assert (int(nbr[ti, 3]) >> (2 * k)) & 3 == back_o[t, k]
        np.testing.assert_array_equal(trans[ti], trans_o[t])
    assert (nbr[:, 3] >> 6).max() == 0  # nothing above the three 2-bit fields


def test_device_calls_reject_host_only_operators(dgsl_lib):
    """The transport and time-step entries check the operator before they touch
    any pointer: on a host-only operator each returns DGSL_ENODEVICE (the
    pointers below are never dereferenced)."""
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(4, 0)
    op = dgsl.Operator(xy, tri, per, 2, host_only=True)
    lib = dgsl.load()
    fake = 8
    codes = [
        lib.dgsl_sl_transport(op.h, 0.1, fake, None, None, 0, None, None, None, None),
        lib.dgsl_sl_transport_imex(op.h, 1, 0.1, fake, None, None, 0, None, None, None, None),
        lib.dgsl_advdiff_step(op.h, 1, 0.1, 0.01, fake, fake, fake, None, None, None),
        lib.dgsl_ns_step(op.h, 0.1, 0.01, fake, fake, None, None, None, None),
        lib.dgsl_ns_imex_step(op.h, 1, 0.1, 0.01, fake, fake, None, None, None, None),
    ]
    assert codes == [dgsl.ENODEVICE] * 5
    nbr, trans = op.sl_tables()  # the host query works on a host-only operator
    assert nbr.shape == (op.n_tri, 4) and np.all(np.abs(trans) <= 1.0)
