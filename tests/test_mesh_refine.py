"""The library's uniform refinement (the paper's uniformrefine, Sec. 2.1) on
the CPU: counts, orientation and areas, the paper's statement that two
refinements of the printed initial mesh give the 8x8 split-square mesh, and
agreement with the oracle's refinement as sets of triangles and boundary
edges (the node numbering of the two may differ)."""
import numpy as np
import pytest

import oracle as O
from paper_1502_02941_gb300 import dg as D
from paper_1502_02941_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__ as g
    g.build()
    return D.load()


def _tris(nodes, elems):
    """Triangles as a set of (cyclically canonical) coordinate triples."""
    out = set()
    for t in elems:
        pts = [tuple(np.round(nodes[v], 12)) for v in t]
        r = min(range(3), key=lambda i: pts[i])
        out.add(tuple(pts[(r + i) % 3] for i in range(3)))
    return out


def _edges(nodes, e, directed=True):
    out = set()
    for a, b in e:
        pa, pb = tuple(np.round(nodes[a], 12)), tuple(np.round(nodes[b], 12))
        out.add((pa, pb) if directed else tuple(sorted((pa, pb))))
    return out


def _area(nodes, elems):
    v = nodes[elems]
    return 0.5 * ((v[:, 1, 0] - v[:, 0, 0]) * (v[:, 2, 1] - v[:, 0, 1]) -
                  (v[:, 1, 1] - v[:, 0, 1]) * (v[:, 2, 0] - v[:, 0, 0]))


def _lshape():
    m = W.lshape_mesh()
    return m.nodes, m.elems, m.dirichlet, m.neumann


def test_two_refinements_of_the_printed_mesh_give_the_8x8_mesh():
    m = (W.FIXTURE_NODES, W.FIXTURE_ELEMS, W.FIXTURE_DIRICHLET, np.zeros((0, 2), np.int32))
    for _ in range(2):
        m = D.dg_mesh_refine(*m)
    s = W.structured_mesh(8)
    assert _tris(m[0], m[1]) == _tris(s.nodes, s.elems)
    assert _edges(m[0], m[2], directed=False) == _edges(s.nodes, s.dirichlet, directed=False)
    assert len(m[3]) == 0 and m[0].shape[0] == 81


@pytest.mark.parametrize("mesh", ["perturbed", "lshape"])
def test_refinement_matches_the_oracle(mesh):
    if mesh == "perturbed":
        p = W.perturbed_mesh(5, seed=4, neumann_sides=("top", "right"))
        m = (p.nodes, p.elems, p.dirichlet, p.neumann)
    else:
        m = _lshape()
    r = D.dg_mesh_refine(*m)
    o = O.refine(*m)
    nv, ne = m[0].shape[0], m[1].shape[0]
    nedges = len({(min(t[f], t[(f + 1) % 3]), max(t[f], t[(f + 1) % 3])) for t in m[1] for f in range(3)})
    assert r[0].shape[0] == nv + nedges and r[1].shape[0] == 4 * ne
    assert (r[2].shape[0], r[3].shape[0]) == (2 * m[2].shape[0], 2 * m[3].shape[0])
    np.testing.assert_array_equal(r[0][:nv], m[0])
    assert _tris(r[0], r[1]) == _tris(o[0], o[1])
    assert _edges(r[0], r[2]) == _edges(o[0], o[2]) and _edges(r[0], r[3]) == _edges(o[0], o[3])
    # counter-clockwise children, each a quarter of its parent
    a0, a1 = _area(m[0], m[1]), _area(r[0], r[1])
    assert (a1 > 0).all()
    np.testing.assert_allclose(a1.reshape(-1, 4), np.repeat(a0[:, None] / 4, 4, 1), rtol=1e-13)
    # the refined arrays form a valid mesh for the oracle's getmesh as well
    om = O.make_mesh(*r)
    assert om.ne == 4 * ne and om.n_bedges == len(r[2]) + len(r[3])


def test_refinement_rejects_bad_input():
    m = W.structured_mesh(2)
    bad = m.elems.copy(); bad[0, 0] = 99
    with pytest.raises(D.DGError) as e:
        D.dg_mesh_refine(m.nodes, bad, m.dirichlet, m.neumann)
    assert e.value.status == D.DG_ERR_MESH
    bd = m.dirichlet.copy(); bd[0] = (0, 8)      # a diagonal of the square, no element edge
    with pytest.raises(D.DGError) as e:
        D.dg_mesh_refine(m.nodes, m.elems, bd, m.neumann)
    assert e.value.status == D.DG_ERR_MESH


@pytest.mark.parametrize("mesh", ["square", "lshape"])
def test_repeated_refinement_counts_and_euler_characteristic(mesh):
    """Each refinement: T' = 4T, E' = 2E + 3T, V' = V + E, boundary edges double;
    so V - E + T (1 for a simply connected polygon) is kept."""
    if mesh == "square":
        m = W.structured_mesh(3, neumann_sides=("left",))
        arrays = (m.nodes, m.elems, m.dirichlet, m.neumann)
    else:
        m = W.lshape_mesh()
        arrays = (m.nodes, m.elems, m.dirichlet, m.neumann)

    def counts(a):
        edges = {tuple(sorted((int(t[f]), int(t[(f + 1) % 3])))) for t in a[1] for f in range(3)}
        used = len(np.unique(a[1]))          # vertices of the triangulation (unused nodes are kept)
        return used, len(edges), a[1].shape[0], a[2].shape[0] + a[3].shape[0]
    V, E, T, B = counts(arrays)
    assert V - E + T == 1
    for _ in range(3):
        arrays = D.dg_mesh_refine(*arrays)
        V2, E2, T2, B2 = counts(arrays)
        assert (V2, E2, T2, B2) == (V + E, 2 * E + 3 * T, 4 * T, 2 * B)
        V, E, T, B = V2, E2, T2, B2
        assert V - E + T == 1
