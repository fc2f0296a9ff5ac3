"""The office generator's recipe: triangle and face counts, closed boxes,
bodies apart from each other and from the transmitters, transmitters off
every face plane and above the furniture, the receiver grid."""
import numpy as np

from paper_2310_10578_gb300 import scenes


def test_office_recipe():
    sc = scenes.office(n_rooms=(4, 3), n_furn=300, n_cyl=20, n_sph=5, n_tx=4, nx=50, ny=40)
    nrx, nry = 4, 3
    walls = 2 * ((nry - 1) * nrx + (nrx - 1) * nry)
    n_box = 1 + walls + 300
    assert sc.tri.shape == (12 * n_box, 3, 3)
    assert sc.tri_face.max() + 1 == 6 * n_box
    assert np.all(np.bincount(sc.tri_face) == 2)                # two triangles a face
    # every box closed: 6 axis-aligned faces, each coplanar pair of triangles
    for f in range(0, 6 * n_box, 97):
        t = sc.tri[sc.tri_face == f].reshape(-1, 3)
        spread = t.max(0) - t.min(0)
        assert np.sum(spread == 0) == 1                          # flat along exactly one axis
    lx, ly = 4 * 5.0, 3 * 4.0
    assert sc.tri[..., 0].min() == 0 and sc.tri[..., 0].max() == lx and sc.tri[..., 2].max() == 3.0
    cyl = sc.bodies[sc.bodies[:, 0] == scenes.BODY_CYLINDER]
    sph = sc.bodies[sc.bodies[:, 0] == scenes.BODY_SPHERE]
    assert len(cyl) == 20 and len(sph) == 5
    assert np.all((cyl[:, 4] >= 0.15) & (cyl[:, 4] <= 0.25)) and np.all((sph[:, 4] >= 0.1) & (sph[:, 4] <= 0.4))
    for i in range(len(cyl)):
        for j in range(i + 1, len(cyl)):
            assert np.hypot(*(cyl[i, 1:3] - cyl[j, 1:3])) >= cyl[i, 4] + cyl[j, 4] + 0.05 - 1e-6
    for s in sph:
        assert np.all(np.hypot(cyl[:, 1] - s[1], cyl[:, 2] - s[2]) >= cyl[:, 4] + s[4] + 0.05 - 1e-6)
    assert sc.txs.shape == (4, 3) and np.all(sc.txs[:, 2] == 2.5)
    furn_top = sc.tri[12 * (1 + walls):, :, 2].max()
    assert furn_top <= 2.0 + 1e-6                                # transmitters above every piece of furniture
    planes = {(ax, float(v)) for t in sc.tri for ax in range(3) if np.all(t[:, ax] == t[0, ax]) for v in [t[0, ax]]}
    for t in sc.txs:
        assert all((ax, float(t[ax])) not in planes for ax in range(3))
        for b in sc.bodies:
            d = np.linalg.norm(t - b[1:4]) if b[0] == scenes.BODY_SPHERE else np.hypot(*(t[:2] - b[1:3]))
            assert d > b[4]
    assert sc.n_rx == 50 * 40 and np.all(sc.rx[:, 2] == np.float32(1.2))
    assert 0 < sc.rx[:, 0].min() and sc.rx[:, 0].max() < lx and sc.rx[:, 1].max() < ly


def test_office_default_size():
    sc = scenes.office(nx=10, ny=10)
    assert 190_000 <= sc.tri.shape[0] <= 200_000 and sc.bodies.shape[0] == 110 and len(sc.txs) == 4
