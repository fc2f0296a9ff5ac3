"""The library's ray launch (host code of the large-scene mode, through the
C ABI with no device: rt_candidates_mesh) against the oracle's own
implementation of the same rule: identical candidate lists for an empty box
and for a small office at several ray counts and orders."""
import numpy as np
import pytest

from paper_2310_10578_gb300 import scenes


@pytest.fixture(scope="module")
def creep():
    from paper_2310_10578_gb300 import creep as c
    c.load()
    return c


@pytest.mark.parametrize("n_rays,order", [(997, 3), (4096, 3), (300, 1), (2000, 2)])
def test_host_ray_launch_equals_oracle(creep, oracle_mod, n_rays, order):
    office = scenes.office(n_rooms=(2, 2), n_furn=40, n_cyl=6, n_sph=3, n_tx=1, nx=4, ny=4)
    tri, face = scenes.box_triangles(10.0, 8.0, 3.0)
    box = scenes.Scene(tri, face, np.zeros((0, 6)), (1.0, 1.0, 2.0), (0, 0, 1.0), [2.4e9],
                       np.zeros((1, 3), dtype=np.float32), "box")
    for sc in (box, office):
        got = creep.candidates_mesh(sc.tri, sc.tri_face, sc.tx, n_rays, order)
        ref = oracle_mod.candidates(sc, n_rays, order)
        assert np.array_equal(got, ref), (sc.name, len(got), len(ref))
        assert len(got) > 0 and (got >= 0).sum(1).max() == order


def test_host_ray_launch_errors(creep):
    tri, face = scenes.box_triangles(10.0, 8.0, 3.0)
    for args in ((tri, face, (1.0, 1.0, 2.0), 0, 3), (tri, face, (1.0, 1.0, 2.0), 100, 4),
                 (tri, face, (1.0, 1.0, 2.0), (1 << 24) + 1, 3)):
        with pytest.raises(creep.CreepError) as e:
            creep.candidates_mesh(*args)
        assert e.value.code == creep.RT_ERR_ARG
