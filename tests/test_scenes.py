"""The seeded synthetic workloads: deterministic, well-formed, and with the sizes they state.

Both the CUDA path and the oracle take their inputs from these generators, so
a generator that drifted between calls, or produced a malformed mesh, would
show up as a parity failure with no bug in either side.
"""
import numpy as np
import pytest

from paper_2012_03939_gb300 import scenes as S

SMALL = ["tiny", "edges", "env", "color_bleed"]


@pytest.mark.parametrize("name", SMALL)
def test_workload_is_deterministic_and_well_formed(name):
    a, b = S.make(name), S.make(name)
    np.testing.assert_array_equal(a.vertices, b.vertices)
    np.testing.assert_array_equal(a.faces, b.faces)
    np.testing.assert_array_equal(a.face_params, b.face_params)
    assert a.vertices.dtype == np.float32 and a.faces.dtype == np.int32
    assert np.isfinite(a.vertices).all() and np.isfinite(a.face_params).all()
    F = a.faces
    assert F.min() >= 0 and F.max() < len(a.vertices)
    assert np.all((F[:, 0] != F[:, 1]) & (F[:, 1] != F[:, 2]) & (F[:, 0] != F[:, 2]))
    area = np.linalg.norm(np.cross(a.vertices[F[:, 1]] - a.vertices[F[:, 0]],
                                   a.vertices[F[:, 2]] - a.vertices[F[:, 0]]), axis=1)
    assert area.min() > 0
    n_tex = len(F) * (a.color_res + 1) * (a.color_res + 2) // 2
    assert a.face_params.shape == (n_tex, 5)
    kd, ks, alpha = a.face_params[:, :3], a.face_params[:, 3], a.face_params[:, 4]
    assert kd.min() >= 0 and kd.max() <= 1 and ks.min() >= 0 and alpha.min() > 0
    # views tile the image rows without gaps or overlaps
    off = 0
    for v in a.views:
        assert v.pixel_offset == off and v.width > 0 and v.height > 0 and v.spp > 0
        off += v.width * v.height
    assert a.n_pixels == off


def test_stated_sizes():
    assert len(S.make("tiny").faces) == 320
    assert len(S.make("edges").faces) == 5120
    assert len(S.make("env").faces) == 50_000
    assert len(S.make("color_bleed").faces) == 384
    env = S.make("env")
    assert env.env.shape == (128, 256, 3) and len(env.views) == 32


def test_small_variant_keeps_the_mesh_and_packs_views():
    sc = S.make("edges")
    sv = S.small_variant(sc, n_views=3, max_res=20, spp=2)
    np.testing.assert_array_equal(sv.vertices, sc.vertices)
    assert len(sv.views) == 3 and all(v.width <= 20 and v.height <= 20 and v.spp == 2 for v in sv.views)
    assert [v.pixel_offset for v in sv.views] == [0, sv.views[0].width * sv.views[0].height,
                                                   sum(v.width * v.height for v in sv.views[:2])]
