"""Failure paths of the C ABI, made on the host: injected allocation and copy faults.

Nothing here faults the GPU. The library's host-side hook (st_inject_fault)
makes one allocation or one host<->device copy report the error the CUDA call
would have returned, without calling it. Each test checks that the failing
call returns the documented status, leaks no device memory, and leaves the
scene usable: the same call succeeds afterwards and gives the image of a
scene that never failed.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2012_03939_gb300 import scenes as S

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ST_ERR_OOM, ST_ERR_CUDA = 2, 3


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03939_gb300 import build
    build.build()
    from paper_2012_03939_gb300 import st as _st
    _st.lib()
    yield _st
    _st.inject_fault("alloc", -1)
    _st.inject_fault("copy", -1)


def _sc():
    sc = S.tiny(res=40, spp=2)
    sc.views = S.ring_views(3, 40, 2)
    return sc


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _reference(st, sc, opts, backward=False):
    scene = st.Scene.from_scene(sc)
    out = _call(st, scene, sc, opts, backward)
    scene.close()
    return out


def _call(st, scene, sc, opts, backward):
    if not backward:
        return scene.render(sc.views, 2, 7, opts).cpu().numpy()
    w = torch.from_numpy(np.random.default_rng(1).normal(size=(sc.n_pixels, 3)).astype(np.float32)).cuda()
    dV, dF = scene.backward(sc.views, 2, 7, w, opts)
    return np.concatenate([dV.cpu().numpy().ravel(), dF.cpu().numpy().ravel()])


def _close_gradients(got, ref):
    # the gradient scatter ends in FP32 atomics whose order varies from call to call
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())


def _sweep(st, site, attempt, expect_status, limit=80):
    """attempt() after arming `site` at n = 0, 1, ...: every failure has the expected status, and some n
    lets the call through. Returns the number of failing events."""
    for n in range(limit):
        st.inject_fault(site, n)
        try:
            attempt()
        except st.StError as e:
            assert e.status == expect_status, (site, n, str(e))
            continue
        finally:
            st.inject_fault(site, -1)
        return n
    raise AssertionError("the call still failed after %d injected events" % limit)


@pytest.mark.parametrize("site,status", [("alloc", ST_ERR_OOM), ("copy", ST_ERR_CUDA)])
def test_scene_create_fails_cleanly_at_every_event(st, site, status):
    sc = _sc()
    ref = _reference(st, sc, None)
    free0 = _free_bytes()
    made = []

    def attempt():
        made.append(st.Scene.from_scene(sc))

    n = _sweep(st, site, attempt, status)
    assert n >= 3                       # a scene makes several allocations and uploads
    scene = made[-1]
    np.testing.assert_array_equal(scene.render(sc.views, 2, 7).cpu().numpy(), ref)
    scene.close()
    assert abs(_free_bytes() - free0) <= 8 << 20     # nothing leaked by the failed creates


@pytest.mark.parametrize("backward", [False, True])
@pytest.mark.parametrize("site,status", [("alloc", ST_ERR_OOM), ("copy", ST_ERR_CUDA)])
@pytest.mark.parametrize("mode", ["batched", "per_view"])
def test_calls_fail_cleanly_and_leave_the_scene_usable(st, site, status, backward, mode):
    # a fresh scene's first call allocates its wavefront buffers and per-call tables, so a fault can hit any
    # of them; after each failure the same call must succeed and match a scene that never failed
    sc = _sc()
    opts = st.make_opts(mode=mode, use_graph=1 if mode == "batched" else 0, edge_term=1 if backward else 0)
    ref = _reference(st, sc, opts, backward)
    free0 = _free_bytes()
    fails = 0
    for n in range(80):
        scene = st.Scene.from_scene(sc)
        st.inject_fault(site, n)
        try:
            _call(st, scene, sc, opts, backward)
            ok = True
        except st.StError as e:
            assert e.status == status, (n, str(e))
            ok = False
        finally:
            st.inject_fault(site, -1)
        got = _call(st, scene, sc, opts, backward)
        if backward:
            _close_gradients(got, ref)
        else:
            np.testing.assert_array_equal(got, ref)
        assert scene.stats()["device_error"] == 0
        scene.close()
        if ok:
            break
        fails += 1
    assert fails >= 1 and ok
    assert abs(_free_bytes() - free0) <= 8 << 20


@pytest.mark.parametrize("site,status", [("alloc", ST_ERR_OOM), ("copy", ST_ERR_CUDA)])
def test_list_builds_fail_cleanly(st, site, status):
    # a call of 2^20 primary rays under a point light builds the primary-visibility and the point-light lists:
    # each allocation or copy of its first call fails in turn; the same call then succeeds with the image of a
    # scene that never failed (the lists are built again, not reused half-made) and nothing leaks
    sc = S.tiny()
    sc.views = S.fibonacci_views(4, [256] * 4, [256] * 4, [4] * 4)
    opts = st.make_opts()
    ref = _reference(st, sc, opts)
    free0 = _free_bytes()
    fails = 0
    for n in range(120):
        scene = st.Scene.from_scene(sc)
        st.inject_fault(site, n)
        try:
            _call(st, scene, sc, opts, False)
            ok = True
        except st.StError as e:
            assert e.status == status, (n, str(e))
            ok = False
        finally:
            st.inject_fault(site, -1)
        np.testing.assert_array_equal(_call(st, scene, sc, opts, False), ref)
        assert scene.stats()["device_error"] == 0
        scene.close()
        if ok:
            break
        fails += 1
    assert fails >= 1 and ok
    assert abs(_free_bytes() - free0) <= 8 << 20


def test_growth_failure_keeps_no_stale_capacity(st):
    # a scene sized by a small call, then a larger call whose buffer growth fails at each allocation in turn:
    # the larger call succeeds on retry and matches a fresh scene
    sc = _sc()
    big = S.ring_views(5, 72, 3)
    big_sc = S.tiny(res=72, spp=3)
    big_sc.views = big
    ref = _reference(st, big_sc, st.make_opts(edge_term=1), backward=True)
    for n in range(40):
        scene = st.Scene.from_scene(sc)
        _call(st, scene, sc, st.make_opts(edge_term=1), True)
        st.inject_fault("alloc", n)
        try:
            _call(st, scene, big_sc, st.make_opts(edge_term=1), True)
            ok = True
        except st.StError as e:
            assert e.status == ST_ERR_OOM
            ok = False
        finally:
            st.inject_fault("alloc", -1)
        _close_gradients(_call(st, scene, big_sc, st.make_opts(edge_term=1), True), ref)
        scene.close()
        if ok:
            return
    raise AssertionError("growth still failing")


def test_statistics_readback_fault(st):
    sc = _sc()
    scene = st.Scene.from_scene(sc)
    scene.render(sc.views, 2, 7)
    st.inject_fault("copy", 0)
    with pytest.raises(st.StError) as e:
        scene.stats()
    assert e.value.status == ST_ERR_CUDA
    assert scene.stats()["device_error"] == 0
    scene.close()


def test_fault_from_the_environment_variable():
    # a process that cannot call st_inject_fault arms it through ST_FAULT
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import torch\n"
            "from paper_2012_03939_gb300 import scenes as S, st\n"
            "sc = S.tiny(res=16, spp=1)\n"
            "try:\n"
            "    st.Scene.from_scene(sc)\n"
            "    print('created')\n"
            "except st.StError as e:\n"
            "    print('status', e.status)\n" % ROOT)
    env = dict(os.environ, ST_FAULT="alloc:0")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "status %d" % ST_ERR_OOM in out.stdout, out.stdout
