"""Failure detection and asset export/import, without any GPU fault: every failure is made on
the host (an injected allocation failure, admission refusal, cancellation or slow request) or
is a bounded device loop that runs out (a BVH with a cycle, whose every index is in range),
and the context stays usable afterwards."""
import os
import subprocess
import sys
import time

import numpy as np
import pytest
import torch

from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tiny(res=48, views=1):
    from paper_2608_24109_b300.render import Renderer
    sc = scenes.config("tiny", res=res, views=views, n_direct=16)
    return sc, Renderer.from_scene(sc)


def _render_with(r, mesh, M):
    from paper_2608_24109_b300 import native as N
    out = torch.empty(r.image_shape(), device="cuda")
    N.exm_render_forward(r.ctx, mesh, M, r.env, r.cams, r.params, r.frame, out)
    return out


@pytest.fixture(autouse=True)
def _clear_faults():
    from paper_2608_24109_b300 import native as N
    yield
    for k in (N.FAULT_ALLOC, N.FAULT_ADMIT, N.FAULT_SLOW, N.FAULT_CANCEL, N.FAULT_CORRUPT):
        N.exm_debug_fault(k, 0)


# ------------------------------------------------------------------ assets

def test_asset_file_round_trip_renders_bit_for_bit(tmp_path):
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc, r = _tiny(64, 2)
    M = torch.as_tensor(sc.maps, device="cuda").to(torch.bfloat16)
    E = torch.as_tensor(sc.env, device="cuda")
    r.prepare_env(E)
    ref = _render_with(r, r.mesh, M).clone()
    vis = r.visbuf()
    path = tmp_path / "asset.exm"
    assets.save_asset(str(path), r.mesh, M, E)
    mesh, M2, E2 = assets.load_asset(str(path), r.ctx)
    assert torch.equal(M2, M) and torch.equal(E2, E)
    out = _render_with(r, mesh, M2)
    r.sync()
    assert torch.equal(out, ref) and torch.equal(r.visbuf(), vis)
    N.exm_mesh_destroy(mesh)
    r.close()


def _root_refs(secs, info):
    """The root's four child references in an exported 4-wide node section (node 0 is stored
    unskewed: after its six plane vectors in 128-byte nodes, after p and step.x in 64-byte ones)."""
    words = secs[4].view(np.int32).reshape(info.n_nodes, info.node_bytes // 4)
    return words[0, 24:28] if info.node_bytes == 128 else words[0, 4:8]


def test_bvh_with_a_cycle_ends_at_the_traversal_cap():
    """The root's node children are made the root again: every index stays in range, so the
    import accepts it; each ray then loops until the traversal stack or step cap ends it, the
    kernels return, exm_sync reports EXM_ERR_TRAVERSAL_LIMIT, and the context renders the
    intact mesh as before."""
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc, r = _tiny()
    M = torch.as_tensor(sc.maps, device="cuda")
    r.prepare_env(torch.as_tensor(sc.env, device="cuda"))
    ref = _render_with(r, r.mesh, M).clone()
    r.sync()
    info, secs = assets.export_mesh(r.mesh)
    refs = _root_refs(secs, info)
    refs[(refs >= 0) & (refs != 0x7FFFFFFF)] = 0
    bad = assets.import_mesh(r.ctx, info, secs)
    _render_with(r, bad, M)
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_TRAVERSAL_LIMIT
    N.exm_mesh_destroy(bad)
    out = _render_with(r, r.mesh, M)
    r.sync()
    assert torch.equal(out, ref)
    r.close()


def test_corrupt_asset_injector_gives_the_same_error():
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc, r = _tiny()
    M = torch.as_tensor(sc.maps, device="cuda")
    r.prepare_env(torch.as_tensor(sc.env, device="cuda"))
    info, secs = assets.export_mesh(r.mesh)
    N.exm_debug_fault(N.FAULT_CORRUPT, 1)
    bad = assets.import_mesh(r.ctx, info, secs)
    _render_with(r, bad, M)
    with pytest.raises(N.ExmError) as e:
        r.sync()
    assert e.value.code == N.EXM_ERR_TRAVERSAL_LIMIT
    good = assets.import_mesh(r.ctx, info, secs)  # the injection was used up
    _render_with(r, good, M)
    r.sync()
    N.exm_mesh_destroy(bad)
    N.exm_mesh_destroy(good)
    r.close()


@pytest.mark.parametrize("what", ["node_ref", "leaf_ref", "leaf_span", "face_index", "version", "node_count"])
def test_import_refuses_out_of_range_assets(what):
    from paper_2608_24109_b300 import assets
    from paper_2608_24109_b300 import native as N
    sc, r = _tiny()
    info, secs = assets.export_mesh(r.mesh)
    if what == "node_ref":
        _root_refs(secs, info)[0] = info.n_nodes + 5
    elif what == "leaf_ref":
        _root_refs(secs, info)[0] = ~(info.nf + 3)
    elif what == "leaf_span":   # a leaf of 4 records from the last one: past the end
        _root_refs(secs, info)[0] = ~((info.nf - 1) | (3 << 28))
    elif what == "node_count":   # more 4-wide nodes than a tree over nf leaves has
        info.n_nodes = info.nf
        secs[4] = np.zeros(info.nf * info.node_bytes, np.uint8)
        info.bytes[4] = secs[4].size
    elif what == "face_index":
        secs[1].view(np.int32)[7] = info.nv
    else:
        info.version = 99
    with pytest.raises(N.ExmError) as e:
        assets.import_mesh(r.ctx, info, secs)
    assert e.value.code == N.EXM_ERR_ARG
    r.close()


# ------------------------------------------------------------------ host-side injectors

def test_allocation_failure_is_reported_and_the_frame_recovers():
    from paper_2608_24109_b300 import native as N
    sc, r = _tiny()
    M = torch.as_tensor(sc.maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    sc2, r2 = _tiny()
    ref = r2.forward(M, E).clone()
    r2.sync()
    N.exm_debug_fault(N.FAULT_ALLOC, 1)  # the frame's first wavefront buffer
    with pytest.raises(N.ExmError) as e:
        r.forward(M, E)
    assert e.value.code == N.EXM_ERR_OOM
    g = torch.ones(r.image_shape(), device="cuda")
    with pytest.raises(N.ExmError):  # no valid forward pass: the backward refuses
        r.backward(M, g, torch.zeros_like(M))
    out = r.forward(M, E)
    r.sync()
    assert torch.equal(out, ref)
    r.close()
    r2.close()


def test_fault_variable_is_read_from_the_environment():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2608_24109_b300 import native as N\n"
            "try:\n    N.exm_create(0)\n    print('created')\n"
            "except N.ExmError as e:\n    print('refused', e.code)\n"
            "c = N.exm_create(0)\nprint('created')\nN.exm_destroy(c)\n") % ROOT
    env = dict(os.environ, EXM_FAULT="alloc:1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.split() == ["refused", str(-2), "created"]


# ------------------------------------------------------------------ serving

def _server(slots=2, budget=2 << 30):
    from paper_2608_24109_b300.serve import RelightServer
    sc = scenes.config("tiny", res=48, views=1, n_direct=16)
    srv = RelightServer(hbm_budget_bytes=budget, max_slots=slots)
    aid = srv.add_asset(sc.V, sc.F, sc.UV, sc.Fuv, torch.as_tensor(sc.maps))
    env = torch.as_tensor(sc.env, device="cuda")
    return srv, aid, env, sc


def test_admission_refusal_and_cancelled_request_injectors():
    from paper_2608_24109_b300 import native as N
    srv, aid, env, sc = _server()
    N.exm_debug_fault(N.FAULT_ADMIT, 1)
    with pytest.raises(N.ExmError) as e:
        srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16))
    assert e.value.code == N.EXM_ERR_BUSY
    N.exm_debug_fault(N.FAULT_CANCEL, 1)
    t = srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16))
    with pytest.raises(N.ExmError) as e:
        srv.wait(t, 10_000)
    assert e.value.code == N.EXM_ERR_CANCELLED
    t = srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16))
    lat, out = srv.wait(t, 30_000)
    assert lat > 0 and float(out.abs().sum()) > 0
    srv.close()


def test_slow_request_wait_times_out_then_completes():
    """A request held 1.5 s on the host: a 0.2-s wait returns EXM_ERR_TIMEOUT and the request
    stays pending; a later wait gets it, with its latency above the hold."""
    from paper_2608_24109_b300 import native as N
    srv, aid, env, sc = _server()
    N.exm_debug_fault(N.FAULT_SLOW, 1500)
    t = srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16))
    N.exm_debug_fault(N.FAULT_SLOW, 0)
    t0 = time.time()
    with pytest.raises(N.ExmError) as e:
        srv.wait(t, 200)
    assert e.value.code == N.EXM_ERR_TIMEOUT and time.time() - t0 < 1.0
    lat, out = srv.wait(t, 30_000)
    assert lat >= 1500 and float(out.abs().sum()) > 0
    srv.close()


def test_cancel_queued_and_in_flight_requests():
    """One slot: the first request (1024^2 pixels x 128 samples, 2^27 shadow rays: tens of
    milliseconds of device work) is launched at once, the second waits in the queue.  Cancelling both while the server
    still reports the first in flight (its completion not yet observed) gives EXM_ERR_CANCELLED
    for each: the launched one finishes on the device and its result is dropped.  The server
    then serves a new request normally."""
    from paper_2608_24109_b300 import native as N
    srv, aid, env, sc = _server(slots=1, budget=8 << 30)
    t1 = srv.submit(srv.request(aid, env, sc.cams, 1024, 1024, 128, seed=1))
    N.exm_debug_fault(N.FAULT_SLOW, 300)
    t2 = srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16, seed=2))
    N.exm_debug_fault(N.FAULT_SLOW, 0)
    st = srv.stats()
    assert st["queued"] == 1 and st["in_flight"] == 1
    srv.cancel(t1)   # no scheduler step between the check and the cancel
    srv.cancel(t2)
    for t in (t1, t2):
        with pytest.raises(N.ExmError) as e:
            srv.wait(t, 30_000)
        assert e.value.code == N.EXM_ERR_CANCELLED
    t3 = srv.submit(srv.request(aid, env, sc.cams, 48, 48, 16, seed=3))
    lat, out = srv.wait(t3, 30_000)
    assert float(out.abs().sum()) > 0
    with pytest.raises(N.ExmError):
        srv.cancel(12345)  # unknown ticket
    srv.close()
