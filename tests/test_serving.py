"""Relight serving: results are the same alone and in a concurrent mix; admission respects
the HBM budget; a relight equals the regular forward render of the same inputs."""
import time

import numpy as np
import pytest
import torch

from paper_2608_24109_b300 import scenes

pytestmark = pytest.mark.gpu


def _assets():
    a = scenes.config("tiny", res=64, views=1)
    b = scenes.blob_scene(n=20, map_res=128, env_w=64, env_h=32, views=1, res=64, n_direct=32, seed=7)
    c = scenes.blob_scene(n=16, map_res=64, env_w=32, env_h=16, views=1, res=48, n_direct=16, n_bounce=2, n_light=2,
                          dents=3, seed=8)
    return [a, b, c]


def _wait(srv, tickets, timeout=60.0):
    outs, lats = {}, {}
    t0 = time.time()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            done, lat, out = srv.poll(t)
            if done:
                outs[t], lats[t] = out, lat
                pending.discard(t)
        assert time.time() - t0 < timeout, "requests did not complete"
    return outs, lats


def _requests(srv, ids, scs, rng):
    reqs = []
    for k in range(8):
        a = int(rng.integers(0, len(ids)))
        sc = scs[a]
        W = int(rng.choice([48, 64, 80]))
        cams = np.stack([scenes.look_at_camera((3 * np.sin(k), 0.5, 3 * np.cos(k)), W, W)])
        envw = int(rng.choice([32, 64]))
        env = torch.as_tensor(scenes.env_map(np.random.default_rng(k), envw, envw // 2, 1.0), device="cuda")
        reqs.append(dict(asset=ids[a], env=env, cams=cams, width=W, height=W, n_direct=sc.n_direct,
                         n_bounce=sc.n_bounce, n_light=sc.n_light, seed=k, wrap_u=sc.wrap_u))
    return reqs


def test_same_alone_and_in_the_mix():
    from paper_2608_24109_b300.serve import RelightServer
    scs = _assets()
    srv = RelightServer(hbm_budget_bytes=4 << 30, max_slots=4)
    ids = [srv.add_asset(s.V, s.F, s.UV, s.Fuv, torch.as_tensor(s.maps).to(torch.bfloat16)) for s in scs]
    reqs = _requests(srv, ids, scs, np.random.default_rng(0))
    alone = []
    for r in reqs:
        t = srv.submit(srv.request(**r))
        outs, _ = _wait(srv, [t])
        alone.append(outs[t].clone())
    from paper_2608_24109_b300 import native as N
    b0, r0 = srv.batches()
    # the first request is held 200 ms on the host, so the others queue behind it (FIFO) and the
    # mix is launched as batches of several requests in flight together
    N.exm_debug_fault(N.FAULT_SLOW, 200)
    tickets = [srv.submit(srv.request(**reqs[0]))]
    N.exm_debug_fault(N.FAULT_SLOW, 0)
    tickets += [srv.submit(srv.request(**r)) for r in reqs[1:]]
    outs, lats = _wait(srv, tickets)
    for k, t in enumerate(tickets):
        assert torch.equal(outs[t], alone[k]), f"request {k} differs in the mix"
        assert outs[t].abs().sum() > 0
        assert lats[t] > 0
    b1, r1 = srv.batches()
    assert r1 - r0 == len(reqs) and b1 - b0 < len(reqs)  # some batch held several requests
    srv.close()


def test_one_batch_of_different_assets_and_sizes():
    """Eight requests over three assets (1280 to 3072 triangles, maps of 64^2 to 256^2 in BF16,
    direct-only and one-bounce), three output sizes and two environment sizes, submitted while
    no batch stream is free, run as one batch: the two persistent tracer launches trace all
    their rays, each through its own asset's BVH, and every image equals the request rendered
    alone."""
    from paper_2608_24109_b300.serve import RelightServer
    from paper_2608_24109_b300 import native as N
    scs = _assets()
    srv = RelightServer(hbm_budget_bytes=8 << 30, max_slots=8)
    ids = [srv.add_asset(s.V, s.F, s.UV, s.Fuv, torch.as_tensor(s.maps).to(torch.bfloat16)) for s in scs]
    reqs = _requests(srv, ids, scs, np.random.default_rng(1))
    alone = []
    for r in reqs:
        t = srv.submit(srv.request(**r))
        outs, _ = _wait(srv, [t])
        alone.append(outs[t].clone())
    # hold the first request on the host for 200 ms: the queue is first in, first out, so the
    # other seven queue up behind it and all eight are ready when a stream takes them
    b0, r0 = srv.batches()
    N.exm_debug_fault(N.FAULT_SLOW, 200)
    held = srv.submit(srv.request(**reqs[0]))
    N.exm_debug_fault(N.FAULT_SLOW, 0)
    tickets = [held] + [srv.submit(srv.request(**r)) for r in reqs[1:]]
    outs, _ = _wait(srv, tickets)
    b1, r1 = srv.batches()
    assert r1 - r0 == 8 and b1 - b0 == 1, (b1 - b0, r1 - r0)
    for k, t in enumerate(tickets):
        assert torch.equal(outs[t], alone[k]), f"request {k} differs in the batch"
    srv.close()


def test_admission_respects_budget():
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300.serve import RelightServer
    scs = _assets()
    probe = RelightServer(hbm_budget_bytes=1 << 40, max_slots=1)
    aid = probe.add_asset(scs[0].V, scs[0].F, scs[0].UV, scs[0].Fuv, torch.as_tensor(scs[0].maps))
    env = torch.as_tensor(scs[0].env, device="cuda")
    one = probe.footprint(probe.request(aid, env, scs[0].cams, 64, 64, 16))
    probe.close()
    # a budget that holds one such request at a time, with four slots
    srv = RelightServer(hbm_budget_bytes=int(one * 1.5), max_slots=4)
    aid = srv.add_asset(scs[0].V, scs[0].F, scs[0].UV, scs[0].Fuv, torch.as_tensor(scs[0].maps))
    tickets = [srv.submit(srv.request(aid, env, scs[0].cams, 64, 64, 16, seed=k)) for k in range(6)]
    st = srv.stats()
    assert st["in_flight"] <= 1 and st["bytes_in_use"] <= int(one * 1.5)
    outs, _ = _wait(srv, tickets)
    assert len(outs) == 6
    # a request larger than the whole budget is refused
    with pytest.raises(N.ExmError) as e:
        big_cams = np.repeat(np.stack([scenes.look_at_camera((0.0, 0.0, 3.0), 1024, 1024)]), 4, 0)
        srv.submit(srv.request(aid, env, big_cams, 1024, 1024, 256))
    assert e.value.code == N.EXM_ERR_BUSY
    srv.close()


def test_relight_equals_forward_render():
    from paper_2608_24109_b300.render import Renderer
    from paper_2608_24109_b300.serve import RelightServer
    sc = scenes.config("tiny", res=64, views=2)
    r = Renderer.from_scene(sc)
    M = torch.as_tensor(sc.maps, device="cuda")
    E = torch.as_tensor(sc.env, device="cuda")
    ref = r.forward(M, E).clone()
    r.sync()
    srv = RelightServer(hbm_budget_bytes=2 << 30, max_slots=2)
    aid = srv.add_asset(sc.V, sc.F, sc.UV, sc.Fuv, M)
    t = srv.submit(srv.request(aid, E, sc.cams, 64, 64, sc.n_direct, seed=sc.seed, wrap_u=True))
    outs, _ = _wait(srv, [t])
    assert torch.equal(outs[t], ref)
    srv.close()
