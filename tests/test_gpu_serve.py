"""Served runs (row a12): continuous batching with admission by device-memory footprint.
A request's result is the same alone and in a mix of concurrent requests; a pool that
holds two runs at a time still completes every request; bad requests fail cleanly."""
import time

import pytest

pytestmark = pytest.mark.gpu

KEYS = ("status", "steps", "particle_steps", "field_energy", "kinetic_energy", "n_particles", "absorbed_object",
        "absorbed_outer", "injected", "current_object", "mg_cycles")


def _req(cpic, **kw):
    base = dict(n1=32, n2=64, particles_per_species=20_000, steps=24, seed=3)
    base.update(kw)
    return cpic.make_request(**base)


def _same(a, b):
    for k in KEYS:
        assert a[k] == b[k], (k, a[k], b[k])


def test_result_same_alone_and_in_mix(cpic):
    target = dict(n1=48, n2=96, particles_per_species=30_000, phi_object=-3.0, steps=30, seed=11)
    sv = cpic.Server(hbm_budget=2 << 30, max_active=8, steps_per_slice=7)
    alone = sv.wait(sv.submit(_req(cpic, **target)))
    assert alone["status"] == 0 and alone["steps"] == 30 and alone["particle_steps"] > 0
    others = [dict(n1=32, n2=64, particles_per_species=50_000, phi_object=-8.0, seed=21),
              dict(n1=64, n2=128, particles_per_species=80_000, phi_object=1.0, temperature=2.0, seed=22),
              dict(n1=16, n2=32, particles_per_species=5_000, density=0.5, seed=23, steps=50),
              dict(n1=32, n2=128, particles_per_species=40_000, seed=24, steps=10)]
    tickets = [sv.submit(_req(cpic, **o)) for o in others[:2]]
    t = sv.submit(_req(cpic, **target))
    tickets += [sv.submit(_req(cpic, **o)) for o in others[2:]]
    mixed = sv.wait(t)
    for tk in tickets:
        assert sv.wait(tk)["status"] == 0
    _same(alone, mixed)
    sv.stop()


def test_admission_by_footprint(cpic):
    """A pool sized for two runs: never more than two active, every request completes with
    the result it has alone."""
    req = _req(cpic, n1=32, n2=64, particles_per_species=60_000, steps=20)
    fp = cpic.Run.footprint(_cfg_of(cpic, req))
    sv = cpic.Server(hbm_budget=int(2.4 * fp), max_active=16, steps_per_slice=5)
    tickets = [sv.submit(_req(cpic, n1=32, n2=64, particles_per_species=60_000, steps=20, seed=100 + i)) for i in range(5)]
    peak = 0
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 300:
        peak = max(peak, sv.stats()["active"])
        for tk in tickets:
            if tk not in results:
                r = sv.poll(tk)
                if r is not None:
                    results[tk] = r
        time.sleep(1e-3)
    assert len(results) == len(tickets)
    assert 1 <= peak <= 2
    assert sv.stats()["pool_free"] == int(2.4 * fp) // 256 * 256
    ref = sv.wait(sv.submit(_req(cpic, n1=32, n2=64, particles_per_species=60_000, steps=20, seed=102)))
    _same(results[tickets[2]], ref)
    sv.stop()


def _cfg_of(cpic, req):
    from paper_1311_2286_gb300 import workloads as wl

    w = wl.cylinder(n1=req.n[0], n2=req.n[1], npart_per_species=req.particles_per_species, host_particles=False)
    return cpic.config_from_workload(w, sort_interval=4)


def test_bad_requests(cpic):
    sv = cpic.Server(hbm_budget=256 << 20, max_active=2)
    with pytest.raises(cpic.CpicError) as e:
        sv.submit(_req(cpic, kind=7))
    assert e.value.status == cpic.CPIC_ERR_INVALID
    with pytest.raises(cpic.CpicError) as e:
        sv.submit(_req(cpic, particles_per_species=0))
    assert e.value.status == cpic.CPIC_ERR_INVALID
    with pytest.raises(cpic.CpicError) as e:
        sv.submit(_req(cpic, particles_per_species=50_000_000))  # larger than the pool
    assert e.value.status == cpic.CPIC_ERR_CAPACITY
    with pytest.raises(cpic.CpicError):
        sv.poll(987654)
    sv.stop()


def test_sphere_requests_in_a_mix(cpic):
    """3D sphere requests run next to cylinder requests and give the same result as alone."""
    sph = dict(kind=cpic.CPIC_REQ_SPHERE, n1=16, n2=16, particles_per_species=40_000, r_outer=30.0, steps=12,
               seed=31)
    sv = cpic.Server(hbm_budget=2 << 30, max_active=8, steps_per_slice=4)
    q = _req(cpic, **sph)
    q.n[2] = 16
    alone = sv.wait(sv.submit(q))
    assert alone["status"] == 0 and alone["steps"] == 12 and alone["injected"][0] > 0
    others = [sv.submit(_req(cpic, seed=40 + i)) for i in range(3)]
    q2 = _req(cpic, **sph)
    q2.n[2] = 16
    mixed = sv.wait(sv.submit(q2))
    for tk in others:
        assert sv.wait(tk)["status"] == 0
    _same(alone, mixed)
    sv.stop()


def test_cancel_queued_and_active_requests(cpic):
    """Host-side failure paths of the server: a queued request cancelled before admission
    and an active one cancelled mid-run both come back with CPIC_ERR_CANCELLED and a message
    saying so (the active one after fewer than its steps), their pool memory returns, a
    cancel of a finished request is refused with CPIC_ERR_STATE, and the requests around
    them still complete with their stand-alone results."""
    long = dict(n1=32, n2=64, particles_per_species=40_000, steps=4000, seed=51)
    fp = cpic.Run.footprint(_cfg_of(cpic, _req(cpic, **long)))
    sv = cpic.Server(hbm_budget=int(1.5 * fp), max_active=4, steps_per_slice=5)  # one run at a time
    t_active = sv.submit(_req(cpic, **long))
    t_queued = sv.submit(_req(cpic, **long))
    t_after = sv.submit(_req(cpic, seed=52))
    t0 = time.time()
    while sv.stats()["active"] < 1 and time.time() - t0 < 60:
        time.sleep(1e-3)
    time.sleep(0.05)
    assert sv.cancel(t_queued) == cpic.CPIC_OK
    assert sv.cancel(t_active) == cpic.CPIC_OK
    rq = sv.wait(t_queued)
    assert rq["status"] == cpic.CPIC_ERR_CANCELLED and rq["steps"] == 0 and "before admission" in rq["message"]
    ra = sv.wait(t_active)
    assert ra["status"] == cpic.CPIC_ERR_CANCELLED and 0 < ra["steps"] < 4000 and "cancelled after" in ra["message"]
    rafter = sv.wait(t_after)
    assert rafter["status"] == 0 and rafter["message"] == ""
    assert sv.cancel(t_after) == cpic.CPIC_ERR_INVALID  # polled: the ticket is retired
    t_done = sv.submit(_req(cpic, seed=53))
    while True:  # one snapshot per test (two calls could straddle the admission)
        st = sv.stats()
        if st["active"] + st["queued"] == 0:
            break
        time.sleep(1e-3)
    assert sv.cancel(t_done) == cpic.CPIC_ERR_STATE
    assert sv.wait(t_done)["status"] == 0
    assert sv.stats()["pool_free"] == int(1.5 * fp) // 256 * 256
    ref = cpic.Server(hbm_budget=2 << 30, max_active=2, steps_per_slice=5)
    _same(rafter, ref.wait(ref.submit(_req(cpic, seed=52))))
    ref.stop()
    sv.stop()


def test_caller_arena_too_small_is_out_of_memory(cpic):
    """Allocation failure without a GPU fault: a caller arena one byte short of the
    footprint (or misaligned) is refused with CPIC_ERR_OOM before anything is launched."""
    import ctypes

    import torch

    cfg = _cfg_of(cpic, _req(cpic))
    need = cpic.Run.footprint(cfg)
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    lib = cpic.load()
    st = lib.cpic_create(ctypes.byref(cfg), ctypes.c_void_p(buf.data_ptr()), need - 1, None, ctypes.byref(h))
    assert st == cpic.CPIC_ERR_OOM and b"arena" in lib.cpic_last_error()
    st = lib.cpic_create(ctypes.byref(cfg), ctypes.c_void_p(buf.data_ptr() + 16), need, None, ctypes.byref(h))
    assert st == cpic.CPIC_ERR_OOM
    st = lib.cpic_create(ctypes.byref(cfg), ctypes.c_void_p(buf.data_ptr()), need, None, ctypes.byref(h))
    assert st == cpic.CPIC_OK
    assert lib.cpic_destroy(h) == cpic.CPIC_OK
