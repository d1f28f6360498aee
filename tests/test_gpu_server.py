"""Serving loop (alb_server_*, alb_submit, alb_poll): requests admitted by a
device-memory budget and stepped in chunks together with whatever else is
resident must give exactly the result of the same request run alone through
alb_step, whatever batch they land in."""
import time

import numpy as np
import pytest

from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS = flows.FlowSpec
TARGET = FS("shear", 64, 48, 2.0, 3.0, 1e-4, 37, "fp32", seed=21)
OTHERS = [
    FS("vortex", 40, 40, 1.2, 2.0, 1e-3, 12, "fp32", seed=22),
    FS("shear", 136, 24, 1.5, 2.0, 1e-5, 60, "fp32", seed=23),
    FS("vortex", 49, 41, 1.0, 1.5, 1e-3, 25, "fp64", seed=24),
    FS("shear", 96, 40, 2.5, 3.0, 1e-4, 9, "fp64", seed=25),
    FS("shear", 44, 40, 0.8, 1.2, 1e-3, 1, "fp32", seed=26),
]


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def cfg_of(alb, sp):
    prec = alb.ALB_FP32_FORM if sp.precision == "fp32" else alb.ALB_FP64_PLAIN
    return dict(nx=sp.nx, ny=sp.ny, nu=sp.nu, precision=prec)


def alone(alb, sp, steps=None):
    fl = alb.Flow(**cfg_of(alb, sp))
    assert fl.init(*sp.fields()) == alb.ALB_OK
    fl.step(sp.steps if steps is None else steps)
    fl.sync()
    m = fl.moments()
    fl.close()
    return m


def wait(srv, rid, timeout=120.0):
    t = time.time()
    while time.time() - t < timeout:
        st, res = srv.poll(rid)
        if res is not None:
            return st, res
        time.sleep(0.005)
    raise AssertionError("request %d not done" % rid)


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_alone_and_in_the_mix_are_identical(alb):
    ref = alone(alb, TARGET)
    refs = [alone(alb, sp) for sp in OTHERS]
    # alone on a server
    srv = alb.Server(chunk_ms=5.0)
    try:
        rid = srv.submit(TARGET.steps, fields=TARGET.fields(), **cfg_of(alb, TARGET))
        st, res = wait(srv, rid)
        assert st == alb.ALB_DONE and res["status"] == alb.ALB_OK
        assert res["steps"] == TARGET.steps
        assert same(res["moments"], ref)
    finally:
        srv.close()
    # in a mix: arrivals spread over the first chunks, small chunks so that the
    # batch composition changes while the target runs
    srv = alb.Server(chunk_ms=2.0, max_chunk=7)
    try:
        ids = [srv.submit(OTHERS[0].steps, fields=OTHERS[0].fields(), **cfg_of(alb, OTHERS[0])),
               srv.submit(OTHERS[1].steps, fields=OTHERS[1].fields(), **cfg_of(alb, OTHERS[1]))]
        time.sleep(0.02)
        tid = srv.submit(TARGET.steps, fill=lambda *o: [a.__setitem__(slice(None), f) for a, f in
                                                        zip(o, TARGET.fields())],
                         **cfg_of(alb, TARGET))
        time.sleep(0.02)
        for sp in OTHERS[2:]:
            ids.append(srv.submit(sp.steps, fields=sp.fields(), **cfg_of(alb, sp)))
        st, res = wait(srv, tid)
        assert st == alb.ALB_DONE and res["status"] == alb.ALB_OK
        assert same(res["moments"], ref)
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        for rid, sp, r in zip(ids, OTHERS, refs):
            st, res = wait(srv, rid)
            assert st == alb.ALB_DONE and res["steps"] == sp.steps
            assert same(res["moments"], r), sp
        srv.drain(10000)
        stats = srv.stats()
        assert stats["completed"] == len(OTHERS) + 1 and stats["failed"] == 0
        assert stats["queued"] == 0 and stats["running"] == 0 and stats["resident_bytes"] == 0
        want = sum(sp.nx * sp.ny * sp.steps for sp in OTHERS + [TARGET])
        assert stats["node_updates"] == want
    finally:
        srv.close()


def test_budget_admission_and_errors(alb):
    big = FS("shear", 256, 256, 2.0, 3.0, 1e-4, 3, "fp32", seed=31)
    small = FS("vortex", 32, 32, 1.0, 1.5, 1e-3, 4, "fp32", seed=32)
    total = torch.cuda.get_device_properties(0).total_memory
    # a budget of about 1.5 flows of 256^2: they run one after the other
    per_flow = 256 * 256 * 460
    srv = alb.Server(hbm_fraction=1.5 * per_flow / total)
    try:
        ids = [srv.submit(big.steps, fields=big.fields(), keep_result=False, **cfg_of(alb, big))
               for _ in range(3)]
        with pytest.raises(alb.AlbError) as ei:
            srv.submit(1, fields=flows.uniform(2048, 2048), nx=2048, ny=2048)
        assert ei.value.code == alb.ALB_ENOMEM
        srv.drain(60000)
        times = []
        for rid in ids:
            st, res = srv.poll(rid)
            assert st == alb.ALB_DONE and "moments" not in res
            times.append((res["t_admit"], res["t_done"]))
        times.sort()
        for (a0, d0), (a1, d1) in zip(times, times[1:]):
            assert a1 >= d0  # never two resident at once
        with pytest.raises(alb.AlbError) as ei:
            srv.poll(ids[0])
        assert ei.value.code == alb.ALB_ENOTFOUND
    finally:
        srv.close()
    srv = alb.Server()
    try:
        def bad_fill(*o):
            raise ValueError("no fields")
        rid = srv.submit(3, fill=bad_fill, **cfg_of(alb, small))
        st, res = wait(srv, rid)
        assert st == alb.ALB_FAILED and res["status"] == alb.ALB_EINVAL
        rid = srv.submit(0, fields=small.fields(), **cfg_of(alb, small))
        st, res = wait(srv, rid)
        assert st == alb.ALB_DONE and res["steps"] == 0
        assert same(res["moments"], alone(alb, small, 0))
        with pytest.raises(alb.AlbError):
            srv.submit(-1, fields=small.fields(), **cfg_of(alb, small))
    finally:
        srv.close()
