"""The serving scheduler's host logic with the GPU classes replaced by a
stand-in (no device work): continuous admission into free slots, requests
that arrive while a class is in flight wait for its step to finish, new
classes only within the memory budget, idle classes evicted for waiting
requests, and every request served for exactly its step count."""
import pytest

serve = pytest.importorskip("paper_2606_06247_gb300.serve")


class _Event:
    def __init__(self):
        self.done = False

    def query(self):
        return self.done


class FakeClass:
    """Stand-in for SizeClass: same slot bookkeeping, a step completes when
    the test says so."""
    created = []

    def __init__(self, key, capacity, prec, device, n_cont=25):
        self.key, self.kind, self.n = key, key[0], key[1]
        self.capacity, self.prec, self.n_cont = capacity, prec, n_cont
        self.d3 = self.kind == "channel3d"
        self.slots = [None] * capacity
        self.pending_event = False
        self.ev1 = _Event()
        self.steps_run = 0
        FakeClass.created.append(self)

    def free_slots(self):
        return [i for i, r in enumerate(self.slots) if r is None]

    def active(self):
        return [i for i, r in enumerate(self.slots) if r is not None]

    def admit(self, slot, req):
        self.slots[slot] = req

    def step(self):
        self.pending_event = True
        self.ev1 = _Event()
        self.steps_run += 1

    def finish_tick(self, now):
        retired = []
        self.pending_event = False
        for i in self.active():
            r = self.slots[i]
            r.done_steps += 1
            if r.done_steps >= r.steps:
                r.result = {"u": None}
                r.t_done = now
                self.slots[i] = None
                retired.append(r)
        return retired


@pytest.fixture
def fake(monkeypatch):
    FakeClass.created = []
    monkeypatch.setattr(serve, "SizeClass", FakeClass)
    return FakeClass


def _finish_all(srv):
    for c in srv.classes.values():
        c.ev1.done = True


def test_every_request_gets_exactly_its_steps_with_continuous_admission(fake):
    srv = serve.Server(prec="f32x2", capacity=2, mem_budget=1 << 40, device="cpu")
    reqs = [serve.Request(i, "cavity", 32, 100.0, 2 + i % 3) for i in range(5)]
    for r in reqs:
        srv.submit(r)
    ticks = 0
    while not srv.idle():
        srv.tick(float(ticks))
        _finish_all(srv)
        ticks += 1
        assert ticks < 100
    assert all(r.done_steps == r.steps and r.result is not None for r in reqs)
    assert len(fake.created) == 1          # one size class for one (kind, n, family)
    # two slots: five requests of 2-4 steps need more than the longest request alone
    assert fake.created[0].steps_run >= 6


def test_a_class_in_flight_takes_new_requests_only_after_its_step(fake):
    srv = serve.Server(prec="f32x2", capacity=4, mem_budget=1 << 40, device="cpu")
    srv.submit(serve.Request(0, "channel", 32, 50.0, 3))
    srv.tick(0.0)                          # admitted and stepping
    cls = fake.created[0]
    assert cls.pending_event and len(cls.active()) == 1
    srv.submit(serve.Request(1, "channel", 32, 50.0, 3))
    srv.tick(0.1)                          # step not finished: the new request waits
    assert len(cls.active()) == 1 and len(srv.queue) == 1
    cls.ev1.done = True
    srv.tick(0.2)                          # step done: admitted, next step launched
    assert len(cls.active()) == 2 and not srv.queue and cls.pending_event


def test_new_classes_respect_the_memory_budget_and_idle_ones_are_evicted(fake):
    one = serve.footprint_bytes(64, 2, "f32x2")
    srv = serve.Server(prec="f32x2", capacity=2, mem_budget=one + one // 2, device="cpu")
    a = serve.Request(0, "cavity", 64, 100.0, 1)
    b = serve.Request(1, "channel", 64, 100.0, 1)   # another class of the same footprint
    srv.submit(a)
    srv.submit(b)
    srv.tick(0.0)
    assert len(srv.classes) == 1 and len(srv.queue) == 1   # b waits for memory
    _finish_all(srv)
    srv.tick(1.0)                          # a retires; its idle class is evicted; b gets a class
    assert a.result is not None
    assert [c.kind for c in srv.classes.values()] == ["channel"]
    while not srv.idle():
        _finish_all(srv)
        srv.tick(2.0)
    assert b.result is not None


def test_smooth_continuation_reaches_the_classes(fake):
    srv = serve.Server(prec="f32x2", capacity=2, mem_budget=1 << 40, device="cpu", fc_cont="smooth")
    srv.submit(serve.Request(0, "cavity", 256, 1000.0, 1))
    srv.submit(serve.Request(1, "cavity", 128, 1000.0, 1))
    srv.tick(0.0)
    assert sorted(c.n_cont for c in fake.created) == [24, 25]
