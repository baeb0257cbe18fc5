"""Host logic of the serving loop, on the CPU.

The server's own admission, packing and completion methods run unchanged;
only what touches the GPU is replaced: streams and events are fakes whose
completion the test controls, the two launch methods record what they were
given, and the memory figure is a number the test sets.  Checked: requests
are admitted in arrival order while the memory they need fits (the first one
always, so a request larger than the device cannot block the queue forever),
finished work gives its memory back, small requests of one dtype are packed
into batches of at most batch_keys keys (a larger one alone), large requests
launch alone, and every request is launched and completed exactly once."""
import collections
import math

import pytest
import torch

from paper_2505_18681_gb300 import serve


class FakeEvent:
    """Completes after `delay` queries (set per test through the class)."""
    delay = 0

    def __init__(self):
        self.left = FakeEvent.delay

    def record(self, stream):
        pass

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True


class FakeStream:
    def synchronize(self):
        pass


class FakeEvo:
    def sync(self):
        pass


def request(rid, n, dtype=torch.int32, need=None):
    r = serve.Request.__new__(serve.Request)
    r.rid, r.keys, r.out, r.arrival = rid, None, None, 0.0
    r.admitted = r.launched = r.done = None
    r.n, r.dtype = n, dtype
    r.nbytes = n * torch.empty(0, dtype=dtype).element_size()
    r.params = None
    r.need = need if need is not None else 2 * r.nbytes + 64
    return r


def server(streams=2, big=1000, batch_keys=500, reserve=10, usable=100, monkeypatch=None):
    srv = serve.SortServer.__new__(serve.SortServer)
    srv.evo = FakeEvo()
    srv.streams = [FakeStream() for _ in range(streams)]
    srv.slots = [None] * streams
    srv.busy = [None] * streams
    srv.big, srv.batch_keys, srv.reserve = big, batch_keys, reserve
    srv.reserved = 0
    srv.waiting, srv.admitted = collections.deque(), collections.deque()
    srv.done, srv.launches = [], 0
    srv.usable_bytes = lambda: usable
    srv.plan = lambda r: None          # the test sets each request's need
    srv.log = []                       # ("big" | "batch", [rids]) per launch
    srv._launch_big = lambda r, s, slot: srv.log.append(("big", [r.rid]))
    srv._launch_batch = lambda batch, s, slot: srv.log.append(("batch", [r.rid for r in batch]))
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    return srv


def test_admission_in_arrival_order_while_memory_fits(monkeypatch):
    srv = server(usable=100, reserve=10, monkeypatch=monkeypatch)
    for rid, need in enumerate([50, 30, 20, 5]):
        srv.submit(request(rid, 10, need=need))
    srv._admit(0.0)
    # 50 always (nothing in flight); 100 - 10 - 50 >= 30; 100 - 10 - 80 < 20 waits,
    # and the smaller request behind it does not overtake it
    assert [r.rid for r in srv.admitted] == [0, 1]
    assert [r.rid for r in srv.waiting] == [2, 3]
    assert srv.reserved == 80


def test_first_request_is_admitted_even_when_larger_than_memory(monkeypatch):
    srv = server(usable=100, reserve=10, monkeypatch=monkeypatch)
    srv.submit(request(0, 10, need=10 ** 12))
    srv.submit(request(1, 10, need=1))
    srv._admit(0.0)
    assert [r.rid for r in srv.admitted] == [0]
    assert [r.rid for r in srv.waiting] == [1]


def test_completion_returns_memory_and_admission_resumes(monkeypatch):
    srv = server(streams=1, usable=100, reserve=10, big=10 ** 9, batch_keys=10 ** 9, monkeypatch=monkeypatch)
    monkeypatch.setattr(FakeEvent, "delay", 1)
    for rid, need in enumerate([60, 60]):
        srv.submit(request(rid, 10, need=need))
    srv.step(0.0)                     # admit 0, launch it
    assert srv.log == [("batch", [0])] and srv.reserved == 60
    assert [r.rid for r in srv.waiting] == [1]
    srv.step(1.0)                     # the event is not done yet
    assert srv.reserved == 60 and [r.rid for r in srv.waiting] == [1]
    srv.step(2.0)                     # done: 0 completes, 1 is admitted and launched
    assert [r.rid for r in srv.done] == [0] and srv.done[0].done == 2.0
    assert srv.log == [("batch", [0]), ("batch", [1])]
    assert srv.reserved == 60


def test_packing_by_dtype_and_batch_size(monkeypatch):
    srv = server(streams=1, big=1000, batch_keys=500, usable=10 ** 12, monkeypatch=monkeypatch)
    reqs = [request(0, 200), request(1, 200, torch.int64), request(2, 200), request(3, 200),
            request(4, 5000), request(5, 50)]
    for r in reqs:
        srv.submit(r)
    srv._admit(0.0)
    srv._launch(0.0)
    # the head's dtype (int32): 0 and 2 fit in 500 keys, 3 would not; 5 (50 keys) still fits
    assert srv.log == [("batch", [0, 2, 5])]
    # the rest keep their order
    assert [r.rid for r in srv.admitted] == [1, 3, 4]


def test_large_requests_launch_alone_and_oversize_small_ones_too(monkeypatch):
    srv = server(streams=3, big=1000, batch_keys=100, usable=10 ** 12, monkeypatch=monkeypatch)
    monkeypatch.setattr(FakeEvent, "delay", 10 ** 6)   # nothing completes: one launch per stream
    for r in (request(0, 5000), request(1, 300), request(2, 20)):
        srv.submit(r)
    srv._admit(0.0)
    srv._launch(0.0)
    # 300 keys exceed batch_keys = 100 but form a batch of their own
    assert srv.log == [("big", [0]), ("batch", [1]), ("batch", [2])]
    assert all(b is not None for b in srv.busy)


@pytest.mark.parametrize("streams,delay", [(1, 0), (2, 2), (4, 5)])
def test_whole_run_launches_and_completes_each_request_once(monkeypatch, streams, delay):
    srv = server(streams=streams, big=1000, batch_keys=2000, usable=60_000, reserve=1000,
                 monkeypatch=monkeypatch)
    monkeypatch.setattr(FakeEvent, "delay", delay)
    g = torch.Generator().manual_seed(streams * 10 + delay)
    sizes = torch.floor(torch.exp(torch.rand(120, generator=g, dtype=torch.float64) * math.log(8000))).long()
    dts = [torch.int32, torch.int64, torch.float64]
    pick = torch.randint(0, 3, (120,), generator=g)
    reqs = [request(i, int(sizes[i]), dts[int(pick[i])]) for i in range(120)]
    srv.run(reqs, [0.0] * len(reqs))
    launched = [rid for _, rids in srv.log for rid in rids]
    assert sorted(launched) == list(range(120))
    assert sorted(r.rid for r in srv.done) == list(range(120))
    assert srv.reserved == 0 and srv.idle()
    by_id = {r.rid: r for r in reqs}
    for kind, rids in srv.log:
        rs = [by_id[i] for i in rids]
        if kind == "big":
            assert len(rs) == 1 and rs[0].n >= 1000
        else:
            assert all(r.n < 1000 for r in rs)
            assert len({r.dtype for r in rs}) == 1
            assert len(rs) == 1 or sum(r.n for r in rs) <= 2000
    for r in reqs:
        assert r.arrival <= r.admitted <= r.launched <= r.done


def test_size_upper_bound():
    assert serve.size_upper_bound(300, 1000, 10 ** 8, None) == 10 ** 8
    assert serve.size_upper_bound(300, 1000, 10 ** 8, 10 ** 12) == 10 ** 8

    def mean(h, lo=1000):
        return (h - lo) / math.log(h / lo)
    for cap in (10 ** 9, 3 * 10 ** 8, 5 * 10 ** 6):
        h = serve.size_upper_bound(300, 1000, 10 ** 8, cap)
        assert 1000 < h < 10 ** 8
        assert 300 * mean(h) <= cap < 300 * mean(h * 1.001)   # the largest bound that fits
