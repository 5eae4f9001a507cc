"""Host-side logic of the server (CPU): memory admission, LRU eviction of idle
sessions, busy sessions never evicted, state carried across eviction, and the
failure cases (a session larger than the whole budget)."""
import pytest

from paper_2601_04860_b300.serve import Server


class FakeData:
    def __init__(self, sid, size):
        self.sid = sid
        self.size = size
        self.n_views = 4


class FakeFusion:
    def __init__(self):
        self.state = None

    def import_state(self, st):
        self.state = st


class FakeSession:
    made = []

    def __init__(self, data, dev):
        self.data = data
        self.fusion = FakeFusion()
        self.views_done = 0
        self.closed = False
        FakeSession.made.append(data.sid)

    def export(self):
        return {"W": f"state-of-{self.data.sid}", "n_views": self.views_done}

    def close(self):
        self.closed = True


def _server(sizes, budget):
    FakeSession.made = []
    data = [FakeData(i, s) for i, s in enumerate(sizes)]
    return Server(data, memory_budget=budget, device="cpu", session_factory=FakeSession,
                  footprint=lambda d: d.size)


def test_admission_and_lru_eviction():
    srv = _server([40, 40, 40], 100)
    assert srv._admit(0, set()) and srv._admit(1, set())
    assert srv.used == 80
    srv.last_use.update({0: 1.0, 1: 2.0})
    assert srv._admit(2, set())            # evicts the least recently used idle session (0)
    assert set(srv.resident) == {1, 2} and srv.stats["evictions"] == 1
    assert 0 in srv.evicted and srv.used == 80
    srv.views_done[0] = 3
    srv.last_use[2] = 5.0
    assert srv._admit(0, set())            # evicts 1 now; 0 comes back with its exported state
    assert srv.resident[0].fusion.state == {"W": "state-of-0", "n_views": 0}
    assert srv.resident[0].views_done == 3


def test_busy_sessions_are_never_evicted():
    srv = _server([60, 60], 100)
    assert srv._admit(0, set())
    assert not srv._admit(1, busy={0})     # the only resident session is in flight: wait
    assert set(srv.resident) == {0} and srv.stats["evictions"] == 0
    assert srv._admit(1, set())            # once idle it can be evicted
    assert set(srv.resident) == {1}


def test_session_larger_than_budget_is_refused():
    srv = _server([150], 100)
    with pytest.raises(ValueError):
        srv._admit(0, set())


def test_admit_all_stops_at_the_budget():
    srv = _server([30, 30, 30, 30], 100)
    assert srv.admit_all() == 3
