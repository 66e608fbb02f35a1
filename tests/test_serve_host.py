"""Host-side bookkeeping of the serving loop (no GPU): the pair arena's first-fit allocator."""
import pytest

from paper_1208_0277_gb300.serve import Arena


def test_arena_first_fit_and_coalescing():
    a = Arena(100)
    s1 = a.take(30)
    s2 = a.take(50)
    assert (s1, s2) == (0, 30) and a.largest() == 20
    with pytest.raises(MemoryError):
        a.take(21)
    a.give(s1, 30)
    assert a.largest() == 30 and a.take(25) == 0           # first fit reuses the freed range
    a.give(0, 25)
    a.give(s2, 50)
    assert a.free == [(0, 100)]                            # neighbours merge back into one range


def test_arena_random_sequence_never_overlaps():
    import random
    rnd = random.Random(3)
    a = Arena(1000)
    held = []
    for _ in range(2000):
        if held and (rnd.random() < 0.5 or a.largest() < 10):
            s, n = held.pop(rnd.randrange(len(held)))
            a.give(s, n)
        else:
            n = rnd.randint(1, min(200, a.largest()))
            held.append((a.take(n), n))
        spans = sorted(held + a.free)
        assert sum(n for _, n in spans) == 1000
        assert all(x[0] + x[1] <= y[0] for x, y in zip(spans, spans[1:]))
    for s, n in held:
        a.give(s, n)
    assert a.free == [(0, 1000)]


def test_ticket_states():
    """A queued ticket can be cancelled (its result then raises); an admitted one cannot; a
    completed one returns its result at once; waiting on an unfinished one times out."""
    import concurrent.futures as cf
    import threading

    from paper_1208_0277_gb300.serve import Job, Ticket

    class Srv:
        cv = threading.Condition()
        done_cv = threading.Condition()

    srv = Srv()
    t = Ticket(Job(0, 5), srv)
    assert t.cancel() and t.cancelled() and t.done()
    with pytest.raises(cf.CancelledError):
        t.result(timeout=0.01)
    u = Ticket(Job(0, 5), srv)
    u._state = 1                                     # admitted to a batch
    assert not u.cancel()
    with pytest.raises(TimeoutError):
        u.result(timeout=0.01)

    def finish():
        u._res = "areas"
        u._state = 2
        with srv.done_cv:
            srv.done_cv.notify_all()
    threading.Timer(0.02, finish).start()
    assert u.result(timeout=5) == "areas" and u.done()
