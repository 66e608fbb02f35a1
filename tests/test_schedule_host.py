"""Stream admission by buffer state (Sec. 4.2's full/empty triggers, GPU streams only), on the host
with simulated task durations: every task runs exactly once under both policies, and a congested
stream (an injected stall) slows the static assignment while the dynamic one moves the smallest
tasks away from it."""
import numpy as np
import pytest

from paper_1208_0277_gb300.schedule import Scheduler, SimExecutor, Task


def uneven_tasks(seed, n=300):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(50), np.log(20_000), n))).astype(int)
    off = np.concatenate([[0], np.cumsum(sizes)])
    return [Task(t, int(off[t]), int(off[t + 1])) for t in range(n)]


@pytest.mark.parametrize("policy", ["static", "dynamic"])
def test_every_task_runs_once(policy):
    tasks = uneven_tasks(1)
    sch = Scheduler(SimExecutor([1.0, 1.0, 1.0, 1.0]), n_streams=4, depth=3, window=2, policy=policy)
    _, done = sch.run(tasks)
    assert sorted(t.tile for t, _ in done) == list(range(len(tasks)))
    assert not any(sch.buf) and not any(sch.flight)


def test_dynamic_admission_routes_around_a_stalled_stream():
    tasks = uneven_tasks(2)
    cost = [8.0, 1.0, 1.0, 1.0]          # stream 0 congested (an injected stall)
    st = Scheduler(SimExecutor(cost), n_streams=4, depth=3, window=2, policy="static")
    t_static, _ = st.run(tasks)
    dy = Scheduler(SimExecutor(cost), n_streams=4, depth=3, window=2, policy="dynamic")
    t_dyn, done = dy.run(tasks)
    assert t_dyn < 0.6 * t_static
    work = np.zeros(4)
    for t, s in done:
        work[s] += t.size
    assert work[0] < work[1:].min()       # the stalled stream got less work


def test_migration_moves_the_smallest_tasks_to_an_idle_stream():
    ex = SimExecutor([1.0, 1.0])
    sch = Scheduler(ex, n_streams=2, depth=4, window=1, policy="dynamic")
    big = Task(0, 0, 1000)
    sch.flight[0].append((big, ex.launch(0, big)))
    for k, n in enumerate((500, 30, 400, 20)):
        sch.buf[0].append(Task(k + 1, 0, n))
    sch._migrate()
    assert sorted(t.size for t in sch.buf[1]) == [20, 30]
    assert sorted(t.size for t in sch.buf[0]) == [400, 500]
    assert sch.migrations == 2
