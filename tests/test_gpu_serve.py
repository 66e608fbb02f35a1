"""Serving loop: every job's result is the same alone and in a mixed stream of batched jobs, and
equals the oracle on its pair slice (tolerance 0: integer areas, correctly rounded Jaccard)."""
import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def resident():
    import paper_1208_0277_gb300 as P
    P.build()
    w = W.batched_uneven(seed=4, n_tiles=24, count_lo=50, count_hi=3000)
    ctx = P.Context(0)
    A, B = ctx.upload(w.A), ctx.upload(w.B)
    pa, pb, tpo = ctx.candidate_pairs(A, B, with_tile_offsets=True)
    # the oracle's own candidate pairs (from its MBRs) are the device's: the oracle is fed these
    _, mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")
    opa, opb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    np.testing.assert_array_equal(pa.cpu().numpy(), opa)
    np.testing.assert_array_equal(pb.cpu().numpy(), opb)
    return P, w, ctx, A, B, pa, pb, tpo


def same(r1, r2):
    np.testing.assert_array_equal(r1.inter, r2.inter)
    np.testing.assert_array_equal(r1.uni, r2.uni)
    for k in ("sum_inter", "sum_union", "n_nonzero", "n_pairs", "J", "Jprime"):
        assert r1.jaccard[k] == r2.jaccard[k], k


def test_results_alone_equal_results_in_the_mix(resident):
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import serve
    srv = serve.Server(A, B, pa, pb, slots=3, max_batch_pairs=40_000, max_batch_jobs=64)
    try:
        rng = np.random.default_rng(0)
        jobs = serve.draw_jobs(rng, tpo, 300, lo=20, hi=5000)
        futs = [srv.submit(serve.Job(j.p0, j.p1, j.tile)) for j in jobs]     # a burst: batched together
        mixed = [f.result(timeout=120) for f in futs]
        assert srv.batches < len(jobs)                                      # jobs really were batched
        assert max(r.batch_jobs for r in mixed) > 1
        for i in rng.choice(len(jobs), 25, replace=False):
            alone = srv.submit(serve.Job(jobs[i].p0, jobs[i].p1, jobs[i].tile)).result(timeout=60)
            assert alone.batch_jobs == 1
            same(alone, mixed[i])
        pa_h, pb_h = O.candidate_pairs(O.polygon_areas(w.A.off, w.A.xy, method="rle")[1], w.A.tile,
                                    O.polygon_areas(w.B.off, w.B.xy, method="rle")[1], w.B.tile)
        for i in rng.choice(len(jobs), 10, replace=False):
            j = jobs[i]
            ri, ru = O.pair_areas(w.A, w.B, pa_h[j.p0:j.p1], pb_h[j.p0:j.p1], method="rle")
            np.testing.assert_array_equal(mixed[i].inter, ri)
            np.testing.assert_array_equal(mixed[i].uni, ru)
            ref = O.jaccard(ri, ru)
            for k in ("sum_inter", "sum_union", "n_nonzero", "J", "Jprime"):
                assert mixed[i].jaccard[k] == ref[k], k
    finally:
        srv.close()


def test_oversized_job_is_refused(resident):
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import serve
    srv = serve.Server(A, B, pa, pb, slots=1, max_batch_pairs=1000, max_batch_jobs=8)
    try:
        with pytest.raises(ValueError):
            srv.submit(serve.Job(0, 1001))
        r = srv.submit(serve.Job(0, 1000)).result(timeout=60)
        assert len(r.inter) == 1000
    finally:
        srv.close()
    with pytest.raises(ValueError):
        serve.Server(A, B, pa, pb, slots=4, max_batch_pairs=1 << 20, mem_budget_bytes=1 << 20)


def test_cancelled_jobs_are_dropped_and_the_server_keeps_serving(resident):
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import serve
    srv = serve.Server(A, B, pa, pb, slots=1, max_batch_pairs=20_000, max_batch_jobs=16)
    try:
        rng = np.random.default_rng(3)
        jobs = serve.draw_jobs(rng, tpo, 200, lo=20, hi=5000)
        futs = [srv.submit(serve.Job(j.p0, j.p1, j.tile)) for j in jobs]
        cancelled = [f.cancel() for f in futs[::2]]          # those still queued are cancelled
        done = [f.result(timeout=120) for f in futs[1::2]]
        assert any(cancelled)
        pa_h, pb_h = O.candidate_pairs(O.polygon_areas(w.A.off, w.A.xy, method="rle")[1], w.A.tile,
                                    O.polygon_areas(w.B.off, w.B.xy, method="rle")[1], w.B.tile)
        j = jobs[1]
        ri, ru = O.pair_areas(w.A, w.B, pa_h[j.p0:j.p1], pb_h[j.p0:j.p1], method="rle")
        np.testing.assert_array_equal(done[0].inter, ri)
        again = srv.submit(serve.Job(jobs[0].p0, jobs[0].p1)).result(timeout=60)
        assert len(again.inter) == jobs[0].p1 - jobs[0].p0
    finally:
        srv.close()


def test_admission_waits_for_device_memory(resident):
    """A pair arena smaller than a burst: jobs are admitted only as completed batches free their
    ranges of it, jobs larger than the arena are refused, and every result stays exact."""
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import serve
    srv = serve.Server(A, B, pa, pb, slots=3, max_batch_pairs=20_000, max_batch_jobs=16, arena_pairs=24_000)
    try:
        rng = np.random.default_rng(7)
        jobs = serve.draw_jobs(rng, tpo, 120, lo=2000, hi=9000)
        res = [f.result(timeout=120) for f in srv.submit_many([serve.Job(j.p0, j.p1, j.tile) for j in jobs])]
        assert srv.waited_for_memory > 0
        assert srv.arena.free == [(0, 24_000)]                  # every range came back
        with pytest.raises(ValueError):
            srv.submit(serve.Job(0, 20_001))                     # more than a slot holds
        pa_h, pb_h = O.candidate_pairs(O.polygon_areas(w.A.off, w.A.xy, method="rle")[1], w.A.tile,
                                    O.polygon_areas(w.B.off, w.B.xy, method="rle")[1], w.B.tile)
        for i in rng.choice(len(jobs), 8, replace=False):
            j = jobs[i]
            ri, ru = O.pair_areas(w.A, w.B, pa_h[j.p0:j.p1], pb_h[j.p0:j.p1], method="rle")
            np.testing.assert_array_equal(res[i].inter, ri)
            np.testing.assert_array_equal(res[i].uni, ru)
    finally:
        srv.close()
    small = serve.Server(A, B, pa, pb, slots=1, max_batch_pairs=20_000, max_batch_jobs=4, arena_pairs=5_000)
    try:
        with pytest.raises(ValueError):
            small.submit(serve.Job(0, 5_001))                    # more than the arena holds
        assert len(small.submit(serve.Job(0, 5_000)).result(timeout=60).inter) == 5_000
    finally:
        small.close()


def test_poisson_replay_stamps_scheduled_arrivals(resident):
    """Latency runs from each job's scheduled arrival: replaying a trace, no result is earlier than
    its arrival, arrivals follow the trace's order, and the achieved rate is reported against the
    offered one."""
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import serve
    srv = serve.Server(A, B, pa, pb, slots=3, max_batch_pairs=40_000, max_batch_jobs=64)
    try:
        rng = np.random.default_rng(11)
        jobs = serve.draw_jobs(rng, tpo, 200, lo=20, hi=3000)
        res, wall = serve.run_load(srv, jobs, 4000.0, rng)
        arr = [r.t_arrival for r in res]
        assert all(b >= a for a, b in zip(arr, arr[1:]))
        assert all(r.t_done >= r.t_arrival for r in res)
        summ = serve.latency_summary(res, wall, 4000.0)
        assert summ["jobs"] == 200 and 0.0 < summ["achieved_over_offered"] < 10.0
        assert summ["p99_ms"] >= summ["p50_ms"] > 0.0
    finally:
        srv.close()


@pytest.mark.parametrize("policy", ["static", "dynamic"])
def test_stream_admission_gives_the_per_tile_results(resident, policy):
    """Tile tasks admitted to four CUDA streams (static round robin, or by buffer state with the
    smallest tasks moved to idle streams): every pair's areas equal the single-launch result."""
    P, w, ctx, A, B, pa, pb, tpo = resident
    from paper_1208_0277_gb300 import schedule
    ref_i, ref_u = ctx.pair_areas(A, B, pa, pb)
    inter = torch.full_like(ref_i, -7)
    uni = torch.full_like(ref_u, -7)
    torch.cuda.synchronize()
    ex = schedule.GpuExecutor(ctx, A, B, pa, pb, inter, uni, n_streams=4)
    sch = schedule.Scheduler(ex, n_streams=4, depth=2, window=1, policy=policy)
    tasks = schedule.tile_tasks(tpo)
    _, done = sch.run(tasks)
    torch.cuda.synchronize()
    assert sorted(t.tile for t, _ in done) == [t.tile for t in tasks]
    assert torch.equal(inter, ref_i) and torch.equal(uni, ref_u)
