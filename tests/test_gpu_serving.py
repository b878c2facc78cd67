"""The continuous-batching server (bem_server_*): results equal bem_eval's,
bit for bit, for a request alone, in a mix of concurrent requests of uneven
size and split across ticks, and match the FP64 oracle within the path's
tolerance; bounded waits, cancellation and statistics."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_03743_gb300 as b
    b.load_library()
    return b


@pytest.fixture(scope="module")
def coax():
    # a small coaxial electrode: 2 x 40 x 50 rectangles + 2 x 40 x 12 ring caps
    return synth.coax_mesh(seed=9, n_phi=40, n_z=50, n_ring=12)


@pytest.mark.parametrize("prec", [0, 1])
def test_alone_and_in_mix_equal_eval(bem, coax, prec):
    reqs = synth.helix_requests(seed=9, n_req=24, max_size=3000)
    with bem.Mesh(coax.types, coax.verts, coax.sigma, precision=prec) as m:
        ref = [m.eval(r) for r in reqs]
        with bem.Server(m, max_points_per_tick=8192) as srv:
            # alone: one request at a time
            alone = []
            for r in reqs[:4]:
                t = srv.submit(r)
                alone.append(srv.wait(t, timeout=120))
            # mixed: everything at once from two threads, uneven sizes
            tickets = [None] * len(reqs)

            def submit(ix):
                for i in ix:
                    tickets[i] = srv.submit(reqs[i])
                    time.sleep(0.001)

            th = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in (0, 1)]
            for x in th:
                x.start()
            for x in th:
                x.join()
            mixed = [srv.wait(t, timeout=120) for t in tickets]
            st = srv.stats()
    for i in range(4):
        assert np.array_equal(alone[i][0], ref[i][0]) and np.array_equal(alone[i][1], ref[i][1])
    for i in range(len(reqs)):
        assert np.array_equal(mixed[i][0], ref[i][0]), i
    # and the server's own results against the oracle (every request, a sample of points each)
    tol = 1e-12 if prec == 0 else 1e-6
    for i, r in enumerate(reqs):
        sub = np.arange(0, len(r), max(1, len(r) // 40))
        rphi, rE, mdr = oracle.eval_field(coax.types, coax.verts, coax.sigma, r[sub], return_min_dr=True)
        far = mdr >= 3
        ephi = np.abs(mixed[i][0][sub] - rphi) / np.abs(rphi)
        eE = np.linalg.norm(mixed[i][1][sub] - rE, axis=1) / np.linalg.norm(rE, axis=1)
        assert ephi[far].max(initial=0) <= tol and eE[far].max(initial=0) <= tol, i
        assert ephi.max() <= max(tol, 1e-5) and eE.max() <= max(tol, 1e-5), i
        assert np.array_equal(mixed[i][1], ref[i][1]), i
    assert st["completed"] == len(reqs) + 4
    assert st["ticks"] >= 2 and st["ticks"] < st["completed"]  # requests were batched together
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_bounded_wait_times_out_while_paused(bem, coax):
    """Failure detection without a GPU fault: a request that cannot finish
    (ticks paused) makes bem_wait return BEM_ERR_TIMEOUT after its bound, and
    the request completes normally once the server resumes."""
    pts = synth.coax_points(seed=10, n=500)
    with bem.Mesh(coax.types, coax.verts, coax.sigma, precision=1) as m:
        ref = m.eval(pts)
        with bem.Server(m) as srv:
            srv.pause(True)
            t = srv.submit(pts)
            t0 = time.perf_counter()
            with pytest.raises(bem.BemError) as e:
                srv.wait(t, timeout=0.2)
            assert e.value.code == -5  # BEM_ERR_TIMEOUT
            assert 0.15 < time.perf_counter() - t0 < 5.0
            done, _, _ = srv.poll(t)
            assert not done
            srv.pause(False)
            phi, E = srv.wait(t, timeout=60)
    assert np.array_equal(phi, ref[0]) and np.array_equal(E, ref[1])


def test_cancel_and_bad_requests(bem, coax):
    with bem.Mesh(coax.types, coax.verts, coax.sigma, precision=1) as m:
        with bem.Server(m, max_points_per_tick=4096) as srv:
            srv.pause(True)
            t1 = srv.submit(synth.coax_points(seed=11, n=100))
            t2 = srv.submit(synth.coax_points(seed=12, n=200))
            srv.cancel(t1)
            with pytest.raises(bem.BemError) as e:
                srv.poll(t1)
            assert e.value.code == -6  # BEM_ERR_NOT_FOUND
            srv.pause(False)
            phi, _ = srv.wait(t2, timeout=60)
            assert phi.shape == (200,)
            bad = synth.coax_points(seed=13, n=10)
            bad[3, 1] = np.nan
            with pytest.raises(bem.BemError):
                srv.submit(bad)


def test_small_budget_shrinks_tick_and_near_overflow_falls_back(bem, coax):
    """A tight near-pair capacity makes ticks overflow; their requests are then
    evaluated one by one and still match bem_eval exactly."""
    pts = synth.coax_points(seed=14, n=3000) * np.array([1.04, 1.04, 1.0])  # hug the inner wall
    with bem.Mesh(coax.types, coax.verts, coax.sigma, precision=1) as m:
        ref = m.eval(pts)
        with bem.Server(m, max_points_per_tick=4096, max_near_pairs_per_tick=64) as srv:
            t = srv.submit(pts)
            phi, E = srv.wait(t, timeout=120)
            st = srv.stats()
    assert st["fallback_ticks"] >= 1
    assert np.array_equal(phi, ref[0]) and np.array_equal(E, ref[1])


def test_large_requests_are_split_across_ticks(bem, coax):
    """A request larger than one tick is evaluated in pieces over several
    ticks; small requests submitted behind it are admitted ahead of its later
    pieces.  Every result equals bem_eval's bit for bit and the oracle's
    within the mixed-path tolerance."""
    big = synth.coax_points(seed=15, n=10000)
    small = [synth.coax_points(seed=16 + k, n=n) for k, n in enumerate((1, 37, 200, 450))]
    with bem.Mesh(coax.types, coax.verts, coax.sigma, precision=1) as m:
        ref_big = m.eval(big)
        ref_small = [m.eval(p) for p in small]
        with bem.Server(m, max_points_per_tick=4096) as srv:
            srv.pause(True)
            tb = srv.submit(big)
            ts = [srv.submit(p) for p in small]
            srv.pause(False)
            phi, E = srv.wait(tb, timeout=120)
            outs = [srv.wait(t, timeout=120) for t in ts]
            st = srv.stats()
            ms, sizes = srv.latencies()
    assert np.array_equal(phi, ref_big[0]) and np.array_equal(E, ref_big[1])
    for (p, e), (rp, re) in zip(outs, ref_small):
        assert np.array_equal(p, rp) and np.array_equal(e, re)
    assert st["ticks"] >= 3  # 10000 points at 4096 per tick
    assert len(ms) == 5 and sorted(sizes.tolist()) == [1, 37, 200, 450, 10000]
    # the small requests finished before the large one's last piece
    assert ms[list(sizes).index(10000)] == ms.max()
    # and against the oracle on a sample of the split request's points
    sub = np.arange(0, len(big), 97)
    rphi, rE, mdr = oracle.eval_field(coax.types, coax.verts, coax.sigma, big[sub], return_min_dr=True)
    far = mdr >= 3
    assert (np.abs(phi[sub] - rphi) / np.abs(rphi))[far].max() <= 1e-6
