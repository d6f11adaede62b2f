"""Batches of steady solves and the serving engine, through the C ABI.

A batch advances all of its running domains in lockstep with one launch per
step.  Each domain of a mixed batch must match the FP64 oracle after the same
number of steps; a domain's result must not depend on what it shares the
launches with (bitwise); FP16 storage must reach the 128 x 128 cavity's steady
state within the reduced-precision bound; and admission must queue requests
that do not fit the device budget and serve them in order.
"""
import os
import time

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from paper_1806_10251_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_at(case, steps, gi_mode=orc.GI_FULL):
    d = orc.Domain(case.nx, case.ny, case.nu, case.gamma, case.sides, gi_mode=gi_mode, solid=case.solid,
                   Fx=case.Fx, Fy=case.Fy)
    d.init_equilibrium()
    d.step(steps)
    return d.fields()


def fluid(case):
    return np.ones((case.ny, case.nx), bool) if case.solid is None else case.solid == 0


def mixed_cases():
    """Cavities, a body-force channel and an obstacle channel of ragged sizes."""
    return [
        wl.cavity(96, 100.0, 0.1, 0.5, ny=70),
        wl.poiseuille(100, 33, 0.05, 0.7, 2e-6),
        wl.channel_obstacle(nx=160, ny=48, D=8, Re=20.0, U0=0.05, gamma=0.4, xc=40),
        wl.couette(70, 40, 0.04, 0.6, 0.08),
        wl.cavity(33, 50.0, 0.1, 1.0),
    ]


def run_fixed(batch, cases, steps):
    """Submit every case for exactly ``steps`` steps (a tolerance no residual meets)."""
    ids = [batch.submit_case(c, tol=1e-300, max_steps=steps) for c in cases]
    batch.run()
    out = []
    for rid, c in zip(ids, cases):
        done, res = batch.poll(rid)
        assert done and res.state == lbm.REQ_NOT_CONVERGED and res.steps == steps, (c.name, res.state, res.steps)
        out.append(batch.fields(rid, c.nx, c.ny))
    return ids, out


@pytest.mark.parametrize("gi_mode", [orc.GI_UNCORRECTED, orc.GI_FULL])
def test_batch_domains_match_oracle(gi_mode):
    """Five domains of different sizes, boundaries and forcing in one FP32 batch,
    200 steps in checks of 50 with 8-row work items: each domain's fields match
    the oracle to the FP32 step tolerance (2e-6 absolute)."""
    cases = mixed_cases()
    b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F32, gi_mode=gi_mode)
    b.set_option("check_every", 50)
    b.set_option("rows_per_item", 8)
    _, fields = run_fixed(b, cases, 200)
    st = b.stats()
    assert st["launches"] == 4 * 50 and st["cell_updates"] == 200 * sum(c.cells for c in cases)
    for c, (rg, ug, vg) in zip(cases, fields):
        ro, uo, vo = oracle_at(c, 200, gi_mode)
        m = fluid(c)
        err = max(np.abs(rg - ro)[m].max(), np.abs(ug - uo)[m].max(), np.abs(vg - vo)[m].max())
        assert err < 2e-6, (c.name, err)
    b.close()


@pytest.mark.parametrize("storage,tol", [(lbm.STORAGE_F64, 1e-11), (lbm.STORAGE_BF16, 5e-3)])
def test_batch_other_storages_match_oracle(storage, tol):
    """The mixed batch in FP64 storage (the one-cell batch kernel; FP64
    arithmetic, so tight) and in BF16 storage (8-bit mantissa deviations with
    stochastic rounding, so loose): 100 steps, fields against the oracle (the
    state itself: no window average of the velocity, which 16-bit batches take
    by default)."""
    cases = mixed_cases()
    b = lbm.Batch(1 << 30, storage=storage)
    b.set_option("check_every", 50)
    b.set_option("rows_per_item", 8)
    b.set_option("average_samples", 0)
    _, fields = run_fixed(b, cases, 100)
    for c, (rg, ug, vg) in zip(cases, fields):
        ro, uo, vo = oracle_at(c, 100)
        m = fluid(c)
        err = max(np.abs(rg - ro)[m].max(), np.abs(ug - uo)[m].max(), np.abs(vg - vo)[m].max())
        print("batch storage", storage, c.name, "max field error", err)
        assert err < tol, (c.name, err)
    b.close()


def test_domain_result_independent_of_batch_mix():
    """A cavity stepped alone, in a mix of forced and unforced domains, and with
    another tile height: bitwise the same (one kernel, per-cell arithmetic that
    does not depend on the work decomposition).  The single-domain solver is a
    separately compiled kernel whose floating-point contraction may differ: it
    agrees to FP32 rounding."""
    a = wl.cavity(80, 200.0, 0.1, 0.6, ny=72)

    def in_batch(cases, rows):
        b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F32)
        b.set_option("check_every", 40)
        b.set_option("rows_per_item", rows)
        ids, f = run_fixed(b, cases, 120)
        b.close()
        return f

    alone = in_batch([a], 8)[0]
    mix = in_batch(mixed_cases()[:3] + [a] + mixed_cases()[3:], 8)[3]
    tall = in_batch([mixed_cases()[1], a], 24)[1]
    g = lbm.solver_from_case(a)
    g.step(120)
    single = g.fields()
    for k in range(3):
        assert np.array_equal(alone[k], mix[k])
        assert np.array_equal(alone[k], tall[k])
        d = np.abs(alone[k] - single[k]).max()
        print("batch vs single-domain kernel, field", k, "max diff", d)
        assert d < 1e-6


def test_fp16_batch_reaches_cavity128_steady_state():
    """FP16 storage (stochastic rounding, the default) in a batch of four
    cavities: the 128 x 128 cavity (Re = 100, gamma = 0.5) runs to a steady
    state within the FP16 criterion (relative L2 change of u between checks
    1000 steps apart below 1e-3: stochastic rounding keeps that change at a
    noise floor of about 4.5e-4, measured on GB300), then 20000 steps more;
    both states are within relative L2 1e-3 of the oracle's steady state
    (measured: 4e-4 to 5e-4 from 20000 to 120000 steps)."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "cavity128_re100_g05_steady.npz"))
    uo, vo = gold["ux"].astype(np.float64), gold["uy"].astype(np.float64)

    def l2(u, v):
        return np.sqrt(((u - uo) ** 2 + (v - vo) ** 2).sum() / (uo**2 + vo**2).sum())

    c = wl.cavity(128, 100.0, 0.1, 0.5)
    others = [wl.cavity(64, 200.0, 0.1, 0.8), wl.cavity(96, 400.0, 0.1, 0.3, ny=80), wl.cavity(160, 100.0, 0.1, 1.0)]
    b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F16)
    b.set_option("check_every", 1000)
    rid = b.submit_case(c, tol=1e-3, max_steps=100000)
    oids = [b.submit_case(o, tol=1e-3, max_steps=200000) for o in others]
    longer = b.submit_case(c, tol=1e-300, max_steps=40000)
    b.run()
    done, res = b.poll(rid)
    print("FP16 batch 128^2: state", res.state, "steps", res.steps, "residual", res.residual)
    assert done and res.state == lbm.REQ_CONVERGED
    _, ug, vg = b.fields(rid, c.nx, c.ny)
    e1 = l2(ug, vg)
    _, ug, vg = b.fields(longer, c.nx, c.ny)
    e2 = l2(ug, vg)
    print("FP16 batch 128^2 steady L2 vs oracle: at convergence", e1, "after 40000 steps", e2)
    assert e1 <= 1e-3 and e2 <= 1e-3, (e1, e2)
    for o in oids:
        assert b.poll(o)[0]
    b.close()


def test_fp16_round_to_nearest_drifts_and_stochastic_rounding_does_not():
    """The same 128 x 128 cavity, 60000 FP16 steps: with round-to-nearest the
    state drifts away from the steady state (measured L2 3.4e-3 against the
    oracle); with stochastic rounding it stays within 1e-3."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "cavity128_re100_g05_steady.npz"))
    uo, vo = gold["ux"].astype(np.float64), gold["uy"].astype(np.float64)
    c = wl.cavity(128, 100.0, 0.1, 0.5)
    err = {}
    for sr in (0, 1):
        b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F16)
        b.set_option("stochastic_rounding", sr)
        b.set_option("check_every", 1000)
        rid = b.submit_case(c, tol=1e-300, max_steps=60000)
        b.run()
        _, ug, vg = b.fields(rid, c.nx, c.ny)
        err[sr] = np.sqrt(((ug - uo) ** 2 + (vg - vo) ** 2).sum() / (uo**2 + vo**2).sum())
        b.close()
    print("FP16 60000 steps, L2 vs oracle: nearest", err[0], "stochastic", err[1])
    assert err[1] <= 1e-3 < err[0]


def test_admission_by_budget_and_release():
    """A budget that holds one 64 x 64 FP16 cavity: the second request waits;
    run() reports that it cannot be admitted while the finished first one holds
    the memory; after release it runs.  A request larger than the budget is
    refused at submission."""
    c = wl.cavity(64, 100.0, 0.1, 0.5)
    one = 2 * 9 * 64 * 64 * 2 + 2 * 64 * 64 * 8  # two FP16 population arrays + the FP64 snapshot
    b = lbm.Batch(one + one // 2, storage=lbm.STORAGE_F16)
    b.set_option("check_every", 100)
    with pytest.raises(lbm.LbmError):
        b.submit_case(wl.cavity(128, 100.0, 0.1, 0.5))
    r1 = b.submit_case(c, tol=1e-3, max_steps=20000)
    r2 = b.submit_case(c, tol=1e-3, max_steps=20000)
    assert b.stats()["queued"] == 2
    with pytest.raises(lbm.LbmError) as e:
        b.run()
    assert e.value.status == lbm.ERR_OOM
    d1, s1 = b.poll(r1)
    d2, s2 = b.poll(r2)
    assert d1 and s1.state == lbm.REQ_CONVERGED and not d2 and s2.state == lbm.REQ_QUEUED
    b.release(r1)
    b.run()
    d2, s2 = b.poll(r2)
    assert d2 and s2.state == lbm.REQ_CONVERGED and s2.steps > 0
    assert s2.t_admit >= s1.t_done
    b.close()


def test_background_engine_serves_a_stream():
    """The engine thread admits, steps and retires requests submitted while it
    runs (FIFO admission under a budget of about three domains); every request
    converges and its latency parts are ordered."""
    cases = [wl.cavity(64 + 32 * (k % 3), 100.0 + 50 * k, 0.1, 0.5 + 0.05 * k) for k in range(8)]
    per = max(2 * 9 * c.nx * c.ny * 2 + 2 * c.nx * c.ny * 8 + 64 * 64 * 9 * 4 for c in cases)
    b = lbm.Batch(3 * per, storage=lbm.STORAGE_F16)
    b.set_option("check_every", 200)
    b.start()
    ids = []
    for c in cases:
        ids.append(b.submit_case(c, tol=1e-3, max_steps=100000))
        time.sleep(0.002)
    pending = set(ids)
    t_end = time.time() + 120
    while pending and time.time() < t_end:
        for rid in list(pending):
            done, res = b.poll(rid)
            if done:
                assert res.state == lbm.REQ_CONVERGED, (rid, res.state)
                assert res.t_submit <= res.t_admit <= res.t_done
                b.release(rid)
                pending.discard(rid)
        time.sleep(0.005)
    b.stop()
    assert not pending
    st = b.stats()
    assert st["running"] == 0 and st["queued"] == 0 and st["device_bytes"] == 0
    b.close()


def test_batch_option_and_request_validation():
    b = lbm.Batch(1 << 26, storage=lbm.STORAGE_F32)
    for key, v in (("check_every", 3), ("check_every", 0), ("rows_per_item", -1), ("nope", 1)):
        with pytest.raises(lbm.LbmError):
            b.set_option(key, v)
    with pytest.raises(lbm.LbmError):
        b.submit(64, 64, nu=-1.0, gamma=0.5)
    with pytest.raises(lbm.LbmError):
        b.submit(64, 64, nu=0.01, gamma=1.5)
    with pytest.raises(lbm.LbmError):
        b.submit(2, 64, nu=0.01, gamma=0.5)
    with pytest.raises(lbm.LbmError):
        b.poll(12345)
    b.close()


def test_fields_and_release_from_two_threads():
    """lbm_batch_fields and lbm_batch_release on the same finished request from
    two host threads: every fields call either returns the full result or is
    refused because the request was released; release waits for reads in
    flight, so no read sees freed memory (ctypes drops the GIL in each call)."""
    import threading

    c = wl.cavity(256, 100.0, 0.1, 0.5)
    for trial in range(3):
        b = lbm.Batch(1 << 28, storage=lbm.STORAGE_F32)
        b.set_option("check_every", 100)
        rid = b.submit_case(c, tol=1e-300, max_steps=200)
        b.run()
        ref = b.fields(rid, c.nx, c.ny)
        outcomes = []

        def reader():
            for _ in range(40):
                try:
                    got = b.fields(rid, c.nx, c.ny)
                    outcomes.append(all(np.array_equal(g, r, equal_nan=True) for g, r in zip(got, ref)))
                except lbm.LbmError as e:
                    outcomes.append(e.status == lbm.ERR_INVALID and "released" in str(e) or
                                    e.status == lbm.ERR_INVALID and "unknown" in str(e))

        t = threading.Thread(target=reader)
        t.start()
        time.sleep(0.001 * trial)
        b.release(rid)
        t.join()
        assert outcomes and all(outcomes), outcomes
        b.close()


def _fixed_tile_batch(storage=lbm.STORAGE_F16, K=500):
    b = lbm.Batch(1 << 30, storage=storage)
    b.set_option("check_every", K)
    b.set_option("rows_per_item", 8)  # no autotuning steps: check points follow the requests' own steps
    return b


def test_fp16_engine_staggered_admission_bitwise_equal_to_alone():
    """Serving as continuous batching: FP16 requests submitted to the running
    background engine at staggered times, while others run, each give exactly
    the result (fields, steps, residual) of the same request run alone.  The
    arithmetic of a domain, its stochastic-rounding bits (a hash of its own step
    and cell), its velocity samples and its checks do not depend on the mix
    (a fixed tile height keeps the autotuner's timing steps out)."""
    cases = [wl.cavity(96, 300.0, 0.1, 0.6), wl.cavity(64, 150.0, 0.1, 0.9), wl.cavity(128, 500.0, 0.1, 0.5, ny=96),
             wl.channel_obstacle(nx=192, ny=48, D=6, Re=20.0, U0=0.05, gamma=0.5, xc=48)]
    alone = []
    for c in cases:
        b = _fixed_tile_batch()
        rid = b.submit_case(c, tol=1e-3, max_steps=20000)
        b.run()
        done, res = b.poll(rid)
        assert done
        alone.append((res.state, res.steps, res.residual, b.fields(rid, c.nx, c.ny)))
        b.close()
    b = _fixed_tile_batch()
    b.start()
    ids = []
    for c in cases:
        ids.append(b.submit_case(c, tol=1e-3, max_steps=20000))
        time.sleep(0.05)  # later requests join while earlier ones run
    t_end = time.time() + 120
    while time.time() < t_end and not all(b.poll(i)[0] for i in ids):
        time.sleep(0.01)
    b.stop()
    for rid, c, (st, steps, r, f) in zip(ids, cases, alone):
        done, res = b.poll(rid)
        assert done and (res.state, res.steps) == (st, steps), (c.name, res.state, res.steps, st, steps)
        assert res.residual == r
        g = b.fields(rid, c.nx, c.ny)
        for a, e in zip(g, f):
            assert np.array_equal(a, e, equal_nan=True), c.name
    b.close()


def test_cancel_queued_and_running_requests_leaves_the_others_unchanged():
    """lbm_batch_cancel: a queued request leaves the queue at once; a running
    one stops between ticks (state CANCELLED, memory kept until release); the
    requests that run on give results bitwise equal to a run without the
    cancelled ones."""
    keep = [wl.cavity(96, 200.0, 0.1, 0.7), wl.cavity(64, 300.0, 0.1, 0.5)]
    drop_running, drop_queued = wl.cavity(128, 400.0, 0.1, 0.4), wl.cavity(160, 100.0, 0.1, 0.8)

    ref = _fixed_tile_batch()
    rids = [ref.submit_case(c, tol=1e-300, max_steps=3000) for c in keep]
    ref.run()
    expect = [ref.fields(r, c.nx, c.ny) for r, c in zip(rids, keep)]
    ref.close()

    one = 2 * 9 * 128 * 128 * 2 + 4 * 128 * 128 * 8  # room for the three smaller domains, not the fourth
    b = lbm.Batch(3 * one, storage=lbm.STORAGE_F16)
    b.set_option("check_every", 500)
    b.set_option("rows_per_item", 8)
    ids = [b.submit_case(c, tol=1e-300, max_steps=3000) for c in keep]
    r_run = b.submit_case(drop_running, tol=1e-300, max_steps=3000)
    r_q = b.submit_case(drop_queued, tol=1e-300, max_steps=3000)
    assert b.stats()["queued"] == 4
    b.cancel(r_q)
    done, res = b.poll(r_q)
    assert done and res.state == lbm.REQ_CANCELLED and res.steps == 0
    b.start()
    t_end = time.time() + 30
    while time.time() < t_end and b.poll(r_run)[1].state == lbm.REQ_QUEUED:
        time.sleep(0.001)
    b.cancel(r_run)
    while time.time() < t_end and not all(b.poll(i)[0] for i in ids + [r_run]):
        time.sleep(0.01)
    b.stop()
    done, res = b.poll(r_run)
    assert done and res.state == lbm.REQ_CANCELLED and 0 <= res.steps < 3000
    with pytest.raises(lbm.LbmError):
        b.cancel(r_run)  # finished
    for rid, c, e in zip(ids, keep, expect):
        done, res = b.poll(rid)
        assert done and res.state == lbm.REQ_NOT_CONVERGED and res.steps == 3000
        for a, x in zip(b.fields(rid, c.nx, c.ny), e):
            assert np.array_equal(a, x, equal_nan=True), c.name
    for rid in ids + [r_run, r_q]:
        b.release(rid)
    assert b.stats()["device_bytes"] == 0
    b.close()


def test_fp16_window_average_reduces_the_steady_error():
    """The 128 x 128 cavity (Re = 100, gamma = 0.5) in FP16 to r < 1e-3 with
    checks 1000 steps apart, with the default 16 velocity samples per check
    window and without: against the oracle's steady state the averaged result is
    closer (stochastic rounding noise removed) and within 6e-4."""
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "cavity128_re100_g05_steady.npz"))
    uo, vo = gold["ux"].astype(np.float64), gold["uy"].astype(np.float64)
    c = wl.cavity(128, 100.0, 0.1, 0.5)
    err = {}
    for m in (0, 16):
        b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F16)
        b.set_option("check_every", 1000)
        b.set_option("average_samples", m)
        rid = b.submit_case(c, tol=1e-3, max_steps=200000)
        b.run()
        done, res = b.poll(rid)
        assert done and res.state == lbm.REQ_CONVERGED
        _, u, v = b.fields(rid, c.nx, c.ny)
        err[m] = np.sqrt(((u - uo) ** 2 + (v - vo) ** 2).sum() / (uo ** 2 + vo ** 2).sum())
        b.close()
    print("FP16 128^2 steady L2 vs oracle: single state", err[0], "window average", err[16])
    assert err[16] < 0.8 * err[0] and err[16] < 6e-4, err


@pytest.mark.parametrize("storage", [lbm.STORAGE_F16, lbm.STORAGE_F32])
def test_persistent_kernel_bitwise_equal_to_per_step_launches(storage):
    """The persistent batch kernel (every step of a tick's segment in one
    cooperative launch, a bounded grid barrier between steps) against a launch
    per step: the same fields bit for bit, for a set of unforced cavities and
    for a set of forced channels (one force variant each), through ticks with
    window samples and domains of different sizes and rows."""
    cavities = [wl.cavity(96, 300.0, 0.1, 0.6), wl.cavity(64, 150.0, 0.1, 0.9),
                wl.cavity(200, 500.0, 0.1, 0.5, ny=70), wl.cavity(33, 50.0, 0.1, 1.0)]
    channels = [wl.poiseuille(100, 33, 0.05, 0.7, 2e-6),
                wl.channel_obstacle(nx=160, ny=48, D=8, Re=20.0, U0=0.05, gamma=0.4, xc=40)]
    for cases in (cavities, channels):
        out = {}
        for mode in (0, 1):
            b = lbm.Batch(1 << 30, storage=storage)
            b.set_option("check_every", 200)
            b.set_option("rows_per_item", 8)
            b.set_option("persistent", mode)
            _, out[mode] = run_fixed(b, cases, 1000)
            b.close()
        for c, f0, f1 in zip(cases, out[0], out[1]):
            for a0, a1 in zip(f0, f1):
                assert np.array_equal(a0, a1, equal_nan=True), (c.name, storage)


def test_persistent_option_with_mixed_force_variants_runs_per_step():
    """A batch holding forced and unforced domains cannot use the one-variant
    persistent kernel: with the option on it runs per-step launches, and the
    domains still match the oracle."""
    cases = mixed_cases()
    b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F32)
    b.set_option("check_every", 50)
    b.set_option("rows_per_item", 8)
    b.set_option("persistent", 1)
    _, fields = run_fixed(b, cases, 100)
    for c, (rg, ug, vg) in zip(cases, fields):
        ro, uo, vo = oracle_at(c, 100)
        m = fluid(c)
        assert max(np.abs(ug - uo)[m].max(), np.abs(vg - vo)[m].max()) < 2e-6, c.name
    b.close()


def test_smallest_first_admission_under_a_cell_cap():
    """admission = 1 with max_running_cells = 2 * 64^2: of a queue holding a
    128^2, two 64^2 and a 96^2 cavity (submitted in that order before the first
    tick), the two 64^2 run first, side by side; the 96^2 (over the cap beside
    them) waits for both to finish, the 128^2 for the 96^2; first come first
    served with the same cap admits the 128^2 first, alone.  The results are
    those of each domain alone."""
    sides = (128, 64, 64, 96)
    cases = [wl.cavity(n, 100.0, 0.1, 0.5) for n in sides]

    def session(admission):
        b = lbm.Batch(1 << 30, storage=lbm.STORAGE_F32)
        b.set_option("check_every", 100)
        b.set_option("rows_per_item", 8)
        b.set_option("admission", admission)
        b.set_option("max_running_cells", 2 * 64 * 64)
        ids = [b.submit_case(c, tol=1e-300, max_steps=400) for c in cases]
        b.run()
        res = [b.poll(r)[1] for r in ids]
        fields = [b.fields(r, c.nx, c.ny) for r, c in zip(ids, cases)]
        b.close()
        return res, fields

    res, fields = session(1)
    big, s1, s2, mid = res
    assert all(r.state == lbm.REQ_NOT_CONVERGED and r.steps == 400 for r in res)
    assert s1.t_admit <= s2.t_admit < min(s1.t_done, s2.t_done)    # side by side
    assert mid.t_admit >= max(s1.t_done, s2.t_done)                 # waits for both
    assert big.t_admit >= mid.t_done
    fifo, _ = session(0)
    assert fifo[0].t_admit <= min(r.t_admit for r in fifo[1:])
    assert min(r.t_admit for r in fifo[1:]) >= fifo[0].t_done
    for c, f in zip(cases, fields):
        alone = lbm.Batch(1 << 30, storage=lbm.STORAGE_F32)
        alone.set_option("check_every", 100)
        alone.set_option("rows_per_item", 8)
        rid = alone.submit_case(c, tol=1e-300, max_steps=400)
        alone.run()
        g = alone.fields(rid, c.nx, c.ny)
        alone.close()
        for a, b_ in zip(f, g):
            assert np.array_equal(a, b_, equal_nan=True), c.name
    with pytest.raises(lbm.LbmError):
        lbm.Batch(1 << 26, storage=lbm.STORAGE_F32).set_option("admission", 2)


def test_large_batch_domains_agree_with_the_single_domain_kernel():
    """Config-4-sized domains in one batch: a 1024^2 cavity, a ragged 1000 x 600
    cavity and a 1024 x 256 obstacle channel (solid row table), 200 FP32 steps,
    against the single-domain kernel (whose 4096^2 launches match the oracle on
    sampled windows, test_gpu_parity): the same fields to FP32 rounding (a
    separately compiled kernel may contract differently)."""
    cases = [wl.cavity(1024, 1000.0, 0.1, 0.3),
             wl.cavity(1000, 400.0, 0.1, 0.7, ny=600),
             wl.channel_obstacle(nx=1024, ny=256, D=16, Re=40.0, U0=0.05, gamma=0.5, xc=128)]
    b = lbm.Batch(8 << 30, storage=lbm.STORAGE_F32)
    b.set_option("check_every", 100)
    b.set_option("rows_per_item", 16)  # no autotuning steps: exactly 200 steps
    _, fields = run_fixed(b, cases, 200)
    b.close()
    for c, f in zip(cases, fields):
        g = lbm.solver_from_case(c)
        g.step(200)
        single = g.fields()
        g.close()
        m = fluid(c)
        for k in range(3):
            d = np.abs(f[k] - single[k])[m].max()
            assert d < 2e-6, (c.name, k, d)
