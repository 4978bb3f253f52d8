"""Misfit requests that join a running forward sweep at its next time step
(hv_engine_*: a slot per model, each with its own step counter, one launch
per tick for all occupied slots): every misfit is bitwise the single-model
misfit (hv_misfit) whatever the tick it joined at, slots are reused, a full
engine refuses with HV_EBUSY, and an empty tick launches nothing."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300.hv import MisfitEngine, kernel_launches
from tests._helpers import f32, oracle_problem
from tests.test_gpu_misfit_models import make, proposals, t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ragged():
    w, P = make(48, 64, 11, 300, 31)
    dobs = O.fwd_model(oracle_problem(w), f32(w.m), nthreads=8)
    return w, P, dobs


def test_joins_at_different_ticks_are_bitwise_the_single_misfit(ragged):
    w, P, dobs = ragged
    ms = proposals(w, 5, 81)
    D = t(dobs)
    E = MisfitEngine(P, 3)
    joins = {0: [0, 1], 5: [2], 299: [3], 301: [4]}     # model 4 joins after model 0 or 1 has left (slot reused)
    phis, slot_of, finished, pending = {}, {}, {}, []
    tick = 0
    while tick < 2000 and (tick <= max(joins) or E.active):
        for i in joins.get(tick, []):
            pending.append(i)
        while pending and E.active < 3:
            i = pending.pop(0)
            slot_of[i], phis[i] = E.join(t(ms[i]), D)
        for j in E.tick():
            i = [i for i, s in slot_of.items() if s == j and i not in finished][0]
            finished[i] = tick
        tick += 1
    assert sorted(finished) == [0, 1, 2, 3, 4]
    assert len(set(slot_of.values())) == 3             # five models through three slots
    for i in range(5):
        assert float(phis[i]) == float(P.misfit(t(ms[i]), D)), i
    ref = O.misfit_grad(oracle_problem(w), f32(ms[2]), f32(dobs), nthreads=8)[0]
    assert abs(float(phis[2]) - ref) < 2e-4 * ref
    E.close()


def test_full_engine_refuses_and_empty_tick_launches_nothing(ragged):
    w, P, dobs = ragged
    ms = proposals(w, 3, 83)
    D = t(dobs)
    E = MisfitEngine(P, 2)
    n0 = kernel_launches()
    assert E.tick() == [] and kernel_launches() == n0
    E.join(t(ms[0]), D)
    E.join(t(ms[1]), D)
    with pytest.raises(_lib.HvError) as ex:
        E.join(t(ms[2]), D)
    assert ex.value.code == _lib.HV_EBUSY
    done = []
    while E.active:
        done += E.tick()
    assert sorted(done) == [0, 1]
    E.close()


def test_one_step_sweeps_and_a_single_slot():
    """nt = 1: a slot joins and finishes in the same tick; one slot reused three times in a row."""
    w, P = make(32, 40, 3, 1, 91)
    dobs = t(synth.normal(93, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr))
    ms = proposals(w, 3, 95)
    E = MisfitEngine(P, 1)
    for i in range(3):
        slot, phi = E.join(t(ms[i]), dobs)
        assert slot == 0 and E.tick() == [0] and E.active == 0
        assert float(phi) == float(P.misfit(t(ms[i]), dobs)), i
    E.close()


def _wait(cond, limit=120.0):
    import time
    t0 = time.perf_counter()
    while not cond():
        assert time.perf_counter() - t0 < limit, "timed out"
        time.sleep(2e-4)


def test_device_loop_admits_posts_while_it_runs(ragged):
    """The device-resident loop: requests posted from another stream join at the loop's next time step
    (here into slots freed while the loop runs); each misfit is bitwise hv_misfit's; the loop ends by itself
    once idle and is relaunched for later posts."""
    w, P, dobs = ragged
    ms = [t(m) for m in proposals(w, 6, 101)]
    D = t(dobs)
    direct = [float(P.misfit(m, D)) for m in ms]
    torch.cuda.synchronize()
    E = MisfitEngine(P, 3)
    loop_st, post_st = torch.cuda.Stream(), torch.cuda.Stream()
    slot_of, phis, finished = {}, {}, []
    pending = list(range(5))

    def post_next():
        i = pending.pop(0)
        s, phi = E.post(ms[i], D, stream=post_st)
        slot_of[s] = i
        phis[i] = phi

    post_next()
    post_next()
    E.serve(loop_st)

    def step():
        done, running = E.poll()
        finished.extend(slot_of.pop(s) for s in done)
        while pending and len(slot_of) < 3:
            post_next()
        if slot_of and not running:
            E.serve(loop_st)
        return len(finished) == 5

    _wait(step)
    assert sorted(finished) == list(range(5))
    assert [float(phis[i]) for i in range(5)] == direct[:5]
    _wait(lambda: not E.poll()[1])                      # idle: the launch ends by itself
    s, phi = E.post(ms[5], D, stream=post_st)            # a later request relaunches the loop
    E.serve(loop_st)
    _wait(lambda: s in E.poll()[0])
    assert float(phi) == direct[5]
    E.close()


def test_device_loop_stop_and_resume(ragged):
    """A stop request ends the loop after its current iteration; the occupied slot keeps its step and the
    next launch finishes it with the same misfit."""
    import time
    w, P, dobs = ragged
    m = t(proposals(w, 1, 103)[0])
    D = t(dobs)
    ref = float(P.misfit(m, D))
    torch.cuda.synchronize()
    E = MisfitEngine(P, 2)
    st = torch.cuda.Stream()
    s, phi = E.post(m, D)
    E.serve(st)
    time.sleep(0.002)
    E.stop()
    seen = []

    def stopped():
        done, running = E.poll()
        seen.extend(done)
        return not running

    _wait(stopped)
    if s not in seen:
        E.serve(st)
        _wait(lambda: bool(seen.extend(E.poll()[0]) or s in seen))
    assert float(phi) == ref
    with pytest.raises(_lib.HvError):
        E.join(m, D)                                     # the engine now serves posted requests only
    E.close()
