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
