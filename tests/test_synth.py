"""Input generators: published test vector of splitmix64 and seed determinism."""
import numpy as np

from paper_2507_10804_gb300 import synth


def test_splitmix64_reference_vector():
    # splitmix64 seeded with 0 (Steele, Lea, Flood 2014; Vigna's reference C code)
    out = synth.splitmix64(0, 3)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_box_muller_moments_and_determinism():
    z = synth.normal(123, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert np.array_equal(z, synth.normal(123, 200000))
    assert not np.array_equal(z[:10], synth.normal(124, 10))


def test_workload_shapes_and_acquisition():
    w = synth.workload(1)
    assert (w.nz, w.nx, w.nb, w.nt, w.ns, w.nr, w.k) == (64, 64, 20, 600, 1, 32, 1)
    assert int(w.acq.src_ix[0]) == 32 and list(w.acq.rec_ix[0][:3]) == [1, 3, 5]
    assert abs(w.vmax * w.dt / w.h - 0.5) < 1e-12
    assert 1300 < w.m.min() and w.m.max() < 2800
    w3 = synth.workload(3)
    assert w3.k == 64 and w3.ns == 32
    assert set(np.unique(w3.v[:48])) == {0.0, 1.0} and set(np.unique(w3.v[48:])) == {-1.0, 1.0}
    w2 = synth.workload(2, nt=10, ns=2)
    assert (w2.nz, w2.nx, w2.nb, w2.ckpt) == (384, 1152, 40, 30)
    assert list(w2.acq.rec_ix[0][:3]) == [1, 4, 7]
    assert 1500 <= w2.m.min() and w2.m.max() <= 5500
