"""The largest axes the C ABI accepts (needs a GPU), each compared with the FP64 oracle: 32,768
phi bins (with layer masks and with counts), 65,535 q/pT rows, 16 layers at the 16-layer
threshold, and a d0 axis whose stacked rows reach 65,535.  Every kernel must pick a launch shape
that fits these sizes; the accumulator, the candidates, the member lists and stage 2 must equal
the oracle's up to the votes it flags, and a batch must equal each event alone.  (The largest
stage-2 grids are covered with the other stage-2 cases in test_gpu_parity.)"""
import numpy as np
import pytest

from paper_1310_7556_gb300 import eventgen as eg

from test_gpu_parity import check_event, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1310_7556_gb300 import binding as b
    b.load()
    return b


G10 = eg.Geometry()
G16 = eg.Geometry(radii_cm=tuple(float(x) for x in np.linspace(4.0, 110.0, 16)))


@pytest.mark.parametrize("acc", [eg.ACC_LAYERS, eg.ACC_COUNTS])
def test_widest_phi_axis(binding, acc):
    """32,768 phi bins on 16 rows: 60 unsmeared helices and 200 noise hits, threshold 2."""
    bn = eg.Binning(n_qpt=16, qpt_min=-0.5, qpt_max=0.5, n_phi=32768, threshold=2, accumulator=acc)
    ev = eg.simulate_event(G10, 60, (2.0, 50.0), 200, seed=5, smear_rphi_cm=0.0)
    r = check_event(binding, G10, bn, ev)
    assert len(r["got"]["candidates"]) > 100


def test_most_qpt_rows(binding):
    """65,535 q/pT rows of 64 phi bins: 7.6M votes from 118 hits."""
    bn = eg.Binning(n_qpt=65535, qpt_min=-2.0, qpt_max=2.0, n_phi=64, threshold=7)
    ev = eg.simulate_event(G10, 10, (0.5, 50.0), 20, seed=6)
    r = check_event(binding, G10, bn, ev)
    assert len(r["got"]["candidates"]) > 50 and r["stage2_checked"] > 0


def test_most_stacked_rows_with_a_d0_axis(binding):
    """5 d0 bins x 13,107 q/pT rows = 65,535 stacked rows."""
    bn = eg.Binning(n_qpt=13107, qpt_min=-1.0, qpt_max=1.0, n_phi=64, threshold=7, n_d0=5, d0_min=-1.0,
                    d0_max=1.0)
    ev = eg.simulate_event(G10, 8, (1.0, 50.0), 10, seed=8, d0_range=(-0.8, 0.8))
    r = check_event(binding, G10, bn, ev)
    assert len(r["got"]["candidates"]) > 50


def test_sixteen_layers(binding):
    """16 layers (4 to 110 cm) at the threshold of all 16, alone and in a batch (whose stage-2
    grids then keep 16-bit masks)."""
    bn = eg.Binning(n_qpt=128, qpt_min=-1.0, qpt_max=1.0, n_phi=512, threshold=16)
    ev = eg.simulate_event(G16, 60, (1.0, 50.0), 300, seed=7)
    r = check_event(binding, G16, bn, ev)
    cands = r["got"]["candidates"]
    assert len(cands) > 40 and np.all(cands["mask"] == 0xFFFF) and r["stage2_checked"] > 0
    other = eg.simulate_event(G16, 30, (1.0, 50.0), 100, seed=17)
    with binding.HoughBatch(G16, bn, max_events=2, max_hits=ev.n_hits + other.n_hits) as b:
        b.run_events([other, ev])
        got, offs = b.candidates()
    assert np.array_equal(got[offs[1]:offs[2]], cands)
    assert np.array_equal(got[offs[0]:offs[1]], run_gpu(binding, G16, bn, other)["candidates"])
