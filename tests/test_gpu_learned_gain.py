"""What the trained damping network gains over the plain method (GPU).

The committed network (trained on instances with seeds 1000..2999 of the
per-cell-resistivity 4-field system, 64^2..128^2 cells) is compared with the
plain hierarchy (damping 0.5, tentative prolongator) on held-out seeds: FGMRES
iterations to 1e-8 with the same FP64 cycle.  The fallback rule (amg_select)
must never end with more iterations than the plain hierarchy.
"""
import numpy as np
import pytest

from paper_2103_07537_gb300 import bamg, learn

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bamg.load()
    torch.cuda.set_device(0)


def test_trained_network_gains_over_the_plain_method():
    weights = learn.load_weights()  # the committed parameters; missing file = failure
    res = learn.evaluate(range(1, 9), 128, weights, cycle_prec=64, log=lambda m: None)
    plain = np.array([r["plain"]["iterations"] for r in res])
    lrn = np.array([r["learned"]["iterations"] for r in res])
    assert all(r["plain"]["converged"] for r in res)
    chosen = np.where([r["choice"] == "learned" for r in res], np.minimum(lrn, plain), plain)
    assert (chosen <= plain).all()
    print(f"plain {plain.mean():.1f}, learned {lrn.mean():.1f}, with fallback {chosen.mean():.1f} iterations")
    assert lrn.mean() < plain.mean()
