"""Fitting the von Karman coupling tensor from random normal initialisations
(Sec. 4.3.3) with the library's full dL/dH: a short version of the
experiment in hfit.py must bring the spectral loss of the best candidate well
below its starting value and move the candidate's response toward the
target's."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2505_05940_gb300 import hfit


def test_coupling_fit_reduces_the_loss():
    res = hfit.fit_coupling(n_phi=12, n_psi=3, steps=4410, iters=80, n_inits=4, lr=0.05,
                            K=512, seed=3)
    print(res)
    assert res["best_loss_ratio"] < 0.5
    assert res["audio_rel_error_2x_length_fit"] < res["audio_rel_error_2x_length_init"]
