"""Host-side logic of the learned proposal (no GPU): parametrisation, the
stability projection, the feature kernel's argument checks and the study's
bookkeeping."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_05940_gb300 import physics, proposal, workloads as W


def _bank_for(insts):
    grid = sorted({float(i.aspect) for i in insts if i.kind == "plate"})
    return proposal._aspect_bank(grid) if grid else {}


def test_fit_parametrisation_reproduces_prepared_model():
    """At the true log-parameters the fit's coefficients equal the ones the
    simulator was prepared with (omega2, gamma, tau, kappa)."""
    wl = W.proposal_draws(4, 6, 256)
    proposal.quantize_aspects(wl.instances, 4)
    bank = _bank_for(wl.instances)
    cp = proposal._bank_coupling(bank)
    preps = [physics.prepare(t, wl.fs, 256, coupling=cp) for t in wl.instances]
    lp = np.stack([proposal.log_params(t) for t in wl.instances])
    w2, gm, tau, kap = proposal._coefficients(preps, lp)
    np.testing.assert_allclose(w2, np.concatenate([p["omega2"] for p in preps]), rtol=1e-12)
    np.testing.assert_allclose(gm, np.concatenate([p["gamma"] for p in preps]), rtol=1e-12)
    np.testing.assert_allclose(tau, [p["tau"] for p in preps], rtol=1e-12)
    ref_k = [p["kappa"] for p in preps if p["kind"] == "plate" and p.get("H") is not None]
    if ref_k:
        np.testing.assert_allclose(kap, np.concatenate(ref_k), rtol=1e-12)


def test_projection_keeps_scheme_stable_and_ratio():
    wl = W.proposal_draws(2, 4, 256)
    proposal.quantize_aspects(wl.instances, 4)
    cp = proposal._bank_coupling(_bank_for(wl.instances))
    preps = [physics.prepare(t, wl.fs, 256, coupling=cp) for t in wl.instances]
    lp = np.stack([proposal.log_params(t) for t in wl.instances])
    lp2 = lp.copy()
    lp2[:, 0] += 3.0
    lp2[:, 1] += 3.0
    out = proposal._project(preps, lp2.copy(), 1.0 / wl.fs)
    for i, p in enumerate(preps):
        lam = np.max(p["lam"])
        w = np.sqrt(np.exp(out[i, 1]) * lam ** 2 + np.exp(out[i, 0]) * lam) / wl.fs
        assert w <= proposal.OMEGA_T_FIT * (1 + 1e-12)
        assert abs((out[i, 0] - out[i, 1]) - (lp2[i, 0] - lp2[i, 1])) < 1e-12
    # inside the region nothing moves
    np.testing.assert_array_equal(proposal._project(preps, lp.copy(), 1.0 / wl.fs), lp)


def test_logmel_rejects_invalid_arguments():
    """mdx_logmel validates its arguments before any device work (no GPU
    needed): NULL buffers, n_fft not a power of two or out of range, a signal
    too short for the reflection padding, fewer frames than segments, a mel
    count outside [1, 512], frequencies outside 0 <= fmin < fmax <= fs / 2."""
    import ctypes
    from paper_2505_05940_gb300 import _native as N
    L = N.load()
    fake = ctypes.c_void_p(16)   # never dereferenced: every call fails validation

    def call(audio=fake, B=1, T=11025, fs=44100.0, n_fft=1024, hop=256, mels=128, fmin=20.0,
             fmax=22050.0, seg=8, out=fake):
        return L.mdx_logmel(audio, B, T, fs, n_fft, hop, mels, fmin, fmax, seg, out, None)

    for kw in (dict(audio=None), dict(out=None), dict(B=0), dict(seg=0), dict(n_fft=1000),
               dict(n_fft=8), dict(n_fft=4096), dict(hop=0), dict(T=512), dict(T=600, seg=8),
               dict(mels=0), dict(mels=513), dict(fmin=-1.0), dict(fmax=20.0),
               dict(fmax=30000.0), dict(fs=0.0)):
        assert call(**kw) == 1, kw
        assert L.mdx_last_error()


def test_summarize_counts_unreached():
    s = proposal.summarize([3, 5, np.inf, 7])
    assert s["success"] == 0.75 and s["median"] in (5.0, 7.0)
    s = proposal.summarize([np.inf, np.inf, 2])
    assert np.isinf(s["median"]) and s["iqr"][0] == 2.0


def test_random_init_keeps_kind_and_aspect():
    wl = W.proposal_draws(7, 10, 256)
    r = proposal.random_init(wl.instances, 1)
    assert r.shape == (10, 6)
    for t, lp in zip(wl.instances, r):
        assert lp[2] == pytest.approx(proposal.log_params(t)[2])




def test_sanitize_estimates_replaces_nonfinite_and_clips():
    Y = np.array([[0.0, 1.0], [2.0, 3.0], [1.0, 2.0]])
    pred = np.array([[np.nan, 10.0], [-5.0, np.inf], [1.5, 2.5]])
    out = proposal.sanitize_estimates(pred, Y, margin=0.5)
    assert np.all(np.isfinite(out))
    np.testing.assert_allclose(out[0], [1.0, 3.5])     # mean for NaN, clip 10 -> 3.5
    np.testing.assert_allclose(out[1], [-0.5, 2.0])    # clip -5 -> -0.5, mean for inf
    np.testing.assert_allclose(out[2], [1.5, 2.5])     # inside the range: unchanged
