"""Host-side logic of the learned proposal (no GPU): parametrisation, the
stability projection, mel filters and the study's bookkeeping."""
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


def test_mel_filterbank_centres_and_peaks():
    fs, n_fft = 44100.0, 1024
    fb = proposal.mel_filterbank(n_fft, fs, 128).numpy()
    assert fb.shape == (128, n_fft // 2 + 1)
    assert np.all(fb >= 0) and np.all(fb.max(1) <= 1 + 1e-6)
    freqs = np.linspace(0, fs / 2, n_fft // 2 + 1)
    centres = freqs[np.argmax(fb, 1)]
    mel = 2595.0 * np.log10(1.0 + centres / 700.0)
    # centres are monotone and evenly spaced on the mel scale (to a bin's width)
    assert np.all(np.diff(centres) >= 0)
    step = (2595.0 * np.log10(1 + (fs / 2) / 700.0) - 2595.0 * np.log10(1 + 20 / 700.0)) / 129
    high = mel[64:]
    assert np.allclose(np.diff(high), step, atol=step * 0.5)


def test_features_cpu_shape():
    audio = torch.zeros(2, 11025)
    audio[:, 100] = 1.0
    f = proposal.features(audio)
    assert f.shape == (2, 1024) and torch.isfinite(f).all()


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


def test_features_match_numpy_definition():
    """Log-mel features (power STFT with a periodic Hann window, hop 256,
    centred frames; HTK-mel triangles; log(mel + 1e-6); mean over 8 equal
    frame segments) recomputed with numpy from the definition."""
    from oracle import stft_oracle as SO
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(11025) * 1e-2).astype(np.float32)
    got = proposal.features(torch.tensor(x[None]), fs=44100.0)[0].numpy()
    n_fft, fs = 1024, 44100.0
    # the STFT oracle's frames use hop n_fft / 4 = 256, as the features do
    P = SO.stft_mag(x.astype(np.float64), n_fft) ** 2
    mel = lambda f: 2595.0 * np.log10(1.0 + f / 700.0)
    imel = lambda m: 700.0 * (10.0 ** (m / 2595.0) - 1.0)
    pts = imel(np.linspace(mel(20.0), mel(fs / 2), 130))
    freqs = np.linspace(0.0, fs / 2, n_fft // 2 + 1)
    fb = np.array([np.clip(np.minimum((freqs - pts[i]) / (pts[i + 1] - pts[i]),
                                      (pts[i + 2] - freqs) / (pts[i + 2] - pts[i + 1])), 0, None)
                   for i in range(128)])
    m = np.log(fb @ P + 1e-6)
    edges = np.linspace(0, m.shape[1], 9).astype(int)
    ref = np.stack([m[:, edges[i]:max(edges[i + 1], edges[i] + 1)].mean(1) for i in range(8)], 1)
    np.testing.assert_allclose(got, ref.reshape(-1), rtol=2e-4, atol=2e-4)
