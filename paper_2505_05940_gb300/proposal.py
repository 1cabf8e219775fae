"""Learned proposal for inverse fitting.

The paper observes that fits of physical parameters are sensitive to their
initialisation (Sec. 4.3.3, Sec. 5) and uses many random starts.  Here a small
network, trained on (audio feature, parameter) pairs that the simulator itself
generates, proposes the starting point, and the adjoint gradient refines it.

  features   log-mel spectrogram (128 bins, n_fft 1024, hop 256, 20 Hz - fs/2),
             log(mel + 1e-6), averaged over 8 equal time segments -> 1024 values
  targets    6 log-parameters: T0/rho, D/rho, aspect (strings: 1), sigma0,
             sigma1, and the nonlinear scale (tau/rho for strings, E/(2 rho_vol)
             for plates)
  network    1024 -> 512 -> 512 -> 512 -> 6, BF16 weights, FP32 accumulation,
             forward / backward / Adam in the library's kernels (mdx_mlp_*)
  fit        Adam on the log-parameters with gradients from the checkpointed
             adjoint (mdx_grad) and the multi-resolution log-STFT loss
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native, coupling, losses, modal, physics
from . import workloads as W

N_PARAMS = 6
PARAM_NAMES = ("T0_hat", "D_hat", "aspect", "sigma0", "sigma1", "nl_scale")


# ----------------------------------------------------------------- parameters

def log_params(inst):
    """Six log-parameters of a string or plate instance (aspect 1 for strings)."""
    if inst.kind == "string":
        nl = inst.EA / (2.0 * inst.length) / inst.rho_lin
        a = 1.0
    else:
        nl = inst.E / (2.0 * inst.rho_vol)
        a = inst.aspect
    return np.log([inst.T0 / inst.rho_lin, inst.D / inst.rho_lin, a, inst.sigma0, inst.sigma1, nl])


# ----------------------------------------------------------------- features

def features(audio, fs=44100.0, n_fft=1024, hop=256, n_mels=128, segments=8):
    """audio [B, T] (GPU) -> [B, n_mels * segments] log-mel features (the
    library's mdx_logmel kernel: power STFT with a periodic Hann window and
    centred frames, HTK-mel triangles from 20 Hz to fs / 2, log(. + 1e-6),
    mean over `segments` equal frame ranges)."""
    return _native.logmel(audio, fs=fs, n_fft=n_fft, hop=hop, n_mels=n_mels, fmin=20.0,
                          segments=segments)


# ----------------------------------------------------------------- network

class MLP:
    """Proposal network on the GPU: FP32 master weights, BF16 copies, Adam
    moments; every product runs in the library's tensor-core kernels."""

    def __init__(self, dims=(1024, 512, 512, 512, 6), device="cuda:0", seed=0):
        self.dims = tuple(dims)
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        self.w, self.wb, self.b = [], [], []
        for l in range(len(dims) - 1):
            bound = math.sqrt(6.0 / dims[l])               # He uniform for ReLU layers
            w = rng.uniform(-bound, bound, size=(dims[l + 1], dims[l])).astype(np.float32)
            if l == len(dims) - 2:
                w *= 0.1
            self.w.append(torch.tensor(w, device=self.device))
            self.wb.append(self.w[-1].to(torch.bfloat16))
            self.b.append(torch.zeros(dims[l + 1], dtype=torch.float32, device=self.device))
        self.params = self.w + self.b
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.dw = [torch.zeros_like(w) for w in self.w]
        self.db = [torch.zeros_like(b) for b in self.b]
        self.t = 0
        self._acts = None

    def _desc(self):
        d = _native.MLPDesc()
        d.n_layers = len(self.dims) - 1
        for i, v in enumerate(self.dims):
            d.dims[i] = v
        for l in range(d.n_layers):
            d.W[l] = self.wb[l].data_ptr()
            d.b[l] = self.b[l].data_ptr()
        return d

    def forward(self, x_bf16):
        L = _native.load()
        B = x_bf16.shape[0]
        d = self._desc()
        n_act = L.mdx_mlp_act_elems(ctypes.byref(d), B)
        acts = torch.empty(max(1, n_act), dtype=torch.bfloat16, device=self.device)
        y = torch.empty(B, self.dims[-1], dtype=torch.float32, device=self.device)
        _native.check(L.mdx_mlp_forward(ctypes.byref(d), B, ctypes.c_void_p(x_bf16.data_ptr()),
                                        ctypes.c_void_p(acts.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), _native._stream()))
        self._acts, self._x = acts, x_bf16
        return y

    def backward(self, dy):
        """Gradients of sum(dy * y) of the last forward into self.dw, self.db."""
        L = _native.load()
        B = dy.shape[0]
        d = self._desc()
        work = torch.empty(max(1, L.mdx_mlp_work_elems(ctypes.byref(d), B)),
                           dtype=torch.bfloat16, device=self.device)
        n = len(self.w)
        dW = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self.dw])
        db = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self.db])
        _native.check(L.mdx_mlp_backward(ctypes.byref(d), B, ctypes.c_void_p(self._x.data_ptr()),
                                         ctypes.c_void_p(self._acts.data_ptr()),
                                         ctypes.c_void_p(dy.contiguous().data_ptr()), dW, db,
                                         ctypes.c_void_p(work.data_ptr()), _native._stream()))

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        L = _native.load()
        self.t += 1
        grads = self.dw + self.db
        bf = self.wb + [None] * len(self.b)
        for p, g, m, v, wb in zip(self.params, grads, self.m, self.v, bf):
            _native.check(L.mdx_adam_step(p.numel(), ctypes.c_void_p(p.data_ptr()),
                                          ctypes.c_void_p(wb.data_ptr()) if wb is not None else None,
                                          ctypes.c_void_p(g.data_ptr()),
                                          ctypes.c_void_p(m.data_ptr()),
                                          ctypes.c_void_p(v.data_ptr()), lr, beta1, beta2, eps,
                                          self.t, _native._stream()))


# ----------------------------------------------------------------- data set

def _aspect_bank(grid, n_phi=200, n_psi=50, area=W.PLATE_AREA):
    """Coupling tensors at the largest size for each grid aspect; smaller plates
    of the same aspect use a prefix (modes sorted by eigenvalue)."""
    bank = {}
    for a in grid:
        Lx, Ly = coupling.sides(area, a)
        labels = physics.mode_labels(W.Instance(kind="plate", n_phi=n_phi, aspect=float(a),
                                                area=area), n_phi)
        airy = coupling.airy_modes(Lx, Ly, n_psi)
        H, z = coupling.coupling_tensor(Lx, Ly, labels, n_psi, airy=airy)
        bank[float(a)] = (labels, H.astype(np.float32), z, coupling.airy_classes(airy[1]))
    return bank


def _bank_coupling(bank):
    def cp(inst, labels, M):
        blabels, H, z, kc = bank[float(inst.aspect)]
        N = len(labels)
        assert np.array_equal(blabels[:N], labels), "mode sets differ from the bank prefix"
        return H[:M, :N, :N], z[:M], kc[:M]
    return cp


def simulate_batch(insts, fs, steps, bank, device="cuda:0"):
    cp = _bank_coupling(bank)
    prep = [physics.prepare(i, fs, steps, coupling=cp) for i in insts]
    sim = modal.Simulator(prep, device=device)
    audio = sim.simulate(steps)["audio"]
    return audio, prep


def quantize_aspects(instances, aspect_points=16):
    """Move every plate's aspect to the nearest of `aspect_points` grid values
    in [0.5, 2] (in place); returns the grid."""
    grid = np.linspace(0.5, 2.0, aspect_points)
    for inst in instances:
        if inst.kind != "string":
            inst.aspect = float(grid[int(np.argmin(np.abs(grid - inst.aspect)))])
    return grid


def make_dataset(n, seed=0, steps=11025, batch=2048, aspect_points=16, device="cuda:0",
                 bank=None):
    """Simulator-generated (features, log-parameters) pairs.  Plate aspects are
    placed on a grid of `aspect_points` values so that coupling tensors can be
    shared (prefix of the largest tensor per aspect)."""
    wl = W.proposal_draws(seed, n, steps)
    grid = quantize_aspects(wl.instances, aspect_points)
    if bank is None:
        bank = _aspect_bank(grid)
    feats, ys = [], []
    for i0 in range(0, n, batch):
        chunk = wl.instances[i0:i0 + batch]
        audio, _ = simulate_batch(chunk, wl.fs, steps, bank, device)
        feats.append(features(audio, wl.fs))
        ys.append(torch.tensor(np.stack([log_params(i) for i in chunk]), dtype=torch.float32,
                               device=device))
    return torch.cat(feats), torch.cat(ys), wl, bank


# ----------------------------------------------------------------- training

class Proposal:
    def __init__(self, net, x_mean, x_std, y_mean, y_std):
        self.net, self.x_mean, self.x_std, self.y_mean, self.y_std = net, x_mean, x_std, y_mean, y_std

    def predict(self, feats):
        x = ((feats - self.x_mean) / self.x_std).to(torch.bfloat16).contiguous()
        return self.net.forward(x) * self.y_std + self.y_mean


def train(X, Y, epochs=30, batch=256, lr=1e-3, seed=0, device="cuda:0", log=None):
    g = torch.Generator(device="cpu").manual_seed(seed)
    x_mean, x_std = X.mean(0), X.std(0) + 1e-3
    y_mean, y_std = Y.mean(0), Y.std(0) + 1e-3
    Xn = ((X - x_mean) / x_std).to(torch.bfloat16)
    Yn = (Y - y_mean) / y_std
    net = MLP((X.shape[1], 512, 512, 512, Y.shape[1]), device=device, seed=seed)
    n = X.shape[0]
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    it = 0
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            y = net.forward(Xn[idx].contiguous())
            diff = y - Yn[idx]
            dy = (2.0 / (idx.numel() * Y.shape[1])) * diff
            net.backward(dy)
            # one-cycle cosine learning rate
            frac = it / max(1, total - 1)
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * frac))
            net.adam(max(cur, lr * 1e-3))
            it += 1
        mse = float((diff ** 2).mean())
        history.append(mse)
        if log:
            log(f"epoch {ep} mse {mse:.4f}")
    return Proposal(net, x_mean, x_std, y_mean, y_std), history


# ----------------------------------------------------------------- fitting

FIT_INDEX = {"string": (0, 1, 3, 4, 5), "plate": (0, 1, 3, 4, 5)}
OMEGA_T_FIT = 1.9


def _coefficients(preps, lp):
    """Plan-order FP64 coefficients at log-parameters lp (Eq. 13-14 with the
    mass normalised to one, i.e. T0_hat = T0/rho and D_hat = D/rho)."""
    w2, gm, tau, kap = [], [], [], []
    for p, l in zip(preps, lp):
        That, Dhat, s0, s1, nl = np.exp(l[[0, 1, 3, 4, 5]])
        o, g = _native.coeffs_from_physics(p["lam"], Dhat, That, 1.0, s0, s1)
        w2.append(o)
        gm.append(g)
        tau.append(nl if p["kind"] == "tension" else 0.0)
        if p["kind"] == "plate" and p.get("H") is not None:
            kap.append(nl / np.asarray(p["zeta4"], np.float64))
    return (np.concatenate(w2), np.concatenate(gm), np.array(tau),
            np.concatenate(kap) if kap else None)


def _project(preps, lp, T):
    """Keep every mode inside the scheme's stability region: scale T_hat and
    D_hat together so that max omega * T <= OMEGA_T_FIT."""
    for i, p in enumerate(preps):
        lam = float(np.max(p["lam"]))
        w2 = np.exp(lp[i, 1]) * lam * lam + np.exp(lp[i, 0]) * lam
        lim = (OMEGA_T_FIT / T) ** 2
        if w2 > lim:
            f = math.log(lim / w2)
            lp[i, 0] += f
            lp[i, 1] += f
    return lp


def _freq_error(preps, lp, true_lp):
    """Largest relative error of the modal frequencies omega_k over each
    instance's modes (the pitch structure the loss sees)."""
    out = np.zeros(len(preps))
    for i, p in enumerate(preps):
        lam = np.asarray(p["lam"], np.float64)
        w2 = np.exp(lp[i, 1]) * lam ** 2 + np.exp(lp[i, 0]) * lam
        w2t = np.exp(true_lp[i, 1]) * lam ** 2 + np.exp(true_lp[i, 0]) * lam
        out[i] = float(np.max(np.abs(np.sqrt(w2 / w2t) - 1.0)))
    return out


def fit(targets, init_lp, bank, fs=44100.0, steps=4410, iters=100, lr=0.05, K=1024, tol=0.01,
        device="cuda:0"):
    """Adam (cosine-decayed learning rate) on the log-parameters of many
    targets at once, gradients from the checkpointed adjoint of the
    multi-resolution log-STFT loss.  Each target's model keeps the target's
    mode set and geometry (aspect fixed); T_hat, D_hat, sigma0, sigma1 and the
    nonlinear scale are fitted.

    Returns dict(reached = first iteration at which every modal frequency is
    within `tol` relative error (inf if never), reached_all = first iteration
    at which every fitted parameter is within `tol`, lp = final estimates,
    loss = final per-target loss, param_err = final |log error| per
    parameter)."""
    cp = _bank_coupling(bank)
    preps = [physics.prepare(t, fs, steps, coupling=cp) for t in targets]
    for t in targets:
        if t.kind not in FIT_INDEX:
            raise ValueError(f"fit supports strings and plates, not {t.kind}")
    sim = modal.Simulator(preps, device=device)
    target_audio = sim.simulate(steps)["audio"].clone()
    true_lp = np.stack([log_params(t) for t in targets])
    n = len(targets)
    mask = np.zeros((n, N_PARAMS), bool)
    for i, t in enumerate(targets):
        mask[i, list(FIT_INDEX[t.kind])] = True
    lp = np.where(mask, np.asarray(init_lp, np.float64), true_lp)
    T = 1.0 / fs
    lp = _project(preps, lp, T)
    m1 = np.zeros_like(lp)
    m2 = np.zeros_like(lp)
    reached = np.full(n, np.inf)
    reached_all = np.full(n, np.inf)   # every fitted parameter within tol
    offs = sim.plan.mode_offset
    kap_off = np.cumsum([0] + [len(p["zeta4"]) if p["kind"] == "plate" and p.get("H") is not None
                               else 0 for p in preps])
    loss_i = None
    for it in range(iters + 1):
        ok = _freq_error(preps, lp, true_lp) <= tol
        reached = np.where(ok & ~np.isfinite(reached), it, reached)
        ok_all = np.all(np.where(mask, np.abs(np.exp(lp - true_lp) - 1.0) <= tol, True), axis=1)
        reached_all = np.where(ok_all & ~np.isfinite(reached_all), it, reached_all)
        w2, gm, tau, kap = _coefficients(preps, lp)
        sim.plan.set_coefficients(omega2=w2, gamma=gm, tau=tau, kappa=kap)
        for tnsr in (sim.omega2, sim.gamma, sim.b, sim.c, sim.tau, sim.kappa, sim.q0, sim.qm1,
                     sim.direction):
            tnsr.grad = None
        audio = modal.simulate_autograd(sim, steps, K=K)
        loss_i = losses.multires_log_stft(audio, target_audio)
        if it == iters:
            break
        loss_i.sum().backward()
        dw2 = sim.omega2.grad.cpu().numpy()
        dgm = sim.gamma.grad.cpu().numpy()
        dtau = sim.tau.grad.cpu().numpy()
        dkap = sim.kappa.grad.cpu().numpy() if sim.kappa.numel() else np.zeros(0)
        g = np.zeros_like(lp)
        for i, p in enumerate(preps):
            sl = slice(offs[i], offs[i] + len(p["lam"]))
            That, Dhat, s0, s1, nl = np.exp(lp[i, [0, 1, 3, 4, 5]])
            v = _native.coeffs_vjp(p["lam"], Dhat, That, 1.0, s0, s1, dw2[sl], dgm[sl])
            g[i, 0], g[i, 1], g[i, 3], g[i, 4] = v["T0"] * That, v["D"] * Dhat, v["s0"] * s0, v["s1"] * s1
            if p["kind"] == "tension":
                g[i, 5] = dtau[i] * nl
            elif kap_off[i + 1] > kap_off[i]:
                ks = slice(kap_off[i], kap_off[i + 1])
                g[i, 5] = float(np.dot(dkap[ks], nl / np.asarray(p["zeta4"], np.float64)))
        # a target whose loss or gradient is not finite keeps its estimate
        g = np.where(mask & np.isfinite(g), g, 0.0)
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        cur = lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * it / max(1, iters))))
        step = cur * (m1 / (1 - 0.9 ** (it + 1))) / (np.sqrt(m2 / (1 - 0.999 ** (it + 1))) + 1e-12)
        lp = _project(preps, lp - np.where(mask, step, 0.0), T)
    return dict(reached=reached, reached_all=reached_all, lp=lp, true_lp=true_lp,
                loss=loss_i.detach().cpu().numpy() if loss_i is not None else None,
                param_err=np.where(mask, np.abs(lp - true_lp), np.nan))


def sanitize_estimates(pred, Y, margin=0.5):
    """Network estimates as fit starting points: non-finite entries take the
    training mean, and every log-parameter is clipped to the training range
    widened by `margin` (an out-of-distribution input must not start a fit
    at an overflowing coefficient)."""
    lo, hi = Y.min(0) - margin, Y.max(0) + margin
    out = np.where(np.isfinite(pred), pred, Y.mean(0))
    return np.clip(out, lo, hi)


def random_init(targets, seed):
    """Baseline initialisation: log-uniform draws from the training prior."""
    draws = W.proposal_draws(seed, 4 * len(targets) + 8).instances
    by_kind = {"string": [d for d in draws if d.kind == "string"],
               "plate": [d for d in draws if d.kind == "plate"]}
    out = []
    for i, t in enumerate(targets):
        d = by_kind[t.kind][i % len(by_kind[t.kind])]
        lp = log_params(d)
        lp[2] = log_params(t)[2]
        out.append(lp)
    return np.stack(out)


def summarize(reached):
    r = np.asarray(reached, np.float64)
    fin = r[np.isfinite(r)]
    # nearest-rank quantiles: unreached fits (inf) stay inf instead of nan
    q = np.percentile(r, [25, 50, 75], method="nearest") if len(r) else [np.nan] * 3
    return dict(success=float(len(fin) / max(1, len(r))), median=float(q[1]),
                iqr=[float(q[0]), float(q[2])])


# ----------------------------------------------------------------- study

def study(n_train=200_000, n_test=1000, train_steps=11025, fit_steps=4410, iters=100,
          epochs=30, batch=2048, seed=0, device="cuda:0", log=print):
    """Train the proposal on simulator samples, then fit held-out targets from
    the proposal's estimate and from random draws of the prior."""
    import time
    t0 = time.perf_counter()
    X, Y, wl, bank = make_dataset(n_train, seed=seed, steps=train_steps, batch=batch,
                                  device=device)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    log(f"data: {n_train} samples in {t_data:.1f} s")
    t0 = time.perf_counter()
    prop, hist = train(X, Y, epochs=epochs, seed=seed, device=device, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    test = W.proposal_draws(seed + 10_007, n_test, train_steps)
    quantize_aspects(test.instances)
    audio, _ = simulate_batch(test.instances, test.fs, train_steps, bank, device)
    feats = features(audio, test.fs)
    # targets whose own simulation or features are not finite cannot be fitted
    ok = (torch.isfinite(audio).all(1) & torch.isfinite(feats).all(1)).cpu().numpy()
    if not ok.all():
        log(f"dropped {int((~ok).sum())} of {len(ok)} targets with non-finite audio")
        test.instances = [t for t, k in zip(test.instances, ok) if k]
        feats = feats[torch.as_tensor(ok, device=feats.device)]
    pred = sanitize_estimates(prop.predict(feats).detach().cpu().numpy().astype(np.float64),
                              Y.detach().cpu().numpy().astype(np.float64))
    true = np.stack([log_params(t) for t in test.instances])
    pred_err = np.median(np.abs(pred - true), axis=0)
    res = {}
    for name, init in (("proposal", pred), ("random", random_init(test.instances, seed + 3))):
        t0 = time.perf_counter()
        r = fit(test.instances, init, bank, fs=test.fs, steps=fit_steps, iters=iters,
                device=device)
        res[name] = dict(summarize(r["reached"]), seconds=time.perf_counter() - t0,
                         all_params=summarize(r["reached_all"]),
                         final_loss_median=float(np.nanmedian(r["loss"])),
                         final_loss_nonfinite=int(np.sum(~np.isfinite(r["loss"]))),
                         final_abs_log_err_median=np.nanmedian(r["param_err"], axis=0).tolist())
        log(f"{name}: {res[name]}")
    return dict(n_train=n_train, n_test=n_test, data_seconds=t_data,
                samples_per_s=n_train / t_data, train_seconds=t_train,
                train_mse=hist[-1], median_abs_log_err=pred_err.tolist(), fits=res)


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200_000)
    ap.add_argument("--test", type=int, default=1000)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--fit-steps", type=int, default=4410)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    out = study(a.train, a.test, iters=a.iters, epochs=a.epochs, fit_steps=a.fit_steps)
    print(json.dumps(out))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)
