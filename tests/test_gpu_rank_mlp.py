"""Learned sample widths through the C ABI: the MLP's FP32 training kernels
and BF16 inference kernel against the NumPy oracle (oracle/mlp.py), and the
gain of the learned form over the adaptive one on the method itself.

Tolerances: the GPU sums in FP32 (unit roundoff 6e-8) over at most a few
hundred terms per value, the oracle in FP64, so loss and gradient agree to
1e-4 relative to their scale.  The BF16 inference rounds weights and
activations to 8-bit significands on both sides; the GPU accumulates in FP32,
the oracle in FP64, so an activation can land one BF16 step (2^-8 relative)
apart: predictions agree within 0.03 * max(1, |prediction|).
"""
import numpy as np
import pytest

from oracle import mlp
from paper_1508_07798_gb300 import dg_inputs as dg

pytestmark = pytest.mark.gpu


def _hss():
    from paper_1508_07798_gb300 import hssnd
    return hssnd


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(3, 9, n), rng.integers(1, 12, n), rng.uniform(0, 2, n),
                         rng.integers(1, 4, n), rng.uniform(0.7, 1.3, n), rng.uniform(0, 0.05, n)])
    t = np.log1p(rng.integers(1, 90, n).astype(float))
    return X.astype(np.float32), t.astype(np.float32)


def _norm_vec(norm):
    mu, sd, tmu, tsd = norm
    return np.concatenate([mu, sd, [tmu, tsd]]).astype(np.float32)


def test_standardisation_loss_and_gradient_match_oracle():
    hs = _hss()
    X, t = _data(333, 1)            # ragged: 10 full tiles of 32 and a tail of 13
    M = hs.RankModel(seed=7)
    M.fit_norm(X, t)
    _, nm = M.get()
    ref = _norm_vec(mlp.standardisation(X.astype(np.float64), t.astype(np.float64)))
    assert np.allclose(nm, ref, rtol=1e-5, atol=1e-6)
    theta = np.random.default_rng(2).normal(0, 0.2, mlp.NPARAMS).astype(np.float32)
    M.set(theta, ref)
    loss, g = M.loss_grad(X, t)
    norm = (ref[:6].astype(np.float64), ref[6:12].astype(np.float64), float(ref[12]), float(ref[13]))
    lo, go = mlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64), norm)
    assert abs(loss - lo) <= 1e-4 * max(1.0, lo)
    assert np.abs(g - go).max() <= 1e-4 * max(1.0, np.abs(go).max())


def test_adam_step_matches_oracle():
    hs = _hss()
    X, t = _data(96, 3)
    norm = mlp.standardisation(X.astype(np.float64), t.astype(np.float64))
    theta = np.random.default_rng(4).normal(0, 0.2, mlp.NPARAMS).astype(np.float32)
    M = hs.RankModel(seed=0)
    M.set(theta, _norm_vec(norm))
    lr = 1e-3
    M.train(X, t, epochs=1, batch=len(t), lr=lr)     # one full-batch step
    th_gpu, _ = M.get()
    _, go = mlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64), norm)
    th_ref, _, _ = mlp.adam_step(theta.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1, lr)
    big = np.abs(go) > 1e-4            # the first step is lr * g / (|g| + eps): sign-like, stable where |g| is not tiny
    assert big.sum() > 1000
    assert np.abs(th_gpu - th_ref)[big].max() <= 0.02 * lr
    assert np.abs(th_gpu - th_ref).max() <= 2.0 * lr


def test_bf16_inference_matches_oracle_and_widths_follow():
    hs = _hss()
    X, t = _data(1000, 5)
    norm = mlp.standardisation(X.astype(np.float64), t.astype(np.float64))
    theta = np.random.default_rng(6).normal(0, 0.15, mlp.NPARAMS).astype(np.float32)
    M = hs.RankModel(seed=0)
    M.set(theta, _norm_vec(norm))
    pred, r = M.predict(X, oversample=10, rmax=96)
    ref = mlp.forward_bf16(theta, X, (norm[0].astype(np.float32), norm[1].astype(np.float32), norm[2], norm[3]))
    assert np.abs(pred - ref).max() <= 0.03 * max(1.0, np.abs(ref).max())
    k = np.maximum(np.expm1(pred.astype(np.float64)), 0)
    expect = np.clip(np.ceil((k + 10) / 8) * 8, 16, 96).astype(np.int32)
    assert np.abs(r - expect).max() <= 8 and (r % 8 == 0).all() and r.min() >= 16 and r.max() <= 96


def _problems(seeds, ps, n=64):
    out = []
    for p in ps:
        for s in seeds:
            mesh, A = dg.helmholtz_2d(n, p, s)
            kap = dg.helmholtz_kappa(n, p)
            out.append(((2, (n, n), p), A, dg.cosine_field(mesh, s), kap / n))
    return out


def test_learned_widths_cut_sampling_rounds_and_keep_convergence():
    """Trained on adaptive runs of the method (64 x 64 Helmholtz, p in
    {1, 2, 3}, seeds 100..103), the model's widths on unseen seeds need fewer
    sampling rounds than the adaptive loop, and the preconditioned solves
    converge with iteration counts within 10% (at least 1) of the adaptive
    form's."""
    import torch
    hs = _hss()
    from paper_1508_07798_gb300 import ranks
    X, t = ranks.training_set(_problems(range(100, 104), (1, 2, 3)), tol=1e-6)
    assert len(t) > 2000
    M = hs.RankModel(seed=1)
    M.fit_norm(X, t)
    l0, _ = M.loss_grad(X, t)
    loss = M.train(X, t, epochs=60, batch=256, lr=2e-3, seed=3)
    assert loss < 0.5 * l0
    for (meshd, A, c, kh) in _problems([0, 1], (2, 3)):
        dA = hs.DeviceBSR.from_host(A)
        tree = hs.nd_order(meshd, dA)
        Fa = hs.hss_factor(dA, tree, tol=1e-6, precision="fp32")
        r0 = ranks.widths(M, hs.rank_features(tree, c, kh))
        Fl = hs.hss_factor(dA, tree, tol=1e-6, precision="fp32", r_init=r0)
        la, ll = Fa.export_log(), Fl.export_log()
        ca, cl = la["r"] > 0, ll["r"] > 0
        assert np.array_equal(ca, cl)
        assert ll["rounds"][cl].sum() < la["rounds"][ca].sum()
        assert (ll["rounds"][cl] == 1).mean() >= 0.8
        mesh = dg.Mesh(2, (meshd[1][0], meshd[1][1], 1), meshd[2])
        b = torch.as_tensor(dg.point_source_rhs(mesh, 0)[:, 0], device="cuda")
        _, sa = hs.fgmres_solve(dA, Fa, b, rtol=1e-8)
        _, sl = hs.fgmres_solve(dA, Fl, b, rtol=1e-8)
        assert sa.converged and sl.converged
        assert abs(sl.iters - sa.iters) <= max(1, round(0.1 * sa.iters)), (sl.iters, sa.iters)
