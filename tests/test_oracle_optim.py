"""Pins of the FP64 oracle of the fused training update (Sec. 3.2 tensor
fusion: global-norm clip, Adam, EMA), each against something other than the
oracle's own formulas:

  * several Adam steps equal torch.optim.Adam's (clipping off, no EMA);
  * under a constant gradient the bias-corrected moments are exactly g and
    g^2, so w_t = w_0 - t lr g / (|g| + eps) for any betas;
  * the global norm equals torch.nn.utils.clip_grad_norm_'s total norm, and
    the clipped gradients its output; the clipped norm equals the threshold;
  * the clip factor is global: one tensor's gradient changes another's;
  * with lr 0 the EMA has the closed form d^t e_0 + (1 - d^t) w;
  * with decay 0 the EMA equals the updated parameters, not the old ones.
"""
import numpy as np
import pytest
import torch

from oracle import optim as O

DT = torch.float64
SHAPES = {"a.w": (7, 5), "a.b": (5,), "b.w": (3, 4, 2)}


def _rand(seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return {k: torch.randn(s, generator=g, dtype=DT) * scale for k, s in SHAPES.items()}


def _zeros():
    return {k: torch.zeros(s, dtype=DT) for k, s in SHAPES.items()}


def test_adam_steps_match_torch_adam():
    h = O.AdamHyper(lr=3e-3, beta1=0.8, beta2=0.99, eps=1e-6, clip_norm=0.0)
    w = _rand(1)
    m, v = _zeros(), _zeros()
    ref = {k: t.clone().requires_grad_(True) for k, t in w.items()}
    opt = torch.optim.Adam(list(ref.values()), lr=h.lr, betas=(h.beta1, h.beta2), eps=h.eps)
    for step in range(1, 6):
        g = _rand(100 + step)
        w, m, v, _, _ = O.train_update(w, g, m, v, None, step, h)
        for k, p in ref.items():
            p.grad = g[k].clone()
        opt.step()
        for k in w:
            assert torch.allclose(w[k], ref[k].detach(), rtol=1e-12, atol=1e-15), (step, k)


@pytest.mark.parametrize("b1,b2", [(0.9, 0.999), (0.5, 0.9), (0.0, 0.0)])
def test_constant_gradient_closed_form(b1, b2):
    h = O.AdamHyper(lr=1e-2, beta1=b1, beta2=b2, eps=1e-3, clip_norm=0.0)
    w0, g = _rand(2), _rand(3, scale=0.1)
    w, m, v = dict(w0), _zeros(), _zeros()
    for t in range(1, 8):
        w, m, v, _, _ = O.train_update(w, g, m, v, None, t, h)
        for k in w:
            exact = w0[k] - t * h.lr * g[k] / (g[k].abs() + h.eps)
            assert torch.allclose(w[k], exact, rtol=0, atol=1e-13), (t, k)


def test_global_norm_and_clip_match_torch():
    g = _rand(4)
    _, G = O.clip_by_global_norm(g, 0.0)
    copies = [t.clone().requires_grad_(True) for t in g.values()]
    for c, t in zip(copies, g.values()):
        c.grad = t.clone()
    total = torch.nn.utils.clip_grad_norm_(copies, max_norm=0.5)
    assert abs(G - float(total)) <= 1e-12 * G
    clipped, _ = O.clip_by_global_norm(g, 0.5)
    # torch divides by (norm + 1e-6): a relative difference of 1e-6 / G
    for c, k in zip(copies, g):
        assert torch.allclose(clipped[k], c.grad, rtol=2e-6 / G, atol=0), k


def test_clipped_norm_is_the_threshold_and_small_gradients_pass():
    g = _rand(5)
    _, G = O.clip_by_global_norm(g, 0.0)
    clipped, _ = O.clip_by_global_norm(g, G / 3)
    assert abs(O.global_norm(clipped) - G / 3) <= 1e-12 * G
    same, _ = O.clip_by_global_norm(g, 2 * G)
    for k in g:
        assert torch.equal(same[k], g[k])


def test_clip_factor_is_global():
    g = _rand(6)
    a, _ = O.clip_by_global_norm(g, 0.1)
    g2 = dict(g)
    g2["a.w"] = 2 * g["a.w"]
    b, _ = O.clip_by_global_norm(g2, 0.1)
    assert not torch.allclose(a["b.w"], b["b.w"])
    # but the direction of every tensor's gradient is kept
    cos = float((a["b.w"] * b["b.w"]).sum() / (a["b.w"].norm() * b["b.w"].norm()))
    assert abs(cos - 1.0) <= 1e-12


def test_ema_closed_form_with_frozen_parameters():
    h = O.AdamHyper(lr=0.0, ema_decay=0.9, clip_norm=0.0)
    w, e0 = _rand(7), _rand(8)
    m, v, e = _zeros(), _zeros(), dict(e0)
    for t in range(1, 6):
        w2, m, v, e, _ = O.train_update(w, _rand(200 + t), m, v, e, t, h)
        for k in w:
            assert torch.equal(w2[k], w[k])
            exact = h.ema_decay ** t * e0[k] + (1 - h.ema_decay ** t) * w[k]
            assert torch.allclose(e[k], exact, rtol=0, atol=1e-14), (t, k)


def test_ema_follows_the_update():
    h = O.AdamHyper(lr=1e-2, ema_decay=0.0, clip_norm=0.0)
    w = _rand(9)
    w2, _, _, e, _ = O.train_update(w, _rand(10), _zeros(), _zeros(), _rand(11), 1, h)
    for k in w:
        assert torch.equal(e[k], w2[k])
        assert not torch.allclose(e[k], w[k])


def test_zero_gradient_leaves_a_fresh_tensor_alone():
    h = O.AdamHyper()
    w = _rand(12)
    g = {k: torch.zeros_like(t) for k, t in w.items()}
    g["a.b"] = torch.ones(SHAPES["a.b"], dtype=DT)
    w2, m, v, _, _ = O.train_update(w, g, _zeros(), _zeros(), None, 1, h)
    assert torch.equal(w2["a.w"], w["a.w"]) and torch.equal(w2["b.w"], w["b.w"])
    assert float(m["a.w"].abs().max()) == 0.0 and float(v["b.w"].abs().max()) == 0.0
    with pytest.raises(ValueError):
        O.train_update(w, g, _zeros(), _zeros(), None, 0, h)


def test_numpy_inputs_are_accepted():
    h = O.AdamHyper()
    w = {k: np.asarray(t, dtype=np.float32) for k, t in _rand(13).items()}
    g = {k: np.asarray(t, dtype=np.float32) for k, t in _rand(14).items()}
    z = {k: np.zeros(s, np.float32) for k, s in SHAPES.items()}
    P, M, V, E, G = O.train_update(w, g, z, z, z, 1, h)
    assert all(P[k].dtype == DT for k in P) and G > 0


def test_adam_state_generator_is_seeded_and_tiles_differ():
    from paper_2207_05477_gb300 import synth
    a, b = synth.make_adam_state(3000, 4), synth.make_adam_state(3000, 4)
    for k in a:
        assert a[k].dtype == np.float32 and a[k].shape == (3000,)
        assert np.array_equal(a[k], b[k]), k
    assert (a["exp_avg_sq"] >= 0).all()
    fresh = synth.make_adam_state(3000, 4, fresh=True)
    assert not fresh["exp_avg"].any() and not fresh["exp_avg_sq"].any()
    assert np.array_equal(fresh["ema"], fresh["params"]) and np.array_equal(fresh["params"], a["params"])
    # longer than one draw: repeats of the draw, each with its own factor
    big = synth.make_adam_state(2500, 4, base=1000)["grad"]
    r1, r2 = big[1000:2000] / big[:1000], big[2000:] / big[:500]
    assert np.allclose(r1, r1[0], rtol=1e-6) and np.allclose(r2, r2[0], rtol=1e-6)
    # ratios of two factors in [0.5, 1.5)
    assert abs(r1[0] - r2[0]) > 1e-3 and 1 / 3 < r1[0] < 3 and 1 / 3 < r2[0] < 3
