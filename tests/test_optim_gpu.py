"""The fused training update (evo_adam_step: global-norm clip, Adam, EMA and
the BF16 shadow copy over one flat buffer, Sec. 3.2 tensor fusion) against the
FP64 oracle, which runs the same stages tensor by tensor.

Tolerance.  Each step is checked on its own: both sides start from the same
FP32 state, the oracle computes in FP64 and the kernel in FP32, so every
output element may differ by the FP32 rounding of the few operations that
make it.  The bounds below follow that arithmetic with u = 2^-24 (the unit
roundoff of FP32) and a factor of two to spare:
  * global norm G: relative 1e-5 (sums of squares of at most ~100 terms per
    FP32 lane, then double);
  * clip factor s: relative |dG| / G + 2u;
  * m: 4 (u + ds) (|b1 m| + (1 - b1) |g s|);  v: 6 (u + ds) (b2 v + (1 - b2) (g s)^2);
  * the step lr m^ / (sqrt(v^) + eps): its absolute error from dm and dv plus
    8u of its size; w: that plus u |w|;
  * EMA: 4u (d |e| + (1 - d) |w|) + (1 - d) |dw|.
The BF16 shadow copy must equal the kernel's own FP32 parameters rounded to
nearest even, bit for bit; padding between tensors must not move at all; and
two runs from the same state must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import optim as O
from paper_2207_05477_gb300 import evo, synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
NORM_RTOL = 1e-5
DEV = "cuda:0"


def _dev(state):
    return {k: torch.tensor(v, device=DEV) for k, v in state.items()}


def _host(state):
    return {k: v.detach().cpu().numpy().astype(np.float64) for k, v in state.items()}


def _run(h, st, ema=True, bf16=True):
    """One evo_adam_step on device copies; returns the new state, G and the BF16 copy."""
    n = st["params"].numel()
    ws = torch.empty(max(evo.adam_workspace_size(n), 1), dtype=torch.uint8, device=DEV)
    pb = torch.empty(n, dtype=torch.bfloat16, device=DEV) if bf16 else None
    gn = torch.zeros(1, device=DEV)
    out = {k: v.clone() for k, v in st.items()}
    evo.adam_step(h, out["params"], out["grad"], out["exp_avg"], out["exp_avg_sq"], ws,
                  ema=out["ema"] if ema else None, params_bf16=pb, grad_norm=gn)
    torch.cuda.synchronize()
    assert evo.get_error() == evo.EVO_OK
    assert torch.equal(out["grad"], st["grad"])  # the gradient is read only
    return out, float(gn), pb


def _tol(h, gs, m, v, e, Mo, Vo, Po, ds):
    """Bounds on |kernel - oracle| for m, v, w and the EMA of one step (gs:
    the clipped gradient)."""
    bc1, bc2 = 1 - h.beta1 ** h.step, 1 - h.beta2 ** h.step
    dm = 4 * (U + ds) * (abs(h.beta1 * m) + (1 - h.beta1) * abs(gs))
    dv = 6 * (U + ds) * (h.beta2 * v + (1 - h.beta2) * gs ** 2)
    root = np.sqrt(Vo / bc2)
    den = root + h.eps
    # change of the square root: dv / (2 root), and never above sqrt(dv)
    droot = np.minimum(dv / bc2 / np.maximum(2 * root, 1e-300), np.sqrt(dv / bc2))
    stepv = h.lr / bc1 * np.abs(Mo) / den
    dstep = h.lr / bc1 * (dm + np.abs(Mo) * droot / den) / den
    dw = 2 * (dstep + 8 * U * stepv) + 2 * U * np.abs(Po)
    de = 4 * U * (h.ema_decay * np.abs(e) + (1 - h.ema_decay) * np.abs(Po)) + (1 - h.ema_decay) * dw
    return dm, dv, dw, de


def _compare(after, Mo, Vo, Po, Eo, tols, where):
    dm, dv, dw, de = tols
    checks = [("m", after["exp_avg"], Mo, dm), ("v", after["exp_avg_sq"], Vo, dv), ("w", after["params"], Po, dw)]
    if Eo is not None:
        checks.append(("ema", after["ema"], Eo, de))
    for lab, got, ref, tol in checks:
        bad = np.abs(got - ref) > tol + 1e-30
        assert not bad.any(), (where, lab, got[bad][:4], ref[bad][:4], tol[bad][:4])


def _hyper(h, clip=None):
    return O.AdamHyper(lr=h.lr, beta1=h.beta1, beta2=h.beta2, eps=h.eps,
                       clip_norm=h.clip_norm if clip is None else clip, ema_decay=h.ema_decay)


def _check_step(h, before, after, G_k, pieces, ema=True):
    """before/after: host FP64 copies of the FP32 state; pieces: name -> index
    array of the elements that form one tensor of the oracle."""
    sel = lambda k: {nm: before[k][ix] for nm, ix in pieces.items()}
    P, M, V, E, G = O.train_update(sel("params"), sel("grad"), sel("exp_avg"), sel("exp_avg_sq"),
                                   sel("ema") if ema else None, h.step, _hyper(h))
    assert abs(G_k - G) <= NORM_RTOL * G, (G_k, G)
    ds = abs(G_k - G) / G + 2 * U
    g_clipped, _ = O.clip_by_global_norm(sel("grad"), h.clip_norm)
    for nm, ix in pieces.items():
        tols = _tol(h, g_clipped[nm].numpy(), before["exp_avg"][ix], before["exp_avg_sq"][ix], before["ema"][ix],
                    M[nm].numpy(), V[nm].numpy(), P[nm].numpy(), ds)
        sub = {k: v[ix] for k, v in after.items()}
        _compare(sub, M[nm].numpy(), V[nm].numpy(), P[nm].numpy(), E[nm].numpy() if ema else None, tols, nm)


def _block_pieces(d, n_blocks, stride):
    lay, _ = synth.param_layout(d)
    pieces = {}
    for b in range(n_blocks):
        for name, off, shape, _ in lay:
            k = int(np.prod(shape))
            pieces[f"{b}:{name}"] = np.arange(b * stride + off, b * stride + off + k)
    return pieces


def test_three_steps_over_a_two_block_buffer():
    d = synth.Dims(n_seq=6, n_res=40)
    cd = evo.cdims(d, evo.EVO_BF16)
    n1 = evo.param_count(cd)
    stride = (n1 + 127) // 128 * 128 + 128
    n = 2 * stride
    pieces = _block_pieces(d, 2, stride)
    used = np.zeros(n, bool)
    for ix in pieces.values():
        used[ix] = True
    st = synth.make_adam_state(n, 51, fresh=True)
    for b in range(2):
        st["params"][b * stride:b * stride + n1] = synth.make_params(d, 51 + b)
    st["params"][~used] = 0.0
    st["ema"] = st["params"].copy()
    dev = _dev(st)
    for step, clip in ((1, 0.1), (2, 0.1), (3, 1e3)):
        g = synth.make_adam_state(n, 60 + step)["grad"]
        g[~used] = 0.0
        dev["grad"] = torch.tensor(g, device=DEV)
        h = evo.adam_hyper(step, clip_norm=clip)
        before = _host(dev)
        dev, G_k, pb = _run(h, dev)
        after = _host(dev)
        assert (G_k > clip) == (step < 3)  # the clip acts in the first two steps only
        _check_step(h, before, after, G_k, pieces)
        assert torch.equal(pb, dev["params"].to(torch.bfloat16))
        for k in ("params", "exp_avg", "exp_avg_sq", "ema"):  # padding does not move
            assert np.array_equal(after[k][~used], before[k][~used]), k


@pytest.mark.parametrize("n", [1, 3, 5, 4099, 1000003])
@pytest.mark.parametrize("ema,bf16,clip", [(True, True, 0.1), (False, False, 0.0), (True, False, 1e3),
                                           (False, True, 0.1)])
def test_ragged_sizes_and_options(n, ema, bf16, clip):
    st = synth.make_adam_state(n, 70 + n)
    dev = _dev(st)
    h = evo.adam_hyper(5, lr=2e-3, beta1=0.8, beta2=0.99, eps=1e-6, clip_norm=clip, ema_decay=0.99)
    before = _host(dev)
    out, G_k, pb = _run(h, dev, ema=ema, bf16=bf16)
    _check_step(h, before, _host(out), G_k, {"flat": np.arange(n)}, ema=ema)
    if not ema:
        assert torch.equal(out["ema"], dev["ema"])
    if bf16:
        assert torch.equal(pb, out["params"].to(torch.bfloat16))


def test_runs_are_bit_identical_and_empty_is_a_no_op():
    st = _dev(synth.make_adam_state(3_000_001, 81))
    h = evo.adam_hyper(2)
    a, Ga, pa = _run(h, st)
    b, Gb, pb = _run(h, st)
    assert Ga == Gb and torch.equal(pa, pb)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    empty = {k: torch.empty(0, device=DEV) for k in st}
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    evo.adam_step(h, empty["params"], empty["grad"], empty["exp_avg"], empty["exp_avg_sq"], ws)
    torch.cuda.synchronize()


def test_full_size_48_block_buffer_sampled():
    """The flat buffer of the 48-block Evoformer stack at the paper's dims
    (each block padded to a multiple of 128 floats), checked on a sample of
    elements against the oracle, whose global norm runs over all of it."""
    cd = evo.cdims(synth.DIMS_TRAIN_CROP, evo.EVO_BF16)
    stride = (evo.param_count(cd) + 127) // 128 * 128
    n = 48 * stride
    st = synth.make_adam_state(n, 91)
    dev = _dev(st)
    h = evo.adam_hyper(7)
    out, G_k, pb = _run(h, dev)
    rng = np.random.default_rng(5)
    ix = np.unique(np.concatenate([rng.integers(0, n, 200_000), np.arange(n - 5, n), np.arange(5)]))
    sel = torch.tensor(ix, device=DEV)
    after = {k: out[k][sel].double().cpu().numpy() for k in out}
    # the clip takes the norm of the whole gradient: the oracle clips all of
    # it, then runs the remaining stages on the sampled elements
    g_clipped, G = O.clip_by_global_norm({"all": st["grad"]}, h.clip_norm)
    assert abs(G_k - G) <= NORM_RTOL * G, (G_k, G)
    ds = abs(G_k - G) / G + 2 * U
    sub = {k: v[ix].astype(np.float64) for k, v in st.items()}
    sub["grad"] = g_clipped["all"].numpy()[ix]
    del g_clipped
    P, M, V, E, _ = O.train_update({"x": sub["params"]}, {"x": sub["grad"]}, {"x": sub["exp_avg"]},
                                   {"x": sub["exp_avg_sq"]}, {"x": sub["ema"]}, h.step, _hyper(h, clip=0.0))
    Mo, Vo, Po, Eo = (t["x"].numpy() for t in (M, V, P, E))
    tols = _tol(h, sub["grad"], sub["exp_avg"], sub["exp_avg_sq"], sub["ema"], Mo, Vo, Po, ds)
    _compare(after, Mo, Vo, Po, Eo, tols, "sample")
    assert torch.equal(pb[sel], out["params"][sel].to(torch.bfloat16))
