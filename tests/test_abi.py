"""The C-ABI library builds for sm_103a, loads, and exports what include/evo.h declares.

Host-only entry points are exercised here; nothing touches a GPU.
"""
import ctypes

import pytest

from paper_2207_05477_gb300 import evo, synth


def test_every_declared_symbol_is_exported(built_lib):
    names = evo.header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(built_lib, n), n


@pytest.mark.parametrize("d", [synth.DIMS_TRAIN_CROP, synth.DIMS_SMALL_FP32, synth.DIMS_EXTRA_MSA])
def test_param_layout_matches_generator_table(built_lib, d):
    cd = evo.cdims(d, evo.EVO_BF16)
    lay = evo.param_layout(cd)
    ref, total = synth.param_layout(d)
    assert [(n, o, s) for n, o, s, _ in ref] == lay
    assert evo.param_count(cd) == total
    assert all(o % 64 == 0 for _, o, _ in lay)  # 256-byte aligned tensors


def test_param_count_at_paper_dims(built_lib):
    assert evo.param_count(evo.cdims(synth.DIMS_TRAIN_CROP, evo.EVO_BF16)) == 1829952


def test_workspace_queries_and_errors(built_lib):
    cd = evo.cdims(synth.DIMS_TRAIN_CROP, evo.EVO_BF16)
    fwd = evo.workspace_size(cd, evo.EVO_MODE_FWD)
    bwd = evo.workspace_size(cd, evo.EVO_MODE_BWD)
    assert 0 < fwd < bwd < 4 * 2 ** 30
    bad = evo.cdims(synth.DIMS_TRAIN_CROP.replace(c_m=100), evo.EVO_BF16)
    with pytest.raises(evo.EvoError) as e:
        evo.workspace_size(bad, evo.EVO_MODE_FWD)
    assert e.value.code == evo.EVO_ERR_UNSUPPORTED
    neg = evo.cdims(synth.DIMS_TRAIN_CROP.replace(n_res=0), evo.EVO_BF16)
    with pytest.raises(evo.EvoError) as e:
        evo.workspace_size(neg, evo.EVO_MODE_FWD)
    assert e.value.code == evo.EVO_ERR_INVALID_ARG
    with pytest.raises(evo.EvoError):
        evo.workspace_size(cd, 7)


def test_pair_slab_field(built_lib):
    """i-slab subbatching (Sec. 3.4.4) shrinks the inference plan's scratch
    (the pair intermediates of one slab instead of the whole grid); it is read
    by the inference plan only, needs the BF16 kernels, and a slab of all the
    rows is the unslabbed plan."""
    d = synth.DIMS_TRAIN_CROP.replace(n_res=1024)
    full = evo.workspace_size(evo.cdims(d, evo.EVO_BF16), evo.EVO_MODE_INFER)
    eighth = evo.workspace_size(evo.cdims(d, evo.EVO_BF16, pair_slab=128), evo.EVO_MODE_INFER)
    assert eighth < 0.5 * full
    assert evo.workspace_size(evo.cdims(d, evo.EVO_BF16, pair_slab=1024), evo.EVO_MODE_INFER) == full
    # the training plans ignore it
    assert evo.workspace_size(evo.cdims(d, evo.EVO_BF16, pair_slab=128), evo.EVO_MODE_FWD) == \
        evo.workspace_size(evo.cdims(d, evo.EVO_BF16), evo.EVO_MODE_FWD)
    with pytest.raises(evo.EvoError) as e:
        evo.workspace_size(evo.cdims(d, evo.EVO_F32, pair_slab=128), evo.EVO_MODE_INFER)
    assert e.value.code == evo.EVO_ERR_UNSUPPORTED
    with pytest.raises(evo.EvoError) as e:
        evo.workspace_size(evo.cdims(d.replace(c_mul=96), evo.EVO_BF16, pair_slab=128), evo.EVO_MODE_INFER)
    assert e.value.code == evo.EVO_ERR_UNSUPPORTED
    with pytest.raises(evo.EvoError) as e:
        evo.workspace_size(evo.cdims(d, evo.EVO_BF16, pair_slab=-1), evo.EVO_MODE_INFER)
    assert e.value.code == evo.EVO_ERR_INVALID_ARG


def test_null_and_misaligned_pointers_are_rejected_before_any_launch(built_lib):
    cd = evo.cdims(synth.DIMS_SMALL_FP32, evo.EVO_F32)
    L = built_lib
    null = ctypes.c_void_p(0)
    r = L.evo_block_fwd(ctypes.byref(cd), null, null, null, null, null, null, null, null, null, 0, null)
    assert r == evo.EVO_ERR_INVALID_ARG
    odd = ctypes.c_void_p(0x1000 + 8)
    r = L.evo_block_fwd(ctypes.byref(cd), odd, null, odd, odd, odd, odd, odd, odd, odd, 1 << 30, null)
    assert r == evo.EVO_ERR_ALIGNMENT


def test_strerror_and_version(built_lib):
    assert evo.strerror(evo.EVO_ERR_TIMEOUT) == "bounded device wait timed out"
    assert b"sm_103a" in built_lib.evo_version()


@pytest.mark.parametrize("d", [synth.DIMS_TEMPLATE, synth.DIMS_TEMPLATE.replace(n_res=37),
                               synth.DIMS_TINY.replace(pair_only=1)])
def test_pair_param_layout_matches_generator_table(built_lib, d):
    cd = evo.cdims(d, evo.EVO_BF16)
    lay = evo.pair_param_layout(cd)
    ref, total = synth.param_layout(d)
    assert [(n, o, s) for n, o, s, _ in ref] == lay
    assert evo.pair_param_count(cd) == total
    assert all(o % 64 == 0 for _, o, _ in lay)


def test_pair_workspace_is_the_pair_share_of_the_block(built_lib):
    d = synth.DIMS_TEMPLATE
    cd = evo.cdims(d, evo.EVO_BF16)
    import ctypes
    n = ctypes.c_size_t(0)
    assert evo.lib().evo_pair_workspace_size(ctypes.byref(cd), evo.EVO_MODE_BWD, ctypes.byref(n)) == evo.EVO_OK
    full = ctypes.c_size_t(0)
    cdf = evo.cdims(d.replace(pair_only=0, n_seq=8), evo.EVO_BF16)
    assert evo.lib().evo_workspace_size(ctypes.byref(cdf), 1, evo.EVO_MODE_BWD, ctypes.byref(full)) == evo.EVO_OK
    assert 0 < n.value < full.value


def test_stack_stride_and_count_are_checked_before_any_launch(built_lib):
    cd = evo.cdims(synth.DIMS_SMALL_FP32, evo.EVO_F32)
    L = built_lib
    null = ctypes.c_void_p(0)
    n = evo.param_count(cd)
    stride = (n + 127) // 128 * 128

    def call(nb, batch, st, sb=None, rb=None, ws=0):
        return L.evo_stack_fwd(ctypes.byref(cd), nb, batch, sb, rb, null, null, ctypes.c_size_t(st), null, null, null,
                               null, null, ctypes.c_size_t(ws), null)

    for nb, st in ((2, stride + 64), (2, stride - 128), (-1, stride)):
        assert call(nb, 1, st) == evo.EVO_ERR_INVALID_ARG, (nb, st)
    # zero blocks is the identity and launches nothing
    assert call(0, 1, stride) == evo.EVO_OK
    # batch sizes: a batch needs its size arrays; sizes within the padded ones;
    # a batch of one is the padded protein itself
    arr = lambda *v: (ctypes.c_int32 * len(v))(*v)
    assert call(2, 0, stride) == evo.EVO_ERR_INVALID_ARG
    assert call(2, 2, stride) == evo.EVO_ERR_INVALID_ARG
    assert call(2, 2, stride, arr(16, 17), arr(64, 64)) == evo.EVO_ERR_INVALID_ARG
    assert call(2, 2, stride, arr(16, 8), arr(0, 64)) == evo.EVO_ERR_INVALID_ARG
    assert call(2, 1, stride, arr(8), arr(64)) == evo.EVO_ERR_INVALID_ARG


def test_stack_workspace_adds_one_staged_protein_for_a_batch(built_lib):
    d = synth.DIMS_SMALL_FP32
    cd = evo.cdims(d, evo.EVO_BF16)
    one = evo.workspace_size(cd, evo.EVO_MODE_FWD)
    two = evo.workspace_size(cd, evo.EVO_MODE_FWD, batch=2)
    assert evo.workspace_size(cd, evo.EVO_MODE_FWD, batch=16) == two
    al = lambda x: (x + 255) // 256 * 256
    S, R = d.n_seq, d.n_res
    staging = al(S * R * d.c_m * 2) + al(R * R * d.c_z * 2) + al(S * R * 4) + al(R * R * 4)
    assert two == one + staging
    with pytest.raises(evo.EvoError):
        evo.workspace_size(cd, evo.EVO_MODE_FWD, batch=0)


def test_adam_step_arguments_are_checked_before_any_launch(built_lib):
    L = built_lib
    null = ctypes.c_void_p(0)
    a = ctypes.c_void_p(0x100000)  # 256-byte aligned, never dereferenced
    odd = ctypes.c_void_p(0x100000 + 16)
    n = 1000
    ws = evo.adam_workspace_size(n)
    assert ws > 0 and evo.adam_workspace_size(0) == 0

    def call(h, n=n, p=a, g=a, m=a, v=a, e=null, pb=null, gn=null, w=a, wsb=ws):
        return L.evo_adam_step(ctypes.byref(h) if h is not None else None, n, p, g, m, v, e, pb, gn, w,
                               ctypes.c_size_t(wsb), null)

    assert call(None) == evo.EVO_ERR_INVALID_ARG
    for bad in (evo.adam_hyper(0), evo.adam_hyper(1, beta1=1.0), evo.adam_hyper(1, beta2=-0.1),
                evo.adam_hyper(1, eps=0.0), evo.adam_hyper(1, lr=float("inf")),
                evo.adam_hyper(1, clip_norm=float("nan"))):
        assert call(bad) == evo.EVO_ERR_INVALID_ARG
    assert call(evo.adam_hyper(1, ema_decay=1.5), e=a) == evo.EVO_ERR_INVALID_ARG
    h = evo.adam_hyper(1)
    assert call(h, n=0, p=null, g=null, m=null, v=null, w=null, wsb=0) == evo.EVO_OK  # empty: nothing to do
    assert call(h, p=null) == evo.EVO_ERR_INVALID_ARG
    assert call(h, w=null) == evo.EVO_ERR_INVALID_ARG
    assert call(h, g=odd) == evo.EVO_ERR_ALIGNMENT
    assert call(h, e=odd) == evo.EVO_ERR_ALIGNMENT
    assert call(h, pb=odd) == evo.EVO_ERR_ALIGNMENT
    assert call(h, wsb=ws - 8) == evo.EVO_ERR_WORKSPACE


def test_infer_plan_is_a_fraction_of_the_forward_plan(built_lib):
    for d in (synth.DIMS_TRAIN_CROP, synth.Dims(n_seq=5, n_res=37), synth.DIMS_EXTRA_MSA):
        for act in (evo.EVO_BF16, evo.EVO_F32):
            cd = evo.cdims(d, act)
            f = evo.workspace_size(cd, evo.EVO_MODE_FWD)
            i = evo.workspace_size(cd, evo.EVO_MODE_INFER)
            assert 0 < i < 0.3 * f, (d, act, i, f)
    # a block at N_res = 8192 (N_seq = 128, BF16): workspace plus m and z
    # (updated in place) stays within one GPU's memory
    d = synth.Dims(n_seq=128, n_res=8192)
    cd = evo.cdims(d, evo.EVO_BF16)
    io = 2 * (d.n_seq * d.n_res * d.c_m + d.n_res * d.n_res * d.c_z)
    assert evo.workspace_size(cd, evo.EVO_MODE_INFER) + io < 260e9
    with pytest.raises(evo.EvoError):
        evo.workspace_size(cd, 3)


def test_infer_arguments_are_checked_before_any_launch(built_lib):
    cd = evo.cdims(synth.DIMS_SMALL_FP32, evo.EVO_F32)
    L = built_lib
    null = ctypes.c_void_p(0)
    a = ctypes.c_void_p(0x100000)
    odd = ctypes.c_void_p(0x100000 + 8)
    need = evo.workspace_size(cd, evo.EVO_MODE_INFER)
    r = L.evo_block_fwd_infer(ctypes.byref(cd), null, null, a, a, a, a, a, a, a, ctypes.c_size_t(need), null)
    assert r == evo.EVO_ERR_INVALID_ARG
    r = L.evo_block_fwd_infer(ctypes.byref(cd), a, null, odd, a, a, a, a, a, a, ctypes.c_size_t(need), null)
    assert r == evo.EVO_ERR_ALIGNMENT
    r = L.evo_block_fwd_infer(ctypes.byref(cd), a, null, a, a, a, a, a, a, a, ctypes.c_size_t(need - 256), null)
    assert r == evo.EVO_ERR_WORKSPACE


def test_binding_declares_every_signature(built_lib):
    """Every function of the header has ctypes argument types in the binding,
    and the ones that return size_t or a string have the matching result
    type (ctypes would otherwise truncate a 64-bit result to int)."""
    import re
    L = built_lib
    txt = re.sub(r"/\*.*?\*/", "", open(evo.HEADER).read(), flags=re.S)
    rets = dict((name, ret.strip()) for ret, name in re.findall(r"(size_t|int|const char \*)\s*(evo_[a-z0-9_]+)\s*\(",
                                                              txt))
    assert set(rets) == set(evo.header_functions())
    for name, ret in rets.items():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        if ret == "size_t":
            assert f.restype is ctypes.c_size_t, name
        elif ret.startswith("const char"):
            assert f.restype is ctypes.c_char_p, name
