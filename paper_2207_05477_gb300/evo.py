"""Thin Python binding of libevo.so (the C ABI in include/evo.h).

Only argument marshalling lives here: every step of the Evoformer block runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.
The library must have been built (``paper_2207_05477_gb300.build.build()``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libevo.so")
HEADER = os.path.join(ROOT, "include", "evo.h")

EVO_OK, EVO_ERR_INVALID_ARG, EVO_ERR_UNSUPPORTED, EVO_ERR_ALIGNMENT = 0, -1, -2, -3
EVO_ERR_WORKSPACE, EVO_ERR_CUDA, EVO_ERR_TIMEOUT = -4, -5, -6
EVO_F32, EVO_BF16 = 0, 1
EVO_COL_ATTENTION, EVO_COL_GLOBAL = 0, 1
EVO_MODE_FWD, EVO_MODE_BWD, EVO_MODE_INFER = 0, 1, 2
EVO_UNIT_GEMM, EVO_UNIT_ATTENTION, EVO_UNIT_TRIMUL, EVO_UNIT_MLP = 0, 1, 2, 3


class EvoError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {code} ({strerror(code)})")


class CDims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_seq", "n_res", "c_m", "c_z", "h_msa", "c_msa", "h_tri", "c_tri",
        "c_mul", "c_opm", "trans_n", "msa_col_mode", "act_dtype", "pair_slab")]


class CProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("calls", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class CParamEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("offset", ctypes.c_int64), ("ndim", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 4)]


class CDropout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("msa_row", "tri_out", "tri_in", "att_start", "att_end")]


class CTuneEntry(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("default_bn", ctypes.c_int32), ("default_splits", ctypes.c_int32), ("bn", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("candidates", ctypes.c_int32)]


class CAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("clip_norm", ctypes.c_float), ("ema_decay", ctypes.c_float),
                ("step", ctypes.c_int32)]


_lib = None
_vp, _sz = ctypes.c_void_p, ctypes.c_size_t


def lib():
    """The loaded libevo.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2207_05477_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.evo_param_count.argtypes = [P(CDims)]
        L.evo_param_count.restype = _sz
        L.evo_param_layout.argtypes = [P(CDims), P(CParamEntry), ctypes.c_int]
        L.evo_params_bf16_size.argtypes = [P(CDims), P(_sz)]
        L.evo_params_to_bf16.argtypes = [P(CDims), _vp, _vp, _vp]
        L.evo_workspace_size.argtypes = [P(CDims), ctypes.c_int, ctypes.c_int, P(_sz)]
        L.evo_block_fwd.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
        L.evo_block_fwd_infer.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
        L.evo_block_bwd.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                    _vp]
        L.evo_block_fwd_dropout.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, P(CDropout), _vp, _sz,
                                            _vp]
        L.evo_block_bwd_dropout.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, P(CDropout), _vp, _vp, _vp, _vp,
                                            _vp, _vp, _sz, _vp]
        L.evo_pair_param_count.argtypes = [P(CDims)]
        L.evo_pair_param_count.restype = _sz
        L.evo_pair_param_layout.argtypes = [P(CDims), P(CParamEntry), ctypes.c_int]
        L.evo_pair_workspace_size.argtypes = [P(CDims), ctypes.c_int, P(_sz)]
        L.evo_pair_params_to_bf16.argtypes = [P(CDims), _vp, _vp, _vp]
        L.evo_pair_block_fwd.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, P(CDropout), _vp, _sz, _vp]
        L.evo_pair_block_bwd.argtypes = [P(CDims), _vp, _vp, _vp, _vp, P(CDropout), _vp, _vp, _vp, _vp, _sz, _vp]
        L.evo_block_fwd_noalloc.argtypes = [P(CDims), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.evo_stack_fwd.argtypes = [P(CDims), ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp, _vp,
                                    _vp, _sz, _vp]
        L.evo_adam_workspace_size.argtypes = [_sz]
        L.evo_adam_workspace_size.restype = _sz
        L.evo_adam_step.argtypes = [P(CAdam), _sz, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
        L.evo_get_error.argtypes = [_vp]
        L.evo_probe_ex2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.evo_debug_wait_timeout.argtypes = [ctypes.c_int, ctypes.c_longlong, _vp]
        L.evo_profile_only.argtypes = [ctypes.c_char_p]
        L.evo_profile_pause.argtypes = [ctypes.c_int]
        L.evo_profile_begin.argtypes = []
        L.evo_profile_end.argtypes = [_vp, P(CProfileEntry), ctypes.c_int]
        L.evo_tune_begin.argtypes = []
        L.evo_tune_end.argtypes = [_vp]
        L.evo_tune_clear.argtypes = []
        L.evo_tune_entries.argtypes = [P(CTuneEntry), ctypes.c_int]
        L.evo_tune_save.argtypes = [ctypes.c_char_p]
        L.evo_tune_load.argtypes = [ctypes.c_char_p]
        L.evo_strerror.argtypes = [ctypes.c_int]
        L.evo_strerror.restype = ctypes.c_char_p
        L.evo_version.argtypes = []
        L.evo_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def header_functions():
    """Names of the functions include/evo.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(evo_[a-z0-9_]+)\s*\(", txt)))


def strerror(code):
    try:
        return lib().evo_strerror(int(code)).decode()
    except Exception:  # during import errors
        return "?"


def _check(code, where):
    if code != EVO_OK:
        raise EvoError(code, where)


def cdims(d, act_dtype, pair_slab=0):
    """ctypes evo_dims from a synth.Dims-like object; pair_slab > 0 runs the
    inference plan's pair stack that many rows at a time (Sec. 3.4.4)."""
    return CDims(d.n_seq, d.n_res, d.c_m, d.c_z, d.h_msa, d.c_msa, d.h_tri, d.c_tri, d.c_mul, d.c_opm,
                 d.trans_n, d.msa_col_mode, act_dtype, pair_slab)


def param_count(cd):
    return int(lib().evo_param_count(ctypes.byref(cd)))


def param_layout(cd):
    n = lib().evo_param_layout(ctypes.byref(cd), None, 0)
    if n < 0:
        raise EvoError(n, "evo_param_layout")
    arr = (CParamEntry * n)()
    lib().evo_param_layout(ctypes.byref(cd), arr, n)
    return [(e.name.decode(), int(e.offset), tuple(int(e.shape[k]) for k in range(e.ndim))) for e in arr]


def workspace_size(cd, mode, batch=1):
    out = _sz(0)
    _check(lib().evo_workspace_size(ctypes.byref(cd), int(batch), mode, ctypes.byref(out)), "evo_workspace_size")
    return int(out.value)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def params_to_bf16(cd, p32, p16, stream=None):
    _check(lib().evo_params_to_bf16(ctypes.byref(cd), _ptr(p32), _ptr(p16), _stream(stream)),
           "evo_params_to_bf16")


def block_fwd(cd, params, params_bf16, m, z, m_out, z_out, msa_mask, pair_mask, ws, stream=None):
    _check(lib().evo_block_fwd(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z), _ptr(m_out),
                               _ptr(z_out), _ptr(msa_mask), _ptr(pair_mask), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream(stream)), "evo_block_fwd")


def _dropout_struct(dropout):
    """CDropout of a dict site -> fp32 device tensor [n_res, channels] (None: no dropout)."""
    if dropout is None:
        return None
    c = CDropout()
    for name, _ in CDropout._fields_:
        t = dropout.get(name)
        setattr(c, name, None if t is None else t.data_ptr())
    return c


def block_fwd_dropout(cd, params, params_bf16, m, z, m_out, z_out, msa_mask, pair_mask, dropout, ws, stream=None):
    """Training-mode block forward: dropout maps site names (msa_row, tri_out, tri_in,
    att_start, att_end) to fp32 scale tensors on the device."""
    c = _dropout_struct(dropout)
    _check(lib().evo_block_fwd_dropout(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z),
                                       _ptr(m_out), _ptr(z_out), _ptr(msa_mask), _ptr(pair_mask),
                                       ctypes.byref(c) if c is not None else None, _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream(stream)), "evo_block_fwd_dropout")


def block_bwd_dropout(cd, params, params_bf16, m, z, msa_mask, pair_mask, dropout, dm_out, dz_out, dm_in, dz_in,
                      dparams, ws, stream=None):
    c = _dropout_struct(dropout)
    _check(lib().evo_block_bwd_dropout(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z),
                                       _ptr(msa_mask), _ptr(pair_mask), ctypes.byref(c) if c is not None else None,
                                       _ptr(dm_out), _ptr(dz_out), _ptr(dm_in), _ptr(dz_in), _ptr(dparams), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream(stream)), "evo_block_bwd_dropout")


def pair_param_count(cd):
    return int(lib().evo_pair_param_count(ctypes.byref(cd)))


def pair_param_layout(cd):
    """[(name, offset, shape)] of the template pair block's flat parameter buffer."""
    n = lib().evo_pair_param_layout(ctypes.byref(cd), None, 0)
    arr = (CParamEntry * n)()
    lib().evo_pair_param_layout(ctypes.byref(cd), arr, n)
    return [(e.name.decode(), e.offset, tuple(e.shape[i] for i in range(e.ndim))) for e in arr]


def pair_workspace(cd, mode, device):
    import torch
    n = _sz(0)
    _check(lib().evo_pair_workspace_size(ctypes.byref(cd), mode, ctypes.byref(n)), "evo_pair_workspace_size")
    return torch.empty(n.value, dtype=torch.uint8, device=device)


def pair_bf16_params(cd, params):
    """BF16 copy of the pair block's flat parameter buffer (None for the FP32 path)."""
    import torch
    if cd.act_dtype != EVO_BF16:
        return None
    p16 = torch.empty(pair_param_count(cd), dtype=torch.bfloat16, device=params.device)
    _check(lib().evo_pair_params_to_bf16(ctypes.byref(cd), _ptr(params), _ptr(p16), _stream(None)),
           "evo_pair_params_to_bf16")
    return p16


def pair_block_fwd(cd, params, params_bf16, z, z_out, pair_mask, ws, dropout=None, stream=None):
    """Template pair stack block forward (AF2 Alg. 16)."""
    c = _dropout_struct(dropout)
    _check(lib().evo_pair_block_fwd(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(z), _ptr(z_out),
                                    _ptr(pair_mask), ctypes.byref(c) if c is not None else None, _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)), "evo_pair_block_fwd")


def pair_block_bwd(cd, params, params_bf16, z, pair_mask, dz_out, dz_in, dparams, ws, dropout=None, stream=None):
    c = _dropout_struct(dropout)
    _check(lib().evo_pair_block_bwd(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(z), _ptr(pair_mask),
                                    ctypes.byref(c) if c is not None else None, _ptr(dz_out), _ptr(dz_in),
                                    _ptr(dparams), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "evo_pair_block_bwd")


def block_fwd_noalloc(cd, params, params_bf16, m, z, m_out, z_out, msa_mask, pair_mask, stream=None):
    """Block forward with the library's own fixed scratch (no workspace, no allocation)."""
    _check(lib().evo_block_fwd_noalloc(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z),
                                       _ptr(m_out), _ptr(z_out), _ptr(msa_mask), _ptr(pair_mask), _stream(stream)),
           "evo_block_fwd_noalloc")


def block_bwd(cd, params, params_bf16, m, z, msa_mask, pair_mask, dm_out, dz_out, dm_in, dz_in, dparams, ws,
              stream=None):
    _check(lib().evo_block_bwd(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z), _ptr(msa_mask),
                               _ptr(pair_mask), _ptr(dm_out), _ptr(dz_out), _ptr(dm_in), _ptr(dz_in), _ptr(dparams),
                               _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "evo_block_bwd")


def block_fwd_infer(cd, params, params_bf16, m, z, m_out, z_out, msa_mask, pair_mask, ws, stream=None):
    """evo_block_fwd_infer: the block forward in the EVO_MODE_INFER workspace."""
    _check(lib().evo_block_fwd_infer(ctypes.byref(cd), _ptr(params), _ptr(params_bf16), _ptr(m), _ptr(z),
                                     _ptr(m_out), _ptr(z_out), _ptr(msa_mask), _ptr(pair_mask), _ptr(ws),
                                     ws.numel() * ws.element_size(), _stream(stream)), "evo_block_fwd_infer")


def stack_fwd(cd, n_blocks, params, params_bf16, param_stride, m, z, msa_mask, pair_mask, ws, stream=None,
              n_seq_b=None, n_res_b=None):
    """n_blocks blocks over m, z in place.  With n_seq_b / n_res_b (lists of
    per-protein sizes) m, z and the masks are padded batches
    [batch, Smax, Rmax, ...] with cd's sizes as Smax, Rmax."""
    batch, sb, rb = 1, None, None
    if n_seq_b is not None:
        batch = len(n_seq_b)
        sb = (ctypes.c_int32 * batch)(*[int(x) for x in n_seq_b])
        rb = (ctypes.c_int32 * batch)(*[int(x) for x in n_res_b])
    _check(lib().evo_stack_fwd(ctypes.byref(cd), n_blocks, batch, sb, rb, _ptr(params), _ptr(params_bf16),
                               param_stride, _ptr(m), _ptr(z), _ptr(msa_mask), _ptr(pair_mask), _ptr(ws),
                               ws.numel() * ws.element_size(), _stream(stream)), "evo_stack_fwd")


def adam_hyper(step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-6, clip_norm=0.1, ema_decay=0.999):
    """evo_adam for step number `step` (defaults: AlphaFold2's training settings)."""
    return CAdam(lr, beta1, beta2, eps, clip_norm, ema_decay, step)


def adam_workspace_size(n):
    return int(lib().evo_adam_workspace_size(n))


def adam_step(h, params, grad, exp_avg, exp_avg_sq, ws, ema=None, params_bf16=None, grad_norm=None, stream=None):
    """evo_adam_step over flat buffers of params.numel() elements."""
    _check(lib().evo_adam_step(ctypes.byref(h), params.numel(), _ptr(params), _ptr(grad), _ptr(exp_avg),
                               _ptr(exp_avg_sq), _ptr(ema), _ptr(params_bf16), _ptr(grad_norm), _ptr(ws),
                               ws.numel() * ws.element_size(), _stream(stream)), "evo_adam_step")


def get_error(stream=None):
    return int(lib().evo_get_error(_stream(stream)))


def probe_ex2(variant, blocks, iters, sink, stream=None):
    """Launches the ex2 throughput probe (variant 0: f32, 1: bf16x2) writing blocks*256 floats to sink."""
    import torch
    assert sink.numel() >= blocks * 256 and sink.dtype == torch.float32 and sink.is_cuda
    _check(lib().evo_probe_ex2(int(variant), int(blocks), int(iters), _ptr(sink), _stream(stream)), "evo_probe_ex2")


def debug_wait_timeout(limit_ns, unit=None, stream=None):
    """One CTA of `unit` (EVO_UNIT_GEMM / _ATTENTION / _TRIMUL / _MLP) whose bounded wait runs out after limit_ns."""
    u = EVO_UNIT_GEMM if unit is None else unit
    _check(lib().evo_debug_wait_timeout(int(u), int(limit_ns), _stream(stream)), "evo_debug_wait_timeout")


def profile_only(kernel_name=None):
    """Restrict the next profile recording to one kernel name (None: all)."""
    _check(lib().evo_profile_only(kernel_name.encode() if kernel_name else None), "evo_profile_only")


def profile_pause(paused=True):
    """Pause or resume launch timing within an open profile session (no synchronisation)."""
    _check(lib().evo_profile_pause(1 if paused else 0), "evo_profile_pause")


def profile_begin():
    _check(lib().evo_profile_begin(), "evo_profile_begin")


def profile_end(stream=None, cap=256):
    """{kernel name: dict(calls, launches, ms, flops, bytes)} recorded since profile_begin."""
    arr = (CProfileEntry * cap)()
    n = lib().evo_profile_end(_stream(stream), arr, cap)
    if n < 0:
        raise EvoError(n, "evo_profile_end")
    return {arr[i].name.decode(): dict(calls=arr[i].calls, launches=arr[i].launches, ms=arr[i].total_ms,
                                       flops=arr[i].flops, bytes=arr[i].bytes) for i in range(min(n, cap))}


def tune_begin():
    """Start a GEMM tile-tuning session (candidates cycle over the launches of each shape)."""
    _check(lib().evo_tune_begin(), "evo_tune_begin")


def tune_end(stream=None):
    """Close the session: keep the fastest candidate per GEMM shape; returns the number of shapes."""
    n = lib().evo_tune_end(_stream(stream))
    if n < 0:
        raise EvoError(n, "evo_tune_end")
    return n


def tune_clear():
    """Drop the tuned table (back to the built-in tile choice)."""
    _check(lib().evo_tune_clear(), "evo_tune_clear")


def tune_save(path):
    """Write the tuned table to a text file."""
    _check(lib().evo_tune_save(str(path).encode()), "evo_tune_save")


def tune_load(path):
    """Replace the tuned table with a file written by tune_save."""
    _check(lib().evo_tune_load(str(path).encode()), "evo_tune_load")


def tune_entries(cap=512):
    """[dict(M, N, K, batch, default_bn, default_splits, bn, splits, candidates)] of the tuned table."""
    arr = (CTuneEntry * cap)()
    n = lib().evo_tune_entries(arr, cap)
    return [{f: getattr(arr[i], f) for f, _ in CTuneEntry._fields_} for i in range(min(n, cap))]


# ------------------------------------------------------------- torch glue

def _torch_dtype(act_dtype):
    import torch
    return torch.bfloat16 if act_dtype == EVO_BF16 else torch.float32


def workspace(cd, mode, device, batch=1):
    import torch
    return torch.empty(workspace_size(cd, mode, batch), dtype=torch.uint8, device=device)


def bf16_params(cd, params):
    """BF16 copy of the flat parameter buffer (None for the FP32 path)."""
    import torch
    if cd.act_dtype != EVO_BF16:
        return None
    p16 = torch.empty(param_count(cd), dtype=torch.bfloat16, device=params.device)
    params_to_bf16(cd, params, p16)
    return p16


def _autograd_fn():
    import torch

    class EvoBlockFn(torch.autograd.Function):
        """One Evoformer block; backward recomputes the block (only m, z saved)."""

        @staticmethod
        def forward(ctx, m, z, params, msa_mask, pair_mask, cd, dropout=None):
            m, z = m.contiguous(), z.contiguous()
            p16 = bf16_params(cd, params)
            m_out, z_out = torch.empty_like(m), torch.empty_like(z)
            ws = workspace(cd, EVO_MODE_FWD, m.device)
            if dropout is None:
                block_fwd(cd, params, p16, m, z, m_out, z_out, msa_mask, pair_mask, ws)
            else:
                block_fwd_dropout(cd, params, p16, m, z, m_out, z_out, msa_mask, pair_mask, dropout, ws)
            ctx.save_for_backward(m, z, params, msa_mask, pair_mask)
            ctx.cd = cd
            ctx.dropout = dropout  # the same draw must be replayed by the recompute
            ctx.mark_non_differentiable(msa_mask, pair_mask)
            return m_out, z_out

        @staticmethod
        def backward(ctx, dm, dz):
            m, z, params, msa_mask, pair_mask = ctx.saved_tensors
            cd = ctx.cd
            dt = _torch_dtype(cd.act_dtype)
            dm = torch.zeros_like(m) if dm is None else dm.to(dt).contiguous()
            dz = torch.zeros_like(z) if dz is None else dz.to(dt).contiguous()
            p16 = bf16_params(cd, params)
            dm_in, dz_in = torch.empty_like(m), torch.empty_like(z)
            dparams = torch.zeros_like(params)
            ws = workspace(cd, EVO_MODE_BWD, m.device)
            if ctx.dropout is None:
                block_bwd(cd, params, p16, m, z, msa_mask, pair_mask, dm, dz, dm_in, dz_in, dparams, ws)
            else:
                block_bwd_dropout(cd, params, p16, m, z, msa_mask, pair_mask, ctx.dropout, dm, dz, dm_in, dz_in,
                                  dparams, ws)
            return dm_in, dz_in, dparams, None, None, None, None

    return EvoBlockFn


_EvoBlockFn = None


def evoformer_block(m, z, params, msa_mask, pair_mask, cd, dropout=None):
    """Differentiable Evoformer block through libevo (forward and backward kernels).
    dropout: None (evaluation mode) or a dict of the site scales (training mode,
    see block_fwd_dropout); the backward replays the same draw."""
    global _EvoBlockFn
    if _EvoBlockFn is None:
        _EvoBlockFn = _autograd_fn()
    return _EvoBlockFn.apply(m, z, params, msa_mask, pair_mask, cd, dropout)


def evoformer_stack(m, z, params_list, msa_mask, pair_mask, cd, dropouts=None):
    """Stack of blocks; each block recomputes itself in backward (per-block recompute).
    dropouts: None or one dropout dict per block."""
    for i, p in enumerate(params_list):
        m, z = evoformer_block(m, z, p, msa_mask, pair_mask, cd, None if dropouts is None else dropouts[i])
    return m, z
