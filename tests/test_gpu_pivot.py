"""Accuracy of the Cholesky pivot routine of the stage factorizations.

The float64 pivot d -> (sqrt(d), 1/sqrt(d)) is built from a float32 reciprocal
square root estimate and a float64 series correction, with the library routines
outside [2^-120, 2^120].  Both results are compared with the exact values
(rounded from extended precision) over the whole exponent range of positive
normal doubles, on both sides of the two switch points: at most 2 ulp.  The
float32 pivot (rsqrtf and one Newton step) is held to 3 ulp over the float32
normal range.  The entry point cyq_pivot_eval runs the device routine itself.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _inputs64(n, seed=0):
    g = np.random.default_rng(seed)
    # random mantissas over every normal exponent
    ex = g.integers(-1021, 1023, size=n)
    d = np.ldexp(g.uniform(1.0, 2.0, size=n), ex)
    # dense sampling around the switch points 2^-120, 2^-119, 2^120, 2^121 and around 1
    edges = []
    for p in (-121, -120, -119, -118, 0, 119, 120, 121, 122):
        base = np.ldexp(1.0, p)
        k = np.arange(-2000, 2000)
        edges.append(base + k * np.spacing(base))
        edges.append(np.nextafter(base, 0.0) - np.arange(0, 50) * np.spacing(np.nextafter(base, 0.0)))
    # mantissa all ones, powers of two, smallest and largest normals
    special = np.concatenate([np.ldexp(np.nextafter(2.0, 0.0), np.arange(-1022, 1023)),
                              np.ldexp(1.0, np.arange(-1022, 1024)),
                              [np.finfo(np.float64).tiny, np.finfo(np.float64).max]])
    d = np.concatenate([d] + edges + [special])
    return d[(d > 0) & np.isfinite(d) & (d >= np.finfo(np.float64).tiny)]


def _ulp_err(x, ref_ld, dtype):
    ref = ref_ld.astype(dtype)
    sp = np.spacing(np.abs(ref)).astype(np.longdouble)
    return np.abs(x.astype(np.longdouble) - ref_ld) / sp


def test_pivot_float64_within_two_ulp_everywhere():
    torch, cyq = require_gpu()
    lib = cyq.load()
    d = _inputs64(1_000_000)
    assert d.size > 1_000_000
    dt = torch.from_numpy(d).cuda()
    l, il = torch.empty_like(dt), torch.empty_like(dt)
    code = lib.cyq_pivot_eval(ctypes.c_void_p(dt.data_ptr()), ctypes.c_void_p(l.data_ptr()),
                              ctypes.c_void_p(il.data_ptr()), None, None, None, d.size,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    l, il = l.cpu().numpy(), il.cpu().numpy()
    dl = d.astype(np.longdouble)
    s_ref = np.sqrt(dl)
    is_ref = 1.0 / s_ref
    e_l = _ulp_err(l, s_ref, np.float64)
    e_il = _ulp_err(il, is_ref, np.float64)
    worst = int(np.argmax(np.maximum(e_l, e_il)))
    assert e_l.max() <= 2.0 and e_il.max() <= 2.0, (float(e_l.max()), float(e_il.max()), d[worst])
    # the series branch (inside [2^-119, 2^120)) alone is also within 2 ulp
    inner = (d >= np.ldexp(1.0, -119)) & (d < np.ldexp(1.0, 120))
    assert inner.sum() > 100_000 and (~inner).sum() > 100_000


def test_pivot_float32_within_three_ulp():
    torch, cyq = require_gpu()
    lib = cyq.load()
    g = np.random.default_rng(1)
    ex = g.integers(-125, 127, size=500_000)
    d = np.ldexp(g.uniform(1.0, 2.0, size=ex.size), ex).astype(np.float32)
    d = np.concatenate([d, np.ldexp(np.float32(1.0), np.arange(-126, 128)).astype(np.float32),
                        np.ldexp(np.nextafter(np.float32(2.0), np.float32(0.0)),
                                 np.arange(-126, 127)).astype(np.float32)])
    d = d[np.isfinite(d) & (d >= np.finfo(np.float32).tiny)]
    dt = torch.from_numpy(d).cuda()
    l, il = torch.empty_like(dt), torch.empty_like(dt)
    code = lib.cyq_pivot_eval(None, None, None, ctypes.c_void_p(dt.data_ptr()), ctypes.c_void_p(l.data_ptr()),
                              ctypes.c_void_p(il.data_ptr()), d.size,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    l, il = l.cpu().numpy(), il.cpu().numpy()
    s_ref = np.sqrt(d.astype(np.longdouble))
    e_l = _ulp_err(l, s_ref, np.float32)
    e_il = _ulp_err(il, 1.0 / s_ref, np.float32)
    assert e_l.max() <= 3.0 and e_il.max() <= 3.0, (float(e_l.max()), float(e_il.max()))
