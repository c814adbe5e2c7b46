"""GB300-native MOFF imaging library -- Python binding of ``libmoff.so``.

Morales (arXiv 0812.3669), Sec. 4, Eq. m6: per channel and time sample,
weight the 4-bit antenna voltages, grid them through each antenna's kernel,
transform the grid to the sky and sum |E|^2 (and the cross-pol products).
All of it runs in the CUDA kernels of ``libmoff.so`` (csrc/); this module
only marshals arguments through ctypes.  Functions carry the C names of
``include/moff.h``; :class:`Plan` wraps them for convenience.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory, passed with ``on_device = 1``).  Complex inputs are converted to
interleaved float32 pairs, the ABI's format.  If the library is not built,
every call raises :class:`MoffError` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

__all__ = [
    "MoffError", "lib", "build", "LIB_PATH", "MOFF_FSTAGE", "MOFF_JONES", "MOFF_PREC_FP32", "MOFF_PREC_FP16TC",
    "moff_plan_create", "moff_set_gains", "moff_set_fstage", "moff_submit", "moff_submit_adc",
    "moff_channelise", "moff_grid_snapshot", "moff_read_image", "moff_sync", "moff_reset",
    "moff_plan_info", "moff_plan_route", "moff_voltage_planes", "moff_plan_destroy", "moff_last_error", "moff_set_timing", "moff_timing",
    "moff_image_noalloc", "moff_tc_selftest", "MOFF_SERVED", "MOFF_AUTOTUNE", "MOFF_GRAPH", "MOFF_PERSIST", "moff_plan_tuning", "moff_plan_dft_tuning",
    "moff_export_accumulators", "moff_import_accumulators",
    "moff_server_create", "moff_server_submit", "moff_server_poll", "moff_server_wait", "moff_server_stats",
    "moff_server_destroy", "moff_set_calibrator", "moff_read_feedback", "moff_feedback_gains",
    "moff_set_autocorr", "moff_read_image_cross", "moff_set_beams", "moff_read_beams", "moff_set_channel_groups",
    "Plan", "Server", "header_symbols", "KERNEL_KINDS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoff.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "moff.h")

MOFF_PREC_FP32 = 0
MOFF_PREC_FP16TC = 1
MOFF_FSTAGE = 1 << 1
MOFF_JONES = 1 << 2
MOFF_SERVED = 1 << 3
MOFF_AUTOTUNE = 1 << 4
MOFF_GRAPH = 1 << 5
MOFF_PERSIST = 1 << 6

KERNEL_KINDS = {0: "pfb_fstage", 1: "grid_rows", 2: "cols_integrate", 3: "volt_prep", 4: "fstage_reorder",
                5: "feedback_corr", 6: "autocorr", 7: "row_transform", 8: "persistent"}

STATUS = {0: "MOFF_OK", -1: "MOFF_EINVAL", -2: "MOFF_ENOMEM", -3: "MOFF_ECUDA",
          -4: "MOFF_ESTATE", -5: "MOFF_ETIMEDOUT", -6: "MOFF_EBUSY"}


class MoffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp, _i, _u, _ll, _f = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_longlong, ctypes.c_float
_SIGS = {
    "moff_plan_create": [ctypes.POINTER(_vp), _i, _vp, _i, _vp, _i, _i, _i, _u, _vp],
    "moff_set_gains": [_vp, _vp, _i],
    "moff_set_channel_groups": [_vp, _i, _vp, _vp, _vp],
    "moff_set_fstage": [_vp, _i, _vp, _f],
    "moff_submit": [_vp, _vp, _i, _i],
    "moff_submit_adc": [_vp, _vp, _ll, _i],
    "moff_channelise": [_vp, _vp, _ll, _i, _vp, _i, _i],
    "moff_grid_snapshot": [_vp, _vp, _i, _i, _vp],
    "moff_read_image": [_vp, _vp, ctypes.POINTER(_ll), _i, _i, _i],
    "moff_sync": [_vp, _i],
    "moff_reset": [_vp],
    "moff_plan_info": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                       ctypes.POINTER(_ll)],
    "moff_plan_route": [_vp, ctypes.POINTER(_i)],
    "moff_voltage_planes": [_vp, _vp, _i, _i, _i, _vp, ctypes.POINTER(_f)],
    "moff_plan_destroy": [_vp],
    "moff_set_timing": [_vp, _i],
    "moff_timing": [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_ll), _i],
    "moff_image_noalloc": [_i, _vp, _i, _vp, _i, _i, _i, _u, _vp, _i, _vp, _vp, _vp],
    "moff_tc_selftest": [_vp, _vp, _vp, _i, _i, _i, _vp],
    "moff_server_create": [ctypes.POINTER(_vp), _ll, _i],
    "moff_server_submit": [_vp, _vp, _vp, _i, _i, ctypes.POINTER(_ll)],
    "moff_server_poll": [_vp, _ll, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double)],
    "moff_server_wait": [_vp, _ll, _i],
    "moff_server_stats": [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_ll), _i],
    "moff_server_destroy": [_vp],
    "moff_set_calibrator": [_vp, _i, _i],
    "moff_set_autocorr": [_vp, _i],
    "moff_read_image_cross": [_vp, _vp, ctypes.POINTER(_ll), _i, _i, _i],
    "moff_set_beams": [_vp, _i, _vp, _vp],
    "moff_read_beams": [_vp, _vp, ctypes.POINTER(_i), _i, _i],
    "moff_read_feedback": [_vp, _vp, _vp, ctypes.POINTER(_ll), _i, _i],
    "moff_feedback_gains": [_vp, _vp, _i],
    "moff_plan_tuning": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i)],
    "moff_export_accumulators": [_vp, _vp, ctypes.POINTER(_ll), _i, _i],
    "moff_import_accumulators": [_vp, _vp, _ll, _i],
    "moff_plan_dft_tuning": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)],
}


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile libmoff.so in-tree (nvcc, sm_103a)."""
    from . import buildlib as _b
    return _b.build(verbose=verbose, force=force)


def lib() -> ctypes.CDLL:
    """Load libmoff.so (raises MoffError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MoffError(-4, f"{LIB_PATH} is not built; call paper_0812_3669_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.moff_last_error.argtypes = []
        L.moff_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Names of the functions declared in include/moff.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:moff_status|const char \*)\s*\n?\s*(moff_\w+)\s*\(", txt, re.M)))


def moff_last_error() -> str:
    return lib().moff_last_error().decode()


def _check(status):
    if status != 0:
        raise MoffError(status, moff_last_error())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _addr(x):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous):
        raise ValueError("array must be a C-contiguous numpy array")
    return ctypes.c_void_p(x.ctypes.data), 0


def _f32_interleaved(z):
    """complex host array -> contiguous float32 (re, im) pairs."""
    z = np.ascontiguousarray(np.asarray(z), dtype=np.complex64)
    return z.view(np.float32)


def _torch_f32_interleaved(t):
    import torch
    if t.is_complex():
        t = torch.view_as_real(t.to(torch.complex64).contiguous())
    return t.contiguous()


# ----------------------------------------------------------------- C-named functions

def moff_plan_create(pos, taps, grid_n, n_chan, n_pol, flags=0, cuda_stream=None):
    """Create a plan; ``pos`` float64 [A][2], ``taps`` complex kernels (see moff.h)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    taps = np.asarray(taps)
    ksize = int(taps.shape[-1])
    t32 = _f32_interleaved(taps)
    out = ctypes.c_void_p()
    st = ctypes.c_void_p(int(cuda_stream)) if cuda_stream else None
    _check(lib().moff_plan_create(ctypes.byref(out), int(pos.shape[0]), pos.ctypes.data, ksize, t32.ctypes.data,
                                  int(grid_n), int(n_chan), int(n_pol), int(flags), st))
    return out


def moff_set_gains(plan, gains):
    if _is_torch(gains):
        g = _torch_f32_interleaved(gains)
        _check(lib().moff_set_gains(plan, ctypes.c_void_p(g.data_ptr()), int(g.is_cuda)))
    else:
        g = _f32_interleaved(gains)
        _check(lib().moff_set_gains(plan, g.ctypes.data, 0))


def moff_set_channel_groups(plan, pos, taps, chan_group=None):
    """Channel-dependent positions and kernels: ``pos`` float64 [G][A][2], ``taps``
    complex [G][A][...] laid out as for moff_plan_create, ``chan_group`` int [C]."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    t32 = _f32_interleaved(taps)
    g = None if chan_group is None else np.ascontiguousarray(chan_group, dtype=np.int32)
    _check(lib().moff_set_channel_groups(plan, int(pos.shape[0]), pos.ctypes.data, t32.ctypes.data,
                                         None if g is None else g.ctypes.data))


def moff_set_fstage(plan, n_taps, coeffs=None, scale=1.0):
    c = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float32)
    _check(lib().moff_set_fstage(plan, int(n_taps), None if c is None else c.ctypes.data, float(scale)))


def moff_submit(plan, volt):
    """``volt`` uint8 [T][C][A][P] (numpy, or a CUDA uint8 tensor)."""
    p, dev = _addr(volt)
    _check(lib().moff_submit(plan, p, int(volt.shape[0]), dev))


def moff_submit_adc(plan, adc):
    """``adc`` int8 [A][P][S]."""
    p, dev = _addr(adc)
    _check(lib().moff_submit_adc(plan, p, int(adc.shape[-1]), dev))


def moff_channelise(plan, adc, out, out_kind=0):
    pi, din = _addr(adc)
    po, dout = _addr(out)
    _check(lib().moff_channelise(plan, pi, int(adc.shape[-1]), din, po, int(out_kind), dout))


def moff_grid_snapshot(plan, volt, chan, out):
    p, dev = _addr(volt)
    o, _ = _addr(out)
    _check(lib().moff_grid_snapshot(plan, p, dev, int(chan), o))


def moff_read_image(plan, out, reset=0, timeout_ms=-1):
    o, dev = _addr(out)
    n = ctypes.c_longlong(0)
    _check(lib().moff_read_image(plan, o, ctypes.byref(n), int(reset), int(timeout_ms), dev))
    return n.value


def moff_sync(plan, timeout_ms=-1):
    _check(lib().moff_sync(plan, int(timeout_ms)))


def moff_reset(plan):
    _check(lib().moff_reset(plan))


def moff_plan_info(plan):
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    e = ctypes.c_longlong()
    _check(lib().moff_plan_info(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                ctypes.byref(e)))
    return dict(n_prod=a.value, rows_per_stripe=b.value, time_chunk=c.value, chan_chunk=d.value,
                device_bytes=e.value)


ROUTES = {0: "fp32", 1: "fp16_rowspec", 2: "fp16_dft", 3: "fp16_tcgrid"}


def moff_plan_route(plan) -> str:
    """The plan's arithmetic route: "fp32", "fp16_rowspec", "fp16_dft" or "fp16_tcgrid" (see MOFF_PREC_FP16TC)."""
    r = ctypes.c_int()
    _check(lib().moff_plan_route(plan, ctypes.byref(r)))
    return ROUTES[r.value]


def moff_voltage_planes(plan, volt, chan, n_ant, n_pol):
    """The row-spectrum route's FP16 voltage planes of one channel (diagnostic):
    returns (complex64 [T][A][P] plane values, the channel's power-of-two scale)."""
    a, dev = _addr(volt)
    T = int(volt.shape[0])
    out = np.empty((T, n_ant, n_pol, 2), dtype=np.float32)
    sc = ctypes.c_float(0.0)
    _check(lib().moff_voltage_planes(plan, a, T, dev, int(chan), out.ctypes.data, ctypes.byref(sc)))
    return out[..., 0] + 1j * out[..., 1], sc.value


def moff_plan_tuning(plan):
    a, b, p, c, w = (ctypes.c_int() for _ in range(5))
    d = ctypes.c_double()
    _check(lib().moff_plan_tuning(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(p), ctypes.byref(c),
                                  ctypes.byref(d), ctypes.byref(w)))
    return dict(time_batch=a.value, staged=b.value, cells_per_lane=p.value, cell_pairs=int(p.value == 2),
                source=c.value, best_ms=d.value,
                wide_rows=w.value)


def moff_plan_dft_tuning(plan):
    w, src = ctypes.c_int(), ctypes.c_int()
    m8, m16 = ctypes.c_double(), ctypes.c_double()
    _check(lib().moff_plan_dft_tuning(plan, ctypes.byref(w), ctypes.byref(src), ctypes.byref(m8), ctypes.byref(m16)))
    return dict(cols_width=w.value, source=src.value, ms_w8=m8.value, ms_w16=m16.value)


def moff_export_accumulators(plan, out, timeout_ms=-1):
    """The plan's FP64 image sums into ``out`` (host float64 array or CUDA tensor,
    [C][n_prod][N][N]); returns the sample count."""
    a, dev = _addr(out)
    n = ctypes.c_longlong(0)
    _check(lib().moff_export_accumulators(plan, a, ctypes.byref(n), dev, int(timeout_ms)))
    return n.value


def moff_import_accumulators(plan, src, n_samples):
    a, dev = _addr(src)
    _check(lib().moff_import_accumulators(plan, a, int(n_samples), dev))


def moff_set_calibrator(plan, kx, ky):
    _check(lib().moff_set_calibrator(plan, int(kx), int(ky)))


def moff_read_feedback(plan, C, A, P, reset=0, timeout_ms=-1):
    """(R complex64 [C, A, P], S float64 [C, P], n_samples) of Sec. 6."""
    corr = np.empty((C, A, P), dtype=np.complex64)
    power = np.empty((C, P), dtype=np.float64)
    n = ctypes.c_longlong(0)
    _check(lib().moff_read_feedback(plan, corr.ctypes.data, power.ctypes.data, ctypes.byref(n), int(reset),
                                    int(timeout_ms)))
    return corr, power, n.value


def moff_feedback_gains(plan, C, A, P, apply=0):
    """Gain-error estimate delta_g complex64 [C, A, P] (Sec. 6); apply=1 adds it to the plan's gains."""
    d = np.empty((C, A, P), dtype=np.complex64)
    _check(lib().moff_feedback_gains(plan, d.ctypes.data, int(apply)))
    return d


def moff_set_autocorr(plan, on):
    _check(lib().moff_set_autocorr(plan, int(on)))


def moff_read_image_cross(plan, out, reset=0, timeout_ms=-1):
    o, dev = _addr(out)
    n = ctypes.c_longlong(0)
    _check(lib().moff_read_image_cross(plan, o, ctypes.byref(n), int(reset), int(timeout_ms), dev))
    return n.value


def moff_set_beams(plan, kx, ky):
    kx = np.ascontiguousarray(kx, dtype=np.int32)
    ky = np.ascontiguousarray(ky, dtype=np.int32)
    if kx.shape != ky.shape:
        raise ValueError("kx and ky must have the same length")
    _check(lib().moff_set_beams(plan, int(kx.size), kx.ctypes.data if kx.size else None,
                                ky.ctypes.data if ky.size else None))


def moff_read_beams(plan, out=None, timeout_ms=-1):
    """Number of samples in the last block's beams; fills ``out`` [T][C][n_beams][P] complex64 if given."""
    n = ctypes.c_int(0)
    o, dev = _addr(out) if out is not None else (None, 0)
    _check(lib().moff_read_beams(plan, o, ctypes.byref(n), int(timeout_ms), dev))
    return n.value


def moff_set_timing(plan, on):
    _check(lib().moff_set_timing(plan, int(on)))


def moff_timing(plan, kind, reset=0):
    """(total device ms, launch count) of one kernel kind since timing was switched on."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    _check(lib().moff_timing(plan, int(kind), ctypes.byref(ms), ctypes.byref(n), int(reset)))
    return ms.value, n.value


def moff_image_noalloc(pos, taps, grid_n, n_chan, n_pol, volt, gains, image, jones=False, cuda_stream=None):
    """Image one block without any GPU allocation by the library.  ``volt``
    (uint8 [T][C][A][P]), ``gains`` (complex [C][A][P]) and ``image`` (float32
    [C][n_prod][N][N]) are CUDA tensors; ``pos``/``taps`` are host arrays."""
    import torch
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    taps = np.asarray(taps)
    t32 = _f32_interleaved(taps)
    g = _torch_f32_interleaved(gains)
    for name, x in (("volt", volt), ("gains", g), ("image", image)):
        if not (_is_torch(x) and x.is_cuda and x.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
    # the library reads and writes exactly these extents: refuse anything else here
    A, P, C, N = int(pos.shape[0]), int(n_pol), int(n_chan), int(grid_n)
    n_prod = 1 if P == 1 else 4
    if pos.ndim != 2 or pos.shape[1] != 2:
        raise ValueError("pos must be float64 [A][2]")
    K = int(taps.shape[-1])
    want_taps = (A, 2, 2, K, K) if jones else (A, P, K, K)
    if tuple(taps.shape) != want_taps:
        raise ValueError(f"taps must have shape {want_taps}, got {tuple(taps.shape)}")
    if volt.dtype != torch.uint8 or volt.dim() != 4 or tuple(volt.shape[1:]) != (C, A, P):
        raise ValueError(f"volt must be uint8 [T][{C}][{A}][{P}], got {volt.dtype} {tuple(volt.shape)}")
    if g.dtype != torch.float32 or g.numel() != C * A * P * 2:
        raise ValueError(f"gains must hold {C}x{A}x{P} complex values")
    if image.dtype != torch.float32 or image.numel() != C * n_prod * N * N:
        raise ValueError(f"image must be float32 with {C}x{n_prod}x{N}x{N} elements")
    if cuda_stream is None:
        cuda_stream = torch.cuda.current_stream().cuda_stream or 1
    _check(lib().moff_image_noalloc(int(pos.shape[0]), pos.ctypes.data, int(taps.shape[-1]), t32.ctypes.data,
                                    int(grid_n), int(n_chan), int(n_pol), MOFF_JONES if jones else 0,
                                    ctypes.c_void_p(volt.data_ptr()), int(volt.shape[0]),
                                    ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(image.data_ptr()),
                                    ctypes.c_void_p(int(cuda_stream))))


def moff_tc_selftest(a, b, d, mode=0, cuda_stream=None):
    """D = A B^T on the tensor cores (diagnostic): ``a`` half [128][k], ``b`` half [n][k], ``d`` float [128][n]
    (CUDA tensors)."""
    if cuda_stream is None:
        import torch
        cuda_stream = torch.cuda.current_stream().cuda_stream or 1
    _check(lib().moff_tc_selftest(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(d.data_ptr()), int(b.shape[0]), int(a.shape[1]), int(mode),
                                  ctypes.c_void_p(int(cuda_stream))))


def moff_plan_destroy(plan):
    _check(lib().moff_plan_destroy(plan))


# ----------------------------------------------------------------- convenience

def moff_server_create(hbm_budget_bytes, n_slots):
    out = ctypes.c_void_p()
    _check(lib().moff_server_create(ctypes.byref(out), int(hbm_budget_bytes), int(n_slots)))
    return out


def moff_server_submit(server, plan, volt):
    """Queue ``volt`` uint8 [T][C][A][P] for a MOFF_SERVED plan; returns the ticket.
    The caller keeps ``volt`` alive until the ticket is done."""
    p, dev = _addr(volt)
    t = ctypes.c_longlong(0)
    _check(lib().moff_server_submit(server, plan, p, int(volt.shape[0]), dev, ctypes.byref(t)))
    return t.value


def moff_server_poll(server, ticket):
    """(state, latency_ms): state 0 queued, 1 on the GPU, 2 done, < 0 failed."""
    st = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(lib().moff_server_poll(server, int(ticket), ctypes.byref(st), ctypes.byref(ms)))
    return st.value, ms.value


def moff_server_wait(server, ticket=0, timeout_ms=-1):
    _check(lib().moff_server_wait(server, int(ticket), int(timeout_ms)))


def moff_server_stats(server, reset=0):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_longlong()
    _check(lib().moff_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n),
                                   int(reset)))
    return dict(p50_ms=a.value, p99_ms=b.value, throughput=c.value, completed=n.value)


def moff_server_destroy(server):
    _check(lib().moff_server_destroy(server))


class Server:
    """Streaming request loop over MOFF_SERVED plans (owns a ``moff_server``).
    Keeps every submitted block referenced until its ticket is seen done."""

    def __init__(self, hbm_budget_bytes, n_slots):
        self.handle = moff_server_create(hbm_budget_bytes, n_slots)
        self._held = {}

    def submit(self, plan, volt):
        h = plan.handle if isinstance(plan, Plan) else plan
        t = moff_server_submit(self.handle, h, volt)
        self._held[t] = volt
        return t

    def poll(self, ticket):
        st, ms = moff_server_poll(self.handle, ticket)
        if st == 2 or st < 0:
            self._held.pop(ticket, None)
        return st, ms

    def wait(self, ticket=0, timeout_ms=-1):
        moff_server_wait(self.handle, ticket, timeout_ms)
        if ticket == 0:
            self._held.clear()
        else:
            self._held.pop(ticket, None)

    def stats(self, reset=False):
        return moff_server_stats(self.handle, int(reset))

    def close(self):
        if getattr(self, "handle", None) is not None:
            moff_server_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """One array's imaging plan (owns a ``moff_plan``)."""

    def __init__(self, pos, taps, grid_n, n_chan, n_pol, jones=False, fstage=False, stream=None, fp16tc=False,
                 served=False, autotune=False, graph=False, persist=False):
        flags = (MOFF_JONES if jones else 0) | (MOFF_FSTAGE if fstage else 0) | (MOFF_PREC_FP16TC if fp16tc else 0)
        flags |= (MOFF_SERVED if served else 0) | (MOFF_AUTOTUNE if autotune else 0) | (MOFF_GRAPH if graph else 0)
        flags |= MOFF_PERSIST if persist else 0
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    # torch's default stream has handle 0, which the ABI reads as
                    # "make a private stream"; pass cudaStreamLegacy (0x1) so work
                    # is ordered with tensors produced on that stream.
                    stream = torch.cuda.current_stream().cuda_stream or 1
            except ImportError:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream or 1
        self.A = int(np.asarray(pos).shape[0])
        self.N, self.C, self.P = int(grid_n), int(n_chan), int(n_pol)
        self.n_prod = 1 if n_pol == 1 else 4
        self.n_taps = 8
        self.handle = moff_plan_create(pos, taps, grid_n, n_chan, n_pol, flags, stream)

    def set_gains(self, gains):
        moff_set_gains(self.handle, gains)

    def set_channel_groups(self, pos, taps, chan_group=None):
        moff_set_channel_groups(self.handle, pos, taps, chan_group)

    def set_fstage(self, n_taps=8, coeffs=None, scale=1.0):
        moff_set_fstage(self.handle, n_taps, coeffs, scale)
        self.n_taps = int(n_taps)

    def submit(self, volt):
        moff_submit(self.handle, volt)

    def submit_adc(self, adc):
        moff_submit_adc(self.handle, adc)

    def channelise(self, adc, kind=0, out=None):
        if out is None:
            F = adc.shape[-1] // (2 * self.C) - self.n_taps + 1
            shape = (F, self.C, self.A, self.P)
            out = np.empty(shape, dtype=np.uint8) if kind == 0 else np.empty(shape, dtype=np.complex64)
        moff_channelise(self.handle, adc, out, kind)
        return out

    def grid_snapshot(self, volt, chan):
        out = np.empty((self.P, self.N, self.N), dtype=np.complex64)
        moff_grid_snapshot(self.handle, volt, chan, out)
        return out

    def read_image(self, reset=False, timeout_ms=-1, out=None):
        if out is None:
            out = np.empty((self.C, self.n_prod, self.N, self.N), dtype=np.float32)
        n = moff_read_image(self.handle, out, int(reset), timeout_ms)
        return out, n

    def sync(self, timeout_ms=-1):
        moff_sync(self.handle, timeout_ms)

    def reset(self):
        moff_reset(self.handle)

    def info(self):
        return moff_plan_info(self.handle)

    def route(self):
        return moff_plan_route(self.handle)

    def voltage_planes(self, volt, chan):
        return moff_voltage_planes(self.handle, volt, chan, self.A, self.P)

    def set_timing(self, on=True):
        moff_set_timing(self.handle, on)

    def tuning(self):
        return moff_plan_tuning(self.handle)

    def dft_tuning(self):
        return moff_plan_dft_tuning(self.handle)

    def _check_acc(self, buf):
        n = self.C * self.n_prod * self.N * self.N
        if _is_torch(buf):
            import torch
            ok = buf.dtype == torch.float64 and buf.numel() == n
        else:
            ok = isinstance(buf, np.ndarray) and buf.dtype == np.float64 and buf.size == n
        if not ok:
            raise ValueError(f"accumulators must be float64 with {n} elements ([C][n_prod][N][N])")

    def export_accumulators(self, out=None, timeout_ms=-1):
        """(float64 [C][n_prod][N][N] sums, sample count): a checkpoint of the integration."""
        if out is None:
            out = np.empty((self.C, self.n_prod, self.N, self.N), dtype=np.float64)
        self._check_acc(out)
        return out, moff_export_accumulators(self.handle, out, timeout_ms)

    def import_accumulators(self, src, n_samples):
        self._check_acc(src)
        moff_import_accumulators(self.handle, src, n_samples)

    def set_calibrator(self, kx, ky):
        moff_set_calibrator(self.handle, kx, ky)

    def read_feedback(self, reset=False, timeout_ms=-1):
        return moff_read_feedback(self.handle, self.C, self.A, self.P, int(reset), timeout_ms)

    def feedback_gains(self, apply=False):
        return moff_feedback_gains(self.handle, self.C, self.A, self.P, int(apply))

    def set_autocorr(self, on=True):
        moff_set_autocorr(self.handle, on)

    def read_image_cross(self, reset=False, timeout_ms=-1, out=None):
        if out is None:
            out = np.empty((self.C, self.n_prod, self.N, self.N), dtype=np.float32)
        n = moff_read_image_cross(self.handle, out, int(reset), timeout_ms)
        return out, n

    def set_beams(self, kx, ky):
        moff_set_beams(self.handle, kx, ky)
        self.n_beams = len(kx)

    def read_beams(self, timeout_ms=-1):
        T = moff_read_beams(self.handle, None, timeout_ms)
        out = np.empty((T, self.C, self.n_beams, self.P), dtype=np.complex64)
        moff_read_beams(self.handle, out, timeout_ms)
        return out

    def timing(self, kind, reset=False):
        return moff_timing(self.handle, kind, reset)

    def close(self):
        if getattr(self, "handle", None) is not None:
            moff_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
