"""Python binding of the C ABI in include/emri_fd.h (argument marshalling only).

Functions with the C names take raw pointers (ints); ``Plan`` wraps them for
torch CUDA tensors / numpy arrays.  Every step of the computation runs in
libemri_fd.so: there is no CPU or PyTorch fallback, and using the binding
without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

EMRI_FD_FP64, EMRI_FD_MIXED, EMRI_FD_FP64X = 0, 1, 2
STATUS = {0: "EMRI_FD_OK", 1: "EMRI_FD_ERR_ARG", 2: "EMRI_FD_ERR_KNOTS", 3: "EMRI_FD_ERR_FREQ",
          4: "EMRI_FD_ERR_MODE", 5: "EMRI_FD_ERR_NONFINITE", 6: "EMRI_FD_ERR_CAPACITY",
          7: "EMRI_FD_ERR_CUDA", 8: "EMRI_FD_ERR_OOM", 9: "EMRI_FD_ERR_TIMEOUT", 10: "EMRI_FD_ERR_INTERNAL"}
EXPORTS = ("emri_fd_plan", "emri_fd_sum_modes", "emri_fd_loglike_and_grad", "emri_fd_sync", "emri_fd_stats",
           "emri_fd_profile", "emri_fd_plan_destroy", "emri_fd_strerror", "emri_fd_sum_modes_noalloc",
           "emri_fd_set_tile", "emri_fd_set_tile_split", "emri_fd_capture", "emri_fd_replay", "emri_fd_graph_destroy",
           "emri_fd_select_modes", "emri_fd_td_sum", "emri_fd_td_spectrum", "emri_fd_fma_probe")


class EmriFdError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        super().__init__("%s: %s (%s)" % (where, STATUS.get(self.code, "?"), _strerror(self.code)))


class emri_fd_desc(C.Structure):
    _fields_ = [("precision", C.c_int), ("conj_partners", C.c_int), ("max_waveforms", C.c_int),
                ("max_knots", C.c_int), ("max_knots_total", C.c_longlong), ("max_modes_total", C.c_longlong),
                ("max_bins_total", C.c_longlong), ("tile_bins", C.c_int), ("likelihood", C.c_int),
                ("spa_form", C.c_int), ("window", C.c_int), ("time_domain", C.c_int), ("tile_split", C.c_int),
                ("reserved", C.c_int * 2)]

SPA_FORMS = {"standard": 0, "extended": 1}
WINDOWS = {None: 0, "none": 0, "hann": 1}


_lib = None


def library_path() -> str:
    """The library this process loads: $EMRI_FD_LIBRARY if set (e.g. the checked build,
    build.LIB_CHECKED), else the in-tree build."""
    return os.environ.get("EMRI_FD_LIBRARY") or _build.LIB


def lib():
    """Load libemri_fd.so (built in-tree by build.build()); raises if absent."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libemri_fd.so is not built (%s); call __graft_entry__.build() -- "
                               "the CUDA library is the only implementation" % path)
        L = C.CDLL(path)
        vp, ll, dp, ip = C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p
        L.emri_fd_plan.argtypes = [C.POINTER(C.c_void_p), C.POINTER(emri_fd_desc), vp]
        L.emri_fd_plan.restype = C.c_int
        L.emri_fd_sum_modes.argtypes = [vp, C.c_int, vp, vp, vp] + [dp] * 5 + [ip] * 3 + [dp] * 5 + [vp, vp]
        L.emri_fd_sum_modes.restype = C.c_int
        L.emri_fd_loglike_and_grad.argtypes = [vp, C.c_int, vp, vp, vp] + [dp] * 5 + [ip] * 3 + [dp] * 5 + [dp] * 10
        L.emri_fd_loglike_and_grad.restype = C.c_int
        L.emri_fd_td_sum.argtypes = [vp, C.c_int, vp, vp, vp] + [dp] * 5 + [ip] * 3 + [dp] * 5 + [vp, vp]
        L.emri_fd_td_sum.restype = C.c_int
        L.emri_fd_td_spectrum.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int, vp, vp, vp, vp]
        L.emri_fd_td_spectrum.restype = C.c_int
        L.emri_fd_select_modes.argtypes = [vp, C.c_int, vp, vp, dp, C.c_double, ip]
        L.emri_fd_select_modes.restype = C.c_int
        L.emri_fd_set_tile.argtypes = [vp, C.c_int]
        L.emri_fd_set_tile.restype = C.c_int
        L.emri_fd_set_tile_split.argtypes = [vp, C.c_int]
        L.emri_fd_set_tile_split.restype = C.c_int
        L.emri_fd_capture.argtypes = [vp, C.c_int, vp, vp, vp] + [dp] * 5 + [ip] * 3 + [dp] * 5 + [vp, vp,
                                                                                          C.POINTER(C.c_void_p)]
        L.emri_fd_capture.restype = C.c_int
        L.emri_fd_replay.argtypes = [vp]
        L.emri_fd_replay.restype = C.c_int
        L.emri_fd_graph_destroy.argtypes = [vp]
        L.emri_fd_graph_destroy.restype = None
        L.emri_fd_sync.argtypes = [vp]
        L.emri_fd_sync.restype = C.c_int
        L.emri_fd_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int]
        L.emri_fd_stats.restype = C.c_int
        L.emri_fd_profile.argtypes = [vp, C.c_int]
        L.emri_fd_profile.restype = C.c_int
        L.emri_fd_sum_modes_noalloc.argtypes = ([C.c_int, C.c_longlong, C.c_longlong, C.c_longlong] + [dp] * 5 +
                                                [ip] * 3 + [dp] + [C.c_double] * 3 + [dp, vp, vp, vp])
        L.emri_fd_sum_modes_noalloc.restype = C.c_int
        L.emri_fd_plan_destroy.argtypes = [vp]
        L.emri_fd_plan_destroy.restype = None
        L.emri_fd_strerror.argtypes = [C.c_int]
        L.emri_fd_strerror.restype = C.c_char_p
        L.emri_fd_fma_probe.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.POINTER(C.c_longlong)]
        L.emri_fd_fma_probe.restype = C.c_int
        _lib = L
    return _lib


def _strerror(code):
    try:
        return lib().emri_fd_strerror(int(code)).decode()
    except Exception:
        return "?"


def _check(code, where):
    if code != 0:
        raise EmriFdError(code, where)


# ---------------------------------------------------------------- C names
def emri_fd_plan(desc: emri_fd_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().emri_fd_plan(C.byref(h), C.byref(desc), C.c_void_p(stream)), "emri_fd_plan")
    return h.value


def emri_fd_sum_modes(plan, n_waveforms, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r,
                      l, m, n, amp, theta, phi, prefactor, freqs, h_plus, h_cross) -> int:
    """All array arguments are raw addresses (ints); returns the status code."""
    return lib().emri_fd_sum_modes(C.c_void_p(plan), int(n_waveforms), *[C.c_void_p(int(x)) for x in (
        knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, theta, phi,
        prefactor, freqs, h_plus, h_cross)])


def emri_fd_loglike_and_grad(plan, n_waveforms, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi,
                             omega_r, l, m, n, amp, theta, phi, prefactor, freqs, data_plus, data_cross, psd, df,
                             loglike, g_phi_phi, g_phi_r, g_omega_phi, g_omega_r, g_amp) -> int:
    """All array arguments are raw addresses (ints, 0 for a skipped gradient); returns the status."""
    return lib().emri_fd_loglike_and_grad(C.c_void_p(plan), int(n_waveforms), *[C.c_void_p(int(x)) for x in (
        knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, theta, phi, prefactor,
        freqs, data_plus, data_cross, psd, df, loglike, g_phi_phi, g_phi_r, g_omega_phi, g_omega_r, g_amp)])


def emri_fd_sum_modes_noalloc(conj_partners, n_knots, n_modes, n_freqs, t, phi_phi, phi_r, omega_phi, omega_r,
                              l, m, n, amp, theta, phi, prefactor, freqs, h_plus, h_cross, stream=0) -> int:
    """The no-allocation single-waveform entry point: for callers that cannot
    allocate device memory (another allocator owns the device's memory, or the
    code path must not call cudaMalloc/cudaFree).  Arrays are device addresses
    (ints); angles and prefactor are floats.  Synchronous; returns the status."""
    return lib().emri_fd_sum_modes_noalloc(int(conj_partners), int(n_knots), int(n_modes), int(n_freqs),
                                           *[C.c_void_p(int(x)) for x in (t, phi_phi, phi_r, omega_phi, omega_r,
                                                                          l, m, n, amp)],
                                           float(theta), float(phi), float(prefactor), C.c_void_p(int(freqs)),
                                           C.c_void_p(int(h_plus)), C.c_void_p(int(h_cross)), C.c_void_p(int(stream)))


def emri_fd_set_tile(plan, tile_bins) -> int:
    return lib().emri_fd_set_tile(C.c_void_p(plan), int(tile_bins))


def emri_fd_set_tile_split(plan, tile_split) -> int:
    return lib().emri_fd_set_tile_split(C.c_void_p(plan), int(tile_split))


def emri_fd_capture(plan, n_waveforms, knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r,
                    l, m, n, amp, theta, phi, prefactor, freqs, h_plus, h_cross):
    """Returns (status, graph handle)."""
    g = C.c_void_p()
    code = lib().emri_fd_capture(C.c_void_p(plan), int(n_waveforms), *[C.c_void_p(int(x)) for x in (
        knot_off, mode_off, freq_off, t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, theta, phi, prefactor,
        freqs, h_plus, h_cross)], C.byref(g))
    return code, g.value


def emri_fd_replay(graph) -> int:
    return lib().emri_fd_replay(C.c_void_p(graph))


def emri_fd_graph_destroy(graph) -> None:
    lib().emri_fd_graph_destroy(C.c_void_p(graph))


def emri_fd_sync(plan) -> int:
    return lib().emri_fd_sync(C.c_void_p(plan))


def emri_fd_stats(plan) -> dict:
    out = (C.c_longlong * 8)()
    _check(lib().emri_fd_stats(C.c_void_p(plan), out, 8), "emri_fd_stats")
    return {"mode_bins": int(out[0]), "runs": int(out[1]), "tiles": int(out[2]),
            "timed_calls": int(out[4]), "spa_ns": int(out[5]), "prep_ns": int(out[6]), "launches": int(out[7])}


def emri_fd_profile(plan, enable: bool) -> None:
    _check(lib().emri_fd_profile(C.c_void_p(plan), int(bool(enable))), "emri_fd_profile")


def emri_fd_strerror(code) -> str:
    return _strerror(code)


def emri_fd_select_modes(plan, n_waveforms, knot_off, mode_off, amp, eps, keep) -> int:
    """Array arguments are raw addresses (ints); returns the status code."""
    return lib().emri_fd_select_modes(C.c_void_p(plan), int(n_waveforms), C.c_void_p(int(knot_off)),
                                      C.c_void_p(int(mode_off)), C.c_void_p(int(amp)), float(eps),
                                      C.c_void_p(int(keep)))


def emri_fd_td_sum(plan, n_waveforms, knot_off, mode_off, sample_off, t, phi_phi, phi_r, omega_phi, omega_r,
                   l, m, n, amp, theta, phi, prefactor, dt, h_plus, h_cross) -> int:
    """Array arguments are raw addresses (ints); returns the status code."""
    return lib().emri_fd_td_sum(C.c_void_p(plan), int(n_waveforms), *[C.c_void_p(int(x)) for x in (
        knot_off, mode_off, sample_off, t, phi_phi, phi_r, omega_phi, omega_r, l, m, n, amp, theta, phi, prefactor,
        dt, h_plus, h_cross)])


def emri_fd_td_spectrum(plan, n_waveforms, sample_off, t0, dt, window, h_plus, h_cross, H_plus, H_cross) -> int:
    """Array arguments are raw addresses (ints); returns the status code."""
    return lib().emri_fd_td_spectrum(C.c_void_p(plan), int(n_waveforms), C.c_void_p(int(sample_off)),
                                     C.c_void_p(int(t0)), C.c_void_p(int(dt)), int(window),
                                     *[C.c_void_p(int(x)) for x in (h_plus, h_cross, H_plus, H_cross)])


def emri_fd_plan_destroy(plan) -> None:
    lib().emri_fd_plan_destroy(C.c_void_p(plan))


def emri_fd_fma_probe(precision, iters, blocks_per_sm, stream=0):
    """Launch the FMA peak probe (precision 0 = FP64, 1 = FP32) on a raw stream
    handle; returns the FMAs the launch executes.  The caller times it."""
    n = C.c_longlong(0)
    _check(lib().emri_fd_fma_probe(int(precision), int(iters), int(blocks_per_sm), C.c_void_p(int(stream)),
                                   C.byref(n)), "emri_fd_fma_probe")
    return n.value


# ---------------------------------------------------------------- wrapper
_KEYS_D = ("t", "phi_phi", "phi_r", "omega_phi", "omega_r", "theta", "phi", "prefactor", "freqs")
_KEYS_I = ("l", "m", "n")


def _addr(x):
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


class Plan:
    """A plan of the C library bound to a torch CUDA stream.

    precision: "fp64" or "fp64x" (complex128 outputs) or "mixed" (complex64 outputs).
    spa: "standard" (Fresnel integral per root) or "extended" (Eq. 10 per root).
    window: None or "hann" (the window's three-term convolution on a uniform grid).
    tile_split: 0/1, 2 or 4 CTAs (a thread-block cluster) per output tile (32- or 64-bin
    tiles; for grids with few tiles).
    Batches are dicts in the layout of synth.concat (numpy or torch)."""

    def __init__(self, precision="fp64", conj_partners=True, max_waveforms=1, max_knots=200,
                 max_modes_total=4096, max_bins_total=1 << 22, max_knots_total=0, tile_bins=0,
                 likelihood=False, device=None, stream=None, spa="standard", window=None, time_domain=False,
                 tile_split=0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.precision = {"fp64": EMRI_FD_FP64, 0: EMRI_FD_FP64, "mixed": EMRI_FD_MIXED, 1: EMRI_FD_MIXED,
                          "fp64x": EMRI_FD_FP64X, 2: EMRI_FD_FP64X}[precision]
        d = emri_fd_desc()
        d.precision = self.precision
        d.conj_partners = int(bool(conj_partners))
        d.max_waveforms = int(max_waveforms)
        d.max_knots = int(max_knots)
        d.max_knots_total = int(max_knots_total)
        d.max_modes_total = int(max_modes_total)
        d.max_bins_total = int(max_bins_total)
        d.tile_bins = int(tile_bins)
        d.likelihood = int(bool(likelihood))
        d.spa_form = SPA_FORMS[spa]
        d.window = WINDOWS[window]
        d.time_domain = int(bool(time_domain))
        d.tile_split = int(tile_split)
        self.spa = spa
        self.window = window
        self.desc = d
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.handle = emri_fd_plan(d, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            emri_fd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def out_dtype(self):
        return self.torch.complex64 if self.precision == EMRI_FD_MIXED else self.torch.complex128

    def upload(self, batch, non_blocking=False):
        """numpy batch -> dict of device tensors (offsets stay on the host)."""
        T = self.torch
        out = {}
        for k in ("knot_off", "mode_off", "freq_off"):
            out[k] = np.ascontiguousarray(np.asarray(batch[k], np.int64))
        for k in _KEYS_D:
            out[k] = T.as_tensor(np.ascontiguousarray(batch[k], np.float64)).to(self.device, non_blocking=non_blocking)
        for k in _KEYS_I:
            out[k] = T.as_tensor(np.ascontiguousarray(batch[k], np.int32)).to(self.device, non_blocking=non_blocking)
        amp = np.ascontiguousarray(batch["amp"], np.complex128).view(np.float64)
        out["amp"] = T.as_tensor(amp).to(self.device, non_blocking=non_blocking)
        return out

    def sum_modes(self, b, out=None, check=True):
        """One call of emri_fd_sum_modes on a device batch; returns (h_plus, h_cross)."""
        T = self.torch
        n_wf = len(b["knot_off"]) - 1
        nf = int(b["freq_off"][-1])
        if out is None:
            out = (T.empty(nf, dtype=self.out_dtype, device=self.device),
                   T.empty(nf, dtype=self.out_dtype, device=self.device))
        ko, mo, fo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off", "freq_off"))
        code = emri_fd_sum_modes(self.handle, n_wf, ko.ctypes.data, mo.ctypes.data, fo.ctypes.data,
                                 _addr(b["t"]), _addr(b["phi_phi"]), _addr(b["phi_r"]), _addr(b["omega_phi"]),
                                 _addr(b["omega_r"]), _addr(b["l"]), _addr(b["m"]), _addr(b["n"]), _addr(b["amp"]),
                                 _addr(b["theta"]), _addr(b["phi"]), _addr(b["prefactor"]), _addr(b["freqs"]),
                                 _addr(out[0]), _addr(out[1]))
        _check(code, "emri_fd_sum_modes")
        if check:
            _check(emri_fd_sync(self.handle), "emri_fd_sum_modes (device checks)")
        return out

    def sum_modes_host(self, b, out=None):
        """emri_fd_sum_modes with HOST buffers (numpy, or pinned torch CPU tensors): the
        library stages inputs and outputs itself and synchronises before returning."""
        n_wf = len(b["knot_off"]) - 1
        nf = int(b["freq_off"][-1])
        cdt = np.complex64 if self.precision == EMRI_FD_MIXED else np.complex128
        if out is None:
            out = (np.empty(nf, cdt), np.empty(nf, cdt))
        ko, mo, fo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off", "freq_off"))
        code = emri_fd_sum_modes(self.handle, n_wf, ko.ctypes.data, mo.ctypes.data, fo.ctypes.data,
                                 *[_addr(b[k]) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r", "l", "m",
                                                         "n", "amp", "theta", "phi", "prefactor", "freqs")],
                                 _addr(out[0]), _addr(out[1]))
        _check(code, "emri_fd_sum_modes")   # host outputs: the call has synchronised and checked
        if any(getattr(x, "is_cuda", False) for x in out):
            _check(emri_fd_sync(self.handle), "emri_fd_sum_modes (device checks)")
        return out

    def td_sum(self, b, dt, n_samples, check=True):
        """emri_fd_td_sum on a device batch: TD samples t_j = t_0 + j dt of every
        waveform (dt and n_samples: one value or one per waveform).  Returns
        (h+, hx, sample_off) with float32 device tensors [sum N_w]."""
        T = self.torch
        ko, mo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off"))
        nw = len(ko) - 1
        ns = np.broadcast_to(np.asarray(n_samples, np.int64), (nw,))
        so = np.zeros(nw + 1, np.int64)
        so[1:] = np.cumsum(ns)
        dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (nw,)))
        hp = T.empty(int(so[-1]), dtype=T.float32, device=self.device)
        hc = T.empty(int(so[-1]), dtype=T.float32, device=self.device)
        code = emri_fd_td_sum(self.handle, nw, ko.ctypes.data, mo.ctypes.data, so.ctypes.data,
                              *[_addr(b[k]) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r", "l", "m", "n",
                                                      "amp", "theta", "phi", "prefactor")],
                              dtv.ctypes.data, hp.data_ptr(), hc.data_ptr())
        _check(code, "emri_fd_td_sum")
        if check:
            _check(emri_fd_sync(self.handle), "emri_fd_td_sum (device checks)")
        self._td_last = (so, dtv)
        return hp, hc, so

    @staticmethod
    def td_freqs(sample_off, dt):
        """The frequencies k/(N_w dt), k = 1 .. N_w/2 - 1, of td_spectrum's bins (numpy)."""
        so = np.asarray(sample_off, np.int64)
        N = np.diff(so)
        dtv = np.broadcast_to(np.asarray(dt, np.float64), N.shape)
        parts = [np.arange(1, Nw // 2) / (Nw * d) for Nw, d in zip(N, dtv) if Nw >= 4]
        return np.concatenate(parts) if parts else np.zeros(0)

    def td_spectrum(self, hp, hc, sample_off, t0, dt, window=None):
        """emri_fd_td_spectrum: complex64 device tensors H+, Hx over the bins
        k = 1 .. N_w/2 - 1 of every waveform (frequencies: td_freqs)."""
        T = self.torch
        so = np.ascontiguousarray(np.asarray(sample_off, np.int64))
        nw = len(so) - 1
        t0v = np.ascontiguousarray(np.broadcast_to(np.asarray(t0, np.float64), (nw,)))
        dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (nw,)))
        N = np.diff(so)
        nb = np.where(N >= 4, N // 2 - 1, 0)
        Hp = T.empty(int(nb.sum()), dtype=T.complex64, device=self.device)
        Hc = T.empty(int(nb.sum()), dtype=T.complex64, device=self.device)
        code = emri_fd_td_spectrum(self.handle, nw, so.ctypes.data, t0v.ctypes.data, dtv.ctypes.data,
                                   WINDOWS[window], hp.data_ptr(), hc.data_ptr(), Hp.data_ptr(), Hc.data_ptr())
        _check(code, "emri_fd_td_spectrum")
        return Hp, Hc

    def select_modes(self, b, eps, check=True):
        """emri_fd_select_modes on a batch (device tensors from upload, or numpy):
        bool tensor [sum N_m] on the plan's device, True for the selected modes."""
        T = self.torch
        ko, mo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off"))
        keep = T.empty(int(mo[-1]), dtype=T.int32, device=self.device)
        code = emri_fd_select_modes(self.handle, len(ko) - 1, ko.ctypes.data, mo.ctypes.data, _addr(b["amp"]),
                                    eps, keep.data_ptr())
        _check(code, "emri_fd_select_modes")
        if check:
            _check(emri_fd_sync(self.handle), "emri_fd_select_modes (device checks)")
        return keep.bool()

    def loglike_and_grad(self, b, data_plus, data_cross, psd, df, grad=True, check=True):
        """emri_fd_loglike_and_grad on a device batch.  data_*: complex128 device tensors,
        psd: float64 device tensor, df: float64 tensor [n_wf].  Returns (loglike [n_wf],
        dict of knot gradients or None)."""
        T = self.torch
        n_wf = len(b["knot_off"]) - 1
        K = int(b["knot_off"][-1])
        namp = int(np.sum(np.diff(b["mode_off"]) * np.diff(b["knot_off"])))
        dev = self.device
        L = T.empty(n_wf, dtype=T.float64, device=dev)
        g = None
        if grad:
            g = {k: T.empty(K, dtype=T.float64, device=dev) for k in ("phi_phi", "phi_r", "omega_phi", "omega_r")}
            g["amp"] = T.empty(namp, dtype=T.complex128, device=dev)
        ko, mo, fo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off", "freq_off"))
        gp = [_addr(g[k]) if g else 0 for k in ("phi_phi", "phi_r", "omega_phi", "omega_r", "amp")]
        code = emri_fd_loglike_and_grad(self.handle, n_wf, ko.ctypes.data, mo.ctypes.data, fo.ctypes.data,
                                        *[_addr(b[k]) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r", "l",
                                                                "m", "n", "amp", "theta", "phi", "prefactor",
                                                                "freqs")],
                                        _addr(data_plus), _addr(data_cross), _addr(psd), _addr(df), _addr(L), *gp)
        _check(code, "emri_fd_loglike_and_grad")
        if check:
            _check(emri_fd_sync(self.handle), "emri_fd_loglike_and_grad (device checks)")
        return L, g

    def set_tile(self, tile_bins):
        _check(emri_fd_set_tile(self.handle, tile_bins), "emri_fd_set_tile")

    def set_tile_split(self, tile_split):
        _check(emri_fd_set_tile_split(self.handle, tile_split), "emri_fd_set_tile_split")

    def capture(self, b, out):
        """Capture emri_fd_sum_modes(b) -> out into a CUDA graph; returns a Graph."""
        ko, mo, fo = (np.ascontiguousarray(np.asarray(b[k], np.int64)) for k in ("knot_off", "mode_off", "freq_off"))
        code, g = emri_fd_capture(self.handle, len(ko) - 1, ko.ctypes.data, mo.ctypes.data, fo.ctypes.data,
                                  *[_addr(b[k]) for k in ("t", "phi_phi", "phi_r", "omega_phi", "omega_r", "l", "m",
                                                          "n", "amp", "theta", "phi", "prefactor", "freqs")],
                                  _addr(out[0]), _addr(out[1]))
        _check(code, "emri_fd_capture")
        return Graph(g, self)

    def sync(self):
        _check(emri_fd_sync(self.handle), "emri_fd_sync")

    def stats(self):
        return emri_fd_stats(self.handle)

    def profile(self, enable=True):
        emri_fd_profile(self.handle, enable)


class Graph:
    """A captured emri_fd_sum_modes call (emri_fd_replay / emri_fd_graph_destroy)."""

    def __init__(self, handle, plan):
        self.handle, self.plan = handle, plan

    def replay(self):
        _check(emri_fd_replay(self.handle), "emri_fd_replay")

    def close(self):
        if self.handle:
            emri_fd_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_batch(batch):
    """numpy copy of a synth.concat batch with the dtypes the C ABI expects."""
    out = dict(batch)
    for k in _KEYS_D:
        out[k] = np.ascontiguousarray(batch[k], np.float64)
    for k in _KEYS_I:
        out[k] = np.ascontiguousarray(batch[k], np.int32)
    out["amp"] = np.ascontiguousarray(batch["amp"], np.complex128).view(np.float64)
    return out


def whittle_loglike(plan, b, data_plus, data_cross, psd, df):
    """Differentiable Whittle log-likelihood (summed over the batch's waveforms).

    The knot tensors b["phi_phi"], b["phi_r"], b["omega_phi"], b["omega_r"]
    (float64) and b["amp"] (float64 view of complex128, [sum N_m K * 2]) may
    require grad.  Forward computes L only; backward calls the C adjoint, which
    recomputes t(f) instead of storing it."""
    return WhittleLogLike.apply(plan, b, data_plus, data_cross, psd, df, b["phi_phi"], b["phi_r"],
                                b["omega_phi"], b["omega_r"], b["amp"])


def _autograd_function():
    import torch

    class _WhittleLogLike(torch.autograd.Function):
        @staticmethod
        def forward(ctx, plan, b, data_plus, data_cross, psd, df, phi_phi, phi_r, omega_phi, omega_r, amp):
            bb = dict(b)
            bb.update(phi_phi=phi_phi.detach(), phi_r=phi_r.detach(), omega_phi=omega_phi.detach(),
                      omega_r=omega_r.detach(), amp=amp.detach())
            L, _ = plan.loglike_and_grad(bb, data_plus, data_cross, psd, df, grad=False)
            # the knot tensors go through save_for_backward, so that autograd's version
            # counters reject a backward after any of them was modified in place
            ctx.save_for_backward(phi_phi, phi_r, omega_phi, omega_r, amp)
            ctx.plan, ctx.b, ctx.data = plan, b, (data_plus, data_cross, psd, df)
            return L.sum()

        @staticmethod
        def backward(ctx, gL):
            phi_phi, phi_r, omega_phi, omega_r, amp = ctx.saved_tensors
            bb = dict(ctx.b)
            bb.update(phi_phi=phi_phi.detach(), phi_r=phi_r.detach(), omega_phi=omega_phi.detach(),
                      omega_r=omega_r.detach(), amp=amp.detach())
            _, g = ctx.plan.loglike_and_grad(bb, *ctx.data, grad=True)
            ga = torch.view_as_real(g["amp"]).reshape(-1)
            return (None, None, None, None, None, None, gL * g["phi_phi"], gL * g["phi_r"], gL * g["omega_phi"],
                    gL * g["omega_r"], gL * ga)

    return _WhittleLogLike


class _LazyFn:
    _fn = None

    def apply(self, *a):
        if _LazyFn._fn is None:
            _LazyFn._fn = _autograd_function()
        return _LazyFn._fn.apply(*a)


WhittleLogLike = _LazyFn()
