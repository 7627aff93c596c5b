"""Python binding of libptycho with torch tensors as device memory.

Each method checks shapes, dtypes and devices, passes raw pointers and the
current torch stream to the C-ABI, and raises PtychoError on failure.  All
arithmetic happens in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

LOSS = {"amplitude": 0, "anscombe": 0, "poisson": 1, "gaussian": 2}
WAVES = {"auto": 0, "store": 1, "recompute": 2}
DFT = {"fft": 0, "tf32x3": 1, "bf16x3": 2, "tf32": 3, "bf16x6": 4}
PREC = {"f32": 0, "f16": 1, "bf16": 2}


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _need(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")


@dataclass
class Geometry:
    S: int
    K: int
    N: int
    H: int
    W: int
    dx: float = 0.1
    lam: float = 0.0197
    dz: tuple = ()
    bandlimit: float = 2.0 / 3.0
    loss: str = "amplitude"
    eps: float = 1e-3
    c: float = 0.0
    waves: str = "auto"
    dft: str = "fft"
    wave_prec: str = "f32"
    deterministic: bool = False

    def to_c(self):
        dz = (C.c_double * max(len(self.dz), 1))(*self.dz) if len(self.dz) else None
        g = _lib.Geom(self.S, self.K, self.N, self.N, self.H, self.W, self.dx, self.lam,
                      C.cast(dz, C.POINTER(C.c_double)) if dz is not None else None,
                      self.bandlimit, LOSS[self.loss], self.eps, self.c, WAVES[self.waves], DFT[self.dft],
                      PREC[self.wave_prec], 1 if self.deterministic else 0)
        return g, dz


def adam_opt(lr_O=1e-3, lr_P=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, update_probe=True, reg_obj_l2=0.0,
             reg_obj_tikhonov=0.0, reg_obj_layers=0.0, reg_probe_l2=0.0, reg_obj_tv=0.0, reg_obj_layers_tv=0.0,
             reg_tv_eps=1e-3) -> _lib.Opt:
    return _lib.Opt(lr_O, lr_P, beta1, beta2, eps, 1 if update_probe else 0, reg_obj_l2, reg_obj_tikhonov,
                    reg_obj_layers, reg_probe_l2, reg_obj_tv, reg_obj_layers_tv, reg_tv_eps)


class AdamState:
    """First/second moments for O and P on the device, step counter t."""

    def __init__(self, geom: Geometry, device="cuda"):
        self.mO = torch.zeros((geom.S, geom.H, geom.W), dtype=torch.complex64, device=device)
        self.vO = torch.zeros((geom.S, geom.H, geom.W), dtype=torch.float32, device=device)
        self.mP = torch.zeros((geom.K, geom.N, geom.N), dtype=torch.complex64, device=device)
        self.vP = torch.zeros((geom.K, geom.N, geom.N), dtype=torch.float32, device=device)
        self.c = _lib.Adam(self.mO.data_ptr(), self.vO.data_ptr(), self.mP.data_ptr(), self.vP.data_ptr(), 0)

    @property
    def t(self) -> int:
        return int(self.c.t)


class Context:
    """One problem geometry on the current CUDA device (ptycho_create)."""

    def __init__(self, geom: Geometry, max_batch: int, scratch_budget: int = 0):
        self.geom = geom
        self.max_batch = int(max_batch)
        g, self._dz = geom.to_c()
        h = C.c_void_p()
        check(lib().ptycho_create(C.byref(g), self.max_batch, scratch_budget, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ptycho_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes
    def _oshape(self):
        g = self.geom
        return (g.S, g.H, g.W)

    def _pshape(self):
        g = self.geom
        return (g.K, g.N, g.N)

    def forward(self, O, P, pos, out=None) -> torch.Tensor:
        g = self.geom
        B = pos.shape[0]
        _need(O, torch.complex64, self._oshape(), "O")
        _need(P, torch.complex64, self._pshape(), "P")
        _need(pos, torch.float32, (B, 2), "pos")
        if out is None:
            out = torch.empty((B, g.N, g.N), dtype=torch.float32, device=O.device)
        check(lib().ptycho_forward(self.h, _ptr(O), _ptr(P), _ptr(pos), B, _ptr(out), _stream()))
        return out

    def adjoint(self, O, P, pos, I_exp, gO=None, gP=None, accumulate=False):
        """Returns (loss [device float64 scalar tensor], gO, gP)."""
        B = pos.shape[0]
        g = self.geom
        _need(O, torch.complex64, self._oshape(), "O")
        _need(P, torch.complex64, self._pshape(), "P")
        _need(pos, torch.float32, (B, 2), "pos")
        _need(I_exp, torch.float32, (B, g.N, g.N), "I_exp")
        if gO is None:
            gO = torch.empty_like(O)
        if gP is None:
            gP = torch.empty_like(P)
        loss = torch.zeros((), dtype=torch.float64, device=O.device)
        check(lib().ptycho_adjoint(self.h, _ptr(O), _ptr(P), _ptr(pos), B, _ptr(I_exp), _ptr(loss),
                                   _ptr(gO), _ptr(gP), 1 if accumulate else 0, _stream()))
        return loss, gO, gP

    def adjoint_positions(self, O, P, pos, I_exp, gO=None, gP=None, gpos=None, accumulate=False):
        """Returns (loss, gO, gP, gpos [B, 2] float64 device tensor)."""
        B = pos.shape[0]
        g = self.geom
        _need(O, torch.complex64, self._oshape(), "O")
        _need(P, torch.complex64, self._pshape(), "P")
        _need(pos, torch.float32, (B, 2), "pos")
        _need(I_exp, torch.float32, (B, g.N, g.N), "I_exp")
        gO = torch.empty_like(O) if gO is None else gO
        gP = torch.empty_like(P) if gP is None else gP
        gpos = torch.empty((B, 2), dtype=torch.float64, device=O.device) if gpos is None else gpos
        loss = torch.zeros((), dtype=torch.float64, device=O.device)
        check(lib().ptycho_adjoint_positions(self.h, _ptr(O), _ptr(P), _ptr(pos), B, _ptr(I_exp), _ptr(loss),
                                             _ptr(gO), _ptr(gP), _ptr(gpos), 1 if accumulate else 0, _stream()))
        return loss, gO, gP, gpos

    def vjp(self, O, P, pos, gI, gO=None, gP=None, accumulate=False):
        B = pos.shape[0]
        g = self.geom
        _need(gI, torch.float32, (B, g.N, g.N), "gI")
        if gO is None:
            gO = torch.empty_like(O)
        if gP is None:
            gP = torch.empty_like(P)
        check(lib().ptycho_vjp(self.h, _ptr(O), _ptr(P), _ptr(pos), B, _ptr(gI), _ptr(gO), _ptr(gP),
                               1 if accumulate else 0, _stream()))
        return gO, gP

    def step(self, O, P, state: AdamState, opt, pos_all, I_exp_all, idx, stats=None):
        """One Adam iteration on the minibatch idx (int32 device tensor);
        returns a device float64 tensor [loss, grad-norm]."""
        B = idx.shape[0]
        _need(idx, torch.int32, (B,), "idx")
        if stats is None:
            stats = torch.zeros(2, dtype=torch.float64, device=O.device)
        g = self.geom
        n_pos = pos_all.shape[0]
        _need(pos_all, torch.float32, (n_pos, 2), "pos_all")
        _need(I_exp_all, torch.float32, (n_pos, g.N, g.N), "I_exp_all")
        check(lib().ptycho_step(self.h, _ptr(O), _ptr(P), C.byref(state.c), C.byref(opt), _ptr(pos_all),
                                _ptr(I_exp_all), n_pos, _ptr(idx), B, _ptr(stats), _stream()))
        return stats

    def epie_step(self, O, P, pos_all, I_exp_all, idx, beta_O=1.0, beta_P=1.0, loss=None):
        """One ePIE / 3PIE update (ptycho_epie_step) of O and P in place from
        the group idx; returns a device float64 tensor [loss before the update]."""
        B = idx.shape[0]
        _need(idx, torch.int32, (B,), "idx")
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float64, device=O.device)
        g = self.geom
        n_pos = pos_all.shape[0]
        _need(pos_all, torch.float32, (n_pos, 2), "pos_all")
        _need(I_exp_all, torch.float32, (n_pos, g.N, g.N), "I_exp_all")
        check(lib().ptycho_epie_step(self.h, _ptr(O), _ptr(P), float(beta_O), float(beta_P), _ptr(pos_all),
                                     _ptr(I_exp_all), n_pos, _ptr(idx), B, _ptr(loss), _stream()))
        return loss

    def lsqml_step(self, O, P, pos_all, I_exp_all, idx, beta_O=1.0, beta_P=1.0, delta_O=0.0, delta_P=0.0,
                   gamma=0.0, illum_prev=None, trans_prev=None, illum_acc=None, trans_acc=None, loss=None):
        """One LSQML update (ptycho_lsqml_step) of O and P in place from the
        group idx; illum_* [S, H, W] and trans_* [N, N] are optional float32
        device tensors (running sums in, the group's sums added out).
        Returns a device float64 tensor [loss before the update]."""
        B = idx.shape[0]
        _need(idx, torch.int32, (B,), "idx")
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float64, device=O.device)
        g = self.geom
        n_pos = pos_all.shape[0]
        _need(pos_all, torch.float32, (n_pos, 2), "pos_all")
        _need(I_exp_all, torch.float32, (n_pos, g.N, g.N), "I_exp_all")
        for t, shape, name in ((illum_prev, (g.S, g.H, g.W), "illum_prev"), (illum_acc, (g.S, g.H, g.W), "illum_acc"),
                               (trans_prev, (g.N, g.N), "trans_prev"), (trans_acc, (g.N, g.N), "trans_acc")):
            if t is not None:
                _need(t, torch.float32, shape, name)
        opt = _lib.LsqmlOpt(beta_O, beta_P, delta_O, delta_P, gamma)
        ptr = lambda t: _ptr(t) if t is not None else None
        check(lib().ptycho_lsqml_step(self.h, _ptr(O), _ptr(P), C.byref(opt), ptr(illum_prev), ptr(trans_prev),
                                      ptr(illum_acc), ptr(trans_acc), _ptr(pos_all), _ptr(I_exp_all), n_pos,
                                      _ptr(idx), B, _ptr(loss), _stream()))
        return loss

    def step_host(self, O, P, state: AdamState, opt, pos_host: np.ndarray, I_exp_host):
        """Step with the group's positions/patterns in host memory (numpy or
        pinned CPU torch tensors); returns (loss, gnorm) as floats."""
        if isinstance(pos_host, torch.Tensor):
            B = pos_host.shape[0]
            pp, ip = pos_host.data_ptr(), I_exp_host.data_ptr()
        else:
            pos_host = np.ascontiguousarray(pos_host, dtype=np.float32)
            I_exp_host = np.ascontiguousarray(I_exp_host, dtype=np.float32)
            B = pos_host.shape[0]
            pp, ip = pos_host.ctypes.data, I_exp_host.ctypes.data
        loss = C.c_double()
        gn = C.c_double()
        check(lib().ptycho_step_host(self.h, _ptr(O), _ptr(P), C.byref(state.c), C.byref(opt), pp, ip, B,
                                     C.byref(loss), C.byref(gn), _stream()))
        return loss.value, gn.value

    def check_status(self):
        check(lib().ptycho_check(self.h, _stream()))

    def set_step_counter(self, t):
        """Keep the Adam step count in the int64 CUDA tensor t (one element,
        ptycho_set_step_counter): steps captured in a CUDA graph then replay
        with the right bias corrections.  None returns to the host count."""
        if t is not None:
            _need(t, torch.int64, (1,), "t")
        check(lib().ptycho_set_step_counter(self.h, _ptr(t)))
        self._t_dev = t

    def set_timing(self, on=True):
        """on: True / 1 (every kernel), 2 (the tile kernels only), False / 0."""
        check(lib().ptycho_set_timing(self.h, int(on)))

    def kernel_times(self, reset=False) -> dict:
        cap = 64
        names = (C.c_char_p * cap)()
        ms = (C.c_double * cap)()
        n_l = (C.c_int32 * cap)()
        n = lib().ptycho_kernel_times(self.h, names, ms, n_l, cap)
        if n < 0:
            check(n)
        out = {names[i].decode(): (ms[i], n_l[i]) for i in range(min(n, cap))}
        if reset:
            lib().ptycho_kernel_times(self.h, None, None, None, -1)
        return out


STATE_NAMES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "admitting"}


class Server:
    """In-process continuous-batching server (ptycho_server_*): requests are
    admitted against an HBM budget, keep their state on the device and have
    their iterations batched into shared launches."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64):
        h = C.c_void_p()
        check(lib().ptycho_server_create(int(hbm_budget_bytes), int(max_active), C.byref(h)))
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ptycho_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, geom: Geometry, pos: np.ndarray, I_exp: np.ndarray, P_init: np.ndarray, O_init=None,
               iterations: int = 1, batch: int = 64, grouping: str = "sparse", seed: int = 0, opt=None) -> int:
        g, dz = geom.to_c()
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        I_exp = np.ascontiguousarray(I_exp, dtype=np.float32)
        P_init = np.ascontiguousarray(P_init, dtype=np.complex64)
        O_ptr = None
        if O_init is not None:
            O_init = np.ascontiguousarray(O_init, dtype=np.complex64)
            O_ptr = O_init.ctypes.data
        req = _lib.Request(g, pos.shape[0], pos.ctypes.data, I_exp.ctypes.data, O_ptr, P_init.ctypes.data,
                           iterations, batch, {"sparse": 0, "compact": 1}[grouping], seed,
                           opt if opt is not None else adam_opt())
        t = C.c_uint64()
        check(lib().ptycho_submit(self.h, C.byref(req), C.byref(t)))  # copies the host arrays
        return int(t.value)

    def poll(self, ticket: int, geom: Geometry | None = None) -> dict:
        st = _lib.Status()
        res = _lib.Result()
        check(lib().ptycho_poll(self.h, ticket, C.byref(st), C.byref(res)))
        out = {"state": STATE_NAMES.get(st.state, st.state), "iterations_done": st.iterations_done,
               "error": st.error, "last_loss": st.last_loss, "submit_ms": st.submit_ms,
               "start_ms": st.start_ms, "finish_ms": st.finish_ms}
        if st.state == 2:
            out["loss"] = np.ctypeslib.as_array(res.loss, shape=(res.n_loss,)).copy() if res.n_loss else np.zeros(0)
            out["iter_ms"] = np.ctypeslib.as_array(res.step_ms, shape=(res.n_step,)).copy() if res.n_step else np.zeros(0)
            if geom is not None:
                nO = geom.S * geom.H * geom.W
                nP = geom.K * geom.N * geom.N
                out["O"] = np.ctypeslib.as_array(C.cast(res.O, C.POINTER(C.c_float)), shape=(2 * nO,)).view(
                    np.complex64).reshape(geom.S, geom.H, geom.W).copy()
                out["P"] = np.ctypeslib.as_array(C.cast(res.P, C.POINTER(C.c_float)), shape=(2 * nP,)).view(
                    np.complex64).reshape(geom.K, geom.N, geom.N).copy()
        return out

    def wait(self, ticket: int, timeout_ms: float = 600e3):
        check(lib().ptycho_wait(self.h, ticket, float(timeout_ms)))

    def release(self, ticket: int):
        check(lib().ptycho_release(self.h, ticket))

    def cancel(self, ticket: int):
        """Ends the request (FAILED, error ECANCELED) without disturbing the others."""
        check(lib().ptycho_cancel(self.h, ticket))

    def inject_stall(self, ms: float):
        """Fault injection for tests: the worker sleeps `ms` before its next tick."""
        check(lib().ptycho_server_inject_stall(self.h, float(ms)))

    def stats(self) -> dict:
        s = _lib.ServerStats()
        check(lib().ptycho_server_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.ServerStats._fields_}


def scratch_bytes(geom: Geometry, B: int, waves: str = "store") -> int:
    g, _dz = geom.to_c()
    return int(lib().ptycho_scratch_bytes(C.byref(g), B, WAVES[waves]))


def fft2(x: torch.Tensor, inverse=False) -> torch.Tensor:
    """Unnormalised 2-D DFT of [count, N, N] complex64 through the tile."""
    assert x.dtype == torch.complex64 and x.is_cuda and x.is_contiguous() and x.dim() == 3
    out = torch.empty_like(x)
    check(lib().ptycho_fft2(x.shape[-1], 1 if inverse else -1, _ptr(x), _ptr(out), x.shape[0], _stream()))
    return out


def fft2_dft(x: torch.Tensor, dft: str = "fft", inverse=False) -> torch.Tensor:
    """fft2 through the tile of a given DFT evaluation (the tensor-core tiles
    exist for N = 192)."""
    assert x.dtype == torch.complex64 and x.is_cuda and x.is_contiguous() and x.dim() == 3
    out = torch.empty_like(x)
    check(lib().ptycho_fft2_dft(x.shape[-1], DFT[dft], 1 if inverse else -1, _ptr(x), _ptr(out), x.shape[0],
                                _stream()))
    return out


TC5 = {"tf32x3": 1, "bf16x3": 2, "tf32": 3}


def dft_rows_tc(x: torch.Tensor, mode: str = "tf32x3", inverse=False, out: torch.Tensor | None = None) -> torch.Tensor:
    """1-D DFT along the last axis of [..., N] complex64 rows on the tcgen05
    tensor cores (unnormalised; see ptycho_dft_rows_tc)."""
    assert x.dtype == torch.complex64 and x.is_cuda and x.is_contiguous()
    N = x.shape[-1]
    if out is None:
        out = torch.empty_like(x)
    check(lib().ptycho_dft_rows_tc(N, TC5[mode], 1 if inverse else -1, _ptr(x), _ptr(out), x.numel() // N,
                                   _stream()))
    return out


def dft_rows_tc_check():
    check(lib().ptycho_dft_rows_tc_check())


def make_groups(P: int, B: int, seed: int, iteration: int, mode: str = "sparse", pos=None) -> np.ndarray:
    out = np.empty(P, dtype=np.int32)
    pp = None
    if pos is not None:
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        pp = pos.ctypes.data
    check(lib().ptycho_make_groups(P, B, seed, iteration, {"sparse": 0, "compact": 1}[mode], pp,
                                   out.ctypes.data))
    return out


def kernels_launched() -> int:
    """Kernels this library has launched in this process."""
    return int(lib().ptycho_kernels_launched())


def version() -> str:
    return lib().ptycho_version().decode()


def fp32_peak(target_ms: float = 300.0, repeats: int = 3) -> dict:
    """Measured FP32 CUDA-core throughput of the current device (TFLOP/s):
    the library's FFMA and FFMA2 microbenchmark kernels, each launched
    `repeats` times at about target_ms per launch after one warm-up launch,
    timed with CUDA events on the current stream; the best launch of each."""
    sink = torch.empty(int(lib().ptycho_fp32_peak_sink_elems()), dtype=torch.float32, device="cuda")
    flops = C.c_double(0.0)
    out = {}
    for packed, name in ((0, "ffma"), (1, "ffma2")):
        iters = 256
        # warm-up, then size the launch to about target_ms
        check(lib().ptycho_fp32_peak_launch(packed, iters, _ptr(sink), C.byref(flops), _stream()))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        check(lib().ptycho_fp32_peak_launch(packed, iters, _ptr(sink), C.byref(flops), _stream()))
        e1.record()
        torch.cuda.synchronize()
        iters = max(1, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        best = 0.0
        ms_best = None
        for _ in range(repeats):
            e0.record()
            check(lib().ptycho_fp32_peak_launch(packed, iters, _ptr(sink), C.byref(flops), _stream()))
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            tf = flops.value / (ms / 1e3) / 1e12
            if tf > best:
                best, ms_best = tf, ms
        out[name] = {"tflops": best, "ms": ms_best, "iters": iters}
    out["tflops"] = max(out["ffma"]["tflops"], out["ffma2"]["tflops"])
    return out
