"""GB300-native machine-learned finite-temperature SP2 (arXiv 2605.08523).

Python binding of the C ABI in ``include/ftsp2.h`` (ctypes; see ``_lib``).
PyTorch provides device memory and streams only; every step of the hot path
(Gershgorin bounds, rescale, the learned recursion on the tensor cores, the
traces and the entropy) runs in the library's CUDA kernels.  There is no CPU
fallback: without the built library or a GB300 every call raises.

Main entry points (same names as the C functions, torch tensors in place of
device pointers):

* ``ModelSet`` -- ``ftsp2_model_set_create`` / ``ftsp2_model_set_builtin``
* ``Solver``   -- a planned batch: workspace, device descriptors, outputs;
                  ``Solver.run()`` issues ``ftsp2_density_entropy`` (or the
                  density-only / entropy-only variants) without allocating.
* ``ftsp2_rescale``, ``ftsp2_train_coeffs``, ``ftsp2_train_residual_jacobian``,
  ``ftsp2_train_normal_equations``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (BF16X3, CLAMP, EPI_DEFERRED, EPI_INLINE, FP16X2, FP32, FULL_OPERANDS, LANCZOS, LAYER_LAUNCHES,
                   MIN_LAYERS, MODES,
                   PAIR_TILES,
                   REFINE1, REFINE2, REFINE_TC, SINGLE_TILES, SYNC,
                   TARGET_ENTROPY, TARGET_FERMI, TF32X3, Ftsp2Error, Instance, RescaleRec, Table, TrainReport,
                   check, lib, status_string)

__all__ = ["ModelSet", "Solver", "ftsp2_rescale", "ftsp2_train_coeffs", "ftsp2_train_coeffs_alt", "ftsp2_alt_to_mlsp2",
           "ftsp2_train_coeffs_skip",
           "ftsp2_train_residual_jacobian",
           "ftsp2_train_normal_equations", "ftsp2_autotune_clear", "kernel_launch_count", "profile_layers",
           "set_wait_limit_ns", "wait_limit_ns", "debug_stall_layer",
           "profile_read", "MODES", "FP32", "TF32X3", "BF16X3", "FP16X2", "SYNC", "CLAMP", "REFINE1", "REFINE2",
           "PAIR_TILES", "SINGLE_TILES", "LANCZOS", "MIN_LAYERS", "REFINE_TC", "EPI_DEFERRED", "EPI_INLINE", "FULL_OPERANDS", "LAYER_LAUNCHES", "TARGET_FERMI", "TARGET_ENTROPY", "Ftsp2Error", "status_string", "lib",
           "REC_DTYPE"]

REC_DTYPE = np.dtype([("e_min", "f8"), ("e_max", "f8"), ("mu_p", "f8"), ("beta_p", "f8"), ("scale", "f8"),
                      ("flip", "i4"), ("model", "i4"), ("status", "i4"), ("layers", "i4"), ("valid", "i4"),
                      ("reserved", "i4")])
INST_DTYPE = np.dtype([("n", "i4"), ("reserved", "i4"), ("offset", "i8"), ("mu", "f8"), ("kT", "f8")])


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def kernel_launch_count() -> int:
    return int(lib().ftsp2_kernel_launch_count())


def set_wait_limit_ns(ns: int):
    """Limit of every bounded device-side wait of the layer kernels (ftsp2_set_wait_limit_ns)."""
    check(lib().ftsp2_set_wait_limit_ns(int(ns)), "ftsp2_set_wait_limit_ns")


def wait_limit_ns() -> int:
    return int(lib().ftsp2_wait_limit_ns())


def debug_stall_layer(layer: int):
    """Test hook: items of this global layer of a multi-layer launch wait for a
    completion that never comes (ftsp2_debug_stall_layer); -1 turns it off."""
    check(lib().ftsp2_debug_stall_layer(int(layer)), "ftsp2_debug_stall_layer")


def profile_layers(enable: bool):
    """Bracket every tensor-core layer launch with CUDA events (ftsp2_profile_layers)."""
    check(lib().ftsp2_profile_layers(int(bool(enable))), "ftsp2_profile_layers")


def profile_read():
    """(summed layer-kernel ms, launches) since the last read (ftsp2_profile_read)."""
    ms, n = C.c_double(), C.c_uint64()
    check(lib().ftsp2_profile_read(C.byref(ms), C.byref(n)), "ftsp2_profile_read")
    return ms.value, int(n.value)


class ModelSet:
    """A set of trained tables (Sec. III A 2).  ``tables`` is a list of dicts
    with keys theta ((L, 4) rows a, b, c, d), beta0, mu0, alpha and optionally
    theta_entropy; ``None`` gives the paper's printed 26-layer table.  A table
    of the one-term form (Eq. mlsp2_alt) gives ``alt`` ((L + 1, 2) rows) instead
    of theta (and ``alt_entropy`` instead of theta_entropy); it is converted by
    ftsp2_alt_to_mlsp2.  A Skip-SP2 table (one stored layer, one accumulator;
    FTSP2_FAMILY_SKIP) gives ``skip`` ((L + 1, 4) rows: (delta, alpha, beta,
    gamma) per layer and the output row (A_0, gamma_L, 0, 0)) and optionally
    ``skip_entropy``.  A Max-SP2 table (FTSP2_FAMILY_MAX; FP32 mode only)
    gives ``max``, the flat table of ``max_nparams(L)`` numbers (blocks
    (delta_i, gamma_i, theta_{i,0..i}), then (c, gamma_L)), and optionally
    ``max_entropy``; ftsp2_mlsp2_to_max and ftsp2_skip_to_max build such tables
    from the other families."""

    def __init__(self, tables=None):
        self._h = C.c_void_p()
        self._keep = []
        if tables is None:
            check(lib().ftsp2_model_set_builtin(C.byref(self._h)), "ftsp2_model_set_builtin")
            self.tables = None
            return
        arr = (Table * len(tables))()
        conv = []
        for i, t in enumerate(tables):
            if t.get("theta") is None and t.get("alt") is not None:
                t = dict(t, theta=ftsp2_alt_to_mlsp2(t["alt"]).tolist())
            if t.get("theta_entropy") is None and t.get("alt_entropy") is not None:
                t = dict(t, theta_entropy=ftsp2_alt_to_mlsp2(t["alt_entropy"]).tolist())
            conv.append(t)
            skip = t.get("skip") is not None
            mx = t.get("max") is not None
            if mx:
                th = np.ascontiguousarray(np.asarray(t["max"], dtype=np.float64).ravel())
                arr[i].family = 2
                arr[i].L = max_layers_of(th.size)
            elif skip:
                th = np.ascontiguousarray(np.asarray(t["skip"], dtype=np.float64).reshape(-1, 4))
                arr[i].family = 1
                arr[i].L = th.shape[0] - 1
            else:
                th = np.ascontiguousarray(np.asarray(t["theta"], dtype=np.float64).reshape(-1, 4))
                arr[i].family = 0
                arr[i].L = th.shape[0]
            self._keep.append(th)
            arr[i].beta0 = float(t["beta0"])
            arr[i].mu0 = float(t["mu0"])
            arr[i].alpha = float(t.get("alpha", 0.842704))
            arr[i].theta = th.ctypes.data_as(C.POINTER(C.c_double))
            te = t.get("max_entropy") if mx else t.get("skip_entropy") if skip else t.get("theta_entropy")
            if te is not None and mx:
                te = np.ascontiguousarray(np.asarray(te, dtype=np.float64).ravel())
                self._keep.append(te)
                arr[i].L_entropy = max_layers_of(te.size)
                arr[i].theta_entropy = te.ctypes.data_as(C.POINTER(C.c_double))
            elif te is not None:
                te = np.ascontiguousarray(np.asarray(te, dtype=np.float64).reshape(-1, 4))
                self._keep.append(te)
                arr[i].L_entropy = te.shape[0] - (1 if skip else 0)
                arr[i].theta_entropy = te.ctypes.data_as(C.POINTER(C.c_double))
            else:
                arr[i].L_entropy = 0
                arr[i].theta_entropy = None
        check(lib().ftsp2_model_set_create(arr, len(tables), C.byref(self._h)), "ftsp2_model_set_create")
        self.tables = conv

    @classmethod
    def from_json(cls, paths):
        """Model set from table files written by train_tables (keys beta0, mu0,
        alpha, and theta / alt / skip / max with the matching entropy key)."""
        import json
        tabs = []
        for p in paths:
            with open(p) as f:
                d = json.load(f)
            tabs.append(dict(theta=d.get("theta"), alt=d.get("alt"), skip=d.get("skip"), max=d.get("max"),
                             beta0=d["beta0"], mu0=d["mu0"], alpha=d.get("alpha", 0.842704),
                             theta_entropy=d.get("theta_entropy"), alt_entropy=d.get("alt_entropy"),
                             skip_entropy=d.get("skip_entropy"), max_entropy=d.get("max_entropy")))
        return cls(tabs)

    @property
    def handle(self):
        return self._h

    def info(self):
        n, L = C.c_int(), C.c_int()
        check(lib().ftsp2_model_set_info(self._h, C.byref(n), C.byref(L)), "ftsp2_model_set_info")
        return n.value, L.value

    def table(self, idx=0):
        """(theta (L, 4), beta0, mu0, alpha) of table idx (ftsp2_model_set_table;
        the flat table for a Max-SP2 table)."""
        L = C.c_int()
        th = (C.c_double * 256)()
        b0, m0, al = C.c_double(), C.c_double(), C.c_double()
        check(lib().ftsp2_model_set_table(self._h, int(idx), C.byref(L), th, C.byref(b0), C.byref(m0),
                                          C.byref(al)), "ftsp2_model_set_table")
        if self.tables is not None and self.tables[idx].get("max") is not None:
            return np.array(th[:max_nparams(L.value)]), b0.value, m0.value, al.value
        return np.array(th[:4 * L.value]).reshape(-1, 4), b0.value, m0.value, al.value

    def close(self):
        if self._h:
            lib().ftsp2_model_set_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _instances(ns, mus, kTs, offsets=None):
    nb = len(ns)
    host = (Instance * nb)()
    offs = []
    o = 0
    for b in range(nb):
        off = o if offsets is None else int(offsets[b])
        host[b].n = int(ns[b])
        host[b].offset = off
        host[b].mu = float(mus[b])
        host[b].kT = float(kTs[b])
        offs.append(off)
        o += int(ns[b]) * int(ns[b])
    return host, offs, o


class Solver:
    """One planned (ragged) batch on the current CUDA device.

    ns, mus, kTs: per-instance order, chemical potential (eV) and temperature
    (eV).  Matrices are packed back to back (offset_b = sum_{b'<b} n_b'^2) in a
    flat FP64 tensor.  want: 1 density, 2 entropy, 3 both.  Allocates the
    workspace, the device descriptor copy and the outputs once; ``run`` then
    only launches kernels (safe to capture in a CUDA graph)."""

    def __init__(self, ns, mus, kTs, model_set: ModelSet, mode="fp16x2", want=3, flags=0, device=None):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        self.want = int(want)
        self.flags = int(flags)
        self.ms = model_set
        self.nb = len(ns)
        self.host_inst, self.offsets, self.total = _instances(ns, mus, kTs)
        self.ns = [int(n) for n in ns]
        raw = np.frombuffer(bytes(self.host_inst), dtype=INST_DTYPE)
        self.d_inst = torch.from_numpy(raw.view(np.uint8).copy()).to(self.device)
        wsz = C.c_size_t()
        check(lib().ftsp2_workspace_size_set(self.host_inst, self.nb, model_set.handle, self.mode, self.want,
                                             C.byref(wsz)), "ftsp2_workspace_size_set")
        self.ws_bytes = wsz.value
        self._ws_raw = torch.empty(self.ws_bytes + 1024, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr()
        self.ws_ptr = (base + 1023) // 1024 * 1024
        self.D = torch.empty(self.total, dtype=torch.float32, device=self.device) if want & 1 else None
        self.trace = torch.empty((self.nb, 2), dtype=torch.float64, device=self.device) if want & 1 else None
        self.S = torch.empty(self.nb, dtype=torch.float64, device=self.device) if want & 2 else None
        self.rec = torch.empty(self.nb * 64, dtype=torch.uint8, device=self.device)

    def set_mu_kT(self, mus, kTs):
        """Change the per-instance mu and kT (host and device copies)."""
        for b in range(self.nb):
            self.host_inst[b].mu = float(mus[b])
            self.host_inst[b].kT = float(kTs[b])
        raw = np.frombuffer(bytes(self.host_inst), dtype=np.uint8).copy()
        self.d_inst.copy_(_torch().from_numpy(raw))

    def run(self, H, stream=None, sync=False):
        """Launch the hot path on the flat FP64 device tensor H (length
        sum n_b^2).  Returns the status of the call (host-side errors raise)."""
        torch = _torch()
        if H.dtype != torch.float64 or not H.is_cuda or H.numel() < self.total:
            raise ValueError("H must be a CUDA float64 tensor with sum(n^2) elements")
        flags = self.flags | (SYNC if sync else 0)
        L = lib()
        args_common = (_ptr(H), self.host_inst, _ptr(self.d_inst), self.nb, self.ms.handle, self.mode, flags)
        if self.want == 1:
            st = L.ftsp2_density(*args_common, _ptr(self.D), _ptr(self.trace), _ptr(self.rec),
                                 C.c_void_p(self.ws_ptr), self.ws_bytes, _stream(stream))
        elif self.want == 2:
            st = L.ftsp2_entropy(*args_common, _ptr(self.S), _ptr(self.rec), C.c_void_p(self.ws_ptr),
                                 self.ws_bytes, _stream(stream))
        else:
            st = L.ftsp2_density_entropy(*args_common, _ptr(self.D), _ptr(self.trace), _ptr(self.S),
                                         _ptr(self.rec), C.c_void_p(self.ws_ptr), self.ws_bytes, _stream(stream))
        if st in (_lib.E_ARG, _lib.E_CUDA, _lib.E_WORKSPACE, _lib.E_NOMODEL, _lib.E_UNSUPPORTED):
            raise Ftsp2Error(st, "ftsp2 hot path")
        return st

    def run_mu(self, H, n_occ, iterations=3, tol=1e-6, stream=None, sync=False):
        """Chemical potentials for prescribed electron counts (ftsp2_density_mu):
        ``iterations`` Newton updates of mu from the current device values,
        then D (and S when the solver has the entropy chain) at the final mu.
        n_occ: per-instance electron counts.  Returns the per-instance number of
        updates taken (int32 tensor); the final mu are in ``mus()``."""
        torch = _torch()
        if self.want == 2:
            raise ValueError("run_mu needs the density chain (want = 1 or 3)")
        if H.dtype != torch.float64 or not H.is_cuda or H.numel() < self.total:
            raise ValueError("H must be a CUDA float64 tensor with sum(n^2) elements")
        nocc = torch.as_tensor(n_occ, dtype=torch.float64, device=self.device).reshape(self.nb).contiguous()
        steps = torch.zeros(self.nb, dtype=torch.int32, device=self.device)
        flags = self.flags | (SYNC if sync else 0)
        S = _ptr(self.S) if self.want == 3 else None
        st = lib().ftsp2_density_mu(_ptr(H), self.host_inst, _ptr(self.d_inst), self.nb, _ptr(nocc), self.ms.handle,
                                    self.mode, flags, int(iterations), float(tol), _ptr(self.D), _ptr(self.trace), S,
                                    _ptr(self.rec), _ptr(steps), C.c_void_p(self.ws_ptr), self.ws_bytes,
                                    _stream(stream))
        if st in (_lib.E_ARG, _lib.E_CUDA, _lib.E_WORKSPACE, _lib.E_NOMODEL, _lib.E_UNSUPPORTED):
            raise Ftsp2Error(st, "ftsp2_density_mu")
        self._nocc_keepalive = nocc
        return steps

    def mus(self):
        """The per-instance mu of the device instance table (after run_mu)."""
        raw = self.d_inst.cpu().numpy().view(INST_DTYPE)
        return raw["mu"].copy()

    def graph(self, H):
        """Record one ``run(H)`` into a CUDA graph and return it
        (``torch.cuda.CUDAGraph``; ``g.replay()`` reruns the whole hot path on
        the current contents of H and of the device instance table, writing
        the same output tensors).  An eager run with the same arguments comes
        first, as the C ABI asks."""
        torch = _torch()
        self.run(H)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(H)
        return g

    def _outputs(self):
        D = _ptr(self.D) if self.want & 1 else None
        T = _ptr(self.trace) if self.want & 1 else None
        S = _ptr(self.S) if self.want & 2 else None
        return D, T, S

    def autotune(self, H, reps=3, stream=None):
        """ftsp2_autotune on this batch: times both tile shapes and records the
        faster for every later call with the same signature.  Returns
        (shape, ms_single, ms_pair); shape 1 = 256 x 256 pairs, 0 = 128 x 128
        single CTAs, -1 = no tensor-core layers (FP32 mode)."""
        torch = _torch()
        if H.dtype != torch.float64 or not H.is_cuda or H.numel() < self.total:
            raise ValueError("H must be a CUDA float64 tensor with sum(n^2) elements")
        choice = C.c_int()
        ms = (C.c_float * 2)()
        D, T, S = self._outputs()
        check(lib().ftsp2_autotune(_ptr(H), self.host_inst, _ptr(self.d_inst), self.nb, self.ms.handle, self.mode,
                                   self.flags, D, T, S, _ptr(self.rec), C.c_void_p(self.ws_ptr), self.ws_bytes,
                                   int(reps), C.byref(choice), ms, _stream(stream)), "ftsp2_autotune")
        return choice.value, float(ms[0]), float(ms[1])

    def tile_shape(self):
        """(shape, from_tuner) that run() uses on the current device
        (ftsp2_tile_shape)."""
        shape, tuned = C.c_int(), C.c_int()
        check(lib().ftsp2_tile_shape(self.host_inst, self.nb, self.mode, self.want, self.flags, C.byref(shape),
                                     C.byref(tuned)), "ftsp2_tile_shape")
        return shape.value, bool(tuned.value)

    def records(self):
        raw = self.rec.cpu().numpy()
        return raw.view(REC_DTYPE)

    def matrix(self, b):
        n, o = self.ns[b], self.offsets[b]
        return self.D[o:o + n * n].view(n, n)


def ftsp2_autotune_clear():
    """Forget every recorded tile-shape choice."""
    check(lib().ftsp2_autotune_clear(), "ftsp2_autotune_clear")


def ftsp2_rescale(H, ns, mus, kTs, model_set: ModelSet, flags=0, stream=None):
    """(a1)+(a2) only; returns the per-instance records (numpy structured)."""
    torch = _torch()
    host, offs, total = _instances(ns, mus, kTs)
    nb = len(ns)
    raw = np.frombuffer(bytes(host), dtype=np.uint8).copy()
    d_inst = torch.from_numpy(raw).to(H.device)
    rec = torch.empty(nb * 64, dtype=torch.uint8, device=H.device)
    wsz = C.c_size_t()
    if int(flags) & LANCZOS:
        # the Lanczos buffers are part of the hot path's workspace
        check(lib().ftsp2_workspace_size(host, nb, FP16X2, 1, C.byref(wsz)), "ftsp2_workspace_size")
    else:
        check(lib().ftsp2_rescale_workspace_size(nb, C.byref(wsz)), "ftsp2_rescale_workspace_size")
    ws = torch.empty(wsz.value + 1024, dtype=torch.uint8, device=H.device)
    wp = (ws.data_ptr() + 1023) // 1024 * 1024
    st = lib().ftsp2_rescale(_ptr(H), host, _ptr(d_inst), nb, model_set.handle, int(flags) | SYNC, _ptr(rec),
                             C.c_void_p(wp), wsz.value, _stream(stream))
    if st in (_lib.E_ARG, _lib.E_CUDA, _lib.E_WORKSPACE, _lib.E_NOMODEL, _lib.E_UNSUPPORTED):
        raise Ftsp2Error(st, "ftsp2_rescale")
    return rec.cpu().numpy().view(REC_DTYPE)


def ftsp2_train_residual_jacobian(target, beta0, mu0, theta, x, alpha=1.0, with_jacobian=True, stream=None):
    """Residuals r (ns,) and augmented Jacobian M ((4L+1), ns) on the GPU."""
    torch = _torch()
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 4))
    L = th.shape[0]
    ns = x.numel()
    r = torch.empty(ns, dtype=torch.float64, device=x.device)
    M = torch.empty((4 * L + 1, ns), dtype=torch.float64, device=x.device) if with_jacobian else None
    check(lib().ftsp2_train_residual_jacobian(int(target), float(beta0), float(mu0), L, float(alpha),
                                              th.ctypes.data_as(C.POINTER(C.c_double)), _ptr(x), ns, _ptr(r),
                                              _ptr(M), _stream(stream)), "ftsp2_train_residual_jacobian")
    return r, M


def ftsp2_train_normal_equations(M, L, stream=None):
    """G = M^T M ((4L+1) x (4L+1)) on the GPU, FP64, fixed reduction order."""
    torch = _torch()
    ns = M.shape[1]
    m = 4 * L + 1
    G = torch.empty((m, m), dtype=torch.float64, device=M.device)
    wb = lib().ftsp2_train_workspace_size(ns, L)
    ws = torch.empty(wb, dtype=torch.uint8, device=M.device)
    check(lib().ftsp2_train_normal_equations(_ptr(M), ns, L, _ptr(G), _ptr(ws), wb, _stream(stream)),
          "ftsp2_train_normal_equations")
    return G


def ftsp2_alt_to_mlsp2(alt):
    """Rows (a, b, c, d) (numpy (L, 4)) of Eq. mlsp2 computing the same function
    as the one-term table alt ((L + 1, 2) rows, Eq. mlsp2_alt)."""
    a = np.ascontiguousarray(np.asarray(alt, dtype=np.float64).reshape(-1, 2))
    L = a.shape[0] - 1
    out = np.zeros((max(L, 1), 4))
    check(lib().ftsp2_alt_to_mlsp2(L, a.ctypes.data_as(C.POINTER(C.c_double)),
                                   out.ctypes.data_as(C.POINTER(C.c_double))), "ftsp2_alt_to_mlsp2")
    return out


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _train(fn, target, beta0, mu0, L, init, width, nrows, nsamples, seed, iterations, accel, alpha, ws_rows, stream):
    torch = _torch()
    p0 = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=np.float64).reshape(-1, width))
    out = np.zeros((nrows, width))
    wb = lib().ftsp2_train_workspace_size(int(nsamples), ws_rows)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    rep = TrainReport()
    check(fn(int(target), float(beta0), float(mu0), int(L), float(alpha), int(nsamples), int(seed), int(iterations),
             int(bool(accel)), None if p0 is None else _dp(p0), _dp(out), C.byref(rep), _ptr(ws), wb,
             _stream(stream)), fn.__name__)
    return out, dict(iterations=rep.iterations, accepted=rep.accepted, cost0=rep.cost0, cost=rep.cost,
                     max_err=rep.max_err, lam=rep.lam)


def ftsp2_train_coeffs(target, beta0, mu0, L=None, theta_init=None, nsamples=100_000, seed=0, iterations=100,
                       accel=True, alpha=1.0, stream=None):
    """Levenberg-Marquardt fit of an Eq. mlsp2 table on the GPU (Sec. II C) on
    the library's own sample set (ftsp2_train_samples(beta0, mu0, nsamples,
    seed)).  theta_init None starts from ftsp2_train_init(L, beta0, mu0).
    Returns (theta (L, 4) numpy, report dict)."""
    if theta_init is not None:
        L = np.asarray(theta_init).reshape(-1, 4).shape[0]
    return _train(lib().ftsp2_train_coeffs, target, beta0, mu0, L, theta_init, 4, L, nsamples, seed, iterations,
                  accel, alpha, L, stream)


def ftsp2_train_coeffs_alt(target, beta0, mu0, L=None, alt_init=None, nsamples=100_000, seed=0, iterations=100,
                           accel=True, alpha=1.0, stream=None):
    """Levenberg-Marquardt fit of a one-term table (Eq. mlsp2_alt) on the GPU.
    Returns (alt (L + 1, 2) numpy, report dict)."""
    if alt_init is not None:
        L = np.asarray(alt_init).reshape(-1, 2).shape[0] - 1
    return _train(lib().ftsp2_train_coeffs_alt, target, beta0, mu0, L, alt_init, 2, L + 1, nsamples, seed,
                  iterations, accel, alpha, L, stream)


def _report(rep):
    return dict(iterations=rep.iterations, accepted=rep.accepted, cost0=rep.cost0, cost=rep.cost,
                max_err=rep.max_err, lam=rep.lam)


def ftsp2_train_coeffs_max(target, beta0, mu0, L=None, max_init=None, nsamples=100_000, seed=0, iterations=100,
                           accel=True, alpha=1.0, stream=None):
    """Levenberg-Marquardt fit of a flat Max-SP2 table on the GPU.  max_init
    None starts from ftsp2_mlsp2_to_max(ftsp2_train_init(L, beta0, mu0)).
    Returns (flat table numpy, report dict)."""
    torch = _torch()
    p0 = None
    if max_init is not None:
        p0 = np.ascontiguousarray(np.asarray(max_init, dtype=np.float64).ravel())
        L = max_layers_of(p0.size)
    out = np.zeros(max_nparams(L))
    wb = lib().ftsp2_train_workspace_size_max(int(nsamples), int(L))
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    rep = TrainReport()
    check(lib().ftsp2_train_coeffs_max(int(target), float(beta0), float(mu0), int(L), float(alpha), int(nsamples),
                                       int(seed), int(iterations), int(bool(accel)), None if p0 is None else _dp(p0),
                                       _dp(out), C.byref(rep), _ptr(ws), wb, _stream(stream)),
          "ftsp2_train_coeffs_max")
    return out, _report(rep)


def skipk_nparams(L, k, K):
    """(1 + k + 2K) L + 2 trainable numbers of a Skip-SP2 table with k stored
    layers and K accumulators."""
    return (1 + int(k) + 2 * int(K)) * int(L) + 2


def ftsp2_train_coeffs_skipk(target, beta0, mu0, L, k, K, skip_init=None, nsamples=100_000, seed=0, iterations=100,
                             accel=True, alpha=1.0, stream=None):
    """Levenberg-Marquardt fit of a Skip-SP2 table with k stored layers and K
    accumulators on the GPU (vector layout of ftsp2_train_coeffs_skipk).
    Returns (vector numpy, report dict)."""
    torch = _torch()
    npar = skipk_nparams(L, k, K)
    p0 = None if skip_init is None else np.ascontiguousarray(np.asarray(skip_init, dtype=np.float64).ravel())
    if p0 is not None and p0.size != npar:
        raise ValueError("skip_init must hold (1 + k + 2K) L + 2 numbers")
    out = np.zeros(npar)
    wb = lib().ftsp2_train_workspace_size_max(int(nsamples), int(L))
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    rep = TrainReport()
    check(lib().ftsp2_train_coeffs_skipk(int(target), float(beta0), float(mu0), int(L), int(k), int(K), float(alpha),
                                         int(nsamples), int(seed), int(iterations), int(bool(accel)),
                                         None if p0 is None else _dp(p0), _dp(out), C.byref(rep), _ptr(ws), wb,
                                         _stream(stream)), "ftsp2_train_coeffs_skipk")
    return out, _report(rep)


def ftsp2_train_init_skipk(L, k, K, beta0, mu0):
    """The library's default start of a Skip-SP2 (k, K) fit (host-only call)."""
    out = np.zeros(skipk_nparams(L, k, K))
    check(lib().ftsp2_train_init_skipk(int(L), int(k), int(K), float(beta0), float(mu0), _dp(out)),
          "ftsp2_train_init_skipk")
    return out


def ftsp2_skipk_to_max(vec, L, k, K):
    """Flat Max-SP2 table of a Skip-SP2 (k, K) vector (host-only call)."""
    v = np.ascontiguousarray(np.asarray(vec, dtype=np.float64).ravel())
    if v.size != skipk_nparams(L, k, K):
        raise ValueError("vector must hold (1 + k + 2K) L + 2 numbers")
    out = np.zeros(max_nparams(L))
    check(lib().ftsp2_skipk_to_max(int(L), int(k), int(K), _dp(v), _dp(out)), "ftsp2_skipk_to_max")
    return out


def ftsp2_train_coeffs_skip(target, beta0, mu0, L=None, skip_init=None, nsamples=100_000, seed=0, iterations=100,
                            accel=True, alpha=1.0, stream=None):
    """Levenberg-Marquardt fit of a Skip-SP2 table (one stored layer, one
    accumulator) on the GPU.  Returns (table (L + 1, 4) numpy, report dict)."""
    if skip_init is not None:
        L = np.asarray(skip_init).reshape(-1, 4).shape[0] - 1
    return _train(lib().ftsp2_train_coeffs_skip, target, beta0, mu0, L, skip_init, 4, L + 1, nsamples, seed,
                  iterations, accel, alpha, L + 1, stream)


def ftsp2_train_samples(beta0, mu0, nsamples, seed=0):
    """The training samples the library builds (numpy, host-only call)."""
    x = np.zeros(int(nsamples))
    check(lib().ftsp2_train_samples(float(beta0), float(mu0), int(nsamples), int(seed), _dp(x)),
          "ftsp2_train_samples")
    return x


def ftsp2_train_init(L, beta0, mu0):
    """The library's starting Eq. mlsp2 table ((L, 4) numpy, host-only call)."""
    th = np.zeros((int(L), 4))
    check(lib().ftsp2_train_init(int(L), float(beta0), float(mu0), _dp(th)), "ftsp2_train_init")
    return th


def ftsp2_train_init_alt(L, mu0):
    """The library's starting one-term table ((L + 1, 2) numpy, host-only call)."""
    a = np.zeros((int(L) + 1, 2))
    check(lib().ftsp2_train_init_alt(int(L), float(mu0), _dp(a)), "ftsp2_train_init_alt")
    return a


def ftsp2_mlsp2_to_skip(theta):
    """Appendix embedding of Eq. mlsp2 rows as a Skip-SP2 table ((L + 1, 4) numpy)."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 4))
    L = th.shape[0]
    out = np.zeros((L + 1, 4))
    check(lib().ftsp2_mlsp2_to_skip(L, _dp(th), _dp(out)), "ftsp2_mlsp2_to_skip")
    return out


def max_nparams(L):
    """Length of a flat Max-SP2 table of L layers: L (L + 5) / 2 + 2."""
    return int(L) * (int(L) + 5) // 2 + 2


def max_layers_of(size):
    """Layer count of a flat Max-SP2 table of `size` numbers."""
    for L in range(1, 64):
        if max_nparams(L) == size:
            return L
    raise ValueError(f"{size} numbers are no flat Max-SP2 table")


def ftsp2_mlsp2_to_max(theta):
    """Flat Max-SP2 table computing the same function as Eq. mlsp2 rows
    (through their Skip-SP2 embedding; host-only call)."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 4))
    L = th.shape[0]
    out = np.zeros(max_nparams(L))
    check(lib().ftsp2_mlsp2_to_max(L, _dp(th), _dp(out)), "ftsp2_mlsp2_to_max")
    return out


def ftsp2_skip_to_max(alpha, beta, gamma, A0, gL=1.0):
    """Flat Max-SP2 table of a Skip-SP2 table with k stored layers and K
    accumulators: alpha (L, k + 1) with the constant last, beta and gamma
    (L, K), A0 (K,), output weight gL of the last layer (host-only call)."""
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    L, k = al.shape[0], al.shape[1] - 1
    be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(L, -1))
    K = be.shape[1]
    ga = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(L, K))
    a0 = np.ascontiguousarray(np.asarray(A0, dtype=np.float64).reshape(K))
    out = np.zeros(max_nparams(L))
    check(lib().ftsp2_skip_to_max(L, k, K, _dp(al), _dp(be) if K else None, _dp(ga) if K else None,
                                  _dp(a0) if K else None, float(gL), _dp(out)), "ftsp2_skip_to_max")
    return out


def ftsp2_layer_count(beta_p):
    """Eq. layer count (host-only call)."""
    return float(lib().ftsp2_layer_count(float(beta_p)))


def ftsp2_train_residuals(target, beta0, mu0, table, x, alpha=1.0, family=0, stream=None):
    """Residuals model - target of a table at the CUDA float64 points x
    (family 0: Eq. mlsp2 rows; 1: Skip-SP2 rows with the output row; 2: a
    flat Max-SP2 table)."""
    torch = _torch()
    if family == 2:
        tb = np.ascontiguousarray(np.asarray(table, dtype=np.float64).ravel())
        L = max_layers_of(tb.size)
    else:
        tb = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 4))
        L = tb.shape[0] - (1 if family == 1 else 0)
    r = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
    check(lib().ftsp2_train_residuals(int(family), int(target), float(beta0), float(mu0), L, float(alpha), _dp(tb),
                                      _ptr(x), x.numel(), _ptr(r), _stream(stream)), "ftsp2_train_residuals")
    return r
