"""Thin ctypes binding of libgwgb.so (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module
converts Python/NumPy/torch arguments into the C ABI of include/gwgb.h and
back.  Device memory for the library comes from PyTorch's caching allocator
and work is enqueued on PyTorch's current CUDA stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwgb.so")

GW_OK, GW_ERR_ARG, GW_ERR_CUDA, GW_ERR_OOM, GW_ERR_NOT_CONVERGED, GW_ERR_SINGULAR, GW_ERR_TIMEOUT, \
    GW_ERR_STATE, GW_ERR_INTERNAL = range(9)
PRECISIONS = {"fp64": 0, "fp32": 1, "split_bf16": 2, "split_tf32": 3, "split_f16": 4}
GW_INPUT_DEVICE, GW_BORROW_V, GW_SKIP_CHECKS, GW_SMALL_TENSOR, GW_SMALL_SIMT, GW_FP64_NATIVE, GW_TRS = \
    1, 2, 4, 8, 16, 32, 64

QUANTITIES = {
    "G_tau": 0, "G_iw": 1, "Sigma_inf": 2, "Sigma_tau": 3, "Sigma_iw": 4, "P0_tau": 5, "P0_iw": 6,
    "P_iw": 7, "P_tau": 8, "gamma": 9, "mu": 10, "TFf": 11, "TBf": 12, "TFb": 13, "TBb": 14,
    "lb": 15, "tau": 16, "n_elec": 17, "Sigma_inf_new": 18,
}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class GwConfig(ctypes.Structure):
    _fields_ = [
        ("nao", ctypes.c_int32), ("naux", ctypes.c_int32), ("kmesh", ctypes.c_int32 * 3),
        ("ntau", ctypes.c_int32), ("beta", ctypes.c_double), ("n_elec", ctypes.c_double),
        ("mu_tol", ctypes.c_double), ("mu_maxit", ctypes.c_int32), ("damping", ctypes.c_double),
        ("contract_prec", ctypes.c_int32), ("spin_factor", ctypes.c_int32),
        ("fermi_n", ctypes.POINTER(ctypes.c_int32)), ("bose_m", ctypes.POINTER(ctypes.c_int32)),
        ("stream", ctypes.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p), ("flags", ctypes.c_uint64),
    ]


class GwGrid(ctypes.Structure):
    _fields_ = [
        ("ntau", ctypes.c_int32), ("nwf", ctypes.c_int32), ("nwb", ctypes.c_int32),
        ("tau", ctypes.c_void_p), ("fermi_n", ctypes.c_void_p), ("bose_m", ctypes.c_void_p),
        ("TFf", ctypes.c_void_p), ("TBf", ctypes.c_void_p), ("TFb", ctypes.c_void_p), ("TBb", ctypes.c_void_p),
        ("lb", ctypes.c_void_p),
    ]


class GwIterStats(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double), ("n_elec", ctypes.c_double), ("mu_steps", ctypes.c_int32),
        ("max_dG", ctypes.c_double), ("max_dSigma", ctypes.c_double), ("ms_total", ctypes.c_float),
        ("ms_polarization", ctypes.c_float), ("ms_screened", ctypes.c_float),
        ("ms_selfenergy", ctypes.c_float), ("ms_dyson", ctypes.c_float), ("ms_hf", ctypes.c_float),
    ]


_lib = None


def load():
    """Load libgwgb.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libgwgb.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2206_07660_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.gw_init.argtypes = [ctypes.POINTER(GwConfig), P, P, P, ctypes.POINTER(P)]
    lib.gw_init_grid.argtypes = [ctypes.POINTER(GwConfig), ctypes.POINTER(GwGrid), P, P, P, ctypes.POINTER(P)]
    lib.gw_destroy.argtypes = [P]
    lib.gw_set.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int]
    lib.gw_get.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t, ctypes.c_int]
    for name in ("gw_hf", "gw_polarization", "gw_screened", "gw_selfenergy", "gw_reset_sigma",
                 "gw_selfenergy_partial", "gw_selfenergy_finish"):
        getattr(lib, name).argtypes = [P]
    lib.gw_set_q_range.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
    lib.gw_save_state.argtypes = [P, ctypes.c_char_p]
    lib.gw_load_state.argtypes = [P, ctypes.c_char_p]
    lib.gw_dyson.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.gw_grand_potential.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.gw_iterate.argtypes = [P, ctypes.c_int32, ctypes.POINTER(GwIterStats)]
    lib.gw_last_error.argtypes = [P]
    lib.gw_last_error.restype = ctypes.c_char_p
    lib.gw_iterate_graph.argtypes = [P, ctypes.c_int32, ctypes.POINTER(GwIterStats)]
    lib.gw_batch_iterate.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32]
    lib.gw_polarization_vjp.argtypes = [P, P, P]
    lib.gw_selfenergy_vjp.argtypes = [P, P, P, P]
    lib.gw_iterate_diis.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_double)]
    lib.gw_polarization_vjp_c64.argtypes = [P, P, P]
    lib.gw_selfenergy_vjp_c64.argtypes = [P, P, P, P]
    lib.gw_polarization_jvp.argtypes = [P, P, P]
    lib.gw_screened_jvp.argtypes = [P, P, P]
    lib.gw_selfenergy_jvp.argtypes = [P, P, P, P]
    lib.gw_sc_jvp.argtypes = [P, P, P, P, P]
    lib.gw_iterate_newton.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.gw_profile.argtypes = [P, ctypes.c_int]
    lib.gw_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.gw_kernel_launches.argtypes = [P]
    lib.gw_kernel_launches.restype = ctypes.c_int64
    for name in ("gw_init", "gw_init_grid", "gw_destroy", "gw_set", "gw_get", "gw_hf", "gw_polarization", "gw_screened",
                 "gw_selfenergy", "gw_dyson", "gw_iterate", "gw_reset_sigma", "gw_profile", "gw_profile_read",
                 "gw_polarization_vjp", "gw_selfenergy_vjp", "gw_iterate_graph", "gw_batch_iterate",
                 "gw_polarization_jvp", "gw_screened_jvp", "gw_selfenergy_jvp", "gw_sc_jvp",
                 "gw_iterate_newton", "gw_selfenergy_partial", "gw_selfenergy_finish", "gw_set_q_range", "gw_save_state",
                 "gw_load_state", "gw_polarization_vjp_c64", "gw_selfenergy_vjp_c64", "gw_iterate_diis"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def batch_iterate(systems, n=1):
    """n captured iterations of several GW contexts, overlapped on their own streams."""
    lib = load()
    arr = (ctypes.c_void_p * len(systems))(*[s.ctx.value if hasattr(s.ctx, "value") else s.ctx for s in systems])
    st = lib.gw_batch_iterate(arr, len(systems), int(n))
    if st != GW_OK:
        raise GWError(st, lib.gw_last_error(None).decode())


class GWError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("gw status %d: %s" % (status, msg))
        self.status = status


def _ptr(x):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data, False
    assert x.is_contiguous()
    return x.data_ptr(), x.is_cuda


class GW:
    """One self-consistent GW problem resident on the GPU.

    H0, S: [nk, nao, nao] complex128; V: [nk, nk, naux, nao, nao] complex128
    (numpy arrays, or CUDA torch tensors with device_inputs=True).
    fermi_n, bose_m: sampled Matsubara integers (length ntau) of the Chebyshev grid.
    grid: optional sparse-sampling grid (an object or dict with tau, fermi_n, bose_m,
    TFf, TBf, TFb, TBb, lb; gw_init_grid) used instead of the Chebyshev grid.
    """

    def __init__(self, H0, S, V, kmesh, ntau, beta, fermi_n=None, bose_m=None, n_elec=None, damping=0.5,
                 mu_tol=1e-9, mu_maxit=400, precision="fp64", spin=2, borrow_V=False,
                 skip_checks=False, torch_alloc=True, small_steps="auto", fp64_gemm="tensor", trs=False,
                 grid=None):
        import torch
        self.lib = load()
        self.torch = torch
        nk, nao = H0.shape[0], H0.shape[1]
        naux = V.shape[2]
        self.nk, self.nao, self.naux, self.ntau = int(nk), int(nao), int(naux), int(ntau)
        gget = (lambda k: grid[k]) if isinstance(grid, dict) else (lambda k: getattr(grid, k))
        if grid is not None:
            fermi_n, bose_m = gget("fermi_n"), gget("bose_m")
        self._fn = np.ascontiguousarray(fermi_n, dtype=np.int32)
        self._bm = np.ascontiguousarray(bose_m, dtype=np.int32)
        self.nwf, self.nwb = int(self._fn.size), int(self._bm.size)
        cfg = GwConfig()
        cfg.nao, cfg.naux, cfg.ntau = self.nao, self.naux, self.ntau
        for i in range(3):
            cfg.kmesh[i] = int(kmesh[i])
        cfg.beta = float(beta)
        cfg.n_elec = float(nao if n_elec is None else n_elec)
        cfg.mu_tol, cfg.mu_maxit, cfg.damping = float(mu_tol), int(mu_maxit), float(damping)
        cfg.contract_prec = PRECISIONS[precision]
        cfg.spin_factor = int(spin)
        cfg.fermi_n = self._fn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        cfg.bose_m = self._bm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self.stream = torch.cuda.current_stream()
        cfg.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.device = torch.cuda.current_device()
        if torch_alloc:
            dev, strm = self.device, self.stream

            def _alloc(user, nbytes):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except Exception:
                    return None

            def _free(user, p):
                torch.cuda.caching_allocator_delete(int(p))
            self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
            cfg.dev_alloc, cfg.dev_free = self._alloc_cb, self._free_cb
        flags = 0
        hp, hdev = _ptr(H0)
        sp, _ = _ptr(S)
        vp, vdev = _ptr(V)
        if hdev:
            flags |= GW_INPUT_DEVICE
        if borrow_V:
            flags |= GW_BORROW_V
            self._V_ref = V
        if skip_checks:
            flags |= GW_SKIP_CHECKS
        flags |= {"auto": 0, "tensor": GW_SMALL_TENSOR, "simt": GW_SMALL_SIMT}[small_steps]
        flags |= {"tensor": 0, "native": GW_FP64_NATIVE}[fp64_gemm]
        if trs:
            flags |= GW_TRS
        cfg.flags = flags
        self._cfg = cfg
        ctx = ctypes.c_void_p()
        if grid is None:
            st = self.lib.gw_init(ctypes.byref(cfg), hp, sp, vp, ctypes.byref(ctx))
        else:
            keep = {k: np.ascontiguousarray(gget(k), dtype=np.complex128) for k in ("TFf", "TBf", "TFb", "TBb")}
            keep["tau"] = np.ascontiguousarray(gget("tau"), dtype=np.float64)
            keep["lb"] = np.ascontiguousarray(np.real(gget("lb")), dtype=np.float64)
            gr = GwGrid()
            gr.ntau, gr.nwf, gr.nwb = self.ntau, self.nwf, self.nwb
            for k, v in keep.items():
                setattr(gr, k, v.ctypes.data)
            gr.fermi_n, gr.bose_m = self._fn.ctypes.data, self._bm.ctypes.data
            st = self.lib.gw_init_grid(ctypes.byref(cfg), ctypes.byref(gr), hp, sp, vp, ctypes.byref(ctx))
        if st != GW_OK:
            raise GWError(st, self.lib.gw_last_error(None).decode())
        self.ctx = ctx

    # -- plumbing
    def _check(self, st):
        if st != GW_OK:
            raise GWError(st, self.lib.gw_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape_of(self, name):
        nk, nao, naux, nt, nf, nb = self.nk, self.nao, self.naux, self.ntau, self.nwf, self.nwb
        return {
            "G_tau": (nt, nk, nao, nao), "G_iw": (nf, nk, nao, nao), "Sigma_inf": (nk, nao, nao),
            "Sigma_inf_new": (nk, nao, nao), "Sigma_tau": (nt, nk, nao, nao), "Sigma_iw": (nf, nk, nao, nao),
            "P0_tau": (nk, nt, naux, naux), "P0_iw": (nk, nb, naux, naux), "P_iw": (nk, nb, naux, naux),
            "P_tau": (nk, nt, naux, naux), "gamma": (nk, nao, nao), "TFf": (nf, nt), "TBf": (nt, nf),
            "TFb": (nb, nt), "TBb": (nt, nb),
        }[name]

    def get(self, name, out=None):
        q = QUANTITIES[name]
        if name in ("mu", "n_elec"):
            v = ctypes.c_double()
            self._check(self.lib.gw_get(self.ctx, q, ctypes.byref(v), 8, 0))
            return v.value
        if name in ("lb", "tau"):
            arr = np.empty(self.ntau, dtype=np.float64)
        else:
            arr = np.empty(self.shape_of(name), dtype=np.complex128) if out is None else out
        p, dev = _ptr(arr)
        self._check(self.lib.gw_get(self.ctx, q, p, arr.nbytes if isinstance(arr, np.ndarray)
                                    else arr.numel() * arr.element_size(), int(dev)))
        return arr

    def set(self, name, value):
        q = QUANTITIES[name]
        if name == "mu":
            v = ctypes.c_double(float(value))
            self._check(self.lib.gw_set(self.ctx, q, ctypes.byref(v), 8, 0))
            return
        if isinstance(value, np.ndarray):
            value = np.ascontiguousarray(value, dtype=np.complex128)
            nbytes = value.nbytes
        else:
            nbytes = value.numel() * value.element_size()
        p, dev = _ptr(value)
        self._check(self.lib.gw_set(self.ctx, q, p, nbytes, int(dev)))

    # -- stages (Eqs. HF_J/HF_K, tilde_P0_tau, tilde_P_omega, tilde_sigma2, Dyson)
    def hf(self):
        self._check(self.lib.gw_hf(self.ctx))

    def polarization(self):
        self._check(self.lib.gw_polarization(self.ctx))

    def screened(self):
        self._check(self.lib.gw_screened(self.ctx))

    def selfenergy(self):
        self._check(self.lib.gw_selfenergy(self.ctx))

    def selfenergy_partial(self):
        self._check(self.lib.gw_selfenergy_partial(self.ctx))

    def selfenergy_finish(self):
        self._check(self.lib.gw_selfenergy_finish(self.ctx))

    def set_q_range(self, q0, q1):
        self._check(self.lib.gw_set_q_range(self.ctx, int(q0), int(q1)))

    def save_state(self, path):
        """Checkpoint G(tau), Sigma_inf, Sigma(i w) and mu to a host file."""
        self._check(self.lib.gw_save_state(self.ctx, os.fsencode(path)))

    def load_state(self, path):
        """Resume from a checkpoint written by save_state (same sizes and beta)."""
        self._check(self.lib.gw_load_state(self.ctx, os.fsencode(path)))

    def dyson(self):
        mu = ctypes.c_double()
        self._check(self.lib.gw_dyson(self.ctx, ctypes.byref(mu)))
        return mu.value

    def grand_potential(self):
        """Phi~ of Eq. tilde_Phi_GW from the current P~0(tau), summed over the context's q range."""
        phi = ctypes.c_double()
        self._check(self.lib.gw_grand_potential(self.ctx, ctypes.byref(phi)))
        return phi.value

    def reset_sigma(self):
        self._check(self.lib.gw_reset_sigma(self.ctx))

    def iterate(self, n=1):
        s = GwIterStats()
        self._check(self.lib.gw_iterate(self.ctx, int(n), ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in GwIterStats._fields_}

    # -- adjoints (device tensors, complex128, contiguous)
    def polarization_vjp(self, Pbar, c64=False):
        """Gbar = VJP of the symmetrised P~0(tau) w.r.t. G(tau) at the current G
        (complex128 arithmetic, or complex64 with c64=True; complex128 storage)."""
        torch = self.torch
        Pbar = Pbar.contiguous()
        Gbar = torch.empty(self.shape_of("G_tau"), dtype=torch.complex128, device=Pbar.device)
        fn = self.lib.gw_polarization_vjp_c64 if c64 else self.lib.gw_polarization_vjp
        self._check(fn(self.ctx, Pbar.data_ptr(), Gbar.data_ptr()))
        return Gbar

    def selfenergy_vjp(self, Sbar, c64=False):
        """(Gbar, Pbar) = VJP of the symmetrised Sigma~(tau) w.r.t. (G(tau), P~(tau))."""
        torch = self.torch
        Sbar = Sbar.contiguous()
        Gbar = torch.empty(self.shape_of("G_tau"), dtype=torch.complex128, device=Sbar.device)
        Pbar = torch.empty(self.shape_of("P_tau"), dtype=torch.complex128, device=Sbar.device)
        fn = self.lib.gw_selfenergy_vjp_c64 if c64 else self.lib.gw_selfenergy_vjp
        self._check(fn(self.ctx, Sbar.data_ptr(), Gbar.data_ptr(), Pbar.data_ptr()))
        return Gbar, Pbar

    def polarization_jvp(self, dG):
        """dP~0(tau) = tangent of the symmetrised P~0(tau) along dG (device complex128)."""
        torch = self.torch
        dG = dG.contiguous()
        dP = torch.empty(self.shape_of("P0_tau"), dtype=torch.complex128, device=dG.device)
        self._check(self.lib.gw_polarization_jvp(self.ctx, dG.data_ptr(), dP.data_ptr()))
        return dP

    def screened_jvp(self, dP0):
        """dP~(tau) = tangent of the screened block (transform, solve, transform back) along dP~0(tau)."""
        torch = self.torch
        dP0 = dP0.contiguous()
        dP = torch.empty(self.shape_of("P_tau"), dtype=torch.complex128, device=dP0.device)
        self._check(self.lib.gw_screened_jvp(self.ctx, dP0.data_ptr(), dP.data_ptr()))
        return dP

    def selfenergy_jvp(self, dG, dP):
        """dSigma~(tau) = tangent of the symmetrised Sigma~(tau) along (dG, dP~(tau))."""
        torch = self.torch
        dG, dP = dG.contiguous(), dP.contiguous()
        dS = torch.empty(self.shape_of("Sigma_tau"), dtype=torch.complex128, device=dG.device)
        self._check(self.lib.gw_selfenergy_jvp(self.ctx, dG.data_ptr(), dP.data_ptr(), dS.data_ptr()))
        return dS

    def sc_jvp(self, dSinf, dSiw):
        """Tangent of the self-consistency map (Sigma_inf, Sigma(i w)) -> (Sigma_inf', Sigma'(i w))."""
        torch = self.torch
        dSinf, dSiw = dSinf.contiguous(), dSiw.contiguous()
        oi = torch.empty(self.shape_of("Sigma_inf"), dtype=torch.complex128, device=dSiw.device)
        ow = torch.empty(self.shape_of("Sigma_iw"), dtype=torch.complex128, device=dSiw.device)
        self._check(self.lib.gw_sc_jvp(self.ctx, dSinf.data_ptr(), dSiw.data_ptr(), oi.data_ptr(), ow.data_ptr()))
        return oi, ow

    def iterate_newton(self, n_outer, m=8, tol=1e-10):
        """Newton-Krylov self-consistency; returns the residual norm of each step."""
        res = (ctypes.c_double * max(1, int(n_outer)))()
        self._check(self.lib.gw_iterate_newton(self.ctx, int(n_outer), int(m), float(tol), res))
        return [float(x) for x in res][:int(n_outer)]

    def iterate_diis(self, n, m=6, mix=0.5, tol=0.0):
        """DIIS self-consistency (see gw_iterate_diis); returns ||F(x) - x||_2 of each step."""
        res = (ctypes.c_double * max(1, int(n)))()
        self._check(self.lib.gw_iterate_diis(self.ctx, int(n), int(m), float(mix), float(tol), res))
        return [float(x) for x in res][:int(n)]

    def profile(self, enable=True):
        self._check(self.lib.gw_profile(self.ctx, int(bool(enable))))

    def profile_read(self):
        """{'simt': (ms, flops, launches), 'tensor': (ms, flops, launches)} since the last read."""
        out = (ctypes.c_double * 6)()
        self._check(self.lib.gw_profile_read(self.ctx, out))
        return {"simt": (float(out[0]), float(out[1]), int(out[2])),
                "tensor": (float(out[3]), float(out[4]), int(out[5]))}

    def iterate_graph(self, n=1):
        """n iterations replayed from a captured CUDA graph (see gw_iterate_graph)."""
        s = GwIterStats()
        self._check(self.lib.gw_iterate_graph(self.ctx, int(n), ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in GwIterStats._fields_}

    def kernel_launches(self):
        return int(self.lib.gw_kernel_launches(self.ctx))
