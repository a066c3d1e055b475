"""Thin ctypes binding of libchi0 (include/chi0.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are numpy arrays; device arrays are torch CUDA tensors
(passed by data_ptr, kept alive by the caller).  Importing this module loads
the library and raises if it has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchi0.so")

CHI0_FP64 = 0
CHI0_MIXED_BF16X3 = 1

STATUS = {
    0: "CHI0_OK", -1: "CHI0_EINVAL", -2: "CHI0_ENOMEM", -3: "CHI0_ECUDA", -4: "CHI0_ESTATE",
    -5: "CHI0_ENOTPD", -6: "CHI0_ESINGULAR", -7: "CHI0_ETIMEOUT", -8: "CHI0_EUNSUPPORTED",
}

EXPORTS = (
    "chi0_create", "chi0_set_wavefunctions", "chi0_set_energies", "chi0_compute_rho",
    "chi0_build_chi0", "chi0_invert_eps", "chi0_build_invert", "chi0_get_response_gvectors", "chi0_get_transitions",
    "chi0_get_rho", "chi0_get_rho_rows", "chi0_synchronize", "chi0_get_stats", "chi0_last_error", "chi0_destroy",
    "chi0_invert_eps_noalloc", "chi0_mlp_nparams", "chi0_mlp_workspace_floats", "chi0_mlp_loss_grad",
    "chi0_mlp_adam", "chi0_mlp_predict", "chi0_term_features", "chi0_set_terminator", "chi0_set_bg_terminator",
    "chi0_batch_create", "chi0_batch_run", "chi0_batch_rho_width", "chi0_batch_destroy",
    "chi0_batch_synchronize", "chi0_batch_info",
    "chi0_ppa_fit", "chi0_ppa_eval", "chi0_build_sigma_i", "chi0_set_pole_grouping", "chi0_set_double_grid",
    "chi0_check_bounded_wait", "chi0_set_band_blocks", "chi0_get_pole_groups",
)


class Chi0Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Chi0Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_double * 9),
        ("kgrid", ctypes.c_int * 3),
        ("nbands", ctypes.c_int),
        ("npw_max", ctypes.c_int),
        ("fft", ctypes.c_int * 3),
        ("ng", ctypes.c_int),
        ("nq", ctypes.c_int),
        ("q_frac", ctypes.POINTER(ctypes.c_double)),
        ("nw", ctypes.c_int),
        ("omega", ctypes.POINTER(ctypes.c_double)),
        ("eta", ctypes.c_double),
        ("spin_factor", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("time_reversal", ctypes.c_int),
        ("occ_drop_tol", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
    ]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libchi0.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.chi0_create.argtypes = [ctypes.POINTER(Chi0Config), ctypes.POINTER(P)]
    lib.chi0_set_wavefunctions.argtypes = [P, I, I, P, P, I, I]
    lib.chi0_set_energies.argtypes = [P, P, P]
    lib.chi0_compute_rho.argtypes = [P, I]
    lib.chi0_build_chi0.argtypes = [P, I, P, I]
    lib.chi0_invert_eps.argtypes = [P, I, P, I]
    lib.chi0_build_invert.argtypes = [P, I, P, P, I]
    lib.chi0_get_response_gvectors.argtypes = [P, I, P]
    lib.chi0_get_transitions.argtypes = [P, ctypes.POINTER(I64), P]
    lib.chi0_get_rho.argtypes = [P, P]
    lib.chi0_get_rho_rows.argtypes = [P, P, I64, P]
    lib.chi0_synchronize.argtypes = [P]
    lib.chi0_get_stats.argtypes = [P, P, P, P, ctypes.POINTER(I64)]
    lib.chi0_last_error.argtypes = [P]
    lib.chi0_last_error.restype = ctypes.c_char_p
    lib.chi0_destroy.argtypes = [P]
    lib.chi0_destroy.restype = None
    lib.chi0_invert_eps_noalloc.argtypes = [P, P, I, I, P, P]
    F = ctypes.c_float
    lib.chi0_mlp_nparams.argtypes = []
    lib.chi0_mlp_workspace_floats.argtypes = [I64]
    lib.chi0_mlp_loss_grad.argtypes = [P, P, P, I64, I, P, P, P, P]
    lib.chi0_mlp_adam.argtypes = [P, P, P, P, I64, F, F, F, F, I, P]
    lib.chi0_mlp_predict.argtypes = [P, P, I64, I, P, P]
    lib.chi0_term_features.argtypes = [P, I, P, P, P, P, P]
    lib.chi0_set_terminator.argtypes = [P, P, I]
    lib.chi0_set_bg_terminator.argtypes = [P, I, D]
    lib.chi0_batch_create.argtypes = [P, P, P, P, I, I, ctypes.POINTER(P)]
    lib.chi0_batch_synchronize.argtypes = [P]
    lib.chi0_batch_info.argtypes = [P, P, P]
    lib.chi0_batch_run.argtypes = [P, P]
    lib.chi0_batch_rho_width.argtypes = [P]
    lib.chi0_batch_destroy.argtypes = [P]
    lib.chi0_ppa_fit.argtypes = [P, P, I, D, P, P, P]
    lib.chi0_build_sigma_i.argtypes = [P, I, I, I, P, I, P, I]
    lib.chi0_set_pole_grouping.argtypes = [P, D]
    lib.chi0_set_double_grid.argtypes = [P, I, P]
    lib.chi0_check_bounded_wait.argtypes = [P]
    lib.chi0_set_band_blocks.argtypes = [P, I, I]
    lib.chi0_get_pole_groups.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I)]
    lib.chi0_ppa_eval.argtypes = [P, P, I, P, I, D, P, P]
    for name in EXPORTS:
        if name not in ("chi0_last_error", "chi0_destroy", "chi0_batch_destroy"):
            getattr(lib, name).restype = I
    lib.chi0_mlp_workspace_floats.restype = I64
    lib.chi0_batch_destroy.restype = None
    del D
    return lib


_lib = load_library()


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(a)}")


def invert_eps_noalloc(chi0, v_sqrt, out, stream=None):
    """chi0_invert_eps_noalloc: eps~^-1 without device allocation.
    chi0, out: contiguous complex128 CUDA tensors [nw][ng][ng]; v_sqrt: host
    float64 [ng].  Raises ValueError on mismatched arguments and Chi0Error on
    a non-zero status."""
    import torch
    for name, t in (("chi0", chi0), ("out", out)):
        if getattr(t, "dtype", None) != torch.complex128:
            raise ValueError(f"{name} must be a complex128 tensor")
        if t.dim() != 3 or t.shape[1] != t.shape[2] or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous [nw][ng][ng] tensor")
    if tuple(out.shape) != tuple(chi0.shape):
        raise ValueError("out must have the shape of chi0")
    v = np.ascontiguousarray(v_sqrt, dtype=np.float64).reshape(-1)
    nw, ng = int(chi0.shape[0]), int(chi0.shape[1])
    if v.size != ng:
        raise ValueError(f"v_sqrt has {v.size} entries, expected ng = {ng}")
    cp, cdev = _ptr(chi0)
    op, odev = _ptr(out)
    if not (cdev and odev):
        raise ValueError("chi0 and out must be device tensors")
    st = _lib.chi0_invert_eps_noalloc(cp, v.ctypes.data, ng, nw, op, stream)
    if st != 0:
        raise Chi0Error(st, "chi0_invert_eps_noalloc failed")
    return out


def ppa_fit(eps_inv_0, eps_inv_p, omega_p, omega_t, R, stream=None):
    """chi0_ppa_fit: plasmon-pole parameters (omega_t, R) of every element from
    eps^-1 at w = 0 and w = i omega_p.  All four are contiguous complex128
    CUDA tensors [ng][ng]."""
    ng = int(eps_inv_0.shape[-1])
    st = _lib.chi0_ppa_fit(_dev(eps_inv_0), _dev(eps_inv_p), ng, float(omega_p), _dev(omega_t), _dev(R), stream)
    if st != 0:
        raise Chi0Error(st, "chi0_ppa_fit failed")


def ppa_eval(omega_t, R, freqs, eta, out, stream=None):
    """chi0_ppa_eval: eps^-1 of the plasmon-pole model at the complex
    frequencies freqs (host) into out, a complex128 CUDA tensor [nf][ng][ng]."""
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.complex128).reshape(-1))
    fr = np.ascontiguousarray(np.stack([f.real, f.imag], axis=1).reshape(-1))
    ng = int(omega_t.shape[-1])
    st = _lib.chi0_ppa_eval(_dev(omega_t), _dev(R), ng, fr.ctypes.data if f.size else None, int(f.size),
                            float(eta), _dev(out), stream)
    if st != 0:
        raise Chi0Error(st, "chi0_ppa_eval failed")


class Batch:
    """chi0_batch: many (context, q index) problems run as one captured graph.
    A context may appear with several q indices (they share its mixed grids).
    eps_out / chi_out: per problem a complex128 CUDA tensor [nw][ng][ng] or
    None; each problem needs at least one of them."""

    def __init__(self, ctxs, iqs, eps_out=None, nstreams=4, chi_out=None):
        n = len(ctxs)
        self._ctxs = list(ctxs)          # keep the contexts alive
        self._outs = list(eps_out) if eps_out is not None else None
        self._chis = list(chi_out) if chi_out is not None else None
        self.n = n
        hs = (ctypes.c_void_p * n)(*[c.h.value for c in ctxs])
        qs = (ctypes.c_int * n)(*[int(q) for q in iqs])
        outs = chis = None
        if eps_out is not None:
            outs = (ctypes.c_void_p * n)(*[(_dev(o) if o is not None else None) for o in eps_out])
        if chi_out is not None:
            chis = (ctypes.c_void_p * n)(*[(_dev(o) if o is not None else None) for o in chi_out])
        h = ctypes.c_void_p()
        st = _lib.chi0_batch_create(hs, qs, chis, outs, n, int(nstreams), ctypes.byref(h))
        if st != 0:
            raise Chi0Error(st, "chi0_batch_create failed: " +
                            "; ".join(_lib.chi0_last_error(c.h).decode(errors="replace") for c in ctxs[:1]))
        self.h = h

    def synchronize(self):
        st = _lib.chi0_batch_synchronize(self.h)
        if st != 0:
            raise Chi0Error(st, "chi0_batch_synchronize reported a device error")

    def info(self):
        """(helper stream of each problem, summed tuned contraction ms)."""
        so = (ctypes.c_int * self.n)()
        ms = ctypes.c_double()
        st = _lib.chi0_batch_info(self.h, so, ctypes.byref(ms))
        if st != 0:
            raise Chi0Error(st, "chi0_batch_info failed")
        return list(so), ms.value

    def run(self, stream=None):
        st = _lib.chi0_batch_run(self.h, stream)
        if st != 0:
            raise Chi0Error(st, "chi0_batch_run failed")

    def rho_width(self):
        return int(_lib.chi0_batch_rho_width(self.h))

    def close(self):
        if getattr(self, "h", None):
            _lib.chi0_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned terminator network (device tensors: float32, contiguous)

def mlp_nparams():
    return int(_lib.chi0_mlp_nparams())


def mlp_workspace_floats(batch):
    return int(_lib.chi0_mlp_workspace_floats(int(batch)))


def _dev(t):
    p, dev = _ptr(t)
    if not dev:
        raise ValueError("device tensor expected")
    return p


def mlp_loss_grad(params, x, t, grad, loss, work, bf16=True, stream=None):
    st = _lib.chi0_mlp_loss_grad(_dev(params), _dev(x), _dev(t), int(x.shape[0]), int(bool(bf16)),
                                 _dev(grad), _dev(loss) if loss is not None else None, _dev(work), stream)
    if st != 0:
        raise Chi0Error(st, "chi0_mlp_loss_grad failed")


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    st = _lib.chi0_mlp_adam(_dev(params), _dev(grad), _dev(m), _dev(v), int(params.numel()), float(lr),
                            float(beta1), float(beta2), float(eps), int(step), stream)
    if st != 0:
        raise Chi0Error(st, "chi0_mlp_adam failed")


def mlp_predict(params, x, y, bf16=True, stream=None):
    st = _lib.chi0_mlp_predict(_dev(params), _dev(x), int(x.shape[0]), int(bool(bf16)), _dev(y), stream)
    if st != 0:
        raise Chi0Error(st, "chi0_mlp_predict failed")


class Chi0:
    """One chi0_ctx.  Method names follow the C entry points."""

    def __init__(self, *, a, kgrid, nbands, npw_max, fft, ng, q_frac, omega, eta,
                 spin_factor=2.0, precision=CHI0_FP64, time_reversal=1, occ_drop_tol=0.0,
                 stream=None):
        cfg = Chi0Config()
        lat = np.eye(3) * float(a)
        cfg.lattice[:] = lat.ravel().tolist()
        cfg.kgrid[:] = [int(v) for v in kgrid]
        cfg.nbands = int(nbands)
        cfg.npw_max = int(npw_max)
        cfg.fft[:] = [int(v) for v in fft]
        cfg.ng = int(ng)
        self._q = np.ascontiguousarray(np.asarray(q_frac, dtype=np.float64).reshape(-1, 3))
        om = np.asarray(omega, dtype=np.complex128).reshape(-1)
        self._om = np.ascontiguousarray(np.stack([om.real, om.imag], axis=1))
        cfg.nq = self._q.shape[0]
        cfg.q_frac = self._q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.nw = self._om.shape[0]
        cfg.omega = self._om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.eta = float(eta)
        cfg.spin_factor = float(spin_factor)
        cfg.precision = int(precision)
        cfg.time_reversal = int(time_reversal)
        cfg.occ_drop_tol = float(occ_drop_tol)
        cfg.cuda_stream = stream
        self.cfg = cfg
        self.nk = int(np.prod(kgrid))
        self.nb = int(nbands)
        self.ng = int(ng)
        self.nw = cfg.nw
        self.precision = int(precision)
        h = ctypes.c_void_p()
        st = _lib.chi0_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise Chi0Error(st, "chi0_create rejected the configuration")
        self.h = h

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise Chi0Error(st, _lib.chi0_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            _lib.chi0_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points
    def set_wavefunctions(self, ik, gvec, coef):
        """gvec [npw][3] int32, coef [nbands][npw] complex64/complex128 (numpy or torch)."""
        gp, gdev = _ptr(gvec)
        cp, cdev = _ptr(coef)
        if gdev != cdev:
            raise ValueError("gvec and coef must both be host or both be device buffers")
        if isinstance(coef, np.ndarray):
            c64 = coef.dtype == np.complex64
            npw = coef.shape[1]
        else:
            import torch
            c64 = coef.dtype == torch.complex64
            npw = coef.shape[1]
        self._check(_lib.chi0_set_wavefunctions(self.h, int(ik), int(npw), gp, cp, int(c64), cdev))

    def set_energies(self, eps, occ):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        self._check(_lib.chi0_set_energies(self.h, eps.ctypes.data, occ.ctypes.data))

    def compute_rho(self, iq):
        self._check(_lib.chi0_compute_rho(self.h, int(iq)))

    def build_chi0(self, iq, out=None):
        """out: None (keep on device), numpy complex128 [nw][ng][ng] or a torch tensor."""
        if out is None:
            self._check(_lib.chi0_build_chi0(self.h, int(iq), None, 1))
            return None
        p, dev = _ptr(out)
        self._check(_lib.chi0_build_chi0(self.h, int(iq), p, dev))
        return out

    def invert_eps(self, iq, out):
        p, dev = _ptr(out)
        self._check(_lib.chi0_invert_eps(self.h, int(iq), p, dev))
        return out

    def set_band_blocks(self, bands_per_block, k_per_block=0):
        """chi0_set_band_blocks: stream the transitions in blocks of k_per_block
        k points (0: all) x bands_per_block bands n; 0 bands = off."""
        self._check(_lib.chi0_set_band_blocks(self.h, int(bands_per_block), int(k_per_block)))

    def pole_groups(self):
        """chi0_get_pole_groups: (number of pole groups, grouped contraction used)."""
        n = ctypes.c_int64()
        g = ctypes.c_int()
        self._check(_lib.chi0_get_pole_groups(self.h, ctypes.byref(n), ctypes.byref(g)))
        return n.value, bool(g.value)

    def set_pole_grouping(self, eps_thresh):
        """chi0_set_pole_grouping: poles within eps_thresh (Ha) share one frequency factor; 0 = off."""
        self._check(_lib.chi0_set_pole_grouping(self.h, float(eps_thresh)))

    def set_double_grid(self, eps_dense):
        """chi0_set_double_grid: eps_dense [nk][nd][nbands] (Ha), or None to switch it off."""
        if eps_dense is None:
            self._check(_lib.chi0_set_double_grid(self.h, 0, None))
            return
        e = np.ascontiguousarray(eps_dense, dtype=np.float64)
        self._check(_lib.chi0_set_double_grid(self.h, int(e.shape[1]), e.ctypes.data))

    def build_sigma_i(self, iq, qp_lo, qp_hi, eps_inv, out):
        """chi0_build_sigma_i: the self-energy kernel I of Eq. (I_c) from eps~^-1
        (a contiguous complex128 CUDA tensor [nw][ng][ng]) into out, numpy or a
        tensor of shape [nw][nk][nbands][nqp][nqp] complex128."""
        p, dev = _ptr(out)
        self._check(_lib.chi0_build_sigma_i(self.h, int(iq), int(qp_lo), int(qp_hi), _dev(eps_inv),
                                            int(eps_inv.shape[0]), p, dev))
        return out

    def build_invert(self, iq, eps_out, chi_out=None):
        """chi0_build_invert: chi0 and eps~^-1 in one pipelined call.  eps_out
        (and chi_out, if given) are both numpy arrays or both device tensors."""
        p, dev = _ptr(eps_out)
        cp = None
        if chi_out is not None:
            cp, cdev = _ptr(chi_out)
            if cdev != dev:
                raise ValueError("chi_out and eps_out must both be host or both be device buffers")
        self._check(_lib.chi0_build_invert(self.h, int(iq), cp, p, dev))
        return eps_out

    def get_response_gvectors(self, iq):
        out = np.zeros((self.ng, 3), dtype=np.int32)
        self._check(_lib.chi0_get_response_gvectors(self.h, int(iq), out.ctypes.data))
        return out

    def get_transitions(self):
        nt = ctypes.c_int64()
        self._check(_lib.chi0_get_transitions(self.h, ctypes.byref(nt), None))
        out = np.zeros((nt.value, 3), dtype=np.int32)
        self._check(_lib.chi0_get_transitions(self.h, ctypes.byref(nt), out.ctypes.data))
        return out

    def get_rho(self):
        nt = ctypes.c_int64()
        self._check(_lib.chi0_get_transitions(self.h, ctypes.byref(nt), None))
        out = np.zeros((nt.value, self.ng), dtype=np.complex128)
        self._check(_lib.chi0_get_rho(self.h, out.ctypes.data))
        return out

    def get_rho_rows(self, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.size, self.ng), dtype=np.complex128)
        self._check(_lib.chi0_get_rho_rows(self.h, rows.ctypes.data, rows.size, out.ctypes.data))
        return out

    def synchronize(self):
        self._check(_lib.chi0_synchronize(self.h))

    def check_bounded_wait(self):
        """chi0_check_bounded_wait: queue a bounded wait that must give up; the
        next synchronize raises Chi0Error with CHI0_ETIMEOUT."""
        self._check(_lib.chi0_check_bounded_wait(self.h))

    def term_features(self, iq, chi_trunc, x, chi_full=None, t=None):
        """Features (and targets) of a truncated chi0 held on the device; returns the scale c."""
        sc = ctypes.c_double()
        self._check(_lib.chi0_term_features(self.h, int(iq), _dev(chi_trunc),
                                            _dev(chi_full) if chi_full is not None else None, _dev(x),
                                            _dev(t) if t is not None else None, ctypes.byref(sc)))
        return sc.value

    def set_bg_terminator(self, eps_bar, on=True):
        """chi0_set_bg_terminator: the Bruneval-Gonze extrapolar correction with
        extrapolar energy eps_bar (Ha); call compute_rho afterwards."""
        self._check(_lib.chi0_set_bg_terminator(self.h, 1 if on else 0, float(eps_bar)))

    def set_terminator(self, params, bf16=True):
        self._check(_lib.chi0_set_terminator(self.h, _dev(params) if params is not None else None,
                                             int(bool(bf16))))

    STAGES = ("wf_grid", "rho", "weights", "contract", "reduce", "dyson")

    def get_stats(self):
        """(ms, bytes, flops) per stage (dicts keyed by STAGES) and the kernel count."""
        ms = np.zeros(6)
        by = np.zeros(6)
        fl = np.zeros(6)
        nl = ctypes.c_int64()
        self._check(_lib.chi0_get_stats(self.h, ms.ctypes.data, by.ctypes.data, fl.ctypes.data,
                                        ctypes.byref(nl)))
        mk = lambda a: dict(zip(self.STAGES, a.tolist()))  # noqa: E731
        return mk(ms), mk(by), mk(fl), nl.value

    # -- convenience: marshal a synthetic system's arrays
    @classmethod
    def for_system(cls, system, precision=CHI0_FP64, stream=None, occ_drop_tol=0.0, **over):
        kw = dict(a=system.spec.a, kgrid=system.spec.kgrid, nbands=system.nb,
                  npw_max=system.npw_max, fft=system.fft, ng=system.ng, q_frac=system.q_frac,
                  omega=system.freqs, eta=system.eta, spin_factor=system.spin_factor,
                  precision=precision, occ_drop_tol=occ_drop_tol, stream=stream)
        kw.update(over)
        return cls(**kw)

    def load_system(self, system):
        for ik in range(system.nk):
            n = int(system.npw[ik])
            self.set_wavefunctions(ik, np.ascontiguousarray(system.gvec[ik, :n]),
                                   np.ascontiguousarray(system.coef[ik, :, :n]))
        self.set_energies(system.eps, system.occ)
