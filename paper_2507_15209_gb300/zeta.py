"""Thin Python binding of libzeta (argument marshalling only).

Every call forwards to the C ABI declared in include/zeta.h with the same name;
PyTorch supplies device memory (torch.empty on CUDA) and the current stream.
All arithmetic of the method runs in the library's CUDA kernels.  If the
library has not been built the import fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libzeta.so")

SUM_NODE, SUM_GAMMA, SUM_PARTICLE = 1, 2, 4
GRAM = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x3": 3, "bf16_fields": 4}
FORM_BITS = {"node": SUM_NODE, "gamma": SUM_GAMMA, "particle": SUM_PARTICLE, "backward": 8, "ss": 16}
_ERR = {0: "ok", -1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "ETIMEOUT", -5: "ENOTSUP", -6: "EWORKSPACE",
        -7: "EDATA"}


class ZetaError(RuntimeError):
    def __init__(self, name: str, code: int):
        super().__init__(f"{name} failed: {_ERR.get(code, code)} ({code})")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("box", ctypes.c_double), ("dsup", ctypes.c_int), ("lmax", ctypes.c_int),
                ("nbins", ctypes.c_int), ("edges", ctypes.POINTER(ctypes.c_double)), ("gram", ctypes.c_int),
                ("radial", ctypes.c_int), ("radii", ctypes.POINTER(ctypes.c_double)), ("tophat", ctypes.c_double),
                ("tophat_primary", ctypes.c_double), ("phi_hat", ctypes.c_int)]


RADIAL = {"shell": 0, "point": 1}


def make_params(n, box, dsup, lmax, edges=None, gram="fp32", radial="shell", radii=None, tophat=0.0,
                tophat_primary=0.0, phi_hat=False):
    """zeta_params from Python values; returns (struct, arrays that must outlive it)."""
    keep = []

    def arr(x):
        if x is None:
            return None
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    nbins = len(radii) if radial == "point" else len(edges) - 1
    p = _Params(int(n), float(box), int(dsup), int(lmax), int(nbins), arr(edges), GRAM[gram], RADIAL[radial],
                arr(radii), float(tophat), float(tophat_primary), 1 if phi_hat else 0)
    return p, keep


_lib = None

_VP, _I64, _INT, _DBL, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "zeta_version": ([], _INT),
    "zeta_strerror": ([_INT], ctypes.c_char_p),
    "zeta_create": ([ctypes.POINTER(_Params), ctypes.POINTER(_VP)], _INT),
    "zeta_destroy": ([_VP], _INT),
    "zeta_workspace_bytes": ([_VP, _I64, _INT], _SZ),
    "zeta_set_workspace": ([_VP, _VP, _SZ], _INT),
    "zeta_tile_count": ([_VP], _I64),
    "zeta_set_gram": ([_VP, _INT], _INT),
    "zeta_assign": ([_VP, _VP, _I64, _VP, _VP, _VP], _INT),
    "zeta_fft_r2c": ([_VP, _VP, _VP, _VP], _INT),
    "zeta_reconstruct_alm": ([_VP, _VP, _INT, _INT, _INT, _INT, _VP, _VP], _INT),
    "zeta_sum_grid": ([_VP, _VP, _VP, _INT, _VP, _VP], _INT),
    "zeta_sort_particles": ([_VP, _VP, _I64, _VP, _VP, _VP], _INT),
    "zeta_sum_particles": ([_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP], _INT),
    "zeta_mass_term": ([_VP, _VP, _INT, _DBL, _VP, _VP], _INT),
    "zeta_zeta_ell": ([_VP, _VP, _I64, _VP, _INT, _VP, _VP], _INT),
    "zeta_zeta_lm": ([_VP, _VP, _I64, _VP, _INT, _INT, _INT, _VP, _VP], _INT),
    "zeta_reduce_lm": ([_VP, _VP, _INT, _VP, _VP], _INT),
    "zeta_lm_slots": ([_VP, _INT], _SZ),
    "zeta_get_status": ([_VP, _VP], _INT),
    "zeta_selftest_wait": ([_VP, _I64, _VP], _INT),
    "zeta_batch": ([_VP, _VP, _VP, _INT, _INT, _VP, _VP], _INT),
    "zeta_backward_node": ([_VP, _VP, _VP, _VP, _VP], _INT),
    "zeta_backward_particles": ([_VP, _VP, _I64, _VP, _VP, _VP], _INT),
    "zeta_autotune": ([_VP, _VP, _I64, _INT, _VP], _INT),
    "zeta_get_tuning": ([_VP, _VP, _INT], _INT),
    "zeta_set_staging": ([_VP, _INT], _INT),
    "zeta_set_tuning": ([_VP, _VP, _INT], _INT),
    "zeta_get_staging": ([_VP], _INT),
    "zeta_assign_noalloc": ([_INT, _DBL, _INT, _VP, _I64, _VP, _VP, _VP], _INT),
    "zeta_profile_enable": ([_VP, _INT], _INT),
    "zeta_profile_read": ([_VP, _VP, _VP, _VP, _INT], _INT),
    "zeta_profile_stage_name": ([_INT], ctypes.c_char_p),
    "zeta_host_jbar": ([_INT, _DBL, _DBL, _DBL, _VP, _I64, _VP], _INT),
    "zeta_host_ylm": ([_INT, _INT, _DBL, _DBL, _DBL], _DBL),
    "zeta_host_jbar_table": ([_INT, _DBL, _INT, _INT, _VP, _VP], _INT),
    "zeta_host_mass_hat": ([_INT, _INT, _VP], _INT),
    "zeta_host_cell_quadrature": ([_INT, _INT, _VP, _VP, _VP], _INT),
    "zeta_host_window_table": ([ctypes.POINTER(_Params), _VP], _INT),
    "zeta_xi": ([_VP, _VP, _I64, _VP, _INT, _VP, _VP], _INT),
    "zeta_zeta_ell_ss": ([_VP, _VP, _I64, _VP, _I64, _INT, _VP, _VP, _VP], _INT),
    "zeta_xi_radii": ([_VP, _VP, _INT, _VP, _VP, _VP], _INT),
    "zeta_host_legendre_sum": ([_INT, _INT, _VP, _INT, _VP, _VP], _INT),
    "zeta_host_reduced_q": ([_INT, _VP, _VP, _VP, _VP, _VP], _INT),
    "zeta_host_phi_hat": ([_INT, _INT, _VP], _INT),
    "zeta_host_daub4_dyadic": ([_INT, _VP], _INT),
    "zeta_set_shapes": ([_VP, _VP, _INT], _INT),
    "zeta_get_shapes": ([_VP, _VP, _INT], _INT),
    "zeta_host_daub4_gamma": ([_VP, _VP, _VP], _INT),
}


def lib():
    """Load libzeta.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libzeta.so not built at {LIB_PATH}; run paper_2507_15209_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(name, rc):
    if rc != 0:
        raise ZetaError(name, rc)


def host_jbar(l: int, box: float, r_lo: float, r_hi: float, n2) -> np.ndarray:
    n2 = np.ascontiguousarray(n2, dtype=np.int64)
    out = np.empty(n2.shape, np.float64)
    _check("zeta_host_jbar", lib().zeta_host_jbar(l, box, r_lo, r_hi, n2.ctypes.data, n2.size, out.ctypes.data))
    return out


def host_ylm(l: int, m: int, vx: float, vy: float, vz: float) -> float:
    return lib().zeta_host_ylm(l, m, vx, vy, vz)


def host_jbar_table(n: int, box: float, lmax: int, edges) -> np.ndarray:
    """The context's window table, float32 (lmax + 1, 3 (n/2 - 1)^2 + 1, 4 ceil(nb / 4))."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(e) - 1
    nbp = 4 * ((nb + 3) // 4)
    h = n // 2 - 1
    out = np.empty((lmax + 1, 3 * h * h + 1, nbp), np.float32)
    _check("zeta_host_jbar_table", lib().zeta_host_jbar_table(n, float(box), lmax, nb, e.ctypes.data,
                                                              out.ctypes.data))
    return out


def host_mass_hat(n: int, dsup: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _check("zeta_host_mass_hat", lib().zeta_host_mass_hat(n, dsup, out.ctypes.data))
    return out


def host_daub4_dyadic(level: int) -> np.ndarray:
    """zeta_host_daub4_dyadic: the Daubechies function at k / 2^level, k = 0 .. 3 * 2^level."""
    out = np.empty(3 * 2 ** int(level) + 1, np.float64)
    _check("zeta_host_daub4_dyadic", lib().zeta_host_daub4_dyadic(int(level), out.ctypes.data))
    return out


def host_daub4_gamma():
    """zeta_host_daub4_gamma: (gamma[5, 5] indexed [a + 2, b + 2], lam[5], u[5, 5] indexed [o, k])."""
    g = np.empty((5, 5), np.float64)
    lam = np.empty(5, np.float64)
    u = np.empty((5, 5), np.float64)
    _check("zeta_host_daub4_gamma", lib().zeta_host_daub4_gamma(g.ctypes.data, lam.ctypes.data, u.ctypes.data))
    return g, lam, u


def host_cell_quadrature(q: int, dsup: int):
    """(t, wq, beta[q, dsup]) of zeta_host_cell_quadrature."""
    t = np.empty(q, np.float64)
    wq = np.empty(q, np.float64)
    beta = np.empty((q, dsup), np.float64)
    _check("zeta_host_cell_quadrature", lib().zeta_host_cell_quadrature(q, dsup, t.ctypes.data, wq.ctypes.data,
                                                                        beta.ctypes.data))
    return t, wq, beta


def assign_noalloc(n: int, box: float, dsup: int, particles, delta=None, wsum=None):
    """zeta_assign_noalloc: B-spline assignment with the library's fixed scratch (no allocation
    inside the call; the caller may pass preallocated delta / wsum tensors).  A non-finite
    particle makes every value of delta and wsum NaN."""
    import torch
    if delta is None:
        delta = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    if wsum is None:
        wsum = torch.empty(1, dtype=torch.float64, device="cuda")
    _check("zeta_assign_noalloc", lib().zeta_assign_noalloc(n, float(box), dsup, _f32(particles, "particles", cols=4),
                                                            particles.shape[0], _f32(delta, "delta", n ** 3),
                                                            _f64(wsum, "wsum", 1), _stream()))
    return delta, wsum


def legendre_sum(zeta_l, mu):
    """zeta_host_legendre_sum: zeta(b1, b2, mu) = sum_l zeta_l P_l(mu); numpy in, numpy (nmu, nb, nb) out."""
    z = np.ascontiguousarray(zeta_l, dtype=np.float64)
    m = np.ascontiguousarray(mu, dtype=np.float64)
    nb = z.shape[-1]
    out = np.empty((len(m), nb, nb))
    _check("zeta_host_legendre_sum", lib().zeta_host_legendre_sum(z.shape[0] - 1, nb, z.ctypes.data_as(ctypes.c_void_p),
                                                                  len(m), m.ctypes.data_as(ctypes.c_void_p),
                                                                  out.ctypes.data_as(ctypes.c_void_p)))
    return out


def reduced_q(zeta, xi1, xi2, xi3):
    """zeta_host_reduced_q: Q = zeta / (xi1 xi2 + xi2 xi3 + xi3 xi1), element-wise (numpy)."""
    arrs = [np.ascontiguousarray(np.broadcast_to(a, np.shape(zeta)), dtype=np.float64).ravel()
            for a in (zeta, xi1, xi2, xi3)]
    q = np.empty(arrs[0].size)
    _check("zeta_host_reduced_q", lib().zeta_host_reduced_q(q.size, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                                            q.ctypes.data_as(ctypes.c_void_p)))
    return q.reshape(np.shape(zeta))


def lm_pairs(lm_rank: int, lm_size: int, lmax: int) -> list:
    """The (l, m) pairs rank lm_rank of lm_size runs in zeta_zeta_lm: index l^2 + l + m, round robin."""
    return [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1) if (l * l + l + m) % lm_size == lm_rank]


def lm_slot(l: int, m: int) -> int:
    """Slot of (l, m) in a zeta_zeta_lm slot array (per form); the uniform term of l is at
    (lmax+1)^2 + l."""
    return l * l + l + m


def interleave(a):
    """Plain stack (nb, n, n, n) -> bin-interleaved (ceil(nb/4), n, n, n, 4), zero-padded (numpy or torch)."""
    nb, n = a.shape[0], a.shape[1]
    g = (nb + 3) // 4
    if hasattr(a, "new_zeros"):
        pad = a.new_zeros((4 * g, n, n, n))
        pad[:nb] = a
        return pad.reshape(g, 4, n, n, n).permute(0, 2, 3, 4, 1).contiguous()
    pad = np.zeros((4 * g, n, n, n), a.dtype)
    pad[:nb] = a
    return np.ascontiguousarray(pad.reshape(g, 4, n, n, n).transpose(0, 2, 3, 4, 1))


def deinterleave(a, nb: int):
    """Bin-interleaved (g, n, n, n, 4) -> plain (nb, n, n, n)."""
    g, n = a.shape[0], a.shape[1]
    if hasattr(a, "permute"):
        return a.permute(0, 4, 1, 2, 3).reshape(4 * g, n, n, n)[:nb]
    return a.transpose(0, 4, 1, 2, 3).reshape(4 * g, n, n, n)[:nb]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _arg(t, name: str, dtype, numel: int = 0, cols: int | None = None):
    """Device pointer of a tensor argument after checking it: a torch tensor of `dtype`,
    contiguous, with at least `numel` elements (or of shape (N, cols)), on the current CUDA
    device.  A host tensor or a short buffer would otherwise reach a kernel as a bad address.
    None passes through (optional arguments)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name}: expected shape (N, {cols}), got {tuple(t.shape)}")
    if t.numel() < numel:
        raise ValueError(f"{name}: needs at least {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor, got one on {t.device}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, name, numel=0, cols=None):
    import torch
    return _arg(t, name, torch.float32, numel, cols)


def _f64(t, name, numel=0):
    import torch
    return _arg(t, name, torch.float64, numel)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """A libzeta context with a torch-allocated workspace."""

    def __init__(self, n: int, box: float, dsup: int, lmax: int, edges, gram: str = "fp32", np_max: int = 0,
                 forms=("node",), radial: str = "shell", radii=None, tophat: float = 0.0,
                 tophat_primary: float = 0.0, phi_hat: bool = False, ws_copies: int = 1):
        """dsup: the basis, 2 or 4 (linear or cubic B-spline) or 3 (the genus-4 Daubechies scaling
        function); edges: bin edges (radial "shell"); radial "point" with radii instead (edges may
        be None); tophat / tophat_primary / phi_hat: the vertex windows of zeta_params; ws_copies:
        whole per-catalogue workspaces to allocate (zeta_batch runs that many catalogues at once)."""
        import torch
        self.n, self.box, self.dsup, self.lmax = int(n), float(box), int(dsup), int(lmax)
        self.edges = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
        p, self._keep = make_params(n, box, dsup, lmax, self.edges, gram, radial, radii, tophat, tophat_primary,
                                    phi_hat)
        self.nbins = int(p.nbins)
        h = ctypes.c_void_p()
        _check("zeta_create", lib().zeta_create(ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self.np_max = int(np_max)
        bits = self.form_bits(forms)
        nbytes = lib().zeta_workspace_bytes(self._h, self.np_max, bits)
        if nbytes == 0:
            raise ZetaError("zeta_workspace_bytes", -1)
        nbytes *= max(1, int(ws_copies))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        _check("zeta_set_workspace", lib().zeta_set_workspace(self._h, self.workspace.data_ptr(), nbytes))

    @staticmethod
    def form_bits(forms) -> int:
        if isinstance(forms, int):
            return forms
        return sum(FORM_BITS[f] for f in set(forms))

    def close(self):
        if getattr(self, "_h", None):
            lib().zeta_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- grid helpers ----
    @property
    def ng(self):
        return self.n ** 3

    def _grid(self, dtype=None):
        import torch
        return torch.empty((self.n, self.n, self.n), dtype=dtype or torch.float32, device="cuda")

    def _alm_numel(self) -> int:
        """Floats in the bin-interleaved fields of all bins: ceil(nb / 4) groups of n^3 x 4."""
        return 4 * ((self.nbins + 3) // 4) * self.ng

    # ---- the C-ABI calls ----
    def assign(self, particles):
        import torch
        delta = self._grid()
        wsum = torch.empty(1, dtype=torch.float64, device="cuda")
        _check("zeta_assign", lib().zeta_assign(self._h, _f32(particles, "particles", cols=4), particles.shape[0],
                                                _ptr(delta), _ptr(wsum), _stream()))
        return delta, wsum

    def fft_r2c(self, delta):
        import torch
        dhat = torch.empty((self.n, self.n, self.n // 2, 2), dtype=torch.float32, device="cuda")
        _check("zeta_fft_r2c", lib().zeta_fft_r2c(self._h, _f32(delta, "delta", self.ng), _ptr(dhat), _stream()))
        return dhat

    def reconstruct_alm(self, delta_hat, l: int, m: int, b0: int = 0, b1: int | None = None, out=None):
        import torch
        b1 = self.nbins if b1 is None else b1
        g = max(0, (b1 - b0 + 3) // 4)
        if out is None:
            out = torch.empty((g, self.n, self.n, self.n, 4), dtype=torch.float32, device="cuda")
        _check("zeta_reconstruct_alm", lib().zeta_reconstruct_alm(self._h, _f32(delta_hat, "delta_hat", self.ng), l, m,
                                                                  b0, b1, _f32(out, "out", 4 * g * self.ng),
                                                                  _stream()))
        return out

    def _gram(self, gram):
        import torch
        if gram is None:
            gram = torch.zeros((self.nbins, self.nbins), dtype=torch.float64, device="cuda")
        return gram

    def sum_grid(self, delta, alm, form: str = "node", gram=None):
        gram = self._gram(gram)
        _check("zeta_sum_grid", lib().zeta_sum_grid(self._h, _f32(delta, "delta", self.ng),
                                                    _f32(alm, "alm", self._alm_numel()), FORM_BITS[form],
                                                    _f64(gram, "gram", self.nbins ** 2), _stream()))
        return gram

    def sort_particles(self, particles):
        import torch
        np_ = particles.shape[0]
        sorted_ = torch.empty((np_, 4), dtype=torch.float32, device="cuda")
        ntile = lib().zeta_tile_count(self._h)
        start = torch.empty(ntile + 1, dtype=torch.int64, device="cuda")
        _check("zeta_sort_particles", lib().zeta_sort_particles(self._h, _f32(particles, "particles", cols=4), np_,
                                                                _ptr(sorted_), _ptr(start), _stream()))
        return sorted_, start

    def sum_particles(self, sorted_, tile_start, wsum, alm, gram=None):
        gram = self._gram(gram)
        import torch
        ntile = lib().zeta_tile_count(self._h)
        _check("zeta_sum_particles", lib().zeta_sum_particles(self._h, _f32(sorted_, "sorted", cols=4),
                                                              _arg(tile_start, "tile_start", torch.int64, ntile + 1),
                                                              sorted_.shape[0], _f64(wsum, "wsum", 1),
                                                              _f32(alm, "alm", self._alm_numel()),
                                                              _f64(gram, "gram", self.nbins ** 2),
                                                              _stream()))
        return gram

    def mass_term(self, delta_hat, l: int, sign: float = 1.0, gram=None):
        gram = self._gram(gram)
        _check("zeta_mass_term", lib().zeta_mass_term(self._h, _f32(delta_hat, "delta_hat", self.ng), l, float(sign),
                                                      _f64(gram, "gram", self.nbins ** 2), _stream()))
        return gram

    def zeta_ell(self, particles=None, delta=None, forms=("particle",), out=None):
        """zeta_l(b1, b2) per form: returns {form: tensor (lmax+1, nb, nb) float64}."""
        import torch
        bits = self.form_bits(forms) & 7
        order = [f for f in ("node", "gamma", "particle") if bits & FORM_BITS[f]]
        if out is None:
            out = torch.empty((len(order), self.lmax + 1, self.nbins, self.nbins), dtype=torch.float64,
                              device="cuda")
        np_ = 0 if particles is None else particles.shape[0]
        per = (self.lmax + 1) * self.nbins ** 2
        _check("zeta_zeta_ell", lib().zeta_zeta_ell(self._h, _f32(particles, "particles", cols=4), np_,
                                                    _f32(delta, "delta", self.ng), bits,
                                                    _f64(out, "out", len(order) * per), _stream()))
        return {f: out[i] for i, f in enumerate(order)}

    def zeta_ell_ss(self, data, randoms, forms=("node",)):
        """zeta_zeta_ell_ss: the Szapudi-Szalay numerator and denominator multipoles,
        ({form: (lmax+1, nb, nb)}, {form: (lmax+1, nb, nb)})."""
        import torch
        bits = self.form_bits(forms) & (SUM_NODE | SUM_GAMMA)
        order = [f for f in ("node", "gamma") if bits & FORM_BITS[f]]
        shape = (len(order), self.lmax + 1, self.nbins, self.nbins)
        num = torch.empty(shape, dtype=torch.float64, device="cuda")
        den = torch.empty(shape, dtype=torch.float64, device="cuda")
        k = len(order) * (self.lmax + 1) * self.nbins ** 2
        _check("zeta_zeta_ell_ss", lib().zeta_zeta_ell_ss(self._h, _f32(data, "data", cols=4), data.shape[0],
                                                          _f32(randoms, "randoms", cols=4), randoms.shape[0], bits,
                                                          _f64(num, "num", k), _f64(den, "den", k), _stream()))
        return {f: num[i] for i, f in enumerate(order)}, {f: den[i] for i, f in enumerate(order)}

    def xi(self, particles=None, delta=None, forms=("node",), out=None):
        """zeta_xi: the 2PCF per bin, {form: tensor (nb,) float64} for the node and particle forms."""
        import torch
        bits = self.form_bits(forms) & (SUM_NODE | SUM_PARTICLE)
        order = [f for f in ("node", "particle") if bits & FORM_BITS[f]]
        if out is None:
            out = torch.empty((len(order), self.nbins), dtype=torch.float64, device="cuda")
        np_ = 0 if particles is None else particles.shape[0]
        _check("zeta_xi", lib().zeta_xi(self._h, _f32(particles, "particles", cols=4), np_,
                                        _f32(delta, "delta", self.ng), bits, _f64(out, "out", len(order) * self.nbins),
                                        _stream()))
        return {f: out[i] for i, f in enumerate(order)}

    def xi_radii(self, delta_hat, radii, out=None):
        """zeta_xi_radii: the node-form 2PCF at the given radii (device float64 tensor)."""
        import torch
        r = np.ascontiguousarray(radii, dtype=np.float64)
        if out is None:
            out = torch.empty(len(r), dtype=torch.float64, device="cuda")
        _check("zeta_xi_radii", lib().zeta_xi_radii(self._h, _f32(delta_hat, "delta_hat", self.ng), len(r),
                                                    r.ctypes.data_as(ctypes.c_void_p), _f64(out, "out", len(r)),
                                                    _stream()))
        return out

    def lm_slots(self, forms=("particle",)) -> int:
        """Number of float64 values in a per-(l, m) slot array (zeta_lm_slots)."""
        return int(lib().zeta_lm_slots(self._h, self.form_bits(forms) & 7))

    def zeta_lm(self, lm_rank: int, lm_size: int, particles=None, delta=None, forms=("particle",), out=None):
        """zeta_zeta_lm: this rank's (l, m) contributions, one slot each (see lm_pairs); returns
        the flat float64 slot array."""
        import torch
        bits = self.form_bits(forms) & 7
        k = self.lm_slots(forms)
        if out is None:
            out = torch.empty(k, dtype=torch.float64, device="cuda")
        np_ = 0 if particles is None else particles.shape[0]
        _check("zeta_zeta_lm", lib().zeta_zeta_lm(self._h, _f32(particles, "particles", cols=4), np_,
                                                  _f32(delta, "delta", self.ng), bits, int(lm_rank), int(lm_size),
                                                  _f64(out, "out", k), _stream()))
        return out

    def reduce_lm(self, slots, forms=("particle",), out=None):
        """zeta_reduce_lm: {form: (lmax+1, nb, nb)} from summed slots, bit-identical to zeta_ell."""
        import torch
        bits = self.form_bits(forms) & 7
        order = [f for f in ("node", "gamma", "particle") if bits & FORM_BITS[f]]
        if out is None:
            out = torch.empty((len(order), self.lmax + 1, self.nbins, self.nbins), dtype=torch.float64,
                              device="cuda")
        per = (self.lmax + 1) * self.nbins ** 2
        _check("zeta_reduce_lm", lib().zeta_reduce_lm(self._h, _f64(slots, "slots", self.lm_slots(forms)), bits,
                                                      _f64(out, "out", len(order) * per), _stream()))
        return {f: out[i] for i, f in enumerate(order)}

    def profile_enable(self, on: bool = True):
        _check("zeta_profile_enable", lib().zeta_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{stage: (milliseconds, kernel launches, calls)} since the last profile_enable."""
        ms = np.zeros(32, np.float64)
        nl = np.zeros(32, np.int64)
        nc = np.zeros(32, np.int64)
        k = lib().zeta_profile_read(self._h, ms.ctypes.data, nl.ctypes.data, nc.ctypes.data, 32)
        if k < 0:
            raise ZetaError("zeta_profile_read", k)
        return {lib().zeta_profile_stage_name(i).decode(): (float(ms[i]), int(nl[i]), int(nc[i])) for i in range(k)}

    def set_gram(self, gram: str):
        _check("zeta_set_gram", lib().zeta_set_gram(self._h, GRAM[gram]))

    def set_staging(self, min_particles: int):
        """zeta_set_staging: tile batches with >= min_particles particles stage their halo."""
        _check("zeta_set_staging", lib().zeta_set_staging(self._h, int(min_particles)))

    def staging(self) -> int:
        return int(lib().zeta_get_staging(self._h))

    def _weights(self, w):
        if hasattr(w, "detach"):
            w = w.detach().double().cpu().numpy()
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.lmax + 1, self.nbins, self.nbins)
        return w

    def backward_node(self, delta, weights, grad=None):
        """zeta_backward_node: dL/d delta of L = sum weights * zeta_node."""
        import torch
        w = self._weights(weights)
        if grad is None:
            grad = torch.empty((self.n, self.n, self.n), dtype=torch.float32, device="cuda")
        _check("zeta_backward_node", lib().zeta_backward_node(self._h, _f32(delta, "delta", self.ng), w.ctypes.data,
                                                              _f32(grad, "grad", self.ng), _stream()))
        return grad

    def backward_particles(self, particles, weights, grad=None):
        """zeta_backward_particles: dL/dx_p (np, 3) of L = sum weights * zeta_particle."""
        import torch
        w = self._weights(weights)
        if grad is None:
            grad = torch.empty((particles.shape[0], 3), dtype=torch.float32, device="cuda")
        _check("zeta_backward_particles", lib().zeta_backward_particles(self._h, _f32(particles, "particles", cols=4),
                                                                        particles.shape[0], w.ctypes.data,
                                                                        _f32(grad, "grad", 3 * particles.shape[0]),
                                                                        _stream()))
        return grad

    def batch(self, particles, offsets, forms=("particle",), out=None):
        """zeta_batch: catalogues particles[offsets[i]:offsets[i+1]] in one CUDA-graph launch.

        Returns a tensor (ncat, nforms, lmax+1, nb, nb); keep `offsets` and `out` to reuse the
        captured graph on later calls."""
        import torch
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        ncat = len(offs) - 1
        bits = self.form_bits(forms)
        nforms = bin(bits).count("1")
        if out is None:
            out = torch.empty((ncat, nforms, self.lmax + 1, self.nbins, self.nbins), dtype=torch.float64,
                              device="cuda")
        self._batch_offsets = offs  # the library keeps a copy; hold ours for the caller's reuse
        if particles.shape[0] < int(offs[-1]):
            raise ValueError(f"particles: offsets reach {int(offs[-1])} rows, got {particles.shape[0]}")
        per = (self.lmax + 1) * self.nbins ** 2
        _check("zeta_batch", lib().zeta_batch(self._h, _f32(particles, "particles", cols=4), offs.ctypes.data, ncat,
                                              bits, _f64(out, "out", ncat * nforms * per), _stream()))
        return out

    def autotune(self, particles, forms=("particle",)) -> list:
        _check("zeta_autotune", lib().zeta_autotune(self._h, _f32(particles, "particles", cols=4), particles.shape[0],
                                                    self.form_bits(forms), _stream()))
        return self.tuning()

    def tuning(self) -> list:
        t = np.zeros(5, np.int32)
        lib().zeta_get_tuning(self._h, t.ctypes.data, 5)
        return [int(x) for x in t]

    def set_tuning(self, ctas_per_sm):
        """zeta_set_tuning: persistent grid sizes [node, particle, Gamma, mass, node-tc]."""
        t = np.ascontiguousarray(ctas_per_sm, dtype=np.int32)
        _check("zeta_set_tuning", lib().zeta_set_tuning(self._h, t.ctypes.data, len(t)))

    def shapes(self) -> list:
        """zeta_get_shapes: tile shape of the z-, y- and x-pass (0 default, 1 the narrower tile)."""
        t = np.zeros(3, np.int32)
        lib().zeta_get_shapes(self._h, t.ctypes.data, 3)
        return [int(x) for x in t]

    def set_shapes(self, shape):
        """zeta_set_shapes: tile shapes [z, y, x] of the field-reconstruction passes (0 or 1)."""
        t = np.ascontiguousarray(shape, dtype=np.int32)
        _check("zeta_set_shapes", lib().zeta_set_shapes(self._h, t.ctypes.data, len(t)))

    def selftest_wait(self, spins: int = 1000):
        _check("zeta_selftest_wait", lib().zeta_selftest_wait(self._h, int(spins), _stream()))

    def get_status(self) -> int:
        return lib().zeta_get_status(self._h, _stream())


def _autograd():
    import torch

    class ZetaNode(torch.autograd.Function):
        """zeta_l of the node form of a contrast grid; differentiable in the grid."""

        @staticmethod
        def forward(fctx, delta, zctx):
            d = delta.detach().contiguous()
            fctx.save_for_backward(d)
            fctx.zctx = zctx
            return zctx.zeta_ell(delta=d, forms=("node",))["node"].clone()

        @staticmethod
        def backward(fctx, g):
            (d,) = fctx.saved_tensors
            return fctx.zctx.backward_node(d, g), None

    class ZetaParticles(torch.autograd.Function):
        """zeta_l of the particle form of a catalogue; differentiable in the positions."""

        @staticmethod
        def forward(fctx, pos, w, zctx):
            parts = torch.cat([pos.detach(), w.detach()[:, None]], 1).contiguous()
            fctx.save_for_backward(parts)
            fctx.zctx = zctx
            return zctx.zeta_ell(particles=parts, forms=("particle",))["particle"].clone()

        @staticmethod
        def backward(fctx, g):
            (parts,) = fctx.saved_tensors
            return fctx.zctx.backward_particles(parts, g), None, None

    return ZetaNode, ZetaParticles


def zeta_node(delta, zctx):
    """Differentiable node-form zeta_l (torch.autograd.Function backed by zeta_backward_node)."""
    return _autograd()[0].apply(delta, zctx)


def zeta_particles(pos, w, zctx):
    """Differentiable particle-form zeta_l in the positions (backed by zeta_backward_particles)."""
    return _autograd()[1].apply(pos, w, zctx)
