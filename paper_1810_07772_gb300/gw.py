"""Python binding of libgw (ctypes).  Argument marshalling only: every step runs in the CUDA
library, which must be built (``__graft_entry__.build()``); there is no CPU fallback.

The names follow the C ABI in ``include/gw.h``: ``load_states``, ``build_P``, ``P_to_G``,
``eps_inv``.  Device buffers are passed as ``torch.Tensor`` (``data_ptr()``) or raw integers; host
buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes
import functools
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB_PATH

GW_OK, GW_E_INVALID, GW_E_NOMEM, GW_E_CUDA, GW_E_NOT_READY, GW_E_NUMERIC, GW_E_TIMEOUT, GW_E_UNSUPPORTED = range(8)
PRECISION = {"tf32x3": 0, "bf16x3": 1, "tf32x1": 2, "fp32_simt": 3, "fp16x3": 4}
INV_METHOD = {"cholesky": 0, "newton": 1, "newton_tc": 2}
HERK_KERNEL = {"single": 0, "pair": 1}
TRANSFORM_KERNEL = {"two_kernel": 0, "fused": 1, "tables": 2}
ZGEMM_MODE = {"fp16x3": 0, "slices": 1}
GW_C64, GW_C128 = 0, 1
BUF = {"P": 0, "F": 1, "PG": 2, "eps": 3, "epsinv": 4, "weights": 5, "psiT": 6}

# Every symbol include/gw.h declares, with its ctypes signature.
_c = ctypes
_vp, _i, _d, _sz = _c.c_void_p, _c.c_int, _c.c_double, _c.c_size_t
SIGNATURES = {
    "gw_status_str": (_c.c_char_p, [_i]),
    "gw_version": (_i, []),
    "gw_create": (_i, [_c.POINTER(_vp), _i, _vp]),
    "gw_destroy": (_i, [_vp]),
    "gw_set_stream": (_i, [_vp, _vp]),
    "gw_last_error": (_i, [_vp, _c.c_char_p, _sz]),
    "gw_load_states": (_i, [_vp, _i, _i, _i, _d, _i, _i, _vp, _i, _i, _vp]),
    "gw_load_states_g": (_i, [_vp, _i, _i, _i, _d, _i, _i, _i, _vp, _vp, _i, _i, _vp]),
    "gw_set_kweight": (_i, [_vp, _d, _i]),
    "gw_pp_modes": (_i, [_vp, _i, _d, _vp, _vp, _vp, _vp]),
    "gw_pp_eval": (_i, [_vp, _d, _i, _vp]),
    "gw_build_P": (_i, [_vp, _i, _vp]),
    "gw_P_to_G": (_i, [_vp, _i, _c.POINTER(_i), _vp, _i, _vp]),
    "gw_build_PG": (_i, [_vp, _i, _i, _c.POINTER(_i), _vp, _i, _vp]),
    "gw_eps_inv": (_i, [_vp, _i, _vp, _vp]),
    "gw_sync": (_i, [_vp]),
    "gw_get_buffer": (_i, [_vp, _i, _c.POINTER(_vp), _c.POINTER(_sz)]),
    "gw_get_dims": (_i, [_vp, _c.POINTER(_i)]),
    "gw_set_timing": (_i, [_vp, _i]),
    "gw_get_times": (_i, [_vp, _c.POINTER(_c.c_float)]),
    "gw_set_wait_limit": (_i, [_vp, _d]),
    "gw_set_q": (_i, [_vp, _c.POINTER(_d)]),
    "gw_set_herk_window": (_i, [_vp, _i, _i]),
    "gw_set_herk_kernel": (_i, [_vp, _i]),
    "gw_set_transform_kernel": (_i, [_vp, _i]),
    "gw_corr_closure": (_i, [_vp, _i, _c.POINTER(_c.c_double), _i, _vp]),
    "gw_corr_train": (_i, [_vp, _vp, _vp, _c.c_long, _vp, _c.POINTER(_c.c_float)]),
    "gw_set_error_target": (_i, [_vp, ctypes.c_double]),
    "gw_reset_times": (_i, [_vp]),
    "gw_get_stats": (_i, [_vp, _c.POINTER(_c.c_double)]),
    "gw_eps_inv_noalloc": (_i, [_vp, _i, _vp, _vp]),
    "gw_zgemm_tc": (_i, [_vp, _i, _i, _i, _i, _vp, _i, _vp, _i, _vp]),
    "gw_zinv_tc": (_i, [_vp, _i, _vp, _vp]),
    "gw_newton_tc_report": (_i, [_vp, _c.POINTER(_c.c_double)]),
    "gw_batch_create": (_i, [_c.POINTER(_vp), _c.POINTER(_vp), _i, _c.POINTER(_i), _i]),
    "gw_batch_destroy": (_i, [_vp]),
    "gw_batch_run": (_i, [_vp, _i]),
    "gw_batch_set_window": (_i, [_vp, _i, _i]),
    "gw_batch_autotune": (_i, [_vp, _c.c_char_p, _d]),
    "gw_batch_stats": (_i, [_vp, _c.POINTER(_c.c_double)]),
    "gw_batch_set_inverse": (_i, [_vp, _i]),
    "gw_batch_last_error": (_i, [_vp, _c.c_char_p, _sz]),
    "gw_mlp_num_params": (_i, [_i, _i, _c.POINTER(_sz)]),
    "gw_mlp_create": (_i, [_c.POINTER(_vp), _i, _i, _i, _i, _vp]),
    "gw_mlp_destroy": (_i, [_vp]),
    "gw_mlp_last_error": (_i, [_vp, _c.c_char_p, _sz]),
    "gw_mlp_set_params": (_i, [_vp, _vp, _i]),
    "gw_mlp_get_params": (_i, [_vp, _vp, _i]),
    "gw_mlp_forward": (_i, [_vp, _vp, _c.c_long, _vp]),
    "gw_mlp_infer": (_i, [_vp, _vp, _c.c_long, _vp]),
    "gw_mlp_check": (_i, [_vp]),
    "gw_mlp_grad": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _vp]),
    "gw_mlp_train_step": (_i, [_vp, _vp, _vp, _vp, _i, _d, _d, _d, _d, _vp]),
    "gw_corr_weight_ratio": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "gw_corr_features": (_i, [_vp, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "gw_corr_targets": (_i, [_vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "gw_corr_apply": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
}

_lib = None


def lib():
    """Load libgw.so (raises if it has not been built: the product path has no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgw.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class GwError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{lib().gw_status_str(status).decode()} ({status}): {message}")
        self.status = status


def _ptr(x):
    """Device or host address of a torch tensor, numpy array or integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a buffer")


def _is_device(x):
    return hasattr(x, "is_cuda") and x.is_cuda


@functools.lru_cache(maxsize=64)
def _sphere_count(dims, gcut):
    axes = [np.arange(-(n // 2), n - n // 2) ** 2 for n in dims]
    m2 = axes[0][:, None, None] + axes[1][None, :, None] + axes[2][None, None, :]
    return int(np.count_nonzero(m2 <= gcut))


def _fits(x, nbytes, what):
    """Reject a tensor or array smaller than the nbytes a call reads or writes through it (the
    library takes plain pointers and trusts the documented sizes; raw integer addresses pass)."""
    if isinstance(x, np.ndarray):
        have = x.nbytes
    elif hasattr(x, "numel") and hasattr(x, "element_size"):
        have = x.numel() * x.element_size()
    else:
        return
    if have < nbytes:
        raise GwError(GW_E_INVALID, f"{what} holds {have} bytes, the call needs {nbytes}")


class DeviceView:
    """Read-only view of a device buffer through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Context:
    """One problem on one GPU; wraps a gw_ctx.  ``stream``: torch.cuda.Stream, raw handle or None
    (torch's current stream at creation)."""

    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._h = ctypes.c_void_p()
        st = lib().gw_create(ctypes.byref(self._h), device, handle)
        if st != GW_OK:
            raise GwError(st, "gw_create failed")
        self.device = device
        self.dims = None
        self.ng = 0
        self.gvec = None
        self._gbuf = np.zeros((1 << 18, 3), dtype=np.int32)  # G-vector output, reused by P_to_G

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gw_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != GW_OK:
            buf = ctypes.create_string_buffer(512)
            lib().gw_last_error(self._h, buf, 512)
            raise GwError(st, buf.value.decode())

    # ------------------------------------------------------------------ the four calls
    def load_states(self, psi, energies_eV, dims, nv, cell_L=1.0):
        """psi: [nv + nc][N_r] complex (torch cuda tensor or numpy host array, complex64/128)."""
        n1, n2, n3 = (int(d) for d in dims)
        nb = psi.shape[0]
        E = np.ascontiguousarray(np.asarray(energies_eV, dtype=np.float64))
        if E.shape != (nb,):
            raise ValueError("energies must have one entry per state")
        dt = str(psi.dtype)
        dtype = GW_C128 if "complex128" in dt else GW_C64
        if "complex" not in dt:
            raise TypeError("psi must be complex64 or complex128")
        if len(psi.shape) < 2 or int(np.prod([int(d) for d in psi.shape[1:]])) != n1 * n2 * n3:
            raise GwError(GW_E_INVALID, f"psi must be [nv + nc][N_r] with N_r = {n1 * n2 * n3}")
        self._check(lib().gw_load_states(self._h, n1, n2, n3, float(cell_L), int(nv), nb - int(nv), _ptr(psi),
                                         dtype, 1 if _is_device(psi) else 0, E.ctypes.data))
        self.dims = (n1, n2, n3)
        self.nv, self.nc = int(nv), nb - int(nv)
        self._E_keep = E

    def load_states_g(self, coef, gvec, energies_eV, dims, nv, cell_L=1.0):
        """States as plane-wave coefficients: coef [nv + nc][npw] complex (torch cuda tensor or numpy
        host array), gvec [npw][3] integer Miller indices (gw_load_states_g)."""
        n1, n2, n3 = (int(d) for d in dims)
        nb, npw = coef.shape
        E = np.ascontiguousarray(np.asarray(energies_eV, dtype=np.float64))
        g = np.ascontiguousarray(np.asarray(gvec, dtype=np.int32))
        if E.shape != (nb,) or g.shape != (npw, 3):
            raise ValueError("energies need one entry per state and gvec one row per plane wave")
        dt = str(coef.dtype)
        if "complex" not in dt:
            raise TypeError("coefficients must be complex64 or complex128")
        dtype = GW_C128 if "complex128" in dt else GW_C64
        self._check(lib().gw_load_states_g(self._h, n1, n2, n3, float(cell_L), int(nv), nb - int(nv), npw,
                                           g.ctypes.data, _ptr(coef), dtype, 1 if _is_device(coef) else 0,
                                           E.ctypes.data))
        self.dims = (n1, n2, n3)
        self.nv, self.nc = int(nv), nb - int(nv)
        self._E_keep = E

    def set_kweight(self, weight, accumulate=False):
        """Weight of the next P~ and whether it adds to the running sum over k-points (gw_set_kweight)."""
        self._check(lib().gw_set_kweight(self._h, float(weight), 1 if accumulate else 0))

    def build_P(self, precision="fp16x3", P_out=None):
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        if self.dims is not None:
            nr = self.dims[0] * self.dims[1] * self.dims[2]
            _fits(P_out, nr * nr * 8, "P_out")
        self._check(lib().gw_build_P(self._h, prec, _ptr(P_out)))

    def P_to_G(self, gcut, PG_out=None):
        """Returns the integer G-vectors (N_g x 3, basis order)."""
        ng = ctypes.c_int(0)
        g = self._gbuf
        self._fits_PG(PG_out, gcut)
        self._check(lib().gw_P_to_G(self._h, int(gcut), ctypes.byref(ng), g.ctypes.data, g.shape[0], _ptr(PG_out)))
        self.ng = ng.value
        self.gvec = g[: ng.value].copy()
        return self.gvec

    def build_PG(self, gcut, precision="fp16x3", PG_out=None):
        """P~ by the g-space route (no P(r,r')); returns the integer G-vectors like P_to_G."""
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        ng = ctypes.c_int(0)
        g = self._gbuf
        self._fits_PG(PG_out, gcut)
        self._check(lib().gw_build_PG(self._h, prec, int(gcut), ctypes.byref(ng), g.ctypes.data, g.shape[0],
                                      _ptr(PG_out)))
        self.ng = ng.value
        self.gvec = g[: ng.value].copy()
        return self.gvec

    def eps_inv(self, method="cholesky", eps_out=None, epsinv_out=None):
        m = INV_METHOD[method] if isinstance(method, str) else int(method)
        _fits(eps_out, self.ng * self.ng * 16, "eps_out")
        _fits(epsinv_out, self.ng * self.ng * 16, "epsinv_out")
        self._check(lib().gw_eps_inv(self._h, m, _ptr(eps_out), _ptr(epsinv_out)))

    def zgemm_tc(self, A, B, mode="slices", C=None):
        """C = A B for device complex128 tensors (A: M x K, B: K x N, rows may be strided) on the
        tensor cores: mode "slices" has FP64 accuracy, "fp16x3" about 1e-6 (gw_zgemm_tc)."""
        import torch
        M, K = A.shape
        K2, N = B.shape
        if K2 != K or A.dtype != torch.complex128 or B.dtype != torch.complex128 or A.stride(1) != 1 or B.stride(1) != 1:
            raise GwError(GW_E_INVALID, "zgemm_tc: complex128 A (M x K), B (K x N) with unit column stride")
        if C is None:
            C = torch.empty((M, N), dtype=torch.complex128, device=A.device)
        m = ZGEMM_MODE[mode] if isinstance(mode, str) else int(mode)
        # rows may be strided (unit column stride checked above), so pass the addresses directly
        self._check(lib().gw_zgemm_tc(self._h, m, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                      _ptr(C)))
        return C

    def zinv_tc(self, A, X=None):
        """A^-1 of a Hermitian positive definite device complex128 matrix by the tensor-core Newton
        iteration (gw_zinv_tc)."""
        import torch
        n = A.shape[0]
        if A.shape != (n, n) or A.dtype != torch.complex128 or not A.is_contiguous():
            raise GwError(GW_E_INVALID, "zinv_tc: contiguous complex128 n x n")
        if X is None:
            X = torch.empty_like(A)
        self._check(lib().gw_zinv_tc(self._h, n, _ptr(A), _ptr(X)))
        return X

    def pp_modes(self, nmodes, tol=1e-12):
        """Plasmon-pole modes of Sec. 5.2 from the last eps^-1 (gw_pp_modes): sigma (ascending),
        omega^2 (Hartree^2), residuals and the eigenvectors A [N_g][nmodes]."""
        sig, w2, res = (np.zeros(nmodes) for _ in range(3))
        A = np.zeros((self.ng, nmodes), dtype=np.complex128)
        self._check(lib().gw_pp_modes(self._h, int(nmodes), float(tol), sig.ctypes.data, w2.ctypes.data,
                                      res.ctypes.data, A.ctypes.data))
        return {"sigma": sig, "omega2": w2, "resid": res, "A": A}

    def pp_eval(self, omega, nuse, S_out=None):
        """S(omega) from the first nuse plasmon-pole modes (gw_pp_eval); a host array unless S_out."""
        out = S_out if S_out is not None else np.zeros((self.ng, self.ng), dtype=np.complex128)
        _fits(out, self.ng * self.ng * 16, "S_out")
        self._check(lib().gw_pp_eval(self._h, float(omega), int(nuse), _ptr(out)))
        return out

    def newton_tc_report(self):
        """Phase-1 steps, residual after phase 1, last measured residual and refinements of the
        last tensor-core Newton inverse (gw_newton_tc_report)."""
        d = (ctypes.c_double * 4)()
        self._check(lib().gw_newton_tc_report(self._h, d))
        return {"steps": int(d[0]), "res_phase1": d[1], "res_last": d[2], "refinements": int(d[3])}

    # ------------------------------------------------------------------ helpers
    def sync(self):
        self._check(lib().gw_sync(self._h))

    def set_timing(self, on=True):
        self._check(lib().gw_set_timing(self._h, 1 if on else 0))

    def times(self):
        t = (ctypes.c_float * 6)()
        self._check(lib().gw_get_times(self._h, t))
        return {"pair": t[0], "herk": t[1], "row_dft": t[2], "col_dft": t[3], "eps_build": t[4], "eps_inv": t[5]}

    def reset_times(self):
        self._check(lib().gw_reset_times(self._h))

    def stats(self):
        d = (ctypes.c_double * 8)()
        self._check(lib().gw_get_stats(self._h, d))
        keys = ["kernel_launches", "newton_iters", "herk_ms_mean", "herk_calls", "fp16_scale_exp", "herk_tiles",
                "window_chunks", "flush_windows"]
        return dict(zip(keys, list(d)))

    def set_herk_window(self, window_chunks, flush_windows):
        self._check(lib().gw_set_herk_window(self._h, int(window_chunks), int(flush_windows)))

    def corr_closure(self, gcut, E_omit_eV, out=None):
        """Closure estimate of the omitted part of P~ from the loaded states and the omitted
        states' energies (gw_corr_closure); returns a complex64 [N_g][N_g] device tensor."""
        import torch
        E = np.ascontiguousarray(np.asarray(E_omit_eV, dtype=np.float64))
        if out is None:
            ng = self._sphere_size(gcut)
            out = torch.empty((ng, ng), dtype=torch.complex64, device=f"cuda:{self.device}")
        else:
            self._fits_PG(out, gcut)
        self._check(lib().gw_corr_closure(self._h, int(gcut), E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          int(E.size), _ptr(out)))
        return out

    def _fits_PG(self, out, gcut):
        """An N_g x N_g complex64 output for the sphere gcut, checked when the grid and the cut are
        valid (otherwise the library rejects the call before writing)."""
        if out is None or self.dims is None or not (0 <= int(gcut) and 4 * int(gcut) < min(self.dims) ** 2):
            return
        ng = self._sphere_size(int(gcut))
        _fits(out, ng * ng * 8, "P~ output")

    def _sphere_size(self, gcut):
        """Number of integer m in the grid's index range with |m|^2 <= gcut (the N_g of the call)."""
        return _sphere_count(tuple(int(n) for n in self.dims), int(gcut))

    def set_transform_kernel(self, kind):
        """Sphere transforms (gw_set_transform_kernel): "two_kernel" (the default; constant
        twiddles where the grid allows), "tables" (the two-kernel form with twiddle tables) or
        "fused" (one kernel per pass)."""
        self._check(lib().gw_set_transform_kernel(self._h, TRANSFORM_KERNEL[kind] if isinstance(kind, str)
                                                  else int(kind)))

    def set_herk_kernel(self, kind):
        """Kernel of the 16-bit r-space update: "single" (one CTA per tile, the default) or "pair"
        (CTA pairs sharing 2-SM MMAs) (gw_set_herk_kernel)."""
        self._check(lib().gw_set_herk_kernel(self._h, HERK_KERNEL[kind] if isinstance(kind, str) else int(kind)))

    def set_error_target(self, target):
        """P~ error target of the 16-bit update; the window follows from it (gw_set_error_target)."""
        self._check(lib().gw_set_error_target(self._h, float(target)))

    def set_q(self, q):
        """Wave vector of eps^q in units of 2 pi / cell_L (gw_set_q)."""
        arr = (ctypes.c_double * 3)(*[float(x) for x in q])
        self._check(lib().gw_set_q(self._h, arr))

    def set_wait_limit(self, ms):
        self._check(lib().gw_set_wait_limit(self._h, float(ms)))

    def buffer(self, which):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        self._check(lib().gw_get_buffer(self._h, BUF[which], ctypes.byref(p), ctypes.byref(n)))
        return p.value, n.value

    def dims8(self):
        d = (ctypes.c_int * 8)()
        self._check(lib().gw_get_dims(self._h, d))
        return list(d)

    def view(self, which, dtype=None):
        """torch tensor sharing an internal device buffer (no copy)."""
        import torch
        ptr, nbytes = self.buffer(which)
        d = self.dims8()
        nr, ng, nr_pad = d[3], d[6], d[7]
        raw = torch.as_tensor(DeviceView(ptr, (nbytes,), "|u1"), device=f"cuda:{self.device}")
        if which == "P":
            return raw.view(torch.complex64).view(nr, nr)
        if which == "PG":
            return raw[: ng * ng * 8].view(torch.complex64).view(ng, ng)
        if which in ("eps", "epsinv"):
            return raw[: ng * ng * 16].view(torch.complex128).view(ng, ng)
        if which == "psiT":
            return raw.view(torch.complex64).view(nr, self.nv + self.nc)
        return raw.view(torch.float32) if nbytes % 4 == 0 else raw


class Batch:
    """Independent systems in one pass (gw_batch_*): contexts with loaded states and their gcuts."""

    def __init__(self, contexts, gcuts, precision="fp16x3"):
        n = len(contexts)
        hs = (ctypes.c_void_p * n)(*[c._h.value for c in contexts])
        gc = (ctypes.c_int * n)(*[int(g) for g in gcuts])
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self._h = ctypes.c_void_p()
        st = lib().gw_batch_create(ctypes.byref(self._h), hs, n, gc, prec)
        if st != GW_OK:
            msg = ""
            for c in contexts:
                buf = ctypes.create_string_buffer(512)
                lib().gw_last_error(c._h, buf, 512)
                msg = msg or buf.value.decode()
            raise GwError(st, "gw_batch_create failed " + msg)
        self.contexts = list(contexts)
        self.gcuts = list(gcuts)

    def _check(self, st):
        if st != GW_OK:
            buf = ctypes.create_string_buffer(512)
            lib().gw_batch_last_error(self._h, buf, 512)
            raise GwError(st, buf.value.decode())

    def run(self, use_graph=True):
        self._check(lib().gw_batch_run(self._h, 1 if use_graph else 0))
        for c in self.contexts:   # each context now holds P~, eps and eps^-1 of its instance
            d = c.dims8()
            c.ng = d[6]

    def set_inverse(self, method):
        """eps^-1 of every instance: "newton_tc" (default) or "cholesky" (gw_batch_set_inverse)."""
        m = INV_METHOD[method] if isinstance(method, str) else int(method)
        self._check(lib().gw_batch_set_inverse(self._h, m))

    def set_window(self, window_chunks, flush_windows):
        self._check(lib().gw_batch_set_window(self._h, int(window_chunks), int(flush_windows)))

    def autotune(self, cache_path=None, target_error=1e-6):
        p = cache_path.encode() if cache_path else None
        self._check(lib().gw_batch_autotune(self._h, p, float(target_error)))
        return self.stats()

    def stats(self):
        d = (ctypes.c_double * 4)()
        self._check(lib().gw_batch_stats(self._h, d))
        return {"herk_ms": d[0], "window_chunks": int(d[1]), "flush_windows": int(d[2]), "tiles": int(d[3])}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gw_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------------------------- learned correction
N_FEATURES = 12


def _stream_handle(device, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _status(st, where):
    if st != GW_OK:
        raise GwError(st, where)


class Mlp:
    """The correction network (gw_mlp_*): n_in -> hidden -> hidden -> hidden -> 2, tanh, FP16 weights."""

    def __init__(self, n_in=N_FEATURES, hidden=256, max_batch=8192, device=0, stream=None):
        import torch
        self.device, self.n_in, self.hidden, self.max_batch = int(device), int(n_in), int(hidden), int(max_batch)
        self.stream = _stream_handle(device, stream)
        n = ctypes.c_size_t()
        _status(lib().gw_mlp_num_params(self.n_in, self.hidden, ctypes.byref(n)), "gw_mlp_num_params")
        self.P = n.value
        self._h = ctypes.c_void_p()
        _status(lib().gw_mlp_create(ctypes.byref(self._h), self.device, self.n_in, self.hidden, self.max_batch,
                                    self.stream), "gw_mlp_create")
        self._dev = torch.device(f"cuda:{self.device}")
        self._loss = torch.zeros(1, dtype=torch.float32, device=self._dev)

    def _check(self, st):
        if st != GW_OK:
            buf = ctypes.create_string_buffer(512)
            lib().gw_mlp_last_error(self._h, buf, 512)
            raise GwError(st, buf.value.decode())

    def set_params(self, theta):
        if _is_device(theta):
            self._check(lib().gw_mlp_set_params(self._h, _ptr(theta), 1))
        else:
            th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
            if th.size != self.P:
                raise ValueError(f"expected {self.P} parameters, got {th.size}")
            self._check(lib().gw_mlp_set_params(self._h, th.ctypes.data, 0))

    def get_params(self):
        th = np.empty(self.P, dtype=np.float32)
        self._check(lib().gw_mlp_get_params(self._h, th.ctypes.data, 0))
        return th

    def forward(self, X, Y=None):
        import torch
        n = X.shape[0]
        if Y is None:
            Y = torch.empty((n, 2), dtype=torch.float32, device=self._dev)
        self._check(lib().gw_mlp_forward(self._h, _ptr(X), n, _ptr(Y)))
        return Y

    def infer(self, X, Y=None):
        """Tensor-core inference (FP16 activations into the 256-wide products)."""
        import torch
        n = X.shape[0]
        if Y is None:
            Y = torch.empty((n, 2), dtype=torch.float32, device=self._dev)
        self._check(lib().gw_mlp_infer(self._h, _ptr(X), n, _ptr(Y)))
        return Y

    def check(self):
        self._check(lib().gw_mlp_check(self._h))

    def grad(self, X, T, rows=None, batch=None):
        """(dL/dtheta as a device tensor, L) for one batch."""
        import torch
        b = int(rows.shape[0]) if rows is not None else (int(batch) if batch else X.shape[0])
        g = torch.empty(self.P, dtype=torch.float32, device=self._dev)
        self._check(lib().gw_mlp_grad(self._h, _ptr(X), _ptr(T), _ptr(rows), b, _ptr(g), _ptr(self._loss)))
        torch.cuda.synchronize(self._dev)
        return g, float(self._loss.item())

    def train_step(self, X, T, rows, lr, beta1=0.9, beta2=0.999, eps=1e-8, loss_accum=None):
        self._check(lib().gw_mlp_train_step(self._h, _ptr(X), _ptr(T), _ptr(rows), int(rows.shape[0]), float(lr),
                                            float(beta1), float(beta2), float(eps), _ptr(loss_accum)))

    def train_corr(self, X, T, epochs, batch, lr, lr_final=1e-5, seed=0, diag_repeat=1, diag_feature=7,
                   beta1=0.9, beta2=0.999, eps=1e-8):
        """Passes of Adam over minibatches of (X, T) in the library's order (gw_corr_train);
        returns the mean loss of each pass."""
        o = CorrTrainOpts(int(epochs), int(batch), float(lr), float(lr_final), float(beta1), float(beta2), float(eps),
                          int(seed), int(diag_repeat), int(diag_feature))
        losses = (ctypes.c_float * int(epochs))()
        self._check(lib().gw_corr_train(self._h, _ptr(X), _ptr(T), int(X.shape[0]), ctypes.byref(o), losses))
        return [float(x) for x in losses]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gw_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class CorrTrainOpts(ctypes.Structure):
    """gw_corr_train_opts of include/gw.h."""
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("lr_final", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("diag_repeat", ctypes.c_int),
                ("diag_feature", ctypes.c_int)]


def _upload(arr, dtype, dev, stream):
    """A host array on the device: staged in pinned memory and copied on the library's stream without
    a host synchronisation (a copy from pageable memory would wait for the stream's earlier work)."""
    import torch
    t = torch.as_tensor(np.ascontiguousarray(np.asarray(arr, dtype=dtype))).pin_memory()
    h = _stream_handle(dev.index, stream)
    s = torch.cuda.ExternalStream(h, device=dev) if h else torch.cuda.default_stream(dev)
    with torch.cuda.stream(s):
        return t.to(dev, non_blocking=True)


def corr_weight_ratio(E_eV, nv, nc_keep, device=0, stream=None):
    """Device float: weight of the omitted pairs relative to the kept ones (gw_corr_weight_ratio).
    E_eV: host energies, or a float64 device tensor."""
    import torch
    dev = torch.device(f"cuda:{device}")
    on_dev = isinstance(E_eV, torch.Tensor) and E_eV.is_cuda and E_eV.dtype == torch.float64
    E = E_eV if on_dev else _upload(E_eV.cpu().numpy() if isinstance(E_eV, torch.Tensor) else E_eV, np.float64, dev,
                                    stream)
    out = torch.empty(1, dtype=torch.float32, device=dev)
    _status(lib().gw_corr_weight_ratio(_ptr(E), int(nv), int(nc_keep), E.shape[0] - int(nv), _ptr(out),
                                       _stream_handle(device, stream)), "gw_corr_weight_ratio")
    return out


def corr_features(PG, gvec, gcut, ratio, clos=None, stream=None):
    """(X [ng(ng+1)/2][12], scale) for a truncated P~ (complex64 ng x ng device tensor); clos is the
    closure estimate of the omitted part (gw_corr_closure) or None."""
    import torch
    dev = PG.device
    ng = PG.shape[0]
    on_dev = isinstance(gvec, torch.Tensor) and gvec.is_cuda and gvec.dtype == torch.int32
    g = gvec if on_dev else _upload(gvec.cpu().numpy() if isinstance(gvec, torch.Tensor) else gvec, np.int32, dev,
                                    stream)
    X = torch.empty((ng * (ng + 1) // 2, N_FEATURES), dtype=torch.float32, device=dev)
    scale = torch.empty(1, dtype=torch.float32, device=dev)
    _status(lib().gw_corr_features(_ptr(PG), ng, _ptr(g), int(gcut), _ptr(ratio), _ptr(clos), _ptr(X), _ptr(scale),
                                   _stream_handle(dev.index, stream)), "gw_corr_features")
    return X, scale


def corr_targets(PG_keep, PG_all, scale, clos=None, stream=None):
    import torch
    ng = PG_keep.shape[0]
    T = torch.empty((ng * (ng + 1) // 2, 2), dtype=torch.float32, device=PG_keep.device)
    _status(lib().gw_corr_targets(_ptr(PG_keep), _ptr(PG_all), _ptr(clos), ng, _ptr(scale), _ptr(T),
                                  _stream_handle(PG_keep.device.index, stream)), "gw_corr_targets")
    return T


def corr_apply(PG, Y, scale, clos=None, stream=None):
    """In place: PG += the closure estimate (if given) and the predicted correction (gw_corr_apply)."""
    _status(lib().gw_corr_apply(_ptr(PG), PG.shape[0], _ptr(Y), _ptr(scale), _ptr(clos),
                                _stream_handle(PG.device.index, stream)), "gw_corr_apply")
