"""Seeded synthetic inputs shaped like the plane-wave GW workloads of Kim et al. (arXiv 1810.07772).

This module draws inputs only: random orthonormal complex states on a cubic real-space grid
and sorted band energies.  It holds none of the polarizability arithmetic, so both the CUDA
path and the FP64 oracle can be fed from it without sharing any of the method's code.

Recipe (the paper's Si supercell states come from a DFT code that is not available here; these
stand in for them with the same shapes):

* ``A = N(0,1) + i N(0,1)`` of shape ``(N_r, N_v + N_c)`` from ``numpy.random.default_rng(seed)``
  (real part drawn first, then the imaginary part), then a reduced QR.  The columns of ``Q``
  are Haar-random and discretely orthonormal, ``sum_r conj(psi_m(r)) psi_n(r) = delta_mn``.
  Columns ``[0, N_v)`` are the occupied states, the rest the unoccupied ones.
* ``E_v ~ U[-10, 0] eV`` and ``E_c ~ U[0.5, 20] eV``, each sorted ascending, drawn after ``A``.
* The real-space index is C order, ``r = (j1 * n2 + j2) * n3 + j3``.

Band-structured states (the learned-correction workload, :func:`make_states_g_structured`): in
Haar-random states every state spreads evenly over all plane waves, so the omitted states of a
band cut are a uniformly random subspace of the complement of the kept ones and nothing about
them is predictable beyond their energies.  Kohn-Sham states are not like that: kinetic energy
rises with band energy, so low bands are smooth and high bands oscillate.  The structured recipe
gives state n plane-wave coefficients ``c_n(m) = env_n(|m|) (a + i b)`` on the sphere of
:func:`psi_sphere`, with ``a, b ~ N(0, 1)`` and a Gaussian shell
``env_n(k) = exp(-(k - k_n)^2 / (2 w^2))`` around ``k_n = k_max sqrt((E_n - E_min) / (E_max - E_min))``
(a free-electron-like ``E ~ k^2``; ``k_max`` = ``kmax_frac`` of half the smallest grid side,
``w`` = ``width`` Miller units), and then a reduced QR of the coefficient matrix with the states in
energy order, which keeps the span of every set of lowest states.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic system: an ``n^3`` grid, ``nv`` occupied and ``nc`` unoccupied states.

    ``gcut`` is the integer sphere cut: the eps basis is every ``G = 2*pi*m/L`` with
    ``|m|^2 <= gcut``.  ``cell_L`` is the cubic cell edge in bohr.
    """

    name: str
    n: int
    nv: int
    nc: int
    gcut: int
    seed: int
    cell_L: float = 1.0

    @property
    def nr(self) -> int:
        return self.n ** 3

    @property
    def k(self) -> int:
        return self.nv * self.nc

    def herk_flop(self) -> float:
        """LAPACK's complex Hermitian rank-k count over one triangle, 4 k N_r (N_r + 1)."""
        return 4.0 * self.k * self.nr * (self.nr + 1)


# The three single-system shapes: the small FP64-checkable case, the plain FP32 case and the
# split-precision case.
SMALL = Workload("grid12_nv4_nc28", 12, 4, 28, 8, 1)
PLAIN = Workload("grid24_nv32_nc480", 24, 32, 480, 29, 2)
SPLIT = Workload("grid36_nv64_nc1000", 36, 64, 1000, 61, 3)


def batch_workloads() -> list[Workload]:
    """Eight independent systems of uneven size (grids 16^3..32^3, N_v 8..48, N_c 100..800).

    The sphere cut follows ``gcut = floor((n / 4.4)^2)`` so every system keeps about 5% of its
    grid in the eps basis, as the single-system shapes do.
    """
    grids = [16, 18, 20, 24, 24, 27, 30, 32]
    out = []
    for i, n in enumerate(grids):
        nv = int(round(8 + 40 * i / 7))
        nc = 100 * (i + 1)
        gcut = int((n / 4.4) ** 2)
        out.append(Workload(f"batch{i}_grid{n}_nv{nv}_nc{nc}", n, nv, nc, gcut, 100 + i))
    return out


def make_states(n: int, nv: int, nc: int, seed: int, dims: tuple[int, int, int] | None = None):
    """Return ``(psi, E_eV)``: ``psi`` complex128 ``[nv + nc][N_r]``, ``E_eV`` float64 ``[nv + nc]``.

    ``dims`` overrides the cubic ``(n, n, n)`` grid for non-cubic test grids.
    """
    if dims is None:
        dims = (n, n, n)
    nr = int(dims[0]) * int(dims[1]) * int(dims[2])
    nb = nv + nc
    if nb > nr:
        raise ValueError("more states than grid points: they cannot be orthonormal")
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nr, nb))
    b = rng.standard_normal((nr, nb))
    q, _ = np.linalg.qr(a + 1j * b, mode="reduced")
    psi = np.ascontiguousarray(q.T)
    ev = np.sort(rng.uniform(-10.0, 0.0, nv))
    ec = np.sort(rng.uniform(0.5, 20.0, nc))
    return psi, np.concatenate([ev, ec])


def psi_sphere(dims, gcut_psi):
    """Plane-wave basis of the states: integer Miller indices m with |m|^2 <= gcut_psi, each
    component in [-n/2, n - n/2), in the order (m1, m2, m3) ascending.  Returns int32 (npw, 3)."""
    pts = [(a, b, c)
           for a in range(-(dims[0] // 2), dims[0] - dims[0] // 2)
           for b in range(-(dims[1] // 2), dims[1] - dims[1] // 2)
           for c in range(-(dims[2] // 2), dims[2] - dims[2] // 2)
           if a * a + b * b + c * c <= gcut_psi]
    return np.array(pts, dtype=np.int32).reshape(-1, 3)


def make_states_g(dims, gcut_psi: int, nv: int, nc: int, seed: int):
    """Return ``(coef, gvec, E_eV)``: random orthonormal plane-wave coefficient sets
    ``coef [nv + nc][npw]`` (complex128; a reduced QR of ``N(0,1) + i N(0,1)`` of shape
    ``(npw, nv + nc)``, real part first), the basis ``gvec`` of :func:`psi_sphere` and energies drawn
    as in :func:`make_states`."""
    gvec = psi_sphere(dims, gcut_psi)
    npw, nb = len(gvec), nv + nc
    if nb > npw:
        raise ValueError("more states than plane waves: they cannot be orthonormal")
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((npw, nb))
    b = rng.standard_normal((npw, nb))
    q, _ = np.linalg.qr(a + 1j * b, mode="reduced")
    ev = np.sort(rng.uniform(-10.0, 0.0, nv))
    ec = np.sort(rng.uniform(0.5, 20.0, nc))
    return np.ascontiguousarray(q.T), gvec, np.concatenate([ev, ec])


def structured_sphere(dims) -> int:
    """The plane-wave sphere of the band-structured states: ``|m| < min(n)/2 - 1/2``."""
    return int(np.floor((min(dims) / 2 - 0.5) ** 2))


def _shell_envelope(gvec, E, dims, width, kmax_frac):
    """env[p, n] = exp(-(|m_p| - k_n)^2 / (2 width^2)), k_n from the energies (see the module notes)."""
    k = np.sqrt(np.sum(np.asarray(gvec, dtype=np.float64) ** 2, axis=1))
    kmax = kmax_frac * min(dims) / 2.0
    kn = kmax * np.sqrt((E - E.min()) / (E.max() - E.min()))
    return np.exp(-0.5 * ((k[:, None] - kn[None, :]) / width) ** 2)


def make_states_g_structured(dims, nv: int, nc: int, seed: int, width: float = 0.8, kmax_frac: float = 0.85):
    """Band-structured states as plane-wave coefficients: ``(coef [nv + nc][npw] complex128, gvec
    [npw][3] int32, E_eV)`` on the sphere of :func:`structured_sphere`.  Energies are drawn first
    (``E_v ~ U[-10, 0]``, ``E_c ~ U[0.5, 20]`` eV, sorted), then ``a`` and ``b`` of shape
    ``(npw, nv + nc)``; see the module notes for the envelope and the QR."""
    gvec = psi_sphere(dims, structured_sphere(dims))
    npw, nb = len(gvec), nv + nc
    if nb > npw:
        raise ValueError("more states than plane waves: they cannot be orthonormal")
    rng = np.random.default_rng(seed)
    E = np.concatenate([np.sort(rng.uniform(-10.0, 0.0, nv)), np.sort(rng.uniform(0.5, 20.0, nc))])
    a = rng.standard_normal((npw, nb))
    b = rng.standard_normal((npw, nb))
    q, _ = np.linalg.qr(_shell_envelope(gvec, E, dims, width, kmax_frac) * (a + 1j * b), mode="reduced")
    return np.ascontiguousarray(q.T), gvec, E


def make_states_g_structured_device(dims, nv: int, nc: int, seed: int, device, width: float = 0.8,
                                    kmax_frac: float = 0.85):
    """Device-drawn variant of :func:`make_states_g_structured` for the full-size learned workload:
    the same energies (``default_rng(seed)``) and envelope, ``a + i b`` from torch's seeded CUDA
    generator (complex64, parts N(0, 1/2)), a reduced QR on the device.  Returns ``(coef [nv + nc]
    [npw] complex64 on device, gvec, E_eV)``."""
    import torch

    gvec = psi_sphere(dims, structured_sphere(dims))
    npw, nb = len(gvec), nv + nc
    rng = np.random.default_rng(seed)
    E = np.concatenate([np.sort(rng.uniform(-10.0, 0.0, nv)), np.sort(rng.uniform(0.5, 20.0, nc))])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    z = torch.randn((npw, nb), dtype=torch.complex64, device=device, generator=gen)
    env = torch.from_numpy(_shell_envelope(gvec, E, dims, width, kmax_frac).astype(np.float32)).to(device)
    q, _ = torch.linalg.qr(z * env, mode="reduced")
    return q.transpose(0, 1).contiguous(), gvec, E


def make_workload_states(w: Workload):
    return make_states(w.n, w.nv, w.nc, w.seed)


def plane_wave_states(dims, m_list, energies_eV):
    """States ``psi_j(r) = exp(i 2 pi m_j . (j1/n1, j2/n2, j3/n3)) / sqrt(N_r)`` for integer ``m_j``.

    Used for closed-form checks: distinct ``m_j`` (mod the grid) give exactly orthonormal states.
    """
    n1, n2, n3 = dims
    j1, j2, j3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    nr = n1 * n2 * n3
    rows = []
    for m in m_list:
        ph = 2.0 * np.pi * (m[0] * j1 / n1 + m[1] * j2 / n2 + m[2] * j3 / n3)
        rows.append((np.exp(1j * ph) / np.sqrt(nr)).reshape(-1))
    return np.array(rows), np.asarray(energies_eV, dtype=np.float64)


def mlp_init(n_in: int, hidden: int, seed: int, n_out: int = 2) -> np.ndarray:
    """Initial parameters of the correction network, flat FP32 ``[W1, b1, W2, b2, W3, b3, W4, b4]``
    with each ``W_l`` of shape ``(out, in)`` row-major: Glorot-uniform weights
    ``U(-a, a), a = sqrt(6 / (fan_in + fan_out))`` and zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for r, c in [(hidden, n_in), (hidden, hidden), (hidden, hidden), (n_out, hidden)]:
        a = np.sqrt(6.0 / (r + c))
        parts.append(rng.uniform(-a, a, r * c))
        parts.append(np.zeros(r))
    return np.concatenate(parts).astype(np.float32)


def make_states_device(n: int, nv: int, nc: int, seed: int, device):
    """Device-drawn variant of :func:`make_states` for workloads that need many large systems:
    ``A`` from torch's seeded CUDA generator (complex64, real and imaginary parts N(0, 1/2)),
    a reduced QR on the device, energies drawn exactly as in :func:`make_states` but from
    ``default_rng(seed)`` directly.  Returns ``(psi [nv + nc][N_r] complex64 on device, E_eV)``."""
    import torch

    nr = n ** 3
    nb = nv + nc
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    a = torch.randn((nr, nb), dtype=torch.complex64, device=device, generator=gen)
    q, _ = torch.linalg.qr(a, mode="reduced")
    psi = q.transpose(0, 1).contiguous()
    rng = np.random.default_rng(seed)
    ev = np.sort(rng.uniform(-10.0, 0.0, nv))
    ec = np.sort(rng.uniform(0.5, 20.0, nc))
    return psi, np.concatenate([ev, ec])
