"""The band-structured input recipe of the learned workload (inputs.make_states_g_structured):
orthonormal coefficient sets on the stated sphere, energies drawn as documented, and the spectral
weight of each state centred where its energy puts it, rising with the band."""
import numpy as np

from paper_1810_07772_gb300 import inputs


def test_structured_states_are_orthonormal_and_band_ordered():
    dims, nv, nc = (12, 12, 12), 4, 120
    coef, gvec, E = inputs.make_states_g_structured(dims, nv, nc, 5)
    assert coef.shape == (nv + nc, len(gvec)) and gvec.shape[1] == 3
    assert np.max(np.abs(coef @ coef.conj().T - np.eye(nv + nc))) <= 1e-12
    k2 = np.sum(gvec.astype(np.int64) ** 2, axis=1)
    assert k2.max() <= inputs.structured_sphere(dims) < (min(dims) / 2) ** 2
    assert np.all(np.diff(E[:nv]) >= 0) and np.all(np.diff(E[nv:]) >= 0) and E[nv - 1] < E[nv]
    assert E[:nv].min() >= -10.0 and E[nv:].max() <= 20.0
    # mean |m| of each state's spectral weight rises with its energy
    mk = np.sum(np.abs(coef) ** 2 * np.sqrt(k2)[None, :], axis=1)
    assert np.corrcoef(E, mk)[0, 1] > 0.9
    assert mk[:nv].mean() < mk[nv:nv + 20].mean() < mk[-20:].mean()
    # the QR in energy order keeps the lowest state on its shell: its weight within 2 widths of k_0 = 0
    assert np.sum(np.abs(coef[0]) ** 2 * (np.sqrt(k2) <= 1.6)) > 0.9


def test_structured_states_are_reproducible():
    a = inputs.make_states_g_structured((8, 8, 8), 2, 20, 11)
    b = inputs.make_states_g_structured((8, 8, 8), 2, 20, 11)
    c = inputs.make_states_g_structured((8, 8, 8), 2, 20, 12)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
