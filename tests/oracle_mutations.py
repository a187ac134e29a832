"""Mutation check of the oracle's pins (a developer script, not collected by pytest).

Each entry below plants one plausible mistake in a copy of the oracle (a flipped sign, a dropped
term or factor, a transposed or unconjugated operand, a wrong index or unit), and the CPU pin tests
run against that copy; every mistake must make at least one of them fail.  The repository's own
oracle files are never modified: the mutants live under tests/_build/mutants/.

    python tests/oracle_mutations.py            # every mutation; exit status 1 if one survives
    python tests/oracle_mutations.py LABEL ...  # only the named ones
"""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G, M, C = "oracle/gw_oracle.py", "oracle/mlp.py", "oracle/rspace.c"

MUTATIONS = [
    (G, 'return np.asarray(E_eV, dtype=np.float64) / HARTREE_EV',
     'return np.asarray(E_eV, dtype=np.float64) / 27.0',
     'to_hartree constant'),
    (G, 'return 2.0 / (E[None, nv:] - E[:nv, None])',
     'return 1.0 / (E[None, nv:] - E[:nv, None])',
     'pair_weights factor 2'),
    (G, 'f = np.conj(psi[:nv])[:, None, :] * psi[nv:][None, :, :]',
     'f = psi[:nv][:, None, :] * np.conj(psi[nv:])[None, :, :]',
     'pair_density conj'),
    (G, 'return -(f.T @ np.conj(f))', 'return (f.T @ np.conj(f))', 'P_from_f sign'),
    (G, 'return -(f.T @ np.conj(f))', 'return -(np.conj(f).T @ f)', 'P_from_f transpose'),
    (G, '/ (E[v] - E[c]))', '/ (E[c] - E[v]))', 'quadruple sign'),
    (G, 'np.conj(psi[v, r]) * psi[c, r] * np.conj(psi[c, rp]) * psi[v, rp]',
     'psi[v, r] * np.conj(psi[c, r]) * psi[c, rp] * np.conj(psi[v, rp])',
     'quadruple conj'),
    (G, 'if a * a + b * b + c * c <= gcut:', 'if a * a + b * b + c * c < gcut:', 'sphere <'),
    (G, '    pts.sort()\n', '', 'sphere unsorted'),
    (G, 'np.exp(2j * np.pi * phase)', 'np.exp(-2j * np.pi * phase)', 'states_from_g sign'),
    (G, '@ np.exp(2j * np.pi * phase)) / np.sqrt(n1 * n2 * n3)',
     '@ np.exp(2j * np.pi * phase)) / (n1 * n2 * n3)',
     'states_from_g norm'),
    (G, 'weights = [1.0 / len(kpoints)] * len(kpoints)', 'weights = [1.0] * len(kpoints)', 'ksum weights'),
    (G, 'rho = 2.0 * np.sum(np.abs(np.asarray(psi)[:nv]) ** 2, axis=0)',
     'rho = np.sum(np.abs(np.asarray(psi)[:nv]) ** 2, axis=0)',
     'density factor 2'),
    (G, 'S = sv[:, None] * (np.asarray(epsinv) - np.eye(len(gvec)))',
     'S = sv[:, None] * (np.asarray(epsinv) + np.eye(len(gvec)))',
     'pp_S minus I'),
    (G, 'return V[:, None] * V[None, :] * (k @ k.T) * rho',
     'return V[:, None] * V[None, :] * (m @ m.T) * rho',
     'pp_omega 2pi/L'),
    (G, '    d = g[:, None, :] - g[None, :, :]\n    rho = rhoG',
     '    d = g[:, None, :] + g[None, :, :]\n    rho = rhoG',
     "pp_omega g+g'"),
    (G, 'np.where(sig != 0, -quad / np.where', 'np.where(sig != 0, quad / np.where', 'pp_modes sign'),
    (G, 'f = sigma * omega2 / (omega2 - w * w)', 'f = sigma * omega2 / (omega2 + w * w)', 'pp_S_omega'),
    (G, 'Phat = np.fft.fftn(np.asarray(P)', 'Phat = np.fft.ifftn(np.asarray(P)', 'P_to_G row sign'),
    (G, 'Pt = np.fft.ifftn(Phat.reshape', 'Pt = np.fft.fftn(Phat.reshape', 'P_to_G col sign'),
    (G, '    return Pt * nr\n', '    return Pt\n', 'P_to_G scale'),
    (G, 'return np.exp(-2j * np.pi * ph)', 'return np.exp(2j * np.pi * ph)', 'dft_matrix sign'),
    (G, 'return D @ np.asarray(P) @ np.conj(D.T)', 'return D @ np.asarray(P) @ D.T', 'P_to_G_direct conj'),
    (G, 'rho = np.conj(psi[v])[None, :] * psi[nv:]',
     'rho = psi[v][None, :] * np.conj(psi[nv:])',
     'matrix_elements conj'),
    (G, 'd = np.concatenate([2.0 / (E[v] - E[nv:]) for v in vs])',
     'd = np.concatenate([2.0 / (E[nv:] - E[v]) for v in vs])',
     'P_gspace sign'),
    (G, 'Pt += (M.T * d[None, :]) @ np.conj(M)', 'Pt += (M.T * d[None, :]) @ M', 'P_gspace conj'),
    (G, 'phases = np.exp(-2j * np.pi', 'phases = np.exp(2j * np.pi', 'entries sign'),
    (G, 'out += (M * d[None, :]) @ np.conj(M.T)', 'out += (M * d[None, :]) @ M.T', 'entries conj'),
    (G, 'return np.sum(2.0 / (E[:nv, None] - Eo[None, :]), axis=1)',
     'return np.sum(2.0 / (Eo[None, :] - E[:nv, None]), axis=1)',
     'closure_weights sign'),
    (G, 'return (T1 - T2) / (nr - n_in)', 'return (T1 + T2) / (nr - n_in)', 'closure T2 sign'),
    (G, 'return (T1 - T2) / (nr - n_in)', 'return (-T2) / (nr - n_in)', 'closure drop T1'),
    (G, 'return (T1 - T2) / (nr - n_in)', 'return (T1) / (nr - n_in)', 'closure drop T2'),
    (G, 'return (T1 - T2) / (nr - n_in)', 'return (T1 - T2) / nr', 'closure denominator'),
    (G, 'T1 = rhoG[d[..., 0] % n1, d[..., 1] % n2, d[..., 2] % n3]',
     'T1 = rhoG[(-d[..., 0]) % n1, (-d[..., 1]) % n2, (-d[..., 2]) % n3]',
     'closure T1 orientation'),
    (G, 'T2 += W[v] * (M.T @ np.conj(M))', 'T2 += W[v] * (M.T @ M)', 'closure T2 conj'),
    (G, 'rhoW = np.sum(W[:, None] * np.abs(psi[:nv]) ** 2, axis=0)',
     'rhoW = np.sum(np.abs(psi[:nv]) ** 2, axis=0)',
     'closure rhoW weights'),
    (G, 'V[nz] = 4.0 * np.pi / (omega * G2[nz])', 'V[nz] = 4.0 * np.pi / G2[nz]', 'coulomb Omega'),
    (G, 'V[nz] = 4.0 * np.pi / (omega * G2[nz])', 'V[nz] = 4.0 * np.pi / (omega * m2[nz])', 'coulomb 2pi/L'),
    (G, 'm = m + np.asarray(q, dtype=np.float64)[None, :]',
     'm = m - np.asarray(q, dtype=np.float64)[None, :]',
     'coulomb q sign'),
    (G, 'return np.eye(Pt.shape[0], dtype=np.complex128) - s[:, None]',
     'return np.eye(Pt.shape[0], dtype=np.complex128) + s[:, None]',
     'eps sign'),
    (G, 'np.asarray(Pt, np.complex128) * s[None, :]',
     'np.asarray(Pt, np.complex128) * s[:, None]',
     'eps scaling transposed'),
    (G, 'L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ np.conj(L[j, :j])) / L[j, j]',
     'L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]',
     'cholesky conj'),
    (G, 'Y[i] = (B[i] - L[i, :i] @ Y[:i]) / L[i, i]', 'Y[i] = (B[i] - L[i, :i] @ Y[:i])', 'forward_substitute pivot'),
    (G, 'return np.conj(Y.T) @ Y', 'return Y @ np.conj(Y.T)', 'inverse_cholesky order'),
    (G, 'X = alpha * np.conj(A.T)', 'X = alpha * A.T', 'newton start conj'),
    (G, 'Xn = X @ (I2 - A @ X)', 'Xn = X @ (I2 - X @ A)', 'newton order'),
    (M, 'd = np.abs(np.real(np.diag(PG_lo)))[1:]', 'd = np.abs(np.real(np.diag(PG_lo)))', 'entry_scale G=0'),
    (M, 'return float(np.sum(w[:, nc_lo:])), float(np.sum(w[:, :nc_lo]))',
     'return float(np.sum(w[:, :nc_lo])), float(np.sum(w[:, nc_lo:]))',
     'omitted_weights swap'),
    (M, 'E = np.asarray(E_eV, dtype=np.float64) / 27.211386245988',
     'E = np.asarray(E_eV, dtype=np.float64)',
     'omitted_weights units'),
    (M, 'np.sum(dm * dm, axis=1) / (4.0 * gcut)', 'np.sum(dm * dm, axis=1) / gcut', 'features dm scale'),
    (M, 's * diag[gi], s * diag[hi]', 's * diag[gi], s * diag[gi]', 'features diag index'),
    (M, '((gi == 0) | (hi == 0))', '((gi == 0) & (hi == 0))', 'features head flag'),
    (M, 'np.full(gi.shape, w_om / w_in)', 'np.full(gi.shape, w_in / w_om)', 'features ratio'),
    (M, 's * np.real(dc), s * np.imag(dc)', 's * np.real(dc), -s * np.imag(dc)', 'features dclos conj'),
    (M, 'D = D - np.asarray(dclos, np.complex128)', 'D = D + np.asarray(dclos, np.complex128)', 'targets dclos sign'),
    (M, 'a = np.tanh(a @ W.T + b)', 'a = np.tanh(a @ W.T) + b', 'forward bias'),
    (M, 'delta = da * (1.0 - acts[l] ** 2)', 'delta = da * (1.0 - acts[l])', 'grad tanh'),
    (M, 'loss = 0.5 * np.sum(r * r) / B', 'loss = np.sum(r * r) / B', 'loss factor'),
    (M, 'grads[l] = (delta.T @ a_in, np.sum(delta, axis=0))',
     'grads[l] = (delta.T @ a_in, np.sum(delta, axis=1)[:delta.shape[1]] * 0)',
     'grad bias'),
    (M, '        o += r * c + r\n    return out', '        o += r * c\n    return out', 'fp16 offsets'),
    (M, 'out[o:o + r * c] = out[o:o + r * c].astype(np.float16)',
     'out[o:o + r * c + r] = out[o:o + r * c + r].astype(np.float16)',
     'fp16 biases rounded'),
    (M, 'P[gi[on], gi[on]] += np.real(d[on])', 'P[gi[on], gi[on]] += d[on]', 'apply diag real'),
    (M, 'P[hi[~on], gi[~on]] += np.conj(d[~on])', 'P[hi[~on], gi[~on]] += d[~on]', 'apply mirror conj'),
    (M, 'keep = (gi != 0) & (hi != 0)', 'keep = gi >= 0', 'apply head'),
    (M, '+ 1j * np.asarray(Y[:, 1], dtype=np.float64)) / s',
     '+ 1j * np.asarray(Y[:, 1], dtype=np.float64)) * s',
     'apply scale'),
    (M, 'mh = m / (1.0 - beta1 ** t)', 'mh = m', 'adam bias m'),
    (M, 'theta - lr * mh / (np.sqrt(vh) + eps)', 'theta - lr * mh / (vh + eps)', 'adam sqrt'),
    (G, "((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (m[:, 2] % n3)",
     "((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (-m[:, 2] % n3)",
     "flat index sign"),
    (G, "vs = list(range(v0, min(nv, v0 + v_chunk)))", "vs = list(range(v0, min(nv, v0 + v_chunk - 1)))",
     "P_gspace drops a state"),
    (G, "    A = A[:, :nmodes]\n", "    A = A[:, -nmodes:]\n", "pp_modes least negative vectors"),
    (G, "    sig = w[:nmodes]\n", "    sig = w[-nmodes:]\n", "pp_modes least negative values"),
    (G, "rho = np.conj(psi[v])[None, :] * psi\n", "rho = psi[v][None, :] * np.conj(psi)\n", "closure M conj"),
    (M, "gi, hi = np.triu_indices(ng)\n    m2 = ", "hi, gi = np.triu_indices(ng)\n    m2 = ", "features lower triangle"),
    (M, "d = D[gi, hi] * s", "d = D[hi, gi] * s", "targets lower triangle"),
    (M, "h2 = f16(np.tanh(h1 @ W2.T + b2))", "h2 = np.tanh(h1 @ W2.T + b2)", "f16act layer 2 unrounded"),
    (M, "h3 = np.tanh(h2 @ W3.T + b3)", "h3 = f16(np.tanh(h2 @ W3.T + b3))", "f16act layer 3 rounded"),
    (M, "sizes = [(hidden, n_in), (hidden, hidden), (hidden, hidden), (n_out, hidden)]",
     "sizes = [(hidden, n_in), (hidden, hidden), (hidden, hidden), (hidden, n_out)]",
     "unpack last shape"),
    (M, "        b = theta[o:o + r]\n        o += r\n", "        b = theta[o:o + r] * 0\n        o += r\n", "unpack biases"),
    (M, "P[gi[~on], hi[~on]] += d[~on]", "P[gi[~on], hi[~on]] += np.conj(d[~on])", "apply upper conj"),
    (G, "        if not d > 0.0:\n", "        if d < 0.0:\n", "cholesky accepts a zero pivot"),
    (G, "alpha = 1.0 / np.max(np.sum(np.abs(A @ np.conj(A.T)), axis=1))",
     "alpha = 1.0 / np.max(np.abs(np.sum(A @ np.conj(A.T), axis=1)))",
     "newton alpha signed sums"),
    (G, "    nz = m2 > 0\n", "    nz = m2 >= 0\n", "coulomb head"),
    (G, "    n_in = psi.shape[0]\n", "    n_in = nv\n", "closure n_in"),
    (C, '/ (E_ha[v] - E_ha[nv + c]);', '/ (E_ha[nv + c] - E_ha[v]);', 'C loop sign'),
    (C, 'acc += 2.0 * conj(pv[r]) * pc[r] * conj(pc[rp]) * pv[rp]',
     'acc += 2.0 * pv[r] * conj(pc[r]) * pc[rp] * conj(pv[rp])',
     'C loop conj'),
    (C, 'acc += 2.0 * conj(pv[r]) * pc[r] * conj(pc[rp]) * pv[rp]',
     'acc += 1.0 * conj(pv[r]) * pc[r] * conj(pc[rp]) * pv[rp]',
     'C loop factor'),
    (C, "for (int c = 0; c < nc; ++c) {", "for (int c = 1; c < nc; ++c) {", "C loop drops the first c"),
    (C, "for (int v = 0; v < nv; ++v) {", "for (int v = 0; v < nv - 1; ++v) {", "C loop drops the last v"),
    (C, "const double complex *pc = psi + (size_t)(nv + c) * nr;", "const double complex *pc = psi + (size_t)c * nr;",
     "C loop unoccupied offset"),
    (C, "out[(size_t)(r - r0) * nr + rp] = acc;", "out[(size_t)(r - r0) * nr + (nr - 1 - rp)] = acc;",
     "C loop column order"),
]


PINS = ["test_oracle_pins.py", "test_oracle_mlp.py", "test_oracle_closure.py"]


def run_one(f, old, new, label, work):
    """Plant one mistake in a fresh copy of oracle/ and run the pins against it; True if caught."""
    if os.path.exists(work):
        shutil.rmtree(work)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    path = os.path.join(work, f)
    text = open(path).read()
    if old not in text:
        raise SystemExit(f"mutation '{label}': anchor not found in {f}")
    with open(path, "w") as fh:
        fh.write(text.replace(old, new, 1))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([work, ROOT]))
    tests = [os.path.join(ROOT, "tests", t) for t in PINS]
    r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-x", "-q", "-p", "no:cacheprovider"], cwd=work,
                       env=env, capture_output=True, text=True, timeout=1800)
    return r.returncode != 0


def main(argv):
    work = os.path.join(ROOT, "tests", "_build", "mutants")
    # the pins must pass on an unmodified copy
    assert not run_one(G, "HARTREE_EV = ", "HARTREE_EV = ", "none", work), "the pins fail on the oracle itself"
    chosen = [m for m in MUTATIONS if not argv or m[3] in argv]
    survivors = []
    for f, old, new, label in chosen:
        caught = run_one(f, old, new, label, work)
        print(f"{'caught  ' if caught else 'SURVIVED'} {label}", flush=True)
        if not caught:
            survivors.append(label)
    shutil.rmtree(work, ignore_errors=True)
    print(f"{len(chosen) - len(survivors)} of {len(chosen)} planted mistakes caught")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
