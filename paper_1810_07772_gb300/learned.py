"""Learned truncation correction of P~(G,G'): training data from the plain method and the
training loop, driving the library's kernels (gw_corr_*, gw_mlp_*).

The arithmetic, the training loop, the minibatch order and the learning-rate schedule run in the
library.  This module calls the C ABI in order:

1. For every seeded system, run the plain method twice: P~ with the nc_keep lowest unoccupied
   states, and P~ with all of them.  The sum over unoccupied states c is the one in
   Eq. (Pstatic).  Both go by the g-space route (gw_build_PG) unless route="rspace" asks for
   P(r,r') and its transforms.  With the kept states loaded, the closure estimate dP~ of the
   omitted part follows from the omitted states' energies alone (gw_corr_closure).
2. Compute the per-entry features of the truncated P~ (with dP~) and the targets
   s (P~_all - P~_keep - dP~), what the closure estimate leaves (gw_corr_features,
   gw_corr_targets).
3. Run Adam on minibatches drawn without replacement from all systems' entries, with a cosine
   learning-rate decay (gw_corr_train).
4. Inference: the closure estimate and the features of a new truncated P~, the forward pass,
   then add both into P~ (gw_corr_apply).  eps and eps^-1 then follow as for any P~.
"""
from __future__ import annotations

import numpy as np

from . import gw


def states_in_real_space(ctx, coef, gvec, E_eV, dims, nv):
    """States given as plane-wave coefficients, loaded through gw_load_states_g (the library's
    transform of the DFT input to the grid) and returned on the grid as a [nv + nc][N_r] complex64
    device tensor (a copy of the context's transposed states)."""
    ctx.load_states_g(coef, gvec, E_eV, dims, nv)
    return ctx.view("psiT").t().contiguous()


def build_PG(ctx, gcut, precision="fp16x3", route="gspace"):
    """P~ of the loaded states by either route; returns the G-vectors."""
    if route == "gspace":
        return ctx.build_PG(gcut, precision)
    ctx.build_P(precision)
    return ctx.P_to_G(gcut)


def truncated_pair(ctx, psi, E_eV, nv, nc_keep, dims, gcut, precision="fp16x3", route="gspace"):
    """(P~_keep, P~_all, dP~, gvec) of one system, dP~ the closure estimate of P~_all - P~_keep from
    the kept states and the omitted energies.  psi: [nv + nc_all][N_r] device tensor."""
    E = np.asarray(E_eV, dtype=np.float64)
    ctx.load_states(psi[: nv + nc_keep], E[: nv + nc_keep], dims, nv)
    gvec = build_PG(ctx, gcut, precision, route)
    PG_keep = ctx.view("PG").clone()
    clos = ctx.corr_closure(gcut, E[nv + nc_keep:])
    ctx.load_states(psi, E, dims, nv)
    build_PG(ctx, gcut, precision, route)
    PG_all = ctx.view("PG").clone()
    return PG_keep, PG_all, clos, gvec


def system_samples(ctx, psi, E_eV, nv, nc_keep, dims, gcut, precision="fp16x3", route="gspace"):
    """Features, targets and the pieces needed to judge a prediction, for one system."""
    PG_keep, PG_all, clos, gvec = truncated_pair(ctx, psi, E_eV, nv, nc_keep, dims, gcut, precision, route)
    ratio = gw.corr_weight_ratio(E_eV, nv, nc_keep, device=PG_keep.device.index)
    X, scale = gw.corr_features(PG_keep, gvec, gcut, ratio, clos)
    T = gw.corr_targets(PG_keep, PG_all, scale, clos)
    return {"X": X, "T": T, "scale": scale, "ratio": ratio, "PG_keep": PG_keep, "PG_all": PG_all, "clos": clos,
            "gvec": gvec}


def training_set(ctx, make_states, seeds, nv, nc_keep, dims, gcut, precision="fp16x3", route="gspace"):
    """Concatenated (X, T) over the seeded systems; make_states(seed) -> (psi on device, E_eV)."""
    import torch

    Xs, Ts = [], []
    for s in seeds:
        psi, E = make_states(s)
        d = system_samples(ctx, psi, E, nv, nc_keep, dims, gcut, precision, route)
        Xs.append(d["X"])
        Ts.append(d["T"])
        del psi, d
    return torch.cat(Xs), torch.cat(Ts)


def train(mlp, X, T, epochs=4, batch=8192, lr=1e-3, lr_final=1e-5, seed=0, beta1=0.9, beta2=0.999, eps=1e-8,
          diag_repeat=1):
    """Adam over `epochs` passes of minibatches without replacement, cosine learning-rate decay from
    lr to lr_final, the diagonal entries (feature 7 set) diag_repeat times in the pool a pass draws
    from (gw_corr_train: the loop, the order and the schedule run in the library).  Diagonal
    entries carry most of the correction's norm but are 1 in ng(ng+1)/2 of the entries, so without
    the repeats their fit is left to few, noisy updates.  Returns the mean loss of each pass."""
    return mlp.train_corr(X, T, epochs, batch, lr, lr_final=lr_final, seed=seed, diag_repeat=diag_repeat,
                          diag_feature=7, beta1=beta1, beta2=beta2, eps=eps)


def correct(mlp, PG_keep, gvec, gcut, E_eV, nv, nc_keep, clos, out=None, tensor_cores=True):
    """Learned form: P~_keep plus the closure estimate clos (gw_corr_closure on the kept states)
    plus the network's prediction of what it leaves (in `out`, or a new tensor).  The prediction
    runs on the tensor cores (gw_mlp_infer) unless tensor_cores=False asks for the FP32 forward of
    training (gw_mlp_forward)."""
    ratio = gw.corr_weight_ratio(E_eV, nv, nc_keep, device=PG_keep.device.index)
    X, scale = gw.corr_features(PG_keep, gvec, gcut, ratio, clos)
    Y = mlp.infer(X) if tensor_cores else mlp.forward(X)
    P = PG_keep.clone() if out is None else out
    if out is not None and out.data_ptr() != PG_keep.data_ptr():
        P.copy_(PG_keep)
    gw.corr_apply(P, Y, scale, clos)
    return P
