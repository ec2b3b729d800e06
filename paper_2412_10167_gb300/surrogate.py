"""J-interpolation surrogate: the network of mw3_mlp_* trained on propagation results.

The cumulative probability of Eq. cumulative-probability needs the probabilities of
every J; the paper computes a coarse set of J and interpolates the rest by
J-shifting (Eq. J-shifting-interpolation). Here a small network learns
P_J(E, v', j') from propagations at training J values (this library's propagation,
one batched context for all of them) and predicts intermediate J. An ensemble of
networks (different seeds) gives both the prediction (the mean) and its uncertainty
(the spread); a held-out J whose spread, times `spread_factor`, exceeds `fallback_dP`
anywhere falls back to propagation, so the decision needs no propagation of the J
values that pass. Energies where the packet's incoming amplitude |a(E)|^2 is below
`a2_floor` of its maximum carry no usable flux information (the probabilities divide
by it) and are left out of training and scoring. A separate propagation of every
held-out J measures the errors of the surrogate, the fallback result and the two
interpolations; it is evaluation, not part of the surrogate path.

State-resolved targets are the product-channel probabilities P_J(E, v', j') (summed over
Omega') of the initial electronic state when the workload enables product channels, else
the reactant-channel (v, j) probabilities projected at R_inf. (At high J the reactant
surface at R_inf = 11.5 bohr is not asymptotic, the centrifugal term there is 0.16 eV at
J = 46, and its elastic |S|^2 exceeds 1; the product surface has no such channel.)
"""
from __future__ import annotations

import copy
import time

import numpy as np

from . import mw3


def propagate_probabilities(cfg: dict, Js, steps: int, precision: str = "fp64", device: int = 0,
                            with_a2: bool = False):
    """Run one batched propagation over the J list; returns (E, P_total[J,E],
    P_state[J, v, j, E] for the initial electronic state (product channels when enabled),
    seconds[, |a(E)|^2])."""
    c = copy.deepcopy(cfg)
    c["J"] = list(Js)
    t0 = time.perf_counter()
    pr = mw3.Propagator(c, device=device, precision=precision)
    pr.propagate(steps)
    E, P, Pst = pr.probabilities()
    if c["analysis"].get("products"):
        Pst = pr.product_probabilities()
    secs = time.perf_counter() - t0
    a2 = pr.incoming_amplitude() if with_a2 else None
    pr.close()
    L0 = c["packet"]["elec0"]
    if with_a2:
        return E, P, Pst[:, L0], secs, a2
    return E, P, Pst[:, L0], secs


def features(J, E, v, j, scale):
    """Network inputs scaled to about [0, 1]: J, E, v', j' and the J-shifted energy
    E - B J(J+1) of the J-shifting model (B fitted on the training propagations), along
    which the probabilities of different J nearly coincide."""
    J = np.asarray(J, float)
    E = np.asarray(E, float)
    Es = E - scale["B"] * J * (J + 1.0)
    return np.stack([J / scale["J"], (E - scale["E0"]) / scale["dE"],
                     np.asarray(v, float) / scale["v"], np.asarray(j, float) / scale["j"],
                     (Es - scale["E0"]) / scale["dE"]], axis=-1).astype(np.float32)


def fit_shift(E, Jtr, Ptr):
    """Mean rotational constant B over the training intervals: least-squares overlay of
    the state-summed curve of J2, shifted by B [J2(J2+1) - J1(J1+1)], on that of J1."""
    from numpy import interp
    Bs = []
    for k in range(len(Jtr) - 1):
        J1, J2 = Jtr[k], Jtr[k + 1]
        dJ = J2 * (J2 + 1) - J1 * (J1 + 1)
        if dJ <= 0:
            continue
        t1, t2 = Ptr[k].sum(axis=(0, 1)), Ptr[k + 1].sum(axis=(0, 1))
        grid = np.linspace(0.0, (E[-1] - E[0]) / dJ, 801)
        err = [np.sum((t1 - interp(E + b * dJ, E, t2, left=t2[0], right=t2[-1])) ** 2) for b in grid]
        Bs.append(grid[int(np.argmin(err))])
    return float(np.mean(Bs)) if Bs else 0.0


def dataset(Js, E, Pst, scale):
    """Flatten P[J, v, j, E] into (X, y)."""
    nJ, nv, nj, nE = Pst.shape
    Jg, vg, jg, Eg = np.meshgrid(np.asarray(Js, float), np.arange(nv), np.arange(nj), E,
                                 indexing="ij")
    X = features(Jg.ravel(), Eg.ravel(), vg.ravel(), jg.ravel(), scale)
    return X, Pst.ravel().astype(np.float32)


def predict(net, Js, E, nv, nj, scale):
    Jg, vg, jg, Eg = np.meshgrid(np.asarray(Js, float), np.arange(nv), np.arange(nj), E,
                                 indexing="ij")
    y = net.forward(features(Jg.ravel(), Eg.ravel(), vg.ravel(), jg.ravel(), scale))
    return y.reshape(len(Js), nv, nj, len(E))


def jshift_baseline(E, Jtr, Ptr, Jte, fit=True):
    """J-shifting interpolation (Eq. J-shifting-interpolation) of every (v, j) curve
    between the bracketing training J values, with B fitted per interval on the
    state-summed probabilities."""
    from numpy import interp

    def shifted(P, dE):
        return interp(E - dE, E, P, left=P[0], right=P[-1])

    out = np.zeros((len(Jte),) + Ptr.shape[1:])
    for t, J in enumerate(Jte):
        k = np.searchsorted(Jtr, J) - 1
        k = min(max(k, 0), len(Jtr) - 2)
        J1, J2 = Jtr[k], Jtr[k + 1]
        tot1, tot2 = Ptr[k].sum(axis=(0, 1)), Ptr[k + 1].sum(axis=(0, 1))
        dJ = J2 * (J2 + 1) - J1 * (J1 + 1)
        B = 0.0
        if fit and dJ > 0:
            grid = np.linspace(0.0, (E[-1] - E[0]) / dJ, 801)
            errs = [np.sum((tot1 - shifted(tot2, -b * dJ)) ** 2) for b in grid]
            B = grid[int(np.argmin(errs))]
        w2 = (J - J1) / (J2 - J1)
        for v in range(Ptr.shape[1]):
            for j in range(Ptr.shape[2]):
                a = shifted(Ptr[k, v, j], B * (J * (J + 1) - J1 * (J1 + 1)))
                b = shifted(Ptr[k + 1, v, j], -B * (J2 * (J2 + 1) - J * (J + 1)))
                out[t, v, j] = (1 - w2) * a + w2 * b
    return out


def linear_baseline(Jtr, Ptr, Jte):
    out = np.zeros((len(Jte),) + Ptr.shape[1:])
    for t, J in enumerate(Jte):
        k = min(max(np.searchsorted(Jtr, J) - 1, 0), len(Jtr) - 2)
        w = (J - Jtr[k]) / (Jtr[k + 1] - Jtr[k])
        out[t] = (1 - w) * Ptr[k] + w * Ptr[k + 1]
    return out


def cumulative(Js, P):
    """Sum_J (2J + 1) P_J(E) summed over final states (Eq. cumulative-probability, one Omega0)."""
    Js = np.asarray(Js, float)
    return np.sum((2 * Js + 1)[:, None] * P.sum(axis=(1, 2)), axis=0)


def run(cfg: dict, J_train, J_test, steps: int, epochs: int = 1500, width: int = 256,
        depth: int = 3, lr: float = 2e-3, batch: int = 512, fallback_dP: float = 0.01,
        ensemble: int = 3, precision: str = "fp64", device: int = 0, seed: int = 10167,
        spread_factor: float = 2.0, a2_floor: float = 0.05, e_stride: int = 1,
        rule: str = "spread"):
    """Train on J_train, predict J_test with the fallback decided by the ensemble spread,
    then score everything against a propagation of J_test; returns a report dictionary.

    Each of `ensemble` networks (different initialisation and shuffling seeds) trains for
    `epochs` at `lr`, then epochs/2 at lr/4 and epochs/2 at lr/16 (the AdamW state carries
    over); the prediction is their mean, the uncertainty their standard deviation. The
    propagations run in `precision` ("fp64" or "mixed"). The networks train on every
    `e_stride`-th kept energy (the probabilities are smooth in E on the energy grid) and
    predict all of them. `rule` decides the fallback without propagating: "spread" (spread
    times `spread_factor` above `fallback_dP`), "linear" (the prediction differs from the
    linear interpolation in J of the neighbouring training values by more than
    `fallback_dP`), or "both" (either)."""
    E_all, _, Ptr_all, t_train, a2 = propagate_probabilities(cfg, J_train, steps, precision,
                                                              device=device, with_a2=True)
    keep = a2 >= a2_floor * np.max(a2)
    E = E_all[keep]
    Ptr = Ptr_all[..., keep]
    nv, nj = Ptr.shape[1], Ptr.shape[2]
    scale = dict(J=max(max(J_train), 1), E0=E[0], dE=max(E[-1] - E[0], 1e-12), v=max(nv - 1, 1),
                 j=max(nj - 1, 1), B=fit_shift(E, np.asarray(J_train, float), Ptr))
    X, y = dataset(J_train, E[::e_stride], Ptr[..., ::e_stride], scale)
    schedule = ((epochs, lr), (epochs // 2, lr / 4), (epochs // 2, lr / 16))
    losses, preds = [], []
    t_fit = t_pred = 0.0
    for k in range(max(1, ensemble)):
        net = mw3.MLP(n_in=X.shape[1], width=width, depth=depth, seed=seed + k, device=device)
        t0 = time.perf_counter()
        for ep, lr_k in schedule:
            if ep > 0:
                loss = net.train(X, y, epochs=ep, batch=batch, lr=lr_k, seed=seed + 7 * k)
        t_fit += time.perf_counter() - t0
        losses.append(loss)
        t0 = time.perf_counter()
        preds.append(predict(net, J_test, E, nv, nj, scale))
        t_pred += time.perf_counter() - t0
        net.close()
    preds = np.asarray(preds)
    Psur = preds.mean(axis=0)
    spread = preds.std(axis=0) if len(preds) > 1 else np.zeros_like(Psur)
    loss = float(np.mean(losses))
    # fallback decided without propagating the held-out J; only those J values are propagated
    Plin = linear_baseline(np.asarray(J_train), Ptr, np.asarray(J_test))
    by_spread = [spread_factor * spread[t].max() > fallback_dP for t in range(len(J_test))]
    by_linear = [np.abs(Psur[t] - Plin[t]).max() > fallback_dP for t in range(len(J_test))]
    flag = {"spread": by_spread, "linear": by_linear,
            "both": [a or b for a, b in zip(by_spread, by_linear)]}[rule]
    bad_J = [J for t, J in enumerate(J_test) if flag[t]]
    final = Psur.astype(np.float64)
    t_fallback = 0.0
    if bad_J:
        _, _, Pfb, t_fallback = propagate_probabilities(cfg, bad_J, steps, precision, device=device)
        for t, J in enumerate(J_test):
            if J in bad_J:
                final[t] = Pfb[bad_J.index(J)][..., keep]
    # evaluation: every held-out J propagated
    _, _, Pte_all, t_test = propagate_probabilities(cfg, J_test, steps, precision, device=device)
    Pte = Pte_all[..., keep]
    Pjs = jshift_baseline(E, np.asarray(J_train), Ptr, np.asarray(J_test))
    err = np.abs(Psur - Pte)
    C_true = cumulative(J_test, Pte)

    def crel(P):
        return float(np.abs(cumulative(J_test, P) - C_true).max() / max(C_true.max(), 1e-30))

    rep = dict(
        train_loss=loss, n_train=int(X.shape[0]), B_shift=scale["B"], ensemble=len(preds),
        energies_scored=int(keep.sum()), energies=int(keep.size), a2_floor=a2_floor,
        mean_abs_dP=dict(surrogate=float(err.mean()), jshift=float(np.abs(Pjs - Pte).mean()),
                         linear=float(np.abs(Plin - Pte).mean()),
                         with_fallback=float(np.abs(final - Pte).mean())),
        max_abs_dP=dict(surrogate=float(err.max()), jshift=float(np.abs(Pjs - Pte).max()),
                        linear=float(np.abs(Plin - Pte).max()),
                        with_fallback=float(np.abs(final - Pte).max())),
        cumulative_rel_err=dict(surrogate=crel(Psur), jshift=crel(Pjs), linear=crel(Plin),
                                with_fallback=crel(final)),
        fallback_J=bad_J, fallback_fraction=len(bad_J) / len(J_test),
        spread_factor=spread_factor, rule=rule, e_stride=e_stride,
        # per held-out J: largest error over largest ensemble spread (calibration of the rule)
        error_over_spread=[float(err[t].max() / max(spread[t].max(), 1e-30))
                           for t in range(len(J_test))],
        passed_J_max_abs_dP=float(max([err[t].max() for t, J in enumerate(J_test) if J not in bad_J],
                                      default=0.0)),
        max_P_propagated=float(Pte.max()),
        # every rule on the same predictions (the evaluation propagation stands in for its
        # fallback propagations)
        rules={name: dict(
            fallback_J=[J for t, J in enumerate(J_test) if f[t]],
            max_abs_dP=float(max(np.abs(np.where(f[t], Pte[t], Psur[t]) - Pte[t]).max()
                                 for t in range(len(J_test)))),
            passed_J_max_abs_dP=float(max([err[t].max() for t in range(len(J_test)) if not f[t]],
                                          default=0.0)),
            cumulative_rel_err=crel(np.asarray([Pte[t] if f[t] else Psur[t]
                                                for t in range(len(J_test))])))
            for name, f in (("spread", by_spread), ("linear", by_linear),
                            ("both", [a or b for a, b in zip(by_spread, by_linear)]))},
        seconds=dict(propagate_train=t_train, fit=t_fit, predict=t_pred,
                     propagate_fallback=t_fallback, propagate_all_test=t_test,
                     surrogate_path=t_fit + t_pred + t_fallback),
    )
    return rep


def c5_config():
    """The J-interpolation workload: the config-3 grid with a single electronic surface,
    Omega up to 15, the configured energy window and final-state ranges."""
    import workloads as W
    c5 = W.C5
    cfg = copy.deepcopy(c5["base"])
    cfg["pes"]["two_state"] = None
    cfg["nelec"] = 1
    cfg["analysis"].update(nE=c5["nE"], E_lo_eV=c5["E_lo_eV"], E_hi_eV=c5["E_hi_eV"],
                           vmax=c5["vmax"], jmax=c5["jmax"])
    return cfg


def main(argv=None):
    """python -m paper_2412_10167_gb300.surrogate [--epochs 60 ...]: the J-interpolation
    workload end to end (training propagations, ensemble training, fallback, evaluation)."""
    import argparse
    import json
    import workloads as W
    ap = argparse.ArgumentParser(description=main.__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--ensemble", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--spread-factor", type=float, default=2.0)
    ap.add_argument("--e-stride", type=int, default=1,
                    help="train on every n-th energy of the grid (all are predicted)")
    ap.add_argument("--rule", default="spread", choices=["spread", "linear", "both"],
                    help="fallback decision made without propagating the held-out J")
    args = ap.parse_args(argv)
    rep = run(c5_config(), W.C5["J_train"], W.C5["J_test"], steps=args.steps,
              epochs=args.epochs, batch=args.batch, ensemble=args.ensemble,
              precision=args.precision, fallback_dP=W.C5["fallback_dP"],
              spread_factor=args.spread_factor, e_stride=args.e_stride, rule=args.rule)
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
