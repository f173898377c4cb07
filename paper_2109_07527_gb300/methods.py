"""Move sets built from invocations of the CR-MC kernels (host orchestration
through the C ABI; every trial runs on the GPU).

The paper's scheme, Eqs. (acid_new)-(salt_new), becomes the conventional
reaction ensemble (RxMC) when X+ = H+ and X- = OH- (pI_X+ = pH, pI_X- = pOH),
and the grand-reaction ensemble when it is applied separately to dissociated
and salt ions (Sec. II.B; App. B: the method invoked repeatedly with
different types of ions).  Types: CR_XP / CR_XM stand for H+ / OH- under
those invocations, CR_SP / CR_SM for the salt ions S+ / S-.

``compare_convergence`` runs the method comparison of Sec. III.A (Fig. 2):
the degree of dissociation of the same random weak-acid configurations
under CR-MC, the grand-reaction ensemble and RxMC, averaged over replicas
that run side by side in one batch per method.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

XP, XM, SP, SM = W.XP, W.XM, W.SP, W.SM


def rxmc_invocation(pH: float, pKw: float = 14.0):
    """(cation, anion, pI_cation, pI_anion, reactions) of RxMC: every move."""
    return (XP, XM, pH, pKw - pH, 7)


def grand_reaction_invocations(pH: float, pIS_plus: float, pIS_minus: float, pKw: float = 14.0,
                               reactions: int = 7):
    """The four invocations of the grand-reaction ensemble with the share of
    the trials each gets so that every reaction is attempted equally often:
    (H+, OH-) and (S+, S-) with the site and salt moves (2 shares each), the
    mixed salt pairs (H+, S-) and (S+, OH-) with the salt move (1 share each).
    `reactions` selects the site moves (acid 1, base 2) of the first two."""
    pOH = pKw - pH
    site = reactions & 3
    return [((XP, XM, pH, pOH, site | 4), 2), ((SP, SM, pIS_plus, pIS_minus, site | 4), 2),
            ((XP, SM, pH, pIS_minus, 4), 1), ((SP, XM, pIS_plus, pOH, 4), 1)]


def compare_convergence(crmc, n_rep=64, blocks=40, m=250, n_acid=500, seed=1, methods=("crmc", "grxmc", "rxmc"),
                        ewald_kmax=0):
    """alpha(trials) of the weak-acid electrolyte (Sec. III.A) under each
    method.  A block is 6 x m trials per replica (6 batch sweeps of m trials:
    all moves of CR-MC and RxMC; the grand-reaction invocations in the shares
    2:2:1:1).  ewald_kmax > 0: Ewald electrostatics (the paper's PPPM energy,
    as a direct Ewald sum with reciprocal vectors |n| <= ewald_kmax) instead of
    DSF.  Returns {"trials": [...], method: mean alpha per block, method +
    "_se": its standard error over the replicas, method + "_sweep_s": the
    wall time of its batch sweeps in the second half of the blocks, after the
    launch-shape tuner's sweeps}."""
    import time
    out = {"trials": [6 * m * (b + 1) for b in range(blocks)]}
    for method in methods:
        ws = [W.weak_acid_electrolyte(n_acid=n_acid, seed=seed + r, trials_per_domain=m) for r in range(n_rep)]
        for w in ws:
            w.params["ewald_kmax"] = int(ewald_kmax)
        ctxs = [crmc.Context(w) for w in ws]
        b = crmc.Batch(ctxs)
        pH = float(ws[0].params["pH"])
        pS = float(ws[0].params["pIS_plus"]), float(ws[0].params["pIS_minus"])
        if method == "rxmc":
            for c in ctxs:
                c.set_invocation(*rxmc_invocation(pH))
        inv = grand_reaction_invocations(pH, *pS, reactions=1)
        alpha = np.zeros((blocks, n_rep))
        k = 0
        t_sweep = 0.0
        for blk in range(blocks):
            t0 = time.perf_counter()
            if method == "grxmc":
                for args, share in inv:
                    for c in ctxs:
                        c.set_invocation(*args)
                    b.sweep(share, 7919 * seed + k)
                    k += 1
            else:
                b.sweep(6, 7919 * seed + k)
                k += 1
            ctxs[0].check()  # the batch's stream is synchronised: the sweeps are done
            if blk >= blocks // 2:
                t_sweep += time.perf_counter() - t0
            for r, c in enumerate(ctxs):
                alpha[blk, r] = c.counts()["alpha"]
        for c in ctxs:
            c.check()
        b.close()
        for c in ctxs:
            c.close()
        out[method] = alpha.mean(axis=1).tolist()
        out[method + "_sweep_s"] = t_sweep
        out[method + "_se"] = (alpha.std(axis=1, ddof=1) / np.sqrt(n_rep)).tolist()
    return out
