"""Exact click-pattern sampling by the chain rule.

The marginal of a Gaussian state on modes 1..j is the Gaussian with the
covariance Sigma_j restricted to those modes' quadratures, so the probability
of a prefix pattern (s_1..s_j) is Eq. 1 in that reduced state:
    p(s_1..s_j) = Tor(O_j restricted to the clicked modes) / sqrt(det Sigma_j),
    O_j = I - Sigma_j^-1.
Mode j is then drawn from p(s_j = 1 | s_1..s_{j-1}), one batched Torontonian
per sample and mode (tor_batch_patterns on O_j), in one of two forms:
  "noclick" (default): p(s_1..s_{j-1}, 0), whose clicked set is the prefix's
      (k clicks, 2^k subsets); p(s_j = 1 | prefix) = 1 - p(prefix, 0) / p(prefix);
  "click": p(s_1..s_{j-1}, 1) (k + 1 clicks, twice the subsets), with
      p(prefix, 0) = p(prefix) - p(prefix, 1).
The no-click form halves the work.  It forms a small click probability as a
difference, so its relative error there is about tol / p(s_j = 1 | prefix).
Probabilities are carried as logarithms.  Samples that exceed k_max clicks stop
early and are drawn again; those below k_min at the end are drawn again too, so
the result is an exact sample of p(S | k_min <= |S| <= k_max) up to the
accuracy of the Torontonians (the tier and tolerance given).
"""
from __future__ import annotations

import numpy as np


def reduced_O(Sigma: np.ndarray, j: int):
    """O_j = I - Sigma_j^-1 (2j x 2j, xxpp) of the first j modes and log det Sigma_j."""
    M = Sigma.shape[0] // 2
    idx = list(range(j)) + list(range(M, M + j))
    S = Sigma[np.ix_(idx, idx)]
    Si = np.linalg.inv(S)
    O = np.eye(2 * j) - 0.5 * (Si + Si.T)
    return O, float(np.linalg.slogdet(S)[1])


def sample(ctx, Sigma: np.ndarray, n: int, seed: int, k_min: int = 0, k_max: int | None = None,
           prec: str = "auto", tol: float = 1e-6, max_rounds: int = 50, form: str = "noclick",
           stats: dict | None = None, evaluate=None):
    """n patterns (uint8 array (n, M)) drawn exactly from p(S | k_min <= |S| <= k_max).
    stats, if given, receives the number of Torontonians and subset determinants evaluated.
    evaluate(j, O_j, cand) -> (Tor values, usable flags) replaces the batched GPU evaluation
    of the Torontonians of O_j restricted to each row's clicks (for tests of this logic)."""
    if form not in ("noclick", "click"):
        raise ValueError("form must be 'noclick' or 'click'")
    M = Sigma.shape[0] // 2
    k_max = M if k_max is None else k_max
    rng = np.random.default_rng(seed)
    mats = [None] + [reduced_O(Sigma, j) for j in range(1, M + 1)]
    if evaluate is None:
        evaluate = _gpu_evaluator(ctx, mats, prec, tol)
    out = []
    for _ in range(max_rounds):
        need = n - sum(len(x) for x in out)
        if need <= 0:
            break
        m = max(need, 64)
        pats = np.zeros((m, M), dtype=np.uint8)
        logp = np.zeros(m)               # log p(prefix); the empty prefix has probability 1
        alive = np.ones(m, dtype=bool)
        for j in range(1, M + 1):
            live = np.nonzero(alive)[0]
            if live.size == 0:
                break
            cand = pats[live, :j].copy()
            cand[:, j - 1] = 1 if form == "click" else 0
            if stats is not None:
                stats["torontonians"] = stats.get("torontonians", 0) + live.size
                stats["subsets"] = stats.get("subsets", 0.0) + float((2.0 ** cand.sum(1)).sum())
            val, ok = evaluate(j, mats[j][0], cand)
            if not np.all(ok):   # every p(S) of a Gaussian state is positive: a failure is an error
                raise RuntimeError(f"{int((~np.asarray(ok)).sum())} prefix Torontonians failed at mode {j}")
            logv = np.log(val) - 0.5 * mats[j][1]
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = np.clip(np.exp(logv - logp[live]), 0.0, 1.0)
                cond = ratio if form == "click" else 1.0 - ratio  # p(s_j = 1 | prefix)
                click = rng.random(live.size) < cond
                pats[live, j - 1] = click
                if form == "click":      # cond = 1 forces a click
                    logp[live] = np.where(click, logv, logp[live] + np.log1p(-cond))
                else:                    # cond = 0 forbids one
                    logp[live] = np.where(click, logp[live] + np.log(cond), logv)
            alive[live[pats[live].sum(1) > k_max]] = False          # over the cap: stop, redraw
        k = pats.sum(1)
        good = alive & (k >= k_min) & (k <= k_max)
        out.append(pats[good][:need])
    res = np.concatenate(out) if out else np.zeros((0, M), dtype=np.uint8)
    if len(res) < n:
        raise RuntimeError(f"only {len(res)} of {n} samples within [{k_min}, {k_max}] clicks")
    return res[:n]


def _gpu_evaluator(ctx, mats, prec, tol):
    """Tor of O_j restricted to each candidate's clicks, one tor_batch_patterns call per mode."""
    import torch
    from . import tor
    dev = [None] + [torch.from_numpy(O).cuda() for O, _ in mats[1:]]

    def evaluate(j, Oj, cand):
        res = tor.results_array(_batch(ctx, dev[j], cand, prec, tol), cand.shape[0])
        val = res["hi"] + res["lo"]
        # a result that misses the tolerance (TOR_EPREC) is still the best value there is
        ok = ((res["status"] == tor.TOR_OK) | (res["status"] == tor.TOR_EPREC)) & (val > 0)
        return val, ok
    return evaluate


def _batch(ctx, Od, cand, prec, tol):
    import torch
    from . import tor
    M = Od.shape[0] // 2
    P = tor.pack_patterns(cand, M).to(Od.device)
    o = torch.zeros(cand.shape[0] * tor.RESULT_BYTES, dtype=torch.uint8, device=Od.device)
    ctx.batch_patterns_async(Od, P, o, prec=prec, tol=tol)
    return o


def exact_log_prob(table_p: np.ndarray, pats: np.ndarray) -> np.ndarray:
    """log p of patterns from a full probability table (index = mask, bit j = mode j)."""
    codes = (pats.astype(np.int64) << np.arange(pats.shape[1])[None, :]).sum(1)
    return np.log(np.maximum(table_p[codes], 1e-300))


def tv_against_table(table_p: np.ndarray, pats: np.ndarray) -> float:
    """Total-variation distance between the empirical distribution of pats and table_p."""
    codes = (pats.astype(np.int64) << np.arange(pats.shape[1])[None, :]).sum(1)
    freq = np.bincount(codes, minlength=table_p.size) / len(codes)
    return 0.5 * float(np.abs(freq - table_p).sum())

