"""The rule behind the candidate x-step, checked on the host against the FP64 oracle.

The GPU x-step first keeps the entries of v above a guess G (from last sweep's threshold) and runs
the operator of Section 2.1 on those candidates alone.  It accepts G only when the operator's
threshold provably lies above it:
- T_s (forms 1, 2): at least s candidates;
- the gamma-targeting rule (forms 5-8 while calibrating): at least s + 1 candidates;
- lambda_s (forms 3, 4): phi(G) = s ||V_G(v)||_2^2 - ||V_G(v)||_1^2 < 0 over the candidates (phi
  has the sign of g'(lambda) for the convex g of Section 2.1, so lambda_s > G);
- a fixed penalty threshold: G is the threshold itself.
Then the x-step on the candidates, scattered back, must be the x-step on all of v: the same x,
F and threshold.  A model of the filter (16 index segments, 64 candidates each, two guesses,
moving a segment to the higher guess when its list would overflow) drives the oracle here, so a
wrong acceptance rule fails this test without a GPU."""
import numpy as np
import pytest

W_CAP, WARPS = 64, 16


def filter_model(v, G_lo, G_hi):
    """(candidate indices, guess) as the filter forms them, or None when a list overflows at G_hi."""
    p = v.size
    seg = ((p + WARPS - 1) // WARPS + 127) // 128 * 128
    a = np.abs(v)
    lists, raised = [], False
    for w in range(WARPS):
        lo, hi = min(p, w * seg), min(p, (w + 1) * seg)
        idx = lo + np.flatnonzero(a[lo:hi] > G_lo)
        if idx.size > W_CAP:
            idx = lo + np.flatnonzero(a[lo:hi] > G_hi)
            raised = True
            if idx.size > W_CAP:
                return None
        lists.append(idx)
    cand = np.concatenate(lists)
    G = G_hi if raised else G_lo
    return cand[a[cand] > G], G


def phi(a, s, G):
    w = a[a > G] - G
    return s * np.sum(w * w) - np.sum(w) ** 2


def accept(form, v, cand, G, s, calibrate):
    a = np.abs(v[cand])
    if form in (1, 2):
        return cand.size >= s
    if form in (3, 4):
        return phi(np.abs(v), s, 0.0) < 0 and cand.size >= 1 and phi(a, s, G) < 0
    if calibrate:
        return cand.size >= s + 1
    return True


def operator_choice(form, v, cand, G_lo, G_hi, used, s, calibrate):
    """The operator's choice: G_hi when valid (cutting a G_lo list), else the list's own guess."""
    if used == G_lo and G_lo != G_hi:
        hi = cand[np.abs(v[cand]) > G_hi]
        if accept(form, v, hi, G_hi, s, calibrate):
            return hi, G_hi
    return (cand, used) if accept(form, v, cand, used, s, calibrate) else (None, None)


def vectors(rng, p):
    yield rng.standard_normal(p)
    yield rng.standard_t(2, p)                              # heavy tails
    v = rng.standard_normal(p); v[::5] = 0.0; yield v       # exact zeros
    v = rng.standard_normal(p); v[100:160] = v[7]; yield v  # a run of equal magnitudes
    v = rng.standard_normal(p) * 0.05; v[rng.choice(p, 40, replace=False)] += rng.choice([-3, 3], 40); yield v


@pytest.mark.parametrize("form", range(1, 9))
def test_candidate_rule_gives_the_full_x_step(oracle, form):
    rng = np.random.default_rng(700 + form)
    p = 5000
    accepted = fallback = 0
    for s in (5, 40, 120):
        for v in vectors(rng, p):
            for calibrate in ((False, True) if form >= 5 else (False,)):
                gamma = 0.0
                if form >= 5 and not calibrate:
                    t_fix = float(np.sort(np.abs(v))[::-1][s])
                    gamma = t_fix * t_fix if form in (5, 6) else t_fix
                full = oracle.xstep(form, v, s, gamma, calibrate)
                t_true = abs(full.thr) if form in (3, 4, 7, 8) else float(np.sort(np.abs(v))[::-1][min(s, p) - 1])
                for ratio in (0.5, 0.8, 0.95, 1.0, 1.1, 1.3, 2.0):       # last sweep's threshold t / this one
                    t = ratio * t_true
                    if form >= 5 and not calibrate:
                        G_lo = G_hi = np.sqrt(gamma) if form in (5, 6) else gamma
                    else:
                        G_lo, G_hi = 0.6 * t, 0.85 * t
                    f = filter_model(v, G_lo, G_hi)
                    if f is None:
                        fallback += 1
                        continue
                    cand, used = f
                    cand, G = operator_choice(form, v, cand, G_lo, G_hi, used, s, calibrate)
                    if cand is None:
                        fallback += 1
                        continue
                    accepted += 1
                    part = oracle.xstep(form, v[cand], s, gamma, calibrate)
                    x = np.zeros(p)
                    x[cand] = part.x
                    assert np.array_equal(x, full.x), (s, ratio, calibrate)
                    assert part.F == full.F and part.nnz == full.nnz and part.thr == full.thr
    assert accepted > 0 and fallback > 0
