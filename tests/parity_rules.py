"""Parity rules shared by the GPU <-> oracle tests of the dilepton kinds, whose FP32
inputs feed an ill-conditioned neutrino solution: each point's tolerance comes from the
oracle's own measure of its conditioning (test_oracle_conditioning.py checks that
measure on the CPU). Test infrastructure: imported by tests only."""
import numpy as np
import pytest


def sensitivity(O, P, T, rec, event_id, perm, seed, idx, d, grid=None):
    """Conditioning of the oracle's weight of point idx: the sum over the coordinates
    of the relative change of the weight when that coordinate of the point's
    unit-cube point moves by 2^-24 (the FP32 spacing of u in [1/2, 1); towards 1/2,
    so that it stays inside the cube), through the VEGAS map when a grid is given."""
    def weight(u):
        if grid is None:
            return O.integrand(P, T, rec, perm, u)
        x, jac, _ = O.vegas_map(grid, u)
        return O.integrand(P, T, rec, perm, x) * jac

    u = O.point_u(seed, event_id, perm, idx, d)
    w = weight(u)
    s = 0.0
    for k in range(d):
        v = u.copy()
        v[k] += 2.0 ** -24 if u[k] < 0.5 else -(2.0 ** -24)
        s += abs(weight(v) / w - 1.0)
    return s


# The kernels round each Breit-Wigner map's output q^2 to FP32; that rounding is
# worth a move of u up to m / (pi Gamma) times the 2^-24 of the sensitivity above
# (the map's slope at the pole: 39 for the top quark, 12 for the W), so a point may
# differ from the oracle by COND_FACTOR times its sensitivity. The cap stays far
# below what a missed or spurious neutrino solution does to a point (one of the 2-4
# summed solutions: an O(1) change) and binds only points whose weight moves by
# more than 5e-4 under a single FP32 step of one coordinate.
COND_FACTOR = 100.0
COND_CAP = 5e-2


def check_conditioned(w_gpu, w_ora, ctx, rel, frac, sum_rel, floor=1e-6):
    """Per-point rule for integrands whose FP32 inputs feed an ill-conditioned FP64
    solution (the dilepton neutrinos next to a branch point): over the points where
    either side is nonzero, the same zero pattern (one edge point allowed), a
    fraction >= frac within rel (plus floor x the mean weight), every point within
    min(COND_CAP, max(rel, COND_FACTOR s_i)) with s_i the oracle's sensitivity
    (computed for the points beyond rel only), and the sum over the points that are
    within rel or well conditioned (COND_FACTOR s_i <= rel) within sum_rel. The
    fraction allows at least one point beyond rel (batches with few points in the
    kinematic region).
    ctx = (O, P, T, rec, event_id, perm, seed, point0, d, grid). Returns the sums of
    both sides and the summed absolute bound of the ill-conditioned points."""
    O, P, T, rec, event_id, perm, seed, point0, d, grid = ctx
    nz = (w_gpu != 0) | (w_ora != 0)
    assert np.count_nonzero((w_gpu == 0) != (w_ora == 0)) <= 1
    scale = np.mean(np.abs(w_ora[nz])) if nz.any() else 0.0
    dw = np.abs(w_gpu - w_ora)
    close = dw <= rel * np.abs(w_ora) + floor * scale
    n_beyond = np.count_nonzero(nz & ~close)
    assert n_beyond <= max(1, int((1.0 - frac) * np.count_nonzero(nz))), (n_beyond, np.count_nonzero(nz))
    keep = nz.copy()
    far_bound = 0.0
    for i in np.flatnonzero(nz & ~close):
        assert w_ora[i] != 0 and w_gpu[i] != 0, i
        s = sensitivity(O, P, T, rec, event_id, perm, seed, point0 + int(i), d, grid)
        bound = min(COND_CAP, max(rel, COND_FACTOR * s))
        assert dw[i] <= bound * abs(w_ora[i]) + floor * scale, (i, dw[i] / abs(w_ora[i]), s)
        if COND_FACTOR * s > rel:
            keep[i] = False
            far_bound += bound * abs(w_ora[i]) + floor * scale
    assert np.sum(w_gpu[keep]) == pytest.approx(np.sum(w_ora[keep]), rel=sum_rel, abs=0)
    return np.sum(w_gpu), np.sum(w_ora), far_bound


def check_frozen_integral(g_prob, o_prob, parts, sum_rel):
    """Frozen-grid integrals of one event from mem_integrate and the oracle, given the
    per-assignment results of check_conditioned on the same points: the integrators
    add nothing to the per-point differences (the ratio of the integrals equals that
    of the point sums to 1e-7: FP32 Kahan sums per thread), and the integrals agree
    within sum_rel plus the ill-conditioned points' bounds."""
    G = sum(p[0] for p in parts)
    Ox = sum(p[1] for p in parts)
    bound = sum(p[2] for p in parts)
    assert g_prob / o_prob == pytest.approx(G / Ox, rel=1e-7, abs=0)
    assert abs(g_prob / o_prob - 1.0) <= sum_rel + bound / Ox, (g_prob / o_prob - 1.0, bound / Ox)
