"""GPU-vs-oracle comparison used by the parity tests.

Tolerances (stated for the FP32 GPU path against the FP64 oracle):
  * cell indices and per-point decisions (outside / fused / rejected / wall)
    bit-exact, except points the oracle flags as marginal: the exact value lies
    within 1e-6 (absolute) plus a few FP32 roundings of the operands of the
    decision's threshold (cell edge, Mahalanobis k, h for the wall rule, range
    limits);
  * heights |dh| <= 1e-5 m, variances relative <= 1e-4, last-update index exact;
  * removed cells (visibility) equal, except cells flagged mark-marginal;
  * normals / smoothing / in-painting <= 1e-5 absolute, except cells whose
    stencil window touches a marginal cell.
Cells that a marginal decision may change (a marginal point's cell and the
cells float32 binning may give it instead; a cell a marginal ray sample may
mark) are excluded from the comparison and counted.  Every comparison bounds
that count as a fraction of the valid cells: 1 % unless a test states a reason
for a wider bound.
"""
from __future__ import annotations

import numpy as np

import oracle

H_TOL = 1e-5
VAR_RTOL = 1e-4
STENCIL_TOL = 1e-5
ABS_BAND = 1e-6


def f32(x: float) -> float:
    return float(np.float32(x))


def oracle_params(P: dict) -> "oracle.Params":
    """The oracle sees the same float32-rounded parameters the library gets."""
    out = {}
    for k, v in P.items():
        out[k] = f32(v) if isinstance(v, float) else v
    return oracle.Params(**out)


def dilate(mask: np.ndarray, r: int) -> np.ndarray:
    out = mask.copy()
    H, W = mask.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sy0, sy1 = max(0, -dy), min(H, H - dy)
            sx0, sx1 = max(0, -dx), min(W, W - dx)
            out[sy0:sy1, sx0:sx1] |= mask[sy0 + dy:sy1 + dy, sx0 + dx:sx1 + dx]
    return out


class Comparison:
    def __init__(self):
        self.notes = {}

    def note(self, k, v):
        self.notes[k] = v


MAX_EXCLUDED = 0.01


def compare_update(om_trace, o_state: dict, g_state: dict, g_trace=None, wall_on: bool = False,
                   check_stencils=("nx", "ny", "nz", "smooth", "inpaint"), prior_valid=None,
                   max_excluded: float = MAX_EXCLUDED) -> Comparison:
    """Assert parity of one update; returns counts of what was excluded.
    max_excluded bounds the value- and mark-marginal cells, each as a fraction
    of the oracle's valid cells after the update."""
    cmp = Comparison()
    tr = om_trace
    value_m = (tr.cflags & oracle.CF_VALUE) != 0
    mark_m = (tr.cflags & oracle.CF_MARK) != 0
    cmp.note("value_marginal_cells", int(value_m.sum()))
    cmp.note("mark_marginal_cells", int(mark_m.sum()))
    n_valid = max(1, int(np.isfinite(o_state["var"]).sum()))
    assert value_m.sum() <= max_excluded * n_valid, \
        f"{value_m.sum()} value-marginal cells of {n_valid} valid exceed {max_excluded:.1%}"
    assert mark_m.sum() <= max_excluded * n_valid, \
        f"{mark_m.sum()} mark-marginal cells of {n_valid} valid exceed {max_excluded:.1%}"

    # ---- per-point cells and decisions
    if g_trace is not None:
        gix, giy, gst = g_trace
        ost = tr.status
        pf = tr.pflags
        exact = pf == 0
        # non-finite is decided without arithmetic: always exact
        assert np.array_equal(gst[ost == 0] == 0, np.ones((ost == 0).sum(), bool)), "non-finite points"
        valid = exact & (ost >= oracle.ST_OUTSIDE)
        bad = valid & ((gix != tr.ix) | (giy != tr.iy))
        assert not bad.any(), f"cell index mismatch on {bad.sum()} points, e.g. {np.flatnonzero(bad)[:5]}"
        dec = exact.copy()
        if wall_on:  # a wall decision depends on the cell's count, which a marginal point may change
            inmap = (ost >= oracle.ST_ACCEPT)
            cell_m = np.zeros_like(dec)
            ix = np.clip(tr.ix, 0, value_m.shape[1] - 1)
            iy = np.clip(tr.iy, 0, value_m.shape[0] - 1)
            cell_m[inmap] = value_m[iy[inmap], ix[inmap]]
            dec &= ~cell_m
        mism = dec & (gst != ost)
        assert not mism.any(), (f"decision mismatch on {mism.sum()} points: "
                                f"gpu {gst[mism][:8]} oracle {ost[mism][:8]}")
        cmp.note("marginal_points", int((~exact).sum()))

    # ---- cell state
    gv = np.isfinite(g_state["var"])
    ov = np.isfinite(o_state["var"])
    excl = value_m | mark_m
    vm = gv != ov
    assert not (vm & ~excl).any(), f"validity mismatch on {(vm & ~excl).sum()} cells"
    both = gv & ov & ~excl
    dh = np.abs(g_state["h"].astype(np.float64) - o_state["h"])
    assert np.all(dh[both] <= H_TOL), f"height error {dh[both].max():.3g} > {H_TOL}"
    rv = np.abs(g_state["var"].astype(np.float64) / o_state["var"] - 1.0)
    assert np.all(rv[both] <= VAR_RTOL), f"variance rel error {rv[both].max():.3g} > {VAR_RTOL}"
    assert np.array_equal(g_state["t_last"][both], o_state["t_last"][both]), "t_last mismatch"
    cmp.note("max_dh", float(dh[both].max()) if both.any() else 0.0)
    cmp.note("max_var_rel", float(rv[both].max()) if both.any() else 0.0)
    cmp.note("cells_compared", int(both.sum()))
    cmp.note("cells_valid", int(ov.sum()))

    # ---- removed cells
    if prior_valid is not None:
        g_cleared = prior_valid & ~gv
        o_cleared = tr.cleared.astype(bool)
        diff = (g_cleared != o_cleared) & ~excl
        assert not diff.any(), f"removal mismatch on {diff.sum()} cells"
        cmp.note("cleared", int(o_cleared.sum()))

    # ---- stencils
    for name, rad in (("nx", 1), ("ny", 1), ("nz", 1), ("smooth", 2), ("inpaint", 10)):
        if name not in check_stencils or name not in g_state or g_state[name] is None:
            continue
        o = o_state[name]
        g = g_state[name].astype(np.float64)
        ex = dilate(excl, rad)
        onan, gnan = np.isnan(o), np.isnan(g)
        nm = (onan != gnan) & ~ex
        assert not nm.any(), f"{name}: NaN pattern differs on {nm.sum()} cells"
        ok = ~onan & ~gnan & ~ex
        err = np.abs(g - o)
        assert np.all(err[ok] <= STENCIL_TOL), f"{name}: error {err[ok].max():.3g} > {STENCIL_TOL}"
        cmp.note(f"max_err_{name}", float(err[ok].max()) if ok.any() else 0.0)
    return cmp


def prior_to_oracle(om, prior: dict):
    f64 = lambda a: None if a is None else np.asarray(a, np.float64)
    om.set_state(h=f64(prior["h"]), var=f64(prior["var"]), t_last=prior["t_last"], nx=f64(prior.get("nx")),
                 ny=f64(prior.get("ny")), nz=f64(prior.get("nz")), t_now=prior["t_now"])


def prior_to_gpu(gm, prior: dict):
    gm.set_state(h=prior["h"], var=prior["var"], t_last=prior["t_last"].astype(np.float32), nx=prior.get("nx"),
                 ny=prior.get("ny"), nz=prior.get("nz"), t_now=prior["t_now"])


def oracle_state_as_prior(om) -> dict:
    """The oracle's state rounded to the library's float32 layers (a seeded prior)."""
    s = om.state()
    out = {k: s[k].astype(np.float32) for k in ("h", "var", "nx", "ny", "nz")}
    out["t_last"] = s["t_last"].astype(np.int32)
    out["t_now"] = om.t_now
    return out
