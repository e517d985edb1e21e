"""Helpers for comparing the CUDA path (through the C ABI) with the oracle."""

from __future__ import annotations

import os

import numpy as np

# (test, rays compared, rays whose GPU visit list differs from the oracle's
# and is explained by the eps margin), printed at the end of the session
VISIT_LOG: list = []

# Tolerances (FP32 kernels vs the FP64 oracle): colour / opacity / intensity
# absolute 1e-4, depth / range absolute 1e-3 m.
TOL_C = 1e-4
TOL_D = 1e-3

# Visit-list validity margin: a ray whose GPU visit list differs from the
# oracle's must be explained by perturbing every voxel box by
# eps = EPS_ABS_CELLS * finest_edge + EPS_REL * distance (FP32 ray geometry:
# directions carry ~1e-7 relative error, positions ~1 ulp of the distance).
EPS_ABS_CELLS = 1e-4
EPS_REL = 4e-6


def to_np(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def gpu_render(gscene, sensor, idx=None, **kw):
    out = gscene.render(sensor, **kw)
    res = {k: to_np(v) for k, v in out.items() if not k.startswith("_")}
    if idx is not None:
        res = {k: v[idx] for k, v in res.items()}
    return res


# Conditioning allowance: FP32 rays carry direction errors up to ~2e-7 rad
# (a few ulps of a unit vector).  Grazing rays amplify that: their outputs
# move by more than the tolerance when the ray turns by KAPPA.  Such rays are
# compared with tolerance + the oracle's own output change under +-KAPPA turns
# of its FP64 ray about two axes normal to it.
KAPPA = 5e-7


def oracle_sensitivity(oracle, osc, sensor, idx, kappa=KAPPA, **kw):
    """Per ray, max |oracle(turned ray) - oracle(ray)| over 4 turns of kappa
    (rgb/opacity/intensity and depth separately).  Oracle-only."""
    rays = oracle.gen_rays(sensor, idx)
    o, d = rays["o"], rays["d"]
    tn, tf = rays["t_near"], np.where(np.isfinite(rays["t_far"]), rays["t_far"], 0.0)
    def render(dd):
        r = np.concatenate([o, dd, tn[:, None], tf[:, None]], axis=1)
        import synth
        return oracle.render(osc, synth.explicit_rays(r, np.float64), **kw)
    base = render(d)
    sc = np.zeros(len(d))
    sd = np.zeros(len(d))
    for ref in (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])):
        a = np.cross(d, ref)
        bad = np.linalg.norm(a, axis=1) < 1e-3
        a[bad] = np.cross(d[bad], np.array([0.0, 1.0, 0.0]))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        for sgn in (-1.0, 1.0):
            d2 = d + sgn * kappa * a
            d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
            p = render(d2)
            dc = np.maximum(np.abs(p["rgb"] - base["rgb"]).max(axis=1),
                            np.abs(p["opacity"] - base["opacity"]))
            dc = np.maximum(dc, np.abs(p["intensity"] - base["intensity"]))
            sc = np.maximum(sc, dc)
            sd = np.maximum(sd, np.abs(p["depth"] - base["depth"]))
    return sc, sd


def compare_outputs(g, o, want_intensity=False, t_min=0.0, term_gap_min=1e-3, sensitivity=None,
                    max_relaxed_frac=0.005):
    """Element-wise comparison with TOL_C / TOL_D.  Rays over tolerance are
    re-checked against tolerance + sensitivity(ray indices) (conditioning,
    see KAPPA) if a callback is given; at most max_relaxed_frac of the rays
    may need it.  Rays whose oracle transmittance came within
    exp(term_gap_min) of t_min at a termination test may also differ by
    t_min * (max |q|): one voxel more or less."""
    valid = o["valid"]
    assert np.array_equal(g["valid"].astype(bool), valid)
    ec = np.maximum(np.abs(g["rgb"] - o["rgb"]).max(axis=1), np.abs(g["opacity"] - o["opacity"]))
    if want_intensity:
        ec = np.maximum(ec, np.abs(g["intensity"] - o["intensity"]))
    ed = np.abs(g["depth"] - o["depth"])
    lim_c = np.full(len(ec), TOL_C)
    lim_d = np.full(len(ed), TOL_D)
    if t_min > 0:
        tie = o["term_gap"] <= term_gap_min
        lim_c[tie] += t_min
        lim_d[tie] += t_min * 500.0
    over = np.where((ec > lim_c) | (ed > lim_d))[0]
    res = dict(max_c=float(ec.max(initial=0)), max_d=float(ed.max(initial=0)),
               n=len(ec), n_over_tol=len(over))
    if len(over) and sensitivity is not None:
        sc, sd = sensitivity(over)
        lim_c[over] += sc
        lim_d[over] += sd
        res["max_c_over_allowance"] = float((ec[over] / lim_c[over]).max())
    bad = np.where((ec > lim_c) | (ed > lim_d))[0]
    assert len(bad) == 0, (f"{len(bad)} rays out of tolerance, e.g. ray {bad[0]}: "
                           f"c {ec[bad[0]]:.3g} / {lim_c[bad[0]]:.3g}, "
                           f"d {ed[bad[0]]:.3g} / {lim_d[bad[0]]:.3g}", res)
    assert len(over) <= max_relaxed_frac * len(ec), res
    return res


def visit_cap(n: int) -> int:
    """Most rays whose GPU visit list may differ from the oracle's (each one
    explained by the eps margin): 0.1% of the rays compared, at least 2."""
    return max(2, n // 1000)


def check_visits(oracle, osc, sensor, scene, g_vis, g_cnt, o_vis, o_cnt, idx):
    """Exact visit-list equality, except rays whose GPU list is explained by an
    eps-perturbation of the voxel boxes (shrunk subset <= GPU <= grown).
    Returns (n_rays, n_explained)."""
    sf = scene.s0 / (1 << scene.max_level)
    cap = g_vis.shape[1]
    assert np.array_equal(g_cnt <= cap, np.ones_like(g_cnt, bool)), "visits_cap too small"
    bad = np.where((g_cnt != o_cnt) | (g_vis != o_vis).any(axis=1))[0]
    for b in bad:
        ray_id = int(idx[b]) if idx is not None else int(b)
        rays = oracle.gen_rays(sensor, [ray_id])
        o, d = rays["o"][0], rays["d"][0]
        tn, tf = rays["t_near"][0], rays["t_far"][0]
        shrunk = oracle.trace_eps(osc, o, d, tn, tf, EPS_ABS_CELLS * sf, EPS_REL, -1)
        grown, g_in, g_out = oracle.trace_eps(osc, o, d, tn, tf, EPS_ABS_CELLS * sf, EPS_REL, +1,
                                              intervals=True)
        gl = [int(v) for v in g_vis[b][:g_cnt[b]]]
        assert set(shrunk) <= set(gl) <= set(grown), (ray_id, gl, shrunk, grown)
        # order: two voxels whose grown intervals overlap may come either way
        # (entered within eps of the same point); otherwise the earlier first
        pos = {v: i for i, v in enumerate(grown)}
        for a, c in zip(gl, gl[1:]):
            assert g_in[pos[a]] <= g_out[pos[c]], (ray_id, gl, grown)
    VISIT_LOG.append((os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], len(g_cnt),
                      len(bad)))
    return len(g_cnt), len(bad)


def conditioned_rays(oracle, osc, sensor, idx, scene, t_min=0.0, term_gap_min=1e-3):
    """Oracle-chosen mask over the rays `idx`: True where the ray's visit list
    is the same for every voxel box shrunk and grown by the visit-list margin
    (EPS_ABS_CELLS finest edges + EPS_REL x distance), and, with early
    termination, its transmittance never came within exp(term_gap_min) of
    t_min at a termination test.  Rays outside the mask have a visit list (or
    a composited count) that FP32 rounding may legitimately change; gradient
    checks give them zero output gradient.  Oracle-only."""
    sf = scene.s0 / (1 << scene.max_level)
    ok = oracle.conditioned(osc, sensor, EPS_ABS_CELLS * sf, EPS_REL, idx)
    if t_min > 0:
        r = oracle.render(osc, sensor, idx=idx, t_min=t_min)
        ok &= r["term_gap"] > term_gap_min
    return ok
