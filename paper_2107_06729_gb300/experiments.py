"""Paper-style experiments on synthetic stand-ins (Sec. III), on the GPU.

    python -m paper_2107_06729_gb300.experiments [--t-end-ps 200] [--only NAME]

prints one JSON line per experiment:

* ``method_sweep`` (Fig. 5(b) analog): every adaptive method of Sec. II at
  e_max = 1e-5, with demag extrapolation of order p and with the exact demag
  at every sub-step; simulated ns per second of both, the speedup factor and
  the error (Eq. 7) of each against a reference run; with --eps-time also
  Eq. 7 over 1 ps samples of the mean magnetisation (extra untimed runs).
* ``order_sweep`` (Fig. 2(a) analog): RKF56 with p = 0 .. 5 and full demag,
  the error against the reference.
* ``fixed_step_sweep``: RK4 at h = 100 .. 500 fs with p = 3 and with full
  demag, the error against the reference.
* ``checker_fixed_step`` (Fig. 3 analog): the checkerboard particle-array
  stand-in (see ``checker_config``), every method at fixed steps of
  100 .. 1000 fs in FP64, full and extrapolated demag, Eq. 7 over the 1 ps
  samples of <m> against an h = 10 fs reference.

The slab stands in for the paper's 3.2 um x 1.6 um x 20 nm Py slab with
5 nm cells (640 x 320 x 4, S-state start, field (-20, 1, 0) kA/m): the mesh
is 512 x 256 x 4 cells of 5 nm (mesh sides are powers of two here), Ms = 800
kA/m, A = 13 pJ/m, alpha = 0.02, the same field, and an S-like start (m
along +x, the end regions tilted towards +y and -y, plus U(-0.02, 0.02)
noise) since the paper does not give its S-state.  The reference is an FP64
run with RKDP54, full demag and e_max = 1e-9.  Everything runs through the
library's C ABI; FP32 fields unless stated.
"""
import argparse
import json
import time

import numpy as np

from . import workloads as W

METHOD_P = [("HEUN12", 1), ("ABM2", 1), ("RK23", 2), ("RKF45", 4), ("RKCK45", 4), ("RKDP54", 4), ("RKF56", 5)]


def slab_config(seed=0):
    """512 x 256 x 4 cells of 5 nm, Py, field (-20, 1, 0) kA/m, S-like start."""
    n = (512, 256, 4)
    d = (5e-9, 5e-9, 5e-9)
    nx, ny, nz = n
    rng = np.random.default_rng(np.random.PCG64(seed))
    x = (np.arange(nx) + 0.5) / nx
    tilt = 0.6 * (np.exp(-((x - 0.0) / 0.08) ** 2) - np.exp(-((x - 1.0) / 0.08) ** 2))
    m = np.zeros((3, nz, ny, nx))
    m[0] = 1.0
    m[1] = tilt.reshape(1, 1, nx)
    m = m + rng.uniform(-0.02, 0.02, size=m.shape)
    m = m / np.linalg.norm(m, axis=0, keepdims=True)
    return {
        "name": "slab_512x256x4_5nm",
        "mesh": {"n": n, "d": d},
        "material": {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0), "alpha": 0.02, "gamma": W.GAMMA},
        "field": {"H0": (-20e3, 1e3, 0.0), "pulse": (0.0, 0.0, 0.0), "t_on": 0.0, "t_off": 0.0},
        "m0": m,
    }


def _adaptive(method, p, tol=1e-5):
    return {"method": method, "extrap_order": p, "adaptive": True, "h": 1e-13, "tol": tol, "hmin": 1e-15,
            "hmax": 3e-12, "cmin": 0.01, "cmax": 2.0}


def _run(pkg, torch, cfg, integ, prec, t_end):
    """One run from the start state; returns (m as float64 numpy, stats,
    device seconds of the run)."""
    dt = torch.float64 if prec == "fp64" else torch.float32
    ctx = pkg.Context(cfg["mesh"], cfg["material"], cfg["field"], integ, prec)
    try:
        m = torch.from_numpy(cfg["m0"]).to("cuda", dt)
        ctx.set_m(m)
        # a short warm-up run builds the graphs; the timed run restarts from
        # the start state (the step the controller proposed is kept)
        ctx.run(1e-13)
        ctx.set_m(m)
        ctx.set_time(0.0)
        s0 = ctx.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.run(t_end)
        e1.record()
        torch.cuda.synchronize()
        out = torch.empty_like(m)
        ctx.get_m(out)
        s1 = ctx.stats()
        st = {k: s1[k] - s0[k] for k in ("accepted", "rejected", "exact_evals", "extrap_evals")}
        return out.double().cpu().numpy(), st, e0.elapsed_time(e1) / 1e3
    finally:
        ctx.close()


def eps(m, ref):
    """Eq. 7: mean over cells of |m - m_ref|."""
    return float(np.linalg.norm(m - ref, axis=0).mean())


def eps_time(mbar, mbar_ref):
    """Eq. 7 with time samples of the mean magnetisation <m> as its points
    (the reading for the paper's error-versus-time curves): [3, S] arrays."""
    return float(np.linalg.norm(np.asarray(mbar) - np.asarray(mbar_ref), axis=0).mean())


def _mean_history(pkg, torch, cfg, integ, prec, t_end, dt=1e-12):
    """<m> every dt up to t_end ([3, S]), from a run in dt chunks (untimed)."""
    tdt = torch.float64 if prec == "fp64" else torch.float32
    ctx = pkg.Context(cfg["mesh"], cfg["material"], cfg["field"], integ, prec)
    try:
        m = torch.from_numpy(cfg["m0"]).to("cuda", tdt)
        ctx.set_m(m)
        out = []
        for k in range(1, int(round(t_end / dt)) + 1):
            ctx.run(k * dt)
            ctx.get_m(m)
            out.append(m.double().mean(dim=(1, 2, 3)).cpu().numpy())
        return np.stack(out, axis=1)
    finally:
        ctx.close()


def method_sweep(pkg, torch, cfg, ref, t_end, ref_hist=None):
    rows = []
    for method, p in METHOD_P:
        mx, sx, tx = _run(pkg, torch, cfg, _adaptive(method, p), "fp32", t_end)
        mf, sf, tf = _run(pkg, torch, cfg, _adaptive(method, -1), "fp32", t_end)
        row = {"method": method, "p": p, "ns_per_s_extrap": round(t_end * 1e9 / tx, 4),
               "ns_per_s_full": round(t_end * 1e9 / tf, 4), "speedup": round(tf / tx, 3),
               "eps_extrap": eps(mx, ref), "eps_full": eps(mf, ref),
               "steps_extrap": sx["accepted"], "steps_full": sf["accepted"],
               "rejected_extrap": sx["rejected"], "rejected_full": sf["rejected"]}
        if ref_hist is not None:
            row["eps_time_extrap"] = eps_time(_mean_history(pkg, torch, cfg, _adaptive(method, p), "fp32", t_end),
                                              ref_hist)
            row["eps_time_full"] = eps_time(_mean_history(pkg, torch, cfg, _adaptive(method, -1), "fp32", t_end),
                                            ref_hist)
        rows.append(row)
    return {"experiment": "method_sweep", "tol": 1e-5, "rows": rows}


def order_sweep(pkg, torch, cfg, ref, t_end):
    rows = []
    for p in [-1, 0, 1, 2, 3, 4, 5]:
        m, st, secs = _run(pkg, torch, cfg, _adaptive("RKF56", p), "fp32", t_end)
        rows.append({"p": p, "eps": eps(m, ref), "steps": st["accepted"], "rejected": st["rejected"],
                     "ns_per_s": round(t_end * 1e9 / secs, 4)})
    return {"experiment": "order_sweep", "method": "RKF56", "tol": 1e-5, "rows": rows}


def fixed_step_sweep(pkg, torch, cfg, ref, t_end):
    rows = []
    for h_fs in (100, 200, 300, 400, 500):
        for p in (3, -1):
            integ = {"method": "RK4", "extrap_order": p, "adaptive": False, "h": h_fs * 1e-15}
            m, st, secs = _run(pkg, torch, cfg, integ, "fp32", t_end)
            rows.append({"h_fs": h_fs, "p": p, "eps": eps(m, ref), "steps": st["accepted"],
                         "ns_per_s": round(t_end * 1e9 / secs, 4)})
    return {"experiment": "fixed_step_sweep", "method": "RK4", "rows": rows}


# ---------------------------------------------------- checkerboard array --
# Fig. 3 analog.  The paper's array: 300 nm x 300 nm x 5 nm, the Standard
# Problem 4 material (Py), particles interacting only through the demag
# field, relaxed at zero field, then field (20, 1, 0) kA/m for 3 ns with
# <m> recorded every 1 ps; fixed steps, FP64, the full-demag and the
# extrapolated result of every method against a reference.  Declared
# stand-in (the particle geometry is not given): 64 x 64 x 1 cells of 5 nm
# (320 nm square), particles of 4 x 4 cells (20 nm) on alternate squares of
# a checkerboard, the cells between them without material (m = 0), so that
# exchange acts inside each particle only; the start relaxed from +x with
# noise at alpha = 0.5 in zero field for 500 ps (FP64, DP54, e_max 1e-8);
# the reference one RKDP54 run with full demag at h = 10 fs.
CHECKER_METHODS = [("HEUN12", 1), ("ABM2", 1), ("RK23", 2), ("RK4", 3), ("RKF45", 4), ("RKCK45", 4),
                   ("RKDP54", 4), ("RKF56", 5)]
CHECKER_H_FS = (100, 200, 250, 500, 1000)  # divide the 1 ps sampling interval


def checker_config(pkg, torch, seed=0):
    n = (64, 64, 1)
    mesh = {"n": n, "d": (5e-9, 5e-9, 5e-9)}
    mat = {"Ms": 8e5, "A": 1.3e-11, "K": 0.0, "ku": (1.0, 0.0, 0.0), "alpha": 0.02, "gamma": W.GAMMA}
    mask = W.checkerboard_mask(n, 4)
    m0 = W.m_uniform_noise(n, direction=(1.0, 0.0, 0.0), noise=0.1, seed=seed) * mask
    relax = dict(mat, alpha=0.5)
    ctx = pkg.Context(mesh, relax, {}, _adaptive("RKDP54", -1, tol=1e-8), "fp64")
    try:
        m = torch.from_numpy(m0).to("cuda", torch.float64)
        ctx.set_m(m)
        ctx.run(500e-12)
        ctx.get_m(m)
        m0 = m.cpu().numpy()
    finally:
        ctx.close()
    return {"name": "checkerboard_64x64x1_5nm_4x4_particles", "mesh": mesh, "material": mat,
            "field": {"H0": (20e3, 1e3, 0.0)}, "m0": m0, "mask": mask}


def _mag_mean_history(pkg, torch, cfg, integ, t_end, dt=1e-12):
    """<m> over the magnetic cells every dt up to t_end ([3, S]), FP64."""
    nmag = float(cfg["mask"].sum())
    ctx = pkg.Context(cfg["mesh"], cfg["material"], cfg["field"], integ, "fp64")
    try:
        m = torch.from_numpy(cfg["m0"]).to("cuda", torch.float64)
        ctx.set_m(m)
        out = []
        for k in range(1, int(round(t_end / dt)) + 1):
            ctx.run(k * dt)
            ctx.get_m(m)
            out.append((m.sum(dim=(1, 2, 3)) / nmag).cpu().numpy())
        return np.stack(out, axis=1), ctx.stats()
    finally:
        ctx.close()


def checker_fixed_step(pkg, torch, cfg, t_end):
    """Every method at fixed steps h (no controller), full demag and Eq. 6
    with p matched to the method order; Eq. 7 over the 1 ps samples of <m>
    against the reference."""
    ref, _ = _mag_mean_history(pkg, torch, cfg, {"method": "RKDP54", "extrap_order": -1, "adaptive": False,
                                                 "h": 10e-15}, t_end)
    rows = []
    for method, p in CHECKER_METHODS:
        for h_fs in CHECKER_H_FS:
            row = {"method": method, "p": p, "h_fs": h_fs}
            for name, pp in (("full", -1), ("extrap", p)):
                integ = {"method": method, "extrap_order": pp, "adaptive": False, "h": h_fs * 1e-15}
                hist, st = _mag_mean_history(pkg, torch, cfg, integ, t_end)
                row["eps_" + name] = eps_time(hist, ref)
                row["steps_" + name] = st["accepted"]
            rows.append(row)
    return {"experiment": "checker_fixed_step", "precision": "fp64", "reference": "RKDP54 full demag, h = 10 fs",
            "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--t-end-ps", type=float, default=200.0)
    ap.add_argument("--only", choices=["method_sweep", "order_sweep", "fixed_step_sweep", "checker_fixed_step"])
    ap.add_argument("--checker-t-end-ps", type=float, default=3000.0,
                    help="horizon of the checkerboard experiment (the paper's 3 ns)")
    ap.add_argument("--eps-time", action="store_true",
                    help="also Eq. 7 over 1 ps samples of <m> in the method sweep (extra untimed chunked runs)")
    args = ap.parse_args(argv)
    import torch
    import paper_2107_06729_gb300 as pkg
    t0 = time.time()
    if args.only in (None, "checker_fixed_step"):
        ccfg = checker_config(pkg, torch)
        out = checker_fixed_step(pkg, torch, ccfg, args.checker_t_end_ps * 1e-12)
        out["workload"] = ccfg["name"]
        out["t_end_ps"] = args.checker_t_end_ps
        print(json.dumps(out), flush=True)
        if args.only:
            print(json.dumps({"experiment": "done", "wall_s": round(time.time() - t0, 1)}), flush=True)
            return
    cfg = slab_config()
    t_end = args.t_end_ps * 1e-12
    ref, rst, rsecs = _run(pkg, torch, cfg, _adaptive("RKDP54", -1, tol=1e-9), "fp64", t_end)
    print(json.dumps({"experiment": "reference", "workload": cfg["name"], "t_end_ps": args.t_end_ps,
                      "method": "RKDP54", "p": -1, "tol": 1e-9, "precision": "fp64", "steps": rst["accepted"],
                      "seconds": round(rsecs, 2)}), flush=True)
    ref_hist = None
    if args.eps_time and args.only in (None, "method_sweep"):
        ref_hist = _mean_history(pkg, torch, cfg, _adaptive("RKDP54", -1, tol=1e-9), "fp64", t_end)
    for name, fn in (("method_sweep", method_sweep), ("order_sweep", order_sweep),
                     ("fixed_step_sweep", fixed_step_sweep)):
        if args.only and args.only != name:
            continue
        out = fn(pkg, torch, cfg, ref, t_end, ref_hist) if name == "method_sweep" else fn(pkg, torch, cfg, ref, t_end)
        out["workload"] = cfg["name"]
        out["t_end_ps"] = args.t_end_ps
        print(json.dumps(out), flush=True)
    print(json.dumps({"experiment": "done", "wall_s": round(time.time() - t0, 1)}), flush=True)


if __name__ == "__main__":
    main()
