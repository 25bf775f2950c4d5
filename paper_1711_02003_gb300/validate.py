"""Validation runs of the configurations on the GPU (physics and precision checks).

    python -m paper_1711_02003_gb300.validate [--only c1,c3,c2,f1,f2,c2scan,c2drip] [--out results.json]

c1  static droplet D2Q9 64^2, R = 16, FP64, 2000 steps: per-component mass drift and the Laplace
    pressure against sigma/R with sigma = 2 A tau / 9 (parity with the oracle is in the tests).
c3  3D Laplace sweep D3Q19 128^3, R in {12, 16, 24, 32}, A in {0.005, 0.01, 0.02}, tau = 1,
    beta = 0.7, 5000 steps: dp against 2 sigma / R and max |u|, FP32-dev for every case and
    FP64 for A = 0.01 (FP32 error of dp and R_eff stated against FP64).
c2  flow-focusing cross junction D2Q9 1024 x 192, FP32-dev, 1e5 steps: droplets detached from
    the dispersed thread (red components whose leftmost site is beyond the side inlets), their
    count, pinch-offs counted as new droplets passing x = 768, and equivalent diameters d/h.
f1  regularized vs BGK relaxation for a resting droplet with relaxation times 1 (continuous) and
    5 (droplet), as in Fig. 1: max |u| ratio, 2D and 3D.
f2  density ratio 1, 2, 5, 10 through alpha_k (D2Q9 128^2 R = 24, D3Q19 96^3 R = 16, 5000 steps):
    Laplace law against the unit-ratio sigma, spurious currents, mass drift, FP32-dev vs FP64.
c2scan / c2drip  flow-focuser regime scans (pinch-off counts, d/h) over A, inlet speeds and
    viscosity ratio.
c4  step emulsifier (768 x 128 x 32, FP32-dev, 2e5 steps, A = 0.1 and 0.3): detached droplets
    beyond the terrace and their equivalent diameters; c4long: 1e6 steps at u_in 0.002 and
    4e5 steps at u_in 0.005, both Ca = 0.01; c4nozzle: a single 24-wide nozzle, 4e5 steps.
c2prec  two dripping flow-focuser cases in FP32-dev and FP64 (pinch-offs, d/h), 2e5 steps each.
f3  d/h against Q_B / (2 Q_Y) in the flow focuser (2e5 steps per case) and its fitted exponent
    (the paper reports 0.5, after Cubaud and Mason).
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import lbcg
from . import workloads as W


def c1() -> dict:
    pb = W.static_droplet(W.D2Q9, 64, 16)
    sim = lbcg.Simulation(pb, lbcg.LBCG_FP64)
    o0 = sim.observables((32, 32))
    out = {"config": "C1 static droplet D2Q9 64^2 R=16 FP64"}
    sim.step(2000)
    o = sim.observables((32, 32))
    sigma = 2 * pb.A * pb.tau_r / 9
    out.update(steps=2000, mass_drift_r=o["mass_r"] / o0["mass_r"] - 1, mass_drift_b=o["mass_b"] / o0["mass_b"] - 1,
               dp=o["dp"], r_eff=o["r_eff"], sigma_closed_form=sigma, dp_times_r_over_sigma=o["dp"] * o["r_eff"] / sigma,
               umax=o["umax"])
    return out


def c3(steps: int = 5000) -> list:
    rows = []
    for A in (0.005, 0.01, 0.02):
        for R in (12, 16, 24, 32):
            pb = W.static_droplet(W.D3Q19, 128, R, A=A)
            rec = {"config": "C3 D3Q19 128^3", "R": R, "A": A, "steps": steps}
            sigma = 2 * A * pb.tau_r / 9
            for prec in ((lbcg.LBCG_FP32_DEV, lbcg.LBCG_FP64) if A == 0.01 else (lbcg.LBCG_FP32_DEV,)):
                sim = lbcg.Simulation(pb, prec)
                t0 = time.perf_counter()
                sim.step(steps)
                o = sim.observables((64, 64, 64))
                dt = time.perf_counter() - t0
                tag = lbcg.PRECISION_NAMES[prec]
                rec[tag] = {"dp": o["dp"], "r_eff": o["r_eff"], "dp_r_over_2sigma": o["dp"] * o["r_eff"] / (2 * sigma),
                            "umax": o["umax"], "mass_drift_r": None, "seconds": dt}
                sim.close()
            if "f64" in rec:
                rec["f32dev_vs_f64"] = {"dp_rel": rec["f32dev"]["dp"] / rec["f64"]["dp"] - 1,
                                        "r_eff_rel": rec["f32dev"]["r_eff"] / rec["f64"]["r_eff"] - 1}
            rows.append(rec)
            print(json.dumps(rec), flush=True)
    return rows


def c2(steps: int = 100000, sample: int = 500, A: float = 0.05, u: float = 0.005, tau_disp: float = 2.0,
       u_cont: float | None = None, precision: int = lbcg.LBCG_FP32_DEV) -> dict:
    u_cont = u if u_cont is None else u_cont
    pb = W.cross_junction(u_disp=u, u_cont=u_cont, A=A, tau_disp=tau_disp)
    sim = lbcg.Simulation(pb, precision)
    nx = pb.nx
    h = 64.0  # main channel width
    side_end = 320
    prev_right = []
    diam = []
    counts = []
    thread = []
    pinch = 0
    t0 = time.perf_counter()
    for t in range(sample, steps + 1, sample):
        sim.step(sample)
        labels, cnts, vols, nd = sim.label(cap=4096)
        if nd == 0:
            counts.append(0)
            continue
        lab = labels.reshape(pb.ny, nx)
        xs = np.arange(nx)[None, :].repeat(pb.ny, 0)
        roots = np.unique(lab[lab >= 0])
        detached = []
        reach = 0
        for k, r in enumerate(roots):
            sel = lab == r
            xmin = xs[sel].min()
            if xmin > side_end:
                cx = xs[sel].mean()
                detached.append((cx, vols[k]))
            else:
                reach = max(reach, int(xs[sel].max()))
        thread.append(reach)
        counts.append(len(detached))
        right = [cx for cx, _ in detached if cx > 768]
        # droplets past x = 768: new ones entering that region count as pinch-offs seen there
        pinch += max(0, len(right) - len(prev_right))
        prev_right = right
        for _, v in detached:
            diam.append(2.0 * math.sqrt(v / math.pi) / h)
    dt = time.perf_counter() - t0
    o = sim.observables((nx / 2, pb.ny / 2), allow_diverged=True)
    return {"config": "C2 flow focuser D2Q9 1024x192 " + lbcg.PRECISION_NAMES[precision], "steps": steps, "A": A,
            "u_max": u,
            "u_max_continuous": u_cont, "q_b_over_2q_y": u / (2 * u_cont),
            "thread_reach_x_mean": float(np.mean(thread)) if thread else None,
            "tau_disp": tau_disp, "tau_cont": pb.tau_b,
            "Ca_estimate": (pb.tau_b - 0.5) / 3 * (2 * u_cont / 3) / (2 * A * pb.tau_b / 9),
            "mean_detached_droplets": float(np.mean(counts)) if counts else 0.0,
            "droplets_passing_x768": pinch, "d_over_h_mean": float(np.mean(diam)) if diam else None,
            "d_over_h_std": float(np.std(diam)) if diam else None, "nonfinite": o["nonfinite"], "seconds": dt}


def f1() -> list:
    out = []
    for lat, n, R, steps, centre in ((W.D2Q9, 64, 16, 3000, None), (W.D3Q19, 64, 16, 2000, (31.5, 31.5, 31.5))):
        umax = {}
        for coll in (W.REG, W.BGK):
            pb = W.static_droplet(lat, n, R, tau_r=5.0, tau_b=1.0, collision=coll, centre=centre)
            sim = lbcg.Simulation(pb, lbcg.LBCG_FP64)
            sim.step(steps)
            c = centre or (n // 2, n // 2, n // 2)
            umax[coll] = sim.observables(c)["umax"]
            sim.close()
        rec = {"config": f"f1 resting droplet {'D2Q9' if lat == W.D2Q9 else 'D3Q19'} {n} R={R} tau 1/5",
               "steps": steps, "umax_reg": umax[W.REG], "umax_bgk": umax[W.BGK],
               "bgk_over_reg": umax[W.BGK] / umax[W.REG]}
        out.append(rec)
        print(json.dumps(rec), flush=True)
    return out


def f2(steps: int = 5000) -> list:
    """Density ratio through alpha_k (Eqs. 7-8): resting droplets holding gamma times the
    surrounding density, Laplace law against the unit-ratio sigma, spurious currents, mass
    drift; FP32-dev against FP64."""
    rows = []
    for lat, n, R, centre in ((W.D2Q9, 128, 24, None), (W.D3Q19, 96, 16, (47.5, 47.5, 47.5))):
        for g in (1.0, 2.0, 5.0, 10.0):
            pb = W.static_droplet(lat, n, R, centre=centre, density_ratio=g)
            sigma = 2 * pb.A * pb.tau_r / 9
            c = centre or (n // 2, n // 2, n // 2)
            rec = {"config": f"f2 {'D2Q9' if lat == W.D2Q9 else 'D3Q19'} {n} R={R}", "density_ratio": g,
                   "alpha_r": pb.alpha_r, "alpha_b": pb.alpha_b, "steps": steps}
            for prec in (lbcg.LBCG_FP32_DEV, lbcg.LBCG_FP64):
                sim = lbcg.Simulation(pb, prec)
                o0 = sim.observables(c, allow_diverged=True)
                sim.step(steps)
                o = sim.observables(c, allow_diverged=True)
                k = 1 if lat == W.D2Q9 else 2
                rec[lbcg.PRECISION_NAMES[prec]] = {
                    "dp": o["dp"], "r_eff": o["r_eff"], "dp_r_over_k_sigma": o["dp"] * o["r_eff"] / (k * sigma),
                    "umax": o["umax"], "mass_drift_r": o["mass_r"] / o0["mass_r"] - 1,
                    "mass_drift_b": o["mass_b"] / o0["mass_b"] - 1, "nonfinite": o["nonfinite"]}
                sim.close()
            rec["f32dev_vs_f64_dp_rel"] = rec["f32dev"]["dp"] / rec["f64"]["dp"] - 1
            rows.append(rec)
            print(json.dumps(rec), flush=True)
    return rows


def f3(steps: int = 200000) -> dict:
    """Droplet size against the flow-rate ratio in the flow focuser (Sec. IV A): continuous
    inlets at u_max 0.01, dispersed inlet swept, Ca 0.05 and 0.025 (A 0.1, 0.2), viscosity
    ratio 2; least-squares exponent of d/h against Q_B / (2 Q_Y) over the cases that pinch off."""
    out = {"cases": [], "fits": {}}
    for A in (0.1, 0.2):
        xs, ys = [], []
        for ud in (0.003, 0.004, 0.005, 0.006, 0.008):
            r = c2(steps, A=A, u=ud, tau_disp=2.0, u_cont=0.01)
            out["cases"].append(r)
            print(json.dumps(r), flush=True)
            if r["droplets_passing_x768"] >= 2 and r["d_over_h_mean"]:
                xs.append(math.log(r["q_b_over_2q_y"]))
                ys.append(math.log(r["d_over_h_mean"]))
        if len(xs) >= 2:
            k, c = np.polyfit(xs, ys, 1)
            out["fits"][f"A={A}"] = {"exponent": float(k), "prefactor": float(math.exp(c)), "points": len(xs)}
    print(json.dumps(out["fits"]), flush=True)
    return out


def c4(steps: int = 200000, sample: int = 10000, cases=((0.1, 0.002), (0.3, 0.002)), nozzle_w=None) -> list:
    """Step emulsifier (Sec. IV B; 768 x 128 x 32, FP32-dev): the dispersed phase enters the
    8-plane terrace at u_max 0.002 and breaks up where the terrace opens into the reservoir.
    Droplets detached from the nozzle thread (red components lying entirely beyond the
    terrace) are counted every `sample` steps; their equivalent diameters D = (6 V / pi)^(1/3)
    are reported against the terrace height h = 8 and the nozzle width w = 126."""
    rows = []
    for A, u_in in cases:
        pb = W.step_emulsifier(A=A, u_in=u_in, nozzle_w=nozzle_w)
        sigma = 2 * A * pb.tau_b / 9
        ca = (pb.tau_b - 0.5) / 3 * (2 * u_in / 3) / sigma
        sim = lbcg.Simulation(pb, lbcg.LBCG_FP32_DEV)
        t0 = time.perf_counter()
        counts, diam = [], []
        last = []
        reach = 0
        for t in range(sample, steps + 1, sample):
            sim.step(sample)
            labels, cnts, vols, nd = sim.label(cap=4096)
            if nd == 0:
                counts.append(0)
                continue
            lab = labels.reshape(pb.nz, pb.ny, pb.nx)
            xs = np.broadcast_to(np.arange(pb.nx)[None, None, :], lab.shape)
            roots = np.unique(lab[lab >= 0])
            det = []
            for k, r in enumerate(roots):
                xr = xs[lab == r]
                if xr.min() > 256:
                    det.append((6.0 * vols[k] / math.pi) ** (1.0 / 3.0))
                else:
                    reach = max(reach, int(xr.max()))
            counts.append(len(det))
            diam += det
            last = det
        dt = time.perf_counter() - t0
        o = sim.observables((384, 64, 16), allow_diverged=True)
        rec = {"config": "C4 step emulsifier 768x128x32 FP32-dev", "nozzle_w": nozzle_w or 126, "A": A,
               "u_in": u_in, "Ca_estimate": ca,
               "steps": steps, "thread_reach_x": reach,
               "detached_max": max(counts) if counts else 0, "detached_final": len(last),
               "D_mean": float(np.mean(diam)) if diam else None, "D_std": float(np.std(diam)) if diam else None,
               "D_over_h": float(np.mean(diam)) / 8 if diam else None,
               "D_over_w": float(np.mean(diam)) / 126 if diam else None,
               "final_diameters": [round(float(d), 2) for d in sorted(last)], "nonfinite": o["nonfinite"],
               "seconds": dt}
        rows.append(rec)
        print(json.dumps(rec), flush=True)
        sim.close()
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="c1,c3,c2,f1")
    ap.add_argument("--out", default=None)
    ap.add_argument("--c3-steps", type=int, default=5000)
    ap.add_argument("--c2-steps", type=int, default=100000)
    args = ap.parse_args(argv)
    lbcg.load()
    res = {}
    for name in args.only.split(","):
        t0 = time.perf_counter()
        if name == "c1":
            res["c1"] = c1()
        elif name == "c3":
            res["c3"] = c3(args.c3_steps)
        elif name == "c2":
            res["c2"] = c2(args.c2_steps)
        elif name == "c2scan":
            res["c2scan"] = []
            # (A, u_max dispersed, u_max continuous, tau dispersed): Ca 0.005-0.05 at the
            # continuous inlet speed, viscosity ratio 1 to 5
            for A, ud, uc, td in ((0.1, 0.002, 0.005, 2.0), (0.1, 0.004, 0.01, 2.0), (0.05, 0.005, 0.01, 2.0),
                                  (0.02, 0.005, 0.01, 2.0), (0.05, 0.01, 0.01, 2.0), (0.02, 0.01, 0.01, 2.0),
                                  (0.01, 0.005, 0.01, 2.0), (0.05, 0.005, 0.01, 5.0), (0.02, 0.005, 0.01, 1.0),
                                  (0.02, 0.003, 0.01, 3.0)):
                r = c2(args.c2_steps, A=A, u=ud, tau_disp=td, u_cont=uc)
                res["c2scan"].append(r)
                print(json.dumps(r), flush=True)
        elif name == "f1":
            res["f1"] = f1()
        elif name == "f2":
            res["f2"] = f2()
        elif name == "c4":
            res["c4"] = c4()
        elif name == "c4nozzle":
            # a single 24-wide nozzle (w / h = 3): step emulsification, Ca 0.01-0.014
            res["c4nozzle"] = c4(400000, 20000, cases=((0.25, 0.005), (0.18, 0.005)), nozzle_w=24)
        elif name == "c4long":
            # Ca = 0.01 reached by A with the config's inlet speed over 10^6 steps, and by a
            # faster inlet over 4 * 10^5 steps
            res["c4long"] = c4(1000000, 50000, cases=((0.1, 0.002),)) + c4(400000, 20000, cases=((0.25, 0.005),))
        elif name == "c2prec":
            # the same dripping cases in FP32-dev and FP64: pinch-off counts and droplet sizes
            res["c2prec"] = []
            for A, ud in ((0.1, 0.003), (0.2, 0.004)):
                for prec in (lbcg.LBCG_FP32_DEV, lbcg.LBCG_FP64):
                    r = c2(2 * args.c2_steps, A=A, u=ud, tau_disp=2.0, u_cont=0.01, precision=prec)
                    res["c2prec"].append(r)
                    print(json.dumps(r), flush=True)
        elif name == "f3":
            res["f3"] = f3(2 * args.c2_steps)
        elif name == "c2drip":
            # dripping-regime search: continuous inlet 0.01 (Ca 0.025-0.05 via A), slower
            # dispersed inlets, viscosity ratio 1-3; 2e5 steps
            res["c2drip"] = []
            for A, ud, td in ((0.1, 0.002, 1.0), (0.1, 0.003, 2.0), (0.1, 0.004, 1.0), (0.2, 0.002, 2.0),
                              (0.2, 0.004, 2.0), (0.2, 0.006, 2.0), (0.1, 0.006, 3.0), (0.15, 0.004, 3.0)):
                r = c2(2 * args.c2_steps, A=A, u=ud, tau_disp=td, u_cont=0.01)
                res["c2drip"].append(r)
                print(json.dumps(r), flush=True)
        print(json.dumps({name: res.get(name), "seconds": time.perf_counter() - t0}, default=float), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1, default=float)


if __name__ == "__main__":
    sys.exit(main())
