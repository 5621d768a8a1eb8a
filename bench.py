#!/usr/bin/env python
"""Benchmark: H_eff matvec TFLOP/s and sweep seconds of two-site DMRG on the spin-1/2
Heisenberg 24x8 square cylinder (periodic width 8, open length 24, snake order, MPO bond
dimension 26) at m = 2000, mixed precision (bf16 tensor-core matvec, FP64 Davidson/SVD).

A step is one two-site bond update in the bulk of the cylinder (form Psi, Davidson with a
fixed number of iterations, SVD + truncation to m, environment update), run through the
library's public C ABI (dmrg_advance).  Inputs are synthetic: a seeded random
mixed-canonical MPS whose U(1) sector dimensions follow a Gaussian profile (sigma = 5 in
2S^z units, ~17 sectors, largest ~320) -- the shape of a ground state's Schmidt spectrum.

Prints one JSON line.  --impl reference times the CPU oracle on the host cores instead.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "H_eff matvec TFLOP/s & sweep s, 24x8 m=2000; mixed vs FP64 GPU at 1e-5 dE/E"
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25     # nominal dense tensor rates (per GPU)



T_START = time.perf_counter()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16", "tf32", "fp64"], default="bf16")
    ap.add_argument("--lattice", choices=["square", "triangular"], default="square",
                    help="Heisenberg cylinder of the sweeps/steps modes (triangular adds the (x,y)-(x+1,y-1) bonds)")
    ap.add_argument("--lx", type=int, default=24)
    ap.add_argument("--ly", type=int, default=8)
    ap.add_argument("--m", type=int, default=2000)
    ap.add_argument("--sigma", type=float, default=5.0)
    ap.add_argument("--dav-iters", type=int, default=4)
    ap.add_argument("--refine-iters", type=int, default=1)
    ap.add_argument("--kmax", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-sample-s", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["steps", "sweeps", "op", "accuracy", "grad", "chain", "observe"],
                    default="sweeps",
                    help="sweeps: a step is one real-space parallel sweep (Fig. 4) over the whole lattice; "
                         "steps: a step is one bulk two-site update (serial); op: repeated H_eff matvecs at "
                         "one bond (random environments, small device footprint, for profiler captures); "
                         "accuracy: the same serial sweeps (m ramped to --acc-m) in FP64 and in --precision "
                         "mode from the same seeded state, energies and sweep times compared")
    ap.add_argument("--acc-m", type=int, default=500)
    ap.add_argument("--acc-tol", type=float, default=1e-8,
                    help="accuracy leg: Davidson residual tolerance of both same-state sweeps")
    ap.add_argument("--acc-iters", type=int, default=12,
                    help="accuracy leg: Davidson iteration cap (FP64; tensor-core iterations of the mixed sweep)")
    ap.add_argument("--acc-refine", type=int, default=12,
                    help="accuracy leg: FP32-accurate refinement iterations of the mixed sweep (after --dav-iters "
                         "tensor-core iterations)")
    ap.add_argument("--time-budget-s", type=float, default=1700.0,
                    help="wall-clock budget of the whole run: the accuracy leg's same-state sweeps are skipped "
                         "(and the reason recorded) when they would end beyond it")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="sweeps mode: skip the FP64 evaluation and the FP64-vs-mixed same-state sweeps")
    ap.add_argument("--env-fp64", action="store_true",
                    help="mixed modes: FP64-accurate environments (default: FP32)")
    ap.add_argument("--edges", type=int, default=2, choices=[0, 1, 2],
                    help="mixed modes: FP64 solves next to the region boundaries and in the merges (1: Davidson, "
                         "2: Davidson and split; 0: mixed precision everywhere)")
    ap.add_argument("--svd-plain-jacobi", action="store_true",
                    help="splits by the one-sided Jacobi on the sector matrices (no QR preconditioning)")
    ap.add_argument("--fp64-emulation", action="store_true",
                    help="FP64 grouped GEMMs on the bf16 tensor cores (FP64-accurate slicing) in the engines of "
                         "the steps, sweeps, observe and chain (FP64 runs) modes")
    ap.add_argument("--obs-m", type=int, default=800,
                    help="observe: bond dimension of the seeded state put in the inverse canonical gauge")
    ap.add_argument("--grad-L", type=int, default=128)
    ap.add_argument("--chain-L", type=int, default=200)
    ap.add_argument("--chain-ramp", default="64,64,128,128,256,256,512,512")
    ap.add_argument("--chain-spin", choices=["half", "one"], default="half")
    ap.add_argument("--chain-warmup", type=int, default=0)
    ap.add_argument("--chain-runs", default="",
                    help="chain: runs to make, comma-separated precision[:svd64][:rN refinement iterations]"
                         "[:e64 FP64-accurate environments][:edge FP64 solves next to the boundaries][:edge2 and FP64 splits there]"
                         "[:dN Davidson iterations][:tz fixed iteration count]"
                         " (default: fp64 and --precision)")
    ap.add_argument("--grad-m", type=int, default=128)
    ap.add_argument("--grad-jq-m", type=int, default=128)
    ap.add_argument("--acc-sweeps", type=int, default=6)
    ap.add_argument("--acc-variants", default="",
                    help="accuracy: extra same-state sweeps, comma-separated precision:refine_iters[:svd64][:davN] "
                         "(e.g. tf32:6, bf16:12:dav1)")
    ap.add_argument("--regions", type=int, default=4)
    ap.add_argument("--region-schedule", choices=list(SCHEDULES), default="lockstep",
                    help="sweeps: concurrent = one host thread and stream per region, overlapping on the GPU; "
                         "serial = the regions one after another, each with the whole GPU; lockstep = every "
                         "region's t-th bond step together, their FP32 splits in one grouped Jacobi launch")
    return ap.parse_args()


SCHEDULES = {"concurrent": 0, "serial": 1, "lockstep": 2}   # dmrg_sweep_params.serial_regions


def op_mode(args, mpo, qn, mps, center):
    """Repeated matvecs at the benchmark bond through dmrg_heff_apply."""
    import torch
    import paper_1301_3494_gb300 as pd
    rng = np.random.default_rng(1)
    j = center
    bl, br = mps.bonds[j], mps.bonds[j + 2]
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]

    def env(bond, flux):
        return np.concatenate([rng.standard_normal(bond[q] * bond[q - int(flux[w])])
                               for q in bond for w in range(len(flux)) if (q - int(flux[w])) in bond])

    Ld = torch.as_tensor(env(bl, f0)).cuda()
    Rd = torch.as_tensor(env(br, f2)).cuda()
    n = sum(bl[qa] * br[qa + qn[a] + qn[b]] for qa in bl for a in range(len(qn)) for b in range(len(qn))
            if qa + qn[a] + qn[b] in br)
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    bond = pd.Bond(qn, bl, br, mpo.W[j], f0, f1, mpo.W[j + 1], f2)
    prec = pd.PRECISIONS[args.precision]
    for _ in range(args.warmup):
        pd.heff_apply(bond, prec, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fl = 0.0
    for _ in range(args.steps):
        fl += pd.heff_apply(bond, prec, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"mode": "op", "workload": f"heisenberg_square_cylinder_{args.lx}x{args.ly}_m{args.m}",
                      "bond": j, "precision": args.precision, "matvec_ms_incl_plan": ms,
                      "flops_per_matvec": fl / args.steps, "tflops_incl_plan": fl / args.steps / ms / 1e9}))


# ------------------------------------------------------------------------------------------
# Workload
# ------------------------------------------------------------------------------------------
def accuracy_mode(args):
    """FP64 vs mixed precision on the 24x8 cylinder: (1) the same serial sweep schedule from the
    same seeded state in both modes; (2) one more sweep from the FP64-converged state in each mode
    and variant.  Every final state is evaluated by an FP64 engine (FP64 environments and Rayleigh
    quotient); energies, their relative differences and sweep seconds are reported."""
    import torch
    import paper_1301_3494_gb300 as pd
    mpo = wl.heisenberg_square_cylinder(args.lx, args.ly)
    qn = list(mpo.site.qn)
    L = mpo.L
    m0 = min(100, args.acc_m)
    mps = wl.isometric_mps(L, qn, 0, m0, args.seed, 0, sigma=args.sigma)
    W, flux, D = wl.pack_mpo(mpo)
    data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn) for j in range(L)])
    ramp = [min(args.acc_m, m0 * 2 ** k) for k in range(args.acc_sweeps)]
    ramp[-2:] = [args.acc_m, args.acc_m]
    res = {}
    state = None
    for prec in ("fp64", args.precision):
        eng = pd.Engine(W, flux, D, qn, 0, prec, args.kmax)
        eng.set_mps(mps.bonds, data, center=0)
        es, ts = [], []
        for m in ramp:
            t0 = time.perf_counter()
            g = eng.sweep(m, dav_tol=1e-9, dav_max_iter=12, refine_iters=0 if prec == "fp64" else 6)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            es.append(g["energy"])
        st = eng.state()
        e_own = eng.energy()
        eng.close()
        if prec == "fp64":
            state = st
            e_true = e_own
        else:
            chk = pd.Engine(W, flux, D, qn, 0, "fp64", args.kmax)
            chk.set_mps(st[0], st[1], center=st[2])
            e_true = chk.energy()
            chk.close()
        res[prec] = {"energies": es, "sweep_s": ts, "final_fp64_rq": e_true, "final_own_rq": e_own,
                     "max_trunc_err": g["max_trunc_err"]}
    # one more sweep in each precision from the same (FP64-converged) state: the precision effect
    # of one sweep, separated from the run-to-run difference of the convergence path
    same = {}
    variants = [("fp64", 0), (args.precision, 6)]
    for v in filter(None, args.acc_variants.split(",")):
        f = v.split(":")
        variants.append((f[0], int(f[1])) + ((f[2],) if len(f) > 2 else ()))
    for var in variants:
        prec, ri = var[0], var[1]
        opts = set(var[2:])
        dav_it = next((int(o[3:]) for o in opts if o.startswith("dav")), 12)
        eng = pd.Engine(W, flux, D, qn, 0, prec, args.kmax, svd_fp64="svd64" in opts)
        eng.set_mps(state[0], state[1], center=state[2])
        e0 = eng.energy()
        t0 = time.perf_counter()
        g = eng.sweep(args.acc_m, dav_tol=1e-9, dav_max_iter=dav_it, refine_iters=ri)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        key = prec if var in (("fp64", 0), (args.precision, 6)) else ":".join(str(x) for x in var)
        e_own = eng.energy()
        st = eng.state()
        eng.close()
        # the state's energy evaluated with FP64 environments (a mixed engine's own Rayleigh
        # quotient uses its FP32 environments)
        chk = pd.Engine(W, flux, D, qn, 0, "fp64", args.kmax)
        chk.set_mps(st[0], st[1], center=st[2])
        same[key] = {"E_start": e0, "E_after_sweep": chk.energy(), "E_own_environments": e_own, "sweep_s": dt,
                     "sweep_energy": g["energy"], "max_trunc_err": g["max_trunc_err"], "dav_nonconv": g["dav_nonconv"]}
        chk.close()
    e64, emx = res["fp64"]["final_fp64_rq"], res[args.precision]["final_fp64_rq"]
    s64, smx = same["fp64"]["E_after_sweep"], same[args.precision]["E_after_sweep"]
    out = {"mode": "accuracy", "workload": f"heisenberg_square_cylinder_{args.lx}x{args.ly}", "m_ramp": ramp,
           "precision": args.precision,
           "same_state_sweep": {"E_fp64": s64, "E_mixed": smx, "dE_over_E": abs(smx - s64) / abs(s64),
                                "sweep_s_fp64": same["fp64"]["sweep_s"], "sweep_s_mixed": same[args.precision]["sweep_s"],
                                "speedup": same["fp64"]["sweep_s"] / same[args.precision]["sweep_s"],
                                "E_start": same["fp64"]["E_start"]},
           "separate_runs": {"E_fp64": e64, "E_mixed": emx, "dE_over_E": abs(emx - e64) / abs(e64)},
           "variants": {k: dict(v, dE_over_E=abs(v["E_after_sweep"] - s64) / abs(s64)) for k, v in same.items()},
           "E_per_site_fp64": s64 / L, "detail": res}
    print(json.dumps(out))


def grad_mode(args):
    """Energy derivatives from the library's gradient (Hellmann-Feynman through dmrg_energy_gradient)
    against central finite differences of converged DMRG energies (step 1e-4) and, for the
    transverse-field Ising chain, the free-fermion closed form; J-Q2 16x8 cylinder: dE/dQ for a
    global scale of the plaquette couplings."""
    import torch
    import paper_1301_3494_gb300 as pd
    out = {"mode": "grad", "tfim": [], "jq2": None}

    def tfim_exact(L_, J_, h_):
        # open chain as free fermions: E0 = -sum of the singular values of the L x L bidiagonal
        # matrix with h on the diagonal and J above it
        M = np.diag(np.full(L_, float(h_))) + np.diag(np.full(L_ - 1, float(J_)), 1)
        return -float(np.sum(np.linalg.svd(M, compute_uv=False)))

    def converge(mpo, m, sweeps=6, seed=2):
        W, flux, D = wl.pack_mpo(mpo)
        qn = list(mpo.site.qn)
        eng = pd.Engine(W, flux, D, qn, mpo.qtot, "fp64", args.kmax)
        mps = wl.random_mps(mpo.L, qn, mpo.qtot, min(16, m), seed=seed)
        data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn) for j in range(mpo.L)])
        eng.set_mps(mps.bonds, data)
        ramp = [min(m, 16 * 2 ** k) for k in range(sweeps)]
        ramp[-2:] = [m, m]
        for mm in ramp:
            eng.sweep(mm, dav_tol=1e-10, dav_max_iter=40)
        torch.cuda.synchronize()
        return eng

    def directional(Wbar, Wp, Wm, step):
        return sum(float(np.sum(g * (a - b))) / (2 * step) for g, a, b in zip(Wbar, Wp.W, Wm.W))

    L, m, fd = args.grad_L, args.grad_m, 1e-4
    for h in (0.5, 1.0, 1.5):
        t0 = time.perf_counter()
        eng = converge(wl.tfim_chain(L, 1.0, h), m)
        Wbar, e = eng.energy_gradient()
        eng.close()
        dh = directional(Wbar, wl.tfim_chain(L, 1.0, h + fd), wl.tfim_chain(L, 1.0, h - fd), fd)
        dJ = directional(Wbar, wl.tfim_chain(L, 1.0 + fd, h), wl.tfim_chain(L, 1.0 - fd, h), fd)
        ep = converge(wl.tfim_chain(L, 1.0, h + fd), m)
        em = converge(wl.tfim_chain(L, 1.0, h - fd), m)
        fd_h = (ep.energy() - em.energy()) / (2 * fd)
        ep.close()
        em.close()
        st = 1e-5
        exact_h = (tfim_exact(L, 1.0, h + st) - tfim_exact(L, 1.0, h - st)) / (2 * st)
        exact_J = (tfim_exact(L, 1.0 + st, h) - tfim_exact(L, 1.0 - st, h)) / (2 * st)
        out["tfim"].append({"L": L, "m": m, "h": h, "E": e, "E_exact": tfim_exact(L, 1.0, h),
                            "dE_dh_gradient": dh, "dE_dh_fd": fd_h, "dE_dh_exact": exact_h,
                            "dE_dJ_gradient": dJ, "dE_dJ_exact": exact_J,
                            "rel_err_dh_vs_exact": abs(dh - exact_h) / abs(exact_h),
                            "rel_err_dJ_vs_exact": abs(dJ - exact_J) / abs(exact_J),
                            "rel_err_dh_vs_fd": abs(dh - fd_h) / abs(fd_h), "seconds": time.perf_counter() - t0})
    # J-Q2 16x8: dE/dQ for Q_p -> s Q_p at s = 1
    t0 = time.perf_counter()
    mpo, Jc, Qc = wl.jq2_cylinder(16, 8, seed=1)
    mj = args.grad_jq_m

    def jq(sc):
        terms, _ = wl.jq2_terms(16, 8, Jc, Qc * sc)
        return wl.build_mpo(16 * 8, wl.spin_half(), terms)

    eng = converge(mpo, mj)
    Wbar, e = eng.energy_gradient()
    eng.close()
    dQ = directional(Wbar, jq(1 + fd), jq(1 - fd), fd)
    ep, em = converge(jq(1 + fd), mj), converge(jq(1 - fd), mj)
    fd_Q = (ep.energy() - em.energy()) / (2 * fd)
    ep.close()
    em.close()
    out["jq2"] = {"lattice": "16x8 cylinder", "m": mj, "D": max(mpo.D), "E": e, "dE_dQscale_gradient": dQ,
                  "dE_dQscale_fd": fd_Q, "rel_diff": abs(dQ - fd_Q) / abs(fd_Q), "seconds": time.perf_counter() - t0}
    print(json.dumps(out))


def observe_mode(args):
    """Inverse canonical gauge (Sec. IV) of a seeded --lx x --ly cylinder state with bond dimension
    --obs-m, then every one- and nearest-neighbour two-site expectation value over the whole lattice
    in one measurement pass (dmrg_local_expectations), timed over --steps passes after --warmup.
    Checks that hold at any size: the S^z sum rule of the sector and, on sampled sites, that psi_j
    carries the Schmidt weights of both its bonds (psi_j is an orthogonality centre)."""
    import torch
    import paper_1301_3494_gb300 as pd
    mpo = wl.heisenberg_square_cylinder(args.lx, args.ly)
    qn = list(mpo.site.qn)
    L = mpo.L
    W, flux, D = wl.pack_mpo(mpo)
    eng = pd.Engine(W, flux, D, qn, mpo.qtot, "fp64", args.kmax, fp64_emulation=args.fp64_emulation)
    mps = wl.random_mps(L, qn, mpo.qtot, args.obs_m, seed=args.seed, sigma=args.sigma)
    data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn) for j in range(L)])
    eng.set_mps(mps.bonds, data)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng.inverse_canonical()
    torch.cuda.synchronize()
    gauge_s = time.perf_counter() - t0
    st = mpo.site
    Sz, Sp, Sm, I2 = st.op("Sz"), st.op("Sp"), st.op("Sm"), np.eye(st.d)
    ops1 = [Sz, Sz @ Sz, Sp + Sm, np.diag(np.arange(1.0, st.d + 1))]
    ops2 = [np.kron(Sz, Sz) + 0.5 * (np.kron(Sp, Sm) + np.kron(Sm, Sp)), np.kron(Sz, I2), np.kron(I2, Sz),
            np.kron(Sp, Sm)]
    for _ in range(args.warmup):
        e1, e2, _ = eng.local_expectations(ops1, ops2)
    ms = []
    for _ in range(args.steps):
        e1, e2, m_ = eng.local_expectations(ops1, ops2)
        ms.append(m_)
    bonds = [eng.icmps_bond(b) for b in range(L + 1)]
    psi_elems = sum(bonds[j][q] * bonds[j + 1][q + s] for j in range(L) for q in bonds[j] for s in qn
                    if q + s in bonds[j + 1])
    theta_elems = sum(bonds[j][q] * bonds[j + 2][q + a + b] for j in range(L - 1) for q in bonds[j] for a in qn
                      for b in qn if q + a + b in bonds[j + 2])
    oc_err = 0.0
    for j in (0, L // 3, L // 2, L - 1):
        blocks = wl.unpack_site(eng.icmps_site(j), bonds[j], bonds[j + 1], qn)
        for side in (0, 1):
            b = j if side == 0 else j + 1
            off = 0
            for q, k in bonds[b].items():
                lam = np.ones(1) if b in (0, L) else 1.0 / eng.icmps_v(b)[off: off + k]
                off += k
                if side == 0:
                    M = sum(x @ x.T for (ql, s), x in blocks.items() if ql == q)
                else:
                    M = sum(x.T @ x for (ql, s), x in blocks.items() if ql + qn[s] == q)
                oc_err = max(oc_err, float(np.abs(M - np.diag(lam ** 2)).max()))
    out = {"mode": "observe", "workload": f"heisenberg_square_cylinder_{args.lx}x{args.ly}_random_m{args.obs_m}",
           "fp64_gemm": "emulated on bf16 tensor cores" if args.fp64_emulation else "FP64 units",
           "sites": L, "max_bond": max(sum(b.values()) for b in bonds), "gauge_s": gauge_s,
           "measure_ms_median": float(np.median(ms)), "measure_ms_all": ms, "n_ops1": len(ops1),
           "n_ops2": len(ops2), "psi_slab_MB": psi_elems * 8 / 1e6, "theta_slab_MB": theta_elems * 8 / 1e6,
           "sz_sum": float(e1[0].sum()), "sz_sum_expected": mpo.qtot / 2, "oc_max_err_sampled": oc_err,
           "bond_energy_sum": float(e2[0].sum())}
    eng.close()
    print(json.dumps(out))


def chain_mode(args):
    """Heisenberg chain with R real-space regions (the paper's Fig. 3 / 200-site setting): the same
    m ramp of parallel sweeps in FP64 and in --precision mode from the same seeded state; per sweep
    the energy, the merge prediction fidelities 1 - |<Psi'|Psi>| and the sweep seconds; the final
    states' energies evaluated with FP64 environments and compared."""
    import torch
    import paper_1301_3494_gb300 as pd
    L = args.chain_L
    mpo = wl.heisenberg_chain(L, spin=args.chain_spin)
    qn = list(mpo.site.qn)
    W, flux, D = wl.pack_mpo(mpo)
    mps = wl.random_mps(L, qn, 0, 16, seed=args.seed)
    data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn) for j in range(L)])
    ramp = [int(x) for x in args.chain_ramp.split(",")]
    res = {}
    finals = {}
    runs = [r for r in args.chain_runs.split(",") if r] or ["fp64", args.precision]
    for run in runs:
        opts = run.split(":")
        prec = opts[0]
        e64 = "e64" in opts
        edges = 2 if "edge2" in opts else (1 if "edge" in opts else 0)
        eng = pd.Engine(W, flux, D, qn, 0, prec, args.kmax, svd_fp64="svd64" in opts,
                        fp64_emulation=(args.fp64_emulation and prec == "fp64") or e64 or edges > 0, env_fp64=e64,
                        accurate_edges=edges)
        eng.set_mps(mps.bonds, data)
        refine = next((int(o[1:]) for o in opts[1:] if o.startswith("r") and o[1:].isdigit()), 6)
        dav_it = next((int(o[1:]) for o in opts[1:] if o.startswith("d") and o[1:].isdigit()), 12)
        dav = dict(dav_tol=0.0 if "tz" in opts else 1e-9, dav_max_iter=dav_it,
                   refine_iters=0 if prec == "fp64" else refine, serial_regions=SCHEDULES[args.region_schedule])
        t0 = time.perf_counter()
        eng.setup_regions(args.regions, args.chain_warmup, ramp[0], **dav)
        t_setup = time.perf_counter() - t0
        rows = []
        for m in ramp:
            t0 = time.perf_counter()
            g = eng.sweep(m, **dav)
            torch.cuda.synchronize()
            rows.append({"m": m, "energy": g["energy"], "fidelity_min": g["min_fidelity"],
                         "fidelity_max": g["max_fidelity"], "max_trunc_err": g["max_trunc_err"],
                         "sweep_s": time.perf_counter() - t0})
        res[run] = {"setup_s": t_setup, "sweeps": rows}
        finals[run] = rows[-1]["energy"]
        eng.close()
    out = {"mode": "chain", "L": L, "spin": args.chain_spin, "regions": args.regions, "warmup": args.chain_warmup,
           "fp64_gemm": "emulated on bf16 tensor cores" if args.fp64_emulation else "FP64 units",
           "m_ramp": ramp, "final_energies": finals, "detail": res}
    if "fp64" in finals and args.precision in finals:
        out["dE_over_E_last_merge"] = abs(finals[args.precision] - finals["fp64"]) / abs(finals["fp64"])
    print(json.dumps(out))


def accuracy_leg(args, eng, W, flux, D, qn, sweep_s=None, t_start=None):
    """The accuracy half of the metric, after the timed sweeps: (1) the timed engine's state,
    exported as one MPS (the regions joined by V = Lambda^-1 at every boundary, Eq. (merge)), is
    canonicalised and evaluated by an FP64 engine; (2) from that canonical state, one FP64 serial
    sweep and one mixed-precision serial sweep (same m; Davidson to the same residual tolerance:
    FP64 iterations, or tensor-core iterations followed by FP32-accurate refinement), both
    timed; the mixed result is evaluated by an FP64 engine.  Returns the record for the JSON line."""
    import torch
    import paper_1301_3494_gb300 as pd
    emu = True      # FP64 GEMMs of the FP64 engines on the tensor cores (FP64-accurate)
    t0 = time.perf_counter()
    if args.mode == "sweeps":
        bonds, data = eng.region_state()
    else:
        bonds, data, _ = eng.state()
    eng.close()                                  # its device memory goes back for the engines below
    f64 = pd.Engine(W, flux, D, qn, 0, "fp64", args.kmax, fp64_emulation=emu)
    f64.set_mps(bonds, data)                     # canonicalised by the engine (FP64 SVDs)
    e_state = f64.energy()
    b0, d0, c0 = f64.state()
    t_canon = time.perf_counter() - t0
    if sweep_s is not None and t_start is not None:
        # the FP64 serial sweep took ~5x a serial-schedule parallel sweep, the mixed one ~1.3x, evaluation
        # ~0.5x; the lockstep schedule speeds up the timed sweeps but not these serial ones (measured
        # together ~340 s at 24x8, m = 2000), so the estimate never drops below that
        projected = time.perf_counter() - t_start + max(7.0 * sweep_s, 420.0)
        if projected > args.time_budget_s:
            f64.close()
            return {"E_fp64_eval_of_timed_state": e_state, "canonicalise_and_evaluate_s": t_canon,
                    "same_state_sweep": {"skipped": f"projected end of run {projected:.0f} s beyond the "
                                                    f"{args.time_budget_s:.0f} s budget"}}
    torch.cuda.synchronize()
    t = time.perf_counter()
    g64 = f64.sweep(args.m, dav_tol=args.acc_tol, dav_max_iter=args.acc_iters, refine_iters=0)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t
    e_fp64 = f64.energy()
    f64.close()
    env64 = args.env_fp64
    mx = pd.Engine(W, flux, D, qn, 0, args.precision, args.kmax, fp64_emulation=True, env_fp64=env64)
    mx.set_mps(b0, d0, center=c0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    gmx = mx.sweep(args.m, dav_tol=args.acc_tol, dav_max_iter=args.dav_iters, refine_iters=args.acc_refine)
    torch.cuda.synchronize()
    mixed_s = time.perf_counter() - t
    b1, d1, c1 = mx.state()
    e_mixed_own = mx.energy()
    mx.close()
    ev = pd.Engine(W, flux, D, qn, 0, "fp64", args.kmax, fp64_emulation=emu)
    ev.set_mps(b1, d1, center=c1)
    e_mixed = ev.energy()
    ev.close()
    return {
        "E_fp64_eval_of_timed_state": e_state,
        "same_state_sweep": {
            "E_start": e_state, "E_fp64": e_fp64, "E_mixed_fp64_eval": e_mixed, "E_mixed_own_environments": e_mixed_own,
            "dE_over_E": abs(e_mixed - e_fp64) / abs(e_fp64), "fp64_sweep_s": fp64_s, "mixed_sweep_s": mixed_s,
            "speedup": fp64_s / mixed_s, "schedule": "serial sweep (L - 1 steps right, L - 1 left), both precisions",
            "davidson": (f"residual <= {args.acc_tol:g} max(1, |E|); FP64: <= {args.acc_iters} iterations; mixed: <= "
                         f"{args.dav_iters} tensor-core + <= {args.acc_refine} FP32-accurate iterations"),
            "dav_nonconverged": {"fp64": g64["dav_nonconv"], "mixed": gmx["dav_nonconv"]},
            "max_trunc_err": {"fp64": g64["max_trunc_err"], "mixed": gmx["max_trunc_err"]},
            "fp64_gemm": "emulated on bf16 tensor cores (FP64-accurate)" if emu else "FP64 units"},
        "canonicalise_and_evaluate_s": t_canon,
    }


def workload(args):
    if args.lattice == "triangular":
        mpo = wl.heisenberg_triangular_cylinder(args.lx, args.ly)
    else:
        mpo = wl.heisenberg_square_cylinder(args.lx, args.ly)
    qn = list(mpo.site.qn)
    L = mpo.L
    if args.mode == "sweeps":
        center = 0
        mps = wl.isometric_mps(L, qn, 0, args.m, args.seed, 0, sigma=args.sigma)
    else:
        center = L // 2 - (args.warmup + args.steps) // 2
        mps = wl.isometric_mps(L, qn, 0, args.m, args.seed, center, sigma=args.sigma)
    return mpo, qn, mps, center


def heff_flops(bl, br, qn, W1, f0, W2, f2):
    """Algorithmic flops of one projected-Hamiltonian application with nonzero blocks and
    nonzero MPO channels only: L stage (2 m_c m_a' m_a per kept block pair), MPO mixing
    (2 flops per element per term), R stage (2 m_c' m_a' m_c per segment).  Counting only."""
    d = len(qn)
    W12 = np.einsum("aijb,bklc->aijklc", W1, W2)
    nz = np.argwhere(W12 != 0)
    used = {(int(w), int(s1p), int(s2p)) for w, _, s1p, _, s2p, _ in nz}
    blocks = [(qa, s1, s2) for qa in bl for s1 in range(d) for s2 in range(d) if qa + qn[s1] + qn[s2] in br]
    fl = 0.0
    X = {}
    for (qa, s1p, s2p) in blocks:
        qc = qa + qn[s1p] + qn[s2p]
        for w in range(W1.shape[0]):
            qab = qa + int(f0[w])
            if (w, s1p, s2p) in used and qab in bl:
                X[(w, qa, s1p, s2p)] = (qab, qc)
                fl += 2.0 * br[qc] * bl[qab] * bl[qa]
    groups = {}
    for w, s1, s1p, s2, s2p, w2 in nz:
        for (qa, a1, a2) in blocks:
            if a1 != s1p or a2 != s2p or (w, qa, a1, a2) not in X:
                continue
            qab, qc = X[(w, qa, a1, a2)]
            qcb = qab + qn[s1] + qn[s2]
            if qcb not in br or (qcb - int(f2[w2])) not in br:
                continue
            g = groups.setdefault((qab, int(s1), int(s2), int(w2)), [0, qab, qc])
            g[0] += 1
    for (qab, s1, s2, w2), (nt, _, qc) in groups.items():
        qcb = qab + qn[s1] + qn[s2]
        fl += 2.0 * bl[qab] * br[qc] * nt + 2.0 * br[qcb] * bl[qab] * br[qc]
    return fl


# ------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ------------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for i, nm in enumerate(names):
                if "Active" in r[5 + i] and "Not" not in r[5 + i]:
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def ncu_traffic(name):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary (profiles/<name>.json), if any."""
    p = os.path.join(ROOT, "profiles", f"{name}.json")
    if os.path.exists(p):
        return json.load(open(p))
    return None


def fp32_peak_tflops(sm_max_mhz):
    """FP32 FMA peak of a GB300 from its unit counts: 152 SMs x 128 FP32 lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_max_mhz * 1e6 / 1e12


# ------------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline field)
# ------------------------------------------------------------------------------------------
def oracle_sample(mpo, qn, mps, j, seed=1):
    """Random environments with the exact block structure of bond j of the benchmark state."""
    from oracle import dmrg as O  # noqa: F401  (test-infrastructure import, CPU baseline only)
    rng = np.random.default_rng(seed)
    bl, br = mps.bonds[j], mps.bonds[j + 2]
    f0, f2 = mpo.flux[j], mpo.flux[j + 2]

    def env(bond, flux):
        return {(q, w): rng.standard_normal((bond[q], bond[q - int(flux[w])]))
                for q in bond for w in range(len(flux)) if (q - int(flux[w])) in bond}

    Lenv, Renv = env(bl, f0), env(br, f2)
    psi = {(qa, s1, s2): rng.standard_normal((bl[qa], br[qa + qn[s1] + qn[s2]]))
           for qa in bl for s1 in range(len(qn)) for s2 in range(len(qn)) if qa + qn[s1] + qn[s2] in br}
    fl = heff_flops(bl, br, qn, mpo.W[j], f0, mpo.W[j + 1], f2)
    return (Lenv, mpo.W[j], f0, mpo.W[j + 1], f2, Renv, psi, qn), fl


def time_oracle(sample, budget_s, min_reps=1):
    from oracle import dmrg as O
    args, fl = sample
    reps, t_tot = 0, 0.0
    while reps < min_reps or t_tot < budget_s:
        t0 = time.perf_counter()
        O.heff_apply(*args)
        t_tot += time.perf_counter() - t0
        reps += 1
    return fl * reps / t_tot / 1e12, reps, t_tot


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


# ------------------------------------------------------------------------------------------
# Distributed helpers (independent replicas, one per GPU)
# ------------------------------------------------------------------------------------------
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        return rank, world, dist
    return rank, world, None


def rooflines(precision, fp64_emulation, prof, rates, pk, pk_kind):
    """Roofline records of the matvec GEMM (the metric's kernel) and of the block-Jacobi SVD kernel
    from the library's profile of the timed steps; returns (roofline, roofline_other): the first is
    whichever of the two took more device time."""
    if precision == "fp64":
        g_ms, g_fl, g_n = prof["f64_gemm_ms"], prof["f64_gemm_flops"], prof["f64_gemm_launches"]
        peak, bound = rates["fp64_fma"], "alu"
        peak_note = "measured FP64 FMA rate (dmrg_probe kind 0: eight independent DFMA chains per thread)"
        if fp64_emulation:
            gemm_kernel = ("k_oz_split + k_tc_gemm (bf16 slices) + k_oz_combine: every FP64 grouped GEMM of the "
                           "step, emulated")
            peak_note += ("; emulated GEMMs are counted in FP64-equivalent flops, so frac > 1 is a rate beyond "
                          "what the FP64 units can deliver")
        else:
            gemm_kernel = "k_gemm_simt<double>: every FP64 grouped GEMM of the step"
    else:
        gemm_kernel = "k_tc_gemm (matvec L and R stages)"
        g_ms, g_fl, g_n = prof["mv_gemm_ms"], prof["mv_gemm_flops"], prof["mv_gemm_launches"]
        peak = pk["bf16_tflops_sustained"] * (1.0 if precision == "bf16" else NOMINAL_TF32_OVER_BF16)
        bound = "tensor"
        peak_note = (f"{pk_kind} bf16 sustained" + ("" if precision == "bf16" else " x nominal tf32/bf16"))
    achieved = g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else 0.0
    tr = ncu_traffic(f"tc_gemm_matvec_{precision}_traffic") if precision != "fp64" else None
    roof_mv = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "traffic": tr["bytes_per_launch"] if tr else None, "kernel": gemm_kernel,
               "launches": g_n, "flops_per_launch": g_fl / max(g_n, 1), "device_ms": g_ms, "peak_source": peak_note}
    roof = roof_mv
    if prof["svd_block_calls"] > 0:
        p32 = rates["fp32_fma"]
        b_ms, b_fl, b_n = prof["svd_block_ms"], prof["svd_block_flops"], prof["svd_block_calls"]
        b_alg, b_bytes = prof["svd_block_alg_flops"], prof["svd_block_alg_bytes"]
        a_alg = b_alg / (b_ms * 1e-3) / 1e12 if b_ms > 0 else 0.0
        a32 = b_fl / (b_ms * 1e-3) / 1e12 if b_ms > 0 else 0.0
        # DRAM bytes per algorithmic byte from a small-case capture of the same kernel, times this
        # run's algorithmic bytes per launch
        trs = ncu_traffic("bjacobi_queue_traffic")
        roof_svd = {"bound": "alu", "achieved": a_alg, "peak": p32, "unit": "TFLOP/s", "frac": a_alg / p32,
                    "traffic": trs["dram_over_algorithmic_bytes"] * b_bytes / b_n if trs else None,
                    "kernel": "k_bjacobi_queue (FP32 block-Jacobi SVD, one launch per batch of splits)",
                    "launches": b_n, "flops_per_launch": b_alg / b_n,
                    "flops_counted": "textbook R-SVD with U and V, 4 p n^2 + 22 n^3 per p x n sector matrix",
                    "algorithmic_bytes_per_launch": b_bytes / b_n,
                    "executed_flops_per_launch": b_fl / b_n, "executed_tflops": a32,
                    "executed_note": "FP32 Gram and rotation flops the Jacobi ran (all its sweeps)",
                    "traffic_source": (f"dram/algorithmic bytes {trs['dram_over_algorithmic_bytes']:.3f} from "
                                       f"{trs['source']}" if trs else None),
                    "device_ms": b_ms,
                    "peak_source": ("measured FP32 FMA rate (dmrg_probe kind 1: eight independent FFMA chains per "
                                    f"thread); unit-count rate {fp32_peak_tflops(2070.0):.1f} TFLOP/s at 2070 MHz")}
        if b_ms > g_ms:
            roof = roof_svd
            roof_other = roof_mv
        else:
            roof_other = roof_svd
    else:
        roof_other = None
    return roof, roof_other


def max_over_ranks(dist, values, device):
    """Each value's maximum over all ranks (a job takes as long as its slowest rank); the values
    themselves on one process."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def main():
    args = parse()
    rank, world, dist = dist_init(args)
    mpo, qn, mps, center = workload(args)
    L = mpo.L
    workload_name = f"heisenberg_{args.lattice}_cylinder_{args.lx}x{args.ly}_m{args.m}"
    if args.impl == "reference":
        if rank != 0:
            return
        sample_bond = L // 2 - 1
        sample = oracle_sample(mpo, qn, mps, sample_bond)
        for _ in range(args.warmup):
            time_oracle(sample, 0.0)
        vals, t_all = [], 0.0
        for _ in range(args.steps):
            v, reps, t = time_oracle(sample, 0.0)
            vals.append(v)
            t_all += t
        value = sum(vals) / len(vals)
        cores = blas_threads()
        out = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"heisenberg_{args.lattice}_cylinder_{args.lx}x{args.ly}_m{args.m}",
                       "D": max(mpo.D), "m": args.m, "bond": sample_bond, "precision": "fp64-oracle"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"one full H_eff matvec of the CPU oracle per step at bond {sample_bond} "
                                       f"of the {args.lx}x{args.ly} m={args.m} state (random environments "
                                       "with that bond's block structure)"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(out))
        return

    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_1301_3494_gb300 as pd
    if not os.path.exists(pd.LIB_PATH):
        from paper_1301_3494_gb300 import build
        build.build()
    if args.mode == "op":
        op_mode(args, mpo, qn, mps, center)
        return
    if args.mode == "accuracy":
        accuracy_mode(args)
        return
    if args.mode == "grad":
        grad_mode(args)
        return
    if args.mode == "observe":
        observe_mode(args)
        return
    if args.mode == "chain":
        chain_mode(args)
        return
    W, flux, D = wl.pack_mpo(mpo)
    mixed = args.precision != "fp64"
    env64 = mixed and args.env_fp64
    edges = args.edges if mixed else 0
    emu = args.fp64_emulation or env64 or edges > 0
    eng = pd.Engine(W, flux, D, qn, 0, args.precision, args.kmax, fp64_emulation=emu,
                    svd_plain_jacobi=args.svd_plain_jacobi, env_fp64=env64, accurate_edges=edges)
    data = np.concatenate([wl.pack_site(mps.sites[j], mps.bonds[j], mps.bonds[j + 1], qn) for j in range(L)])
    t_setup = time.perf_counter()
    eng.set_mps(mps.bonds, data, center=center)
    # a fixed number of Davidson steps: tensor-core iterations, then an FP32-accurate refinement
    dav = dict(dav_tol=0.0, dav_max_iter=args.dav_iters, refine_iters=args.refine_iters)
    if args.mode == "sweeps":
        dav["serial_regions"] = SCHEDULES[args.region_schedule]
        eng.setup_regions(args.regions, 0, args.m, **dav)
        run_step = lambda: eng.sweep(args.m, **dav)
    else:
        run_step = lambda: eng.advance(1, args.m, **dav)
    t_setup = time.perf_counter() - t_setup
    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()
    pd.profile_reset()
    pd.profile_enable(True)
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    w0 = time.perf_counter()
    ev0.record()
    for _ in range(args.steps):
        stats.append(run_step())    # host parameters in, host statistics out, every step
    ev1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = clk.stop()
    pd.profile_enable(False)
    prof = pd.profile_read()
    dev_s = ev0.elapsed_time(ev1) * 1e-3
    dev_s, wall = max_over_ranks(dist, [dev_s, wall], "cuda")
    mv_flops = sum(s["matvec_flops"] for s in stats)
    mv_s = sum(s["matvec_seconds"] for s in stats)
    value = world * mv_flops / mv_s / 1e12
    ms_step = 1e3 * dev_s / args.steps
    # roofline of the matvec GEMM and of the block-Jacobi SVD kernel
    pk, pk_kind = peaks()
    rates = {"fp64_fma": pd.probe(0), "fp32_fma": pd.probe(1), "bf16_tc_gemm_8192": pd.probe(2),
             "tf32_tc_gemm_8192": pd.probe(3)}
    roof, roof_other = rooflines(args.precision, args.fp64_emulation, prof, rates, pk, pk_kind)
    e2e_value = world * mv_flops / wall / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": workload_name, "D": max(mpo.D),
                   "m": args.m, "sectors_at_centre": len(mps.bonds[L // 2]), "step": args.mode,
                   "dav_iters": args.dav_iters, "refine_iters": args.refine_iters, "kmax": args.kmax,
                   "precision": args.precision, "regions": args.regions if args.mode == "sweeps" else 1,
                   "region_schedule": args.region_schedule if args.mode == "sweeps" else None,
                   "l2": "inputs larger than L2 (environments and intermediates > 129 MB)",
                   "fp64_gemm": "emulated on bf16 tensor cores" if emu else "FP64 units",
                   "environments": "FP64" if (env64 or not mixed) else "FP32",
                   "boundary_solves": {0: "mixed precision", 1: "FP64 Davidson next to region boundaries and in merges",
                                       2: "FP64 Davidson and split next to region boundaries and in merges"}[edges],
                   "svd": "one-sided Jacobi on W" if args.svd_plain_jacobi else "one-sided Jacobi on R^T (Householder QR)",
                   "setup_s": t_setup},
        "sweep_s": ms_step / 1e3 if args.mode == "sweeps" else ms_step * 2 * (L - 1) / 1e3,
        "sweep_s_note": ("one real-space parallel sweep, measured" if args.mode == "sweeps"
                         else "bulk step time at m=2000 x 2(L-1) steps"),
        "merge_fidelity_max": max(s["max_fidelity"] for s in stats) if args.mode == "sweeps" else None,
        "matvecs": sum(s["n_matvec"] for s in stats),
        "refine_matvecs": sum(s["n_refine_matvec"] for s in stats),
        "refine_matvec_ms": 1e3 * sum(s["refine_seconds"] for s in stats) / max(1, sum(s["n_refine_matvec"] for s in stats)),
        "matvec_ms": 1e3 * mv_s / max(1, sum(s["n_matvec"] for s in stats)),
        "energy_last_step": stats[-1]["energy"],
        "max_trunc_err": max(s["max_trunc_err"] for s in stats),
        "roofline": roof,
        "roofline_other": roof_other,
        "e2e": {"value": e2e_value, "unit": "TFLOP/s",
                "h2d_bytes_per_step": ctypes.sizeof(pd.SweepParams),
                "d2h_bytes_per_step": ctypes.sizeof(pd.SweepStats)},
        "svd": {"calls": prof["svd_calls"], "bonds": prof["svd_bonds"], "sweeps_per_call": prof["svd_sweeps"] / max(1, prof["svd_calls"]),
                "ms_per_call": prof["svd_ms"] / max(1, prof["svd_calls"]),
                "block_calls": prof["svd_block_calls"], "block_ms": prof["svd_block_ms"],
                "fp64_calls": prof["svd_fp64_calls"], "fp64_ms": prof["svd_fp64_ms"],
                "max_sector_rows": prof["svd_max_rows"], "fp64_fallbacks": prof["svd_fp64_fallbacks"],
                "rotated_pairs_per_sweep": [h for h in prof["svd_rot_hist"] if h > 0]},
        "env_update_ms_per_step": ((prof["env_gemm_ms"] if env64 else prof["f32_gemm_ms"]) / args.steps
                                   if args.precision != "fp64" else None),
        "gpu_launches": prof["launches"],
        "measured_rates_tflops": dict(rates, source="dmrg_probe (the library's own probe kernels), CUDA events"),
        "gemm_autotuner": {"shape_classes_timed": prof["tune_classes"], "overruled_cost_model": prof["tune_changed"]},
        "clocks": clocks,
    }
    if rank == 0 and args.mode in ("sweeps", "steps") and not args.no_accuracy and args.precision != "fp64":
        out["accuracy"] = accuracy_leg(args, eng, W, flux, D, qn, sweep_s=ms_step / 1e3 * (
            1.0 if args.mode == "sweeps" else 2 * (L - 1)), t_start=T_START)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_bond = L // 2 - 1
        sample = oracle_sample(mpo, qn, mps, sample_bond)
        v, reps, t = time_oracle(sample, args.cpu_sample_s)
        out["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": blas_threads(), "kind": "oracle",
                               "sample": f"{reps} H_eff matvecs of the CPU oracle ({t:.1f} s) at bond {sample_bond} "
                                         "with random environments of that bond's block structure"}
    if rank == 0:
        print(json.dumps(out))
    eng.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
