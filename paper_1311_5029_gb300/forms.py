"""Evaluate the solver forms on the paper-shaped synthetic workloads (one GPU).

    python -m paper_1311_5029_gb300.forms [--form multi|net|large|all] [--quick]

Each form prints one JSON line:

* ``multi``: 20^3 x 64, am0 in {0.3, 1.0, 2.5}: the 12 spin-colour point sources of one propagator
  solved as one multi-RHS batch (FP16 W, FP32 fields, FP64 reliable updates, CUDA-graph-captured
  iteration) against twelve plain FP64 BiCGStab solves; time to a true FP64 residual below 1e-10
  for every source.
* ``net``: 16^3 x 32, the learned right preconditioner: trained on (source, solution) pairs that
  this library's solver generates on 20 synthetic gauge fields with link roughness eps in
  [0.1, 0.3], then evaluated on 10 held-out fields against the unpreconditioned solver
  (iterations, wall time) and against plain FP64 BiCGStab.
* ``large``: 28^3 x 96 (2.1 M sites): memory held and time to 1e-10 for the 12 sources with the
  multi-RHS mixed-precision solve, without and with a learned preconditioner (trained for this
  mass and roughness on 16^3 x 32 fields); plain FP64 timed on two sources and scaled to twelve.

Inputs are seeded synthetic fields (no gauge ensemble is available); times are wall-clock around
the library call after one untimed warm-up solve, with the device synchronised on both sides.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import synth
import paper_1311_5029_gb300 as ok

# Reliable-update threshold of the timed mixed-precision solves (the FP32 residual must drop by
# this factor before an FP64 residual is recomputed); set by --delta.
DELTA = 1e-4


def _sync():
    import torch
    torch.cuda.synchronize()


def _timed(fn):
    _sync()
    t0 = time.perf_counter()
    out = fn()
    _sync()
    return out, 1e3 * (time.perf_counter() - t0)


def spin_colour_sources(dims, site=0):
    """The 12 unit sources at one site, [12, T, Z, Y, X, 4, 3] complex128 on the device."""
    import torch
    V = int(np.prod(dims))
    b = torch.zeros((12, V, 12), dtype=torch.complex128, device="cuda")
    for k in range(12):
        b[k, site, k] = 1.0
    return b.reshape((12,) + synth.lattice_shape(dims) + (4, 3))


def _gaussian_sources(dims, n, seed):
    """n Gaussian complex sources (re, im iid N(0, 1)) drawn on the device from a seeded generator;
    the training pairs need many, and drawing them on the host would dominate the run."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    shape = (n,) + synth.lattice_shape(dims) + (4, 3, 2)
    r = torch.randn(shape, generator=g, device="cuda", dtype=torch.float64)
    return torch.view_as_complex(r)


def _links(dims, eps, seed):
    import torch
    return torch.from_numpy(synth.random_links(dims, eps, seed)).cuda()


def form_multi(quick=False):
    w = synth.WORKLOADS["20^3x64"]
    dims = w["dims"]
    U = _links(dims, w["eps"], w["seed"])
    out = {"form": "multi_rhs", "workload": "20^3x64, 12 spin-colour point sources", "tol": 1e-10, "masses": []}
    for am0 in ((1.0,) if quick else (0.3, 1.0, 2.5)):
        W = ok.precompute_W(U, synth.placeholder_coeffs(am0), (1, 1, 1, 1), ok.W_F64 | ok.W_F16)
        b = spin_colour_sources(dims)
        nr, us = ok.autotune(W, ok.F32_W16, nrhs=12)
        ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=DELTA, check_every=8)
        (x, infos), t_multi = _timed(lambda: ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=DELTA,
                                                               check_every=8))
        worst = max(ok.true_residual(W, b[k].contiguous(), x[k].contiguous()) for k in range(12))
        nplain = 2 if quick else 12
        ok.bicgstab(W, b[0].contiguous(), tol=1e-10, mode=ok.SOLVE_F64)
        plain = []
        _sync()
        t0 = time.perf_counter()
        for k in range(nplain):
            _, ik = ok.bicgstab(W, b[k].contiguous(), tol=1e-10, mode=ok.SOLVE_F64)
            plain.append(ik["iters"])
        _sync()
        t_plain = 1e3 * (time.perf_counter() - t0) * 12 / nplain
        out["masses"].append({"am0": am0, "multi_ms": round(t_multi, 1), "plain_f64_12_ms": round(t_plain, 1),
                              "speedup_vs_plain_f64": round(t_plain / t_multi, 2),
                              "multi_iters": [i["iters"] for i in infos], "plain_f64_iters": plain,
                              "worst_true_relres": worst, "rhs_per_thread": nr, "apply_us": round(us, 1),
                              "plain_sources_timed": nplain})
        del W, b, x
    return out


def train_net(dims, am0, eps_list, per_field, layers=4, epochs=6, lr=1e-2, seed0=20000):
    """Generate (source, solution) pairs with this library's multi-RHS solver on one synthetic field
    per entry of eps_list and train a preconditioner network on them.  Returns (net, report)."""
    import torch
    c = synth.placeholder_coeffs(am0)
    t_gen0 = time.perf_counter()
    pairs = []
    for f, eps in enumerate(eps_list):
        W = ok.precompute_W(_links(dims, eps, seed0 + f), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F16 | ok.W_LINKS)
        bs, xs = [], []
        for j in range(0, per_field, 12):
            n = min(12, per_field - j)
            b = _gaussian_sources(dims, n, 10 * seed0 + 1000 * f + j)
            x, _ = ok.bicgstab_multi(W, b, tol=1e-8, mode=ok.SOLVE_MIXED16, delta=1e-2, check_every=8)
            bs.append(b.to(torch.complex64))
            xs.append(x.to(torch.complex64))
            del b, x
        pairs.append((W, torch.cat(bs), torch.cat(xs)))
    t_gen = time.perf_counter() - t_gen0
    net = ok.Net(layers)
    batch = 4
    steps = [(f, j) for f in range(len(pairs)) for j in range(0, per_field - batch + 1, batch)]
    rng = np.random.default_rng(0)
    per_epoch = []
    t_train0 = time.perf_counter()
    first = last = None
    nsteps = epochs * len(steps)
    k = 0
    for e in range(epochs):
        for i in rng.permutation(len(steps)):
            f, j = steps[i]
            W, b, x = pairs[f]
            rate = lr * (0.1 ** (k / max(nsteps - 1, 1)))  # exponential decay to lr / 10
            loss = ok.net_train_step(net, W, b[j:j + batch], x[j:j + batch], lr=rate)
            first = loss if first is None else first
            last = loss
            k += 1
        per_epoch.append(float(last))
    t_train = time.perf_counter() - t_train0
    del pairs
    torch.cuda.empty_cache()
    return net, {"layers": layers, "train_fields": len(eps_list), "pairs": len(eps_list) * per_field, "epochs": epochs,
                 "pair_generation_s": round(t_gen, 1), "training_s": round(t_train, 1), "loss_first": first,
                 "loss_last": last, "loss_per_epoch": per_epoch}


def form_net(quick=False, layers=4, epochs=6, lr=1e-2):
    import torch
    w = synth.WORKLOADS["16^3x32"]
    dims = w["dims"]
    c = synth.placeholder_coeffs(w["am0"])
    nfields, per_field, nheld = (4, 24, 3) if quick else (20, 100, 10)
    eps_list = [0.1 + 0.2 * f / max(nfields - 1, 1) for f in range(nfields)]
    net, report = train_net(dims, w["am0"], eps_list, per_field, layers, epochs, lr)
    evals = []
    for h in range(nheld):
        eps = 0.1 + 0.2 * h / max(nheld - 1, 1)
        W = ok.precompute_W(_links(dims, eps, 40000 + h), c, (1, 1, 1, 1), ok.W_F64 | ok.W_F32 | ok.W_F16 | ok.W_LINKS)
        b = torch.from_numpy(synth.gaussian_source(dims, 50000 + h)).cuda()
        if h == 0:
            ok.bicgstab(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-4)
            ok.bicgstab_net(W, net, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-4)
        (xp, ip), tp = _timed(lambda: ok.bicgstab(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-4))
        (xn, inn), tn = _timed(lambda: ok.bicgstab_net(W, net, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=1e-4))
        (x64, i64), t64 = _timed(lambda: ok.bicgstab(W, b, tol=1e-10, mode=ok.SOLVE_F64))
        evals.append({"eps": round(eps, 3), "plain_mixed16": [ip["iters"], round(tp, 1)],
                      "net_mixed16": [inn["iters"], round(tn, 1)], "plain_f64": [i64["iters"], round(t64, 1)],
                      "net_true_relres": ok.true_residual(W, b, xn)})
        del W, b
    mean = lambda key, i: float(np.mean([e[key][i] for e in evals]))  # noqa: E731
    out = {"form": "learned_preconditioner", "workload": "16^3x32", "held_out": nheld}
    out.update(report)
    out.update({"mean_iters": {"plain_mixed16": mean("plain_mixed16", 0), "net_mixed16": mean("net_mixed16", 0),
                               "plain_f64": mean("plain_f64", 0)},
                "mean_ms": {"plain_mixed16": mean("plain_mixed16", 1), "net_mixed16": mean("net_mixed16", 1),
                            "plain_f64": mean("plain_f64", 1)},
                "held_out_fields": evals})
    return out


def form_large(quick=False):
    import torch
    w = synth.WORKLOADS["28^3x96"]
    dims = w["dims"]
    # the network for this mass and roughness, trained on 16^3 x 32 fields (it is local and
    # translation invariant, so it carries over to the larger lattice)
    small = synth.WORKLOADS["16^3x32"]["dims"]
    nf = 3 if quick else 6
    net, report = train_net(small, w["am0"], [w["eps"]] * nf, 24 if quick else 48, seed0=60000)
    free0, total = torch.cuda.mem_get_info()
    W = ok.precompute_W(_links(dims, w["eps"], w["seed"]), synth.placeholder_coeffs(w["am0"]), (1, 1, 1, 1),
                        ok.W_F64 | ok.W_F16 | ok.W_LINKS)
    b = spin_colour_sources(dims)
    nr, _ = ok.autotune(W, ok.F32_W16, nrhs=12)
    (x, infos), t_multi = _timed(lambda: ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=DELTA,
                                                           check_every=8))
    worst = max(ok.true_residual(W, b[k].contiguous(), x[k].contiguous()) for k in range(12))
    free1, _ = torch.cuda.mem_get_info()
    del x
    (xn, infn), t_net = _timed(lambda: ok.bicgstab_multi(W, b, tol=1e-10, mode=ok.SOLVE_MIXED16, delta=DELTA,
                                                         check_every=8, net=net))
    worst_net = max(ok.true_residual(W, b[k].contiguous(), xn[k].contiguous()) for k in range(12))
    del xn
    nplain = 1 if quick else 2
    _sync()
    t0 = time.perf_counter()
    iters = []
    for k in range(nplain):
        _, ik = ok.bicgstab(W, b[k].contiguous(), tol=1e-10, mode=ok.SOLVE_F64)
        iters.append(ik["iters"])
    _sync()
    t_plain = 1e3 * (time.perf_counter() - t0) * 12 / nplain
    return {"form": "large_lattice", "workload": "28^3x96, 12 spin-colour point sources",
            "sites": int(np.prod(dims)), "W_bytes": W.nbytes, "device_bytes_in_use_after_solve": int(total - free1),
            "device_bytes_total": int(total), "multi_ms": round(t_multi, 1), "multi_iters": [i["iters"] for i in infos],
            "worst_true_relres": worst, "multi_net_ms": round(t_net, 1), "multi_net_iters": [i["iters"] for i in infn],
            "worst_true_relres_net": worst_net, "net_training": report,
            "plain_f64_12_ms_scaled": round(t_plain, 1), "plain_f64_iters": iters, "plain_sources_timed": nplain,
            "speedup_vs_plain_f64": round(t_plain / t_multi, 2), "speedup_net_vs_plain_f64": round(t_plain / t_net, 2),
            "rhs_per_thread": nr}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--form", default="all", choices=["multi", "net", "large", "all"])
    ap.add_argument("--quick", action="store_true", help="smaller samples (a smoke run)")
    ap.add_argument("--delta", type=float, default=DELTA, help="reliable-update threshold of the timed solves")
    a = ap.parse_args(argv)
    globals()["DELTA"] = a.delta
    forms = ["multi", "net", "large"] if a.form == "all" else [a.form]
    for f in forms:
        res = {"multi": form_multi, "net": form_net, "large": form_large}[f](quick=a.quick)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
