"""Training and evaluation of the learned initial guess (include/gcmg_cnn.h).

Data: seeded star domains phi = r - R0 (1 + a sin(k theta + p)) on a 513^2
grid (the star generator with seeds 0, 1, ... for training and 10^6 + i for
testing), f a sum of 1-4 seeded Gaussians, g = 0 on both boundary parts, a
Dirichlet/Neumann split by a seeded line.  Targets are the discrete
solutions computed by this library's own batched solver (FP32 V-cycles in
FP64 refinement, relative residual 1e-10).

Network input (4 channels): phi, f / F_SCALE on Omega_h (0 elsewhere), g at
the ghosts (0 here), and the boundary-type mask (+1 Dirichlet ghost, -1
Neumann ghost, 0 elsewhere).  Output channel 0 is u / U_SCALE, trained with
the squared error over Omega_h u Gamma_h plus LAP_WEIGHT times the squared
h^2-scaled residual of that error on Omega_h; channel 1 is not trained.

The solve keeps the network's guess only if its FP64 defect is smaller than
that of u = 0 (guessed_start): the V-cycle remains the fallback and decides
whether the guess is used, so the converged result never depends on the
network.  evaluate() also reports, outside the timed solves, the defect one
cycle leaves when started from the guess and from u = 0 (first_cycle_defects):
the stopping test is a defect, and the BF16 network's pixel-scale noise,
amplified by the 1/h^2 of the Laplacian, keeps the guess's defect far above
that of u = 0 even after a cycle, although its error is well below ||u||.

    python -m paper_1111_0983_gb300.learn --train 4096 --steps 6000 --out weights.npz
"""
import argparse
import json
import os
import time

import numpy as np

from . import cnn, gcmg, inputs

N_GRID = 513
N_COARSE = 33
F_SCALE = 10.0
U_SCALE = 1.0
LAP_WEIGHT = 0.0
TEST_BASE = 10 ** 6
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "guess513.npz")


def problem(i, n=N_GRID):
    """(Problem, f grid) of learning domain i (n overrides the drawn size)."""
    sp = dict(inputs.star_params(i, base=0))
    sp["n"] = n
    P = inputs.star(i, base=0, params=sp)
    return P, inputs.gaussian_rhs(i, n, sp["R0"], base=0)


def network_input(S, P, f, n=N_GRID):
    """[4][n][n] FP32 input of a domain whose solver S has its bc types set,
    and its masks: unknowns (Omega_h u Gamma_h) and inside nodes (Omega_h)."""
    T = S.node_types(0) & 3
    G = S.ghosts(0)
    bc = P.bc_types(G["B"])
    x = np.zeros((4, n, n), np.float32)
    x[0] = P.phi_grid(n)
    x[1] = np.where(T == 1, f / F_SCALE, 0.0)
    mask = np.zeros(n * n, np.float32)
    mask[G["node"]] = np.where(bc, -1.0, 1.0)
    x[3] = mask.reshape(n, n)
    return x, np.stack([T > 0, T == 1])


def solve_chunk(ids, stream=None, n=N_GRID, rtol=1e-10):
    """Inputs, solutions and unknown masks of domains `ids`, solved as one batch."""
    import torch
    probs = [problem(i, n) for i in ids]
    B = gcmg.Batch([P.phi_grid(n) for P, _ in probs], N_COARSE, stream=stream, rtol=rtol, max_cycles=100)
    xs, ms = [], []
    try:
        for S, (P, f) in zip(B.domains, probs):
            for l in range(S.nlev):
                S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
            g = np.zeros(S.num_ghosts(0))
            S.set_rhs(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
            x, m = network_input(S, P, f, n)
            xs.append(x)
            ms.append(m)
        stats, _ = B.solve()
        us = []
        for k in range(len(ids)):
            u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            B.solution(k, u)
            us.append(u.float())
    finally:
        B.close()
    ok = [s["converged"] for s in stats]
    return np.stack(xs), torch.stack(us), np.stack(ms), ok


def make_dataset(ids, chunk=128, stream=None, log=print, n=N_GRID):
    """Device tensors X [N][4][n][n], U [N][n][n], M [N][2][n][n] (FP32: the
    unknowns, the inside nodes) of the domains whose solve converged, and the
    number left out."""
    import torch
    X, U, M = [], [], []
    t0 = time.perf_counter()
    bad = 0
    for s in range(0, len(ids), chunk):
        x, u, m, ok = solve_chunk(ids[s:s + chunk], stream, n)
        keep = [k for k, o in enumerate(ok) if o]   # a target must be a converged solution
        bad += len(ok) - len(keep)
        X.append(torch.from_numpy(x[keep]).cuda())
        U.append(u[torch.tensor(keep, dtype=torch.long, device=u.device)])
        M.append(torch.from_numpy(m[keep].astype(np.float32)).cuda())
        log(f"data {s + len(ok)}/{len(ids)} {time.perf_counter() - t0:.1f}s")
    return torch.cat(X), torch.cat(U), torch.cat(M), bad


def train(X, U, M, steps, batch=8, lr=1e-3, seed=0, log=print, params=None, lap_weight=LAP_WEIGHT):
    """Adam on the GPU kernels; returns (parameter vector, loss history).  The
    loss is the squared error of u on the unknowns plus lap_weight times the
    squared h^2-scaled residual of that error on the inside nodes."""
    import torch
    n = X.shape[-1]
    net = cnn.Net(batch, n, n)
    if params is None:
        rng = np.random.default_rng(seed)
        parts = []
        for ci, co in cnn.LAYERS:
            parts.append((rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci)), np.zeros(co)))
        params = cnn.pack_params(parts)
    net.set_params(params)
    rng = np.random.default_rng(seed + 1)
    tgt = torch.zeros((batch, 2, n, n), dtype=torch.float32, device="cuda")
    msk = torch.zeros((batch, 2, n, n), dtype=torch.float32, device="cuda")
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        idx = torch.from_numpy(rng.integers(0, X.shape[0], batch)).cuda()
        xb = X.index_select(0, idx).contiguous()
        tgt[:, 0] = U.index_select(0, idx) / U_SCALE
        msk.copy_(M.index_select(0, idx))
        # cosine decay of the learning rate
        lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        loss = net.train_step(xb, tgt, msk, float(msk[:, 0].sum().item()), lr_t, lap_weight,
                              float(msk[:, 1].sum().item()))
        hist.append(loss)
        if it % 500 == 0 or it == steps - 1:
            log(f"step {it} loss {loss:.3e} lr {lr_t:.2e} {time.perf_counter() - t0:.1f}s")
    p = net.get_params()
    net.close()
    return p, hist


def guessed_start(S, net, xd, md, out, fd, g0, r):
    """Initial u from the network, kept only if its FP64 defect is below the
    defect of u = 0; the V-cycle that follows converges from either start.
    Returns (u, kept, relative defect of the guess)."""
    import torch
    net.forward(xd, out)
    u = torch.where(md, out[0, 0].double() * U_SCALE, torch.zeros_like(r))
    rg = S.defect(0, u, fd, g0, r)
    r0 = S.defect(0, torch.zeros_like(u), fd, g0, r)
    if not rg < r0:
        u.zero_()
    return u, bool(rg < r0), rg / r0


def first_cycle_defects(S, u_guess, max_cycles=100):
    """Relative FP64 defect after one solver cycle started from u_guess and
    from u = 0 (untimed diagnostic; gcmg_set_max_cycles limits the solve)."""
    import torch
    S.set_max_cycles(1)
    try:
        ug = u_guess.clone()
        sg = S.solve(ug)
        uz = torch.zeros_like(u_guess)
        sz = S.solve(uz)
    finally:
        S.set_max_cycles(max_cycles)
    return float(sg["rel"][-1]), float(sz["rel"][-1])


def evaluate(params, ids, rtol=1e-10, precision=1, log=print, n=N_GRID):
    """Per test domain: cycles and device time to rtol from u = 0 and from the
    network's guess (guess time included), and the guess's relative error."""
    import torch
    net = cnn.Net(1, n, n)
    net.set_params(params)
    out = torch.zeros((1, 2, n, n), dtype=torch.float32, device="cuda")
    rows = []
    for i in ids:
        P, f = problem(i, n)
        S = gcmg.Solver(P.phi_grid(n), N_COARSE, precision=precision, rtol=rtol, max_cycles=100)
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        S.set_rhs(torch.from_numpy(f).cuda(), torch.zeros(S.num_ghosts(0), dtype=torch.float64, device="cuda"))
        x, masks = network_input(S, P, f, n)
        m = masks[0]
        xd = torch.from_numpy(x[None]).cuda()
        md = torch.from_numpy(m).cuda()
        fd = torch.from_numpy(f).cuda()
        g0 = torch.zeros(S.num_ghosts(0), dtype=torch.float64, device="cuda")
        r = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        rg = float("nan")
        res = {}
        for name in ("zero", "zero", "guess", "guess"):   # second of each pair is timed warm
            u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            kept = False
            if name == "guess":
                u, kept, rg = guessed_start(S, net, xd, md, out, fd, g0, r)
            st = S.solve(u)
            b.record()
            torch.cuda.synchronize()
            res[name] = (st["cycles"], a.elapsed_time(b), st["converged"], u, kept)
        u_star = res["zero"][3]
        u0 = torch.where(md, out[0, 0].double() * U_SCALE, torch.zeros_like(u_star))
        err = float((u0 - u_star).abs().max() / u_star.abs().max())
        err2 = float((u0 - u_star).norm() / u_star.norm())
        d1g, d1z = first_cycle_defects(S, u0)
        rows.append(dict(id=int(i), cycles_zero=res["zero"][0], cycles_guess=res["guess"][0],
                         ms_zero=res["zero"][1], ms_guess=res["guess"][1],
                         converged=bool(res["zero"][2] and res["guess"][2]), guess_rel_err=err,
                         guess_rel_err_l2=err2, guess_rel_residual=float(rg),
                         guess_rel_residual_after_cycle=d1g, zero_rel_residual_after_cycle=d1z,
                         guess_kept=res["guess"][4], unknowns=int(m.sum()),
                         solution_rel_diff=float((res["guess"][3] - u_star).abs().max() / u_star.abs().max())))
        S.close()
    net.close()
    return rows


def summary(rows):
    cz = np.array([r["cycles_zero"] for r in rows])
    cg = np.array([r["cycles_guess"] for r in rows])
    tz = np.array([r["ms_zero"] for r in rows])
    tg = np.array([r["ms_guess"] for r in rows])
    unk = np.array([r["unknowns"] for r in rows])
    return dict(domains=len(rows), cycles_zero_mean=float(cz.mean()), cycles_guess_mean=float(cg.mean()),
                ms_zero_mean=float(tz.mean()), ms_guess_mean=float(tg.mean()),
                unknowns_per_s_zero=float(unk.sum() / (tz.sum() / 1e3)),
                unknowns_per_s_guess=float(unk.sum() / (tg.sum() / 1e3)),
                guess_rel_err_median=float(np.median([r["guess_rel_err"] for r in rows])),
                guess_rel_err_l2_median=float(np.median([r["guess_rel_err_l2"] for r in rows])),
                guess_rel_residual_median=float(np.median([r["guess_rel_residual"] for r in rows])),
                after_one_cycle_guess_median=float(np.median([r["guess_rel_residual_after_cycle"] for r in rows])),
                after_one_cycle_zero_median=float(np.median([r["zero_rel_residual_after_cycle"] for r in rows])),
                guesses_kept=int(sum(r["guess_kept"] for r in rows)),
                solution_rel_diff_max=float(max(r["solution_rel_diff"] for r in rows)),
                all_converged=bool(all(r["converged"] for r in rows)))


def compare_forms(params, ids, rtol=1e-10, n=N_GRID):
    """Device time and cycles to rtol on domains `ids` for the three forms:
    plain FP64 V-cycles from u = 0, FP32 V-cycles inside FP64 refinement from
    u = 0, and the same started from the learned guess (inference and its
    defect check included)."""
    f64 = evaluate(params, ids, rtol, precision=0, n=n)
    mix = evaluate(params, ids, rtol, precision=1, n=n)
    unk = sum(r["unknowns"] for r in mix)

    def form(rows, key):
        ms = sum(r["ms_" + key] for r in rows)
        return dict(ms_per_solve=ms / len(rows), unknowns_per_s=unk / (ms / 1e3),
                    cycles_mean=float(np.mean([r["cycles_" + key] for r in rows])))
    return dict(domains=len(ids), grid=n, unknowns=unk, rtol=rtol,
                f64=form(f64, "zero"), mixed=form(mix, "zero"), mixed_learned=form(mix, "guess"),
                guesses_kept=int(sum(r["guess_kept"] for r in mix)),
                guess_rel_err_median=float(np.median([r["guess_rel_err"] for r in mix])),
                guess_rel_err_l2_median=float(np.median([r["guess_rel_err_l2"] for r in mix])),
                guess_rel_residual_median=float(np.median([r["guess_rel_residual"] for r in mix])),
                after_one_cycle_guess_median=float(np.median([r["guess_rel_residual_after_cycle"] for r in mix])),
                after_one_cycle_zero_median=float(np.median([r["zero_rel_residual_after_cycle"] for r in mix])),
                cycles_per_domain=[(r["cycles_zero"], r["cycles_guess"]) for r in mix],
                all_converged=bool(all(r["converged"] for r in f64 + mix)))


def load_weights(path=WEIGHTS):
    return np.load(path)["params"].astype(np.float32)


VAL_BASE = 2 * 10 ** 6


def time_forward(reps, batch=8, n=N_GRID):
    """Device time of the network's forward pass on `batch` images (seeded
    inputs), with the tensor-core FLOPs of the six layers (padding included)."""
    import torch
    net = cnn.Net(batch, n, n)
    net.set_params(load_weights())
    x = torch.from_numpy(np.random.default_rng(0).standard_normal((batch, 4, n, n)).astype(np.float32)).cuda()
    out = torch.zeros((batch, 2, n, n), dtype=torch.float32, device="cuda")
    for _ in range(3):
        net.forward(x, out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        net.forward(x, out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    pad = 2 * max(cnn.DILATIONS)
    pix = batch * (n + pad) ** 2
    # MMA shapes: K = 16 (layer 1, 4 channels padded) or 32 input channels,
    # N = 32 output channels (16 for the last layer)
    flops = 2 * 9 * pix * (16 * 32 + 4 * 32 * 32 + 32 * 16)
    net.close()
    return dict(batch=batch, grid=n, ms_per_forward=ms, tensor_tflops=flops / (ms / 1e3) / 1e12)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lap-weights", default="0",
                    help="residual-term weights to train; the one whose guesses save most time on the "
                         "validation seeds is kept")
    ap.add_argument("--val", type=int, default=16)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--forward-only", type=int, default=0,
                    help="only time this many forward passes of a batch at 513^2 with the stored weights")
    args = ap.parse_args()
    if args.forward_only:
        print(json.dumps(time_forward(args.forward_only, args.batch)), flush=True)
        return
    X, U, M, bad = make_dataset(list(range(args.train)))
    best = None
    for beta in [float(b) for b in args.lap_weights.split(",")]:
        params, hist = train(X, U, M, args.steps, args.batch, args.lr, lap_weight=beta)
        sm = summary(evaluate(params, [VAL_BASE + i for i in range(args.val)]))
        print(json.dumps(dict(lap_weight=beta, final_loss=float(np.mean(hist[-50:])), **sm)), flush=True)
        if best is None or sm["ms_guess_mean"] < best[0]:
            best = (sm["ms_guess_mean"], beta, params, hist)
    _, beta, params, hist = best
    del X, U, M
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=params, loss=np.array(hist, np.float32), train=args.train, steps=args.steps,
             batch=args.batch, lr=args.lr, lap_weight=beta, unconverged_targets=bad)
    rows = evaluate(params, [TEST_BASE + i for i in range(args.test)])
    print(json.dumps(dict(summary(rows), train=args.train, steps=args.steps, lap_weight=beta,
                          final_loss=float(np.mean(hist[-50:])), unconverged_targets=bad)), flush=True)


if __name__ == "__main__":
    main()
