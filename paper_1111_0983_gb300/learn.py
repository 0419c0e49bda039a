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
the squared error over Omega_h u Gamma_h; channel 1 is not trained.

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
    """[4][n][n] FP32 input of a domain whose solver S has its bc types set."""
    T = S.node_types(0) & 3
    G = S.ghosts(0)
    bc = P.bc_types(G["B"])
    x = np.zeros((4, n, n), np.float32)
    x[0] = P.phi_grid(n)
    x[1] = np.where(T == 1, f / F_SCALE, 0.0)
    mask = np.zeros(n * n, np.float32)
    mask[G["node"]] = np.where(bc, -1.0, 1.0)
    x[3] = mask.reshape(n, n)
    return x, (T > 0)


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


def make_dataset(ids, chunk=128, stream=None, log=print):
    """Device tensors X [N][4][n][n], U [N][n][n], M [N][n][n] (FP32) of the
    domains whose solve converged, and the number left out."""
    import torch
    X, U, M = [], [], []
    t0 = time.perf_counter()
    bad = 0
    for s in range(0, len(ids), chunk):
        x, u, m, ok = solve_chunk(ids[s:s + chunk], stream)
        keep = [k for k, o in enumerate(ok) if o]   # a target must be a converged solution
        bad += len(ok) - len(keep)
        X.append(torch.from_numpy(x[keep]).cuda())
        U.append(u[torch.tensor(keep, dtype=torch.long, device=u.device)])
        M.append(torch.from_numpy(m[keep].astype(np.float32)).cuda())
        log(f"data {s + len(ok)}/{len(ids)} {time.perf_counter() - t0:.1f}s")
    return torch.cat(X), torch.cat(U), torch.cat(M), bad


def train(X, U, M, steps, batch=8, lr=1e-3, seed=0, log=print, params=None):
    """Adam on the GPU kernels; returns (parameter vector, loss history)."""
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
        msk[:, 0] = M.index_select(0, idx)
        # cosine decay of the learning rate
        lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        loss = net.train_step(xb, tgt, msk, float(msk.sum().item()), lr_t)
        hist.append(loss)
        if it % 500 == 0 or it == steps - 1:
            log(f"step {it} loss {loss:.3e} lr {lr_t:.2e} {time.perf_counter() - t0:.1f}s")
    p = net.get_params()
    net.close()
    return p, hist


def evaluate(params, ids, rtol=1e-10, precision=1, log=print):
    """Per test domain: cycles and device time to rtol from u = 0 and from the
    network's guess (guess time included), and the guess's relative error."""
    import torch
    n = N_GRID
    net = cnn.Net(1, n, n)
    net.set_params(params)
    out = torch.zeros((1, 2, n, n), dtype=torch.float32, device="cuda")
    rows = []
    for i in ids:
        P, f = problem(i)
        S = gcmg.Solver(P.phi_grid(n), N_COARSE, precision=precision, rtol=rtol, max_cycles=100)
        for l in range(S.nlev):
            S.set_bc_types(l, P.bc_types(S.ghosts(l)["B"]))
        S.set_rhs(torch.from_numpy(f).cuda(), torch.zeros(S.num_ghosts(0), dtype=torch.float64, device="cuda"))
        x, m = network_input(S, P, f)
        xd = torch.from_numpy(x[None]).cuda()
        md = torch.from_numpy(m).cuda()
        res = {}
        for name in ("zero", "zero", "guess", "guess"):   # second of each pair is timed warm
            u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if name == "guess":
                net.forward(xd, out)
                u.copy_(torch.where(md, out[0, 0].double() * U_SCALE, torch.zeros_like(u)))
            st = S.solve(u)
            b.record()
            torch.cuda.synchronize()
            res[name] = (st["cycles"], a.elapsed_time(b), st["converged"], u)
        u_star = res["zero"][3]
        u0 = torch.where(md, out[0, 0].double() * U_SCALE, torch.zeros_like(u_star))
        err = float((u0 - u_star).abs().max() / u_star.abs().max())
        rows.append(dict(id=int(i), cycles_zero=res["zero"][0], cycles_guess=res["guess"][0],
                         ms_zero=res["zero"][1], ms_guess=res["guess"][1],
                         converged=bool(res["zero"][2] and res["guess"][2]), guess_rel_err=err,
                         unknowns=int(m.sum())))
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
                all_converged=bool(all(r["converged"] for r in rows)))


def load_weights(path=WEIGHTS):
    return np.load(path)["params"].astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    X, U, M, bad = make_dataset(list(range(args.train)))
    params, hist = train(X, U, M, args.steps, args.batch, args.lr)
    del X, U, M
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=params, loss=np.array(hist, np.float32), train=args.train, steps=args.steps,
             batch=args.batch, lr=args.lr, unconverged_targets=bad)
    rows = evaluate(params, [TEST_BASE + i for i in range(args.test)])
    print(json.dumps(dict(summary(rows), train=args.train, steps=args.steps, final_loss=hist[-1],
                          unconverged_targets=bad)), flush=True)


if __name__ == "__main__":
    main()
