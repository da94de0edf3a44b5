"""Training and evaluation of the learned preconditioner (an extension of
the paper's solver; the paper has no network).

The preconditioner is M(v) = s net(features(v / s)) + P v with s the RMS of
v over the unknowns and P = diag(1 / (D + 1/h)) (pn_cnn_output).  Three
training modes, every step in the library's kernels (pn_cnn_forward,
pn_cnn_backward, pn_cnn_adam_step, pn_cnn_train_step, pn_apply, pn_apply_t):

* hard (default): supervised pairs (r_k, e_k) where r_k is the residual that
  plain GMRES(15) leaves after k = 0, 1, 3, 6, 10, 20 restart cycles from zero
  and e_k = x* - x_k its exact error (x* solved to 1e-8): the components a
  restarted Krylov method converges slowly on, with targets (e - P r) / s;
* residual: the loss |A M(r) - r|^2 / |r|^2 over residual pools (sources,
  partial-solve residuals, Krylov powers A^j Q, random combinations, and
  optionally the residuals FGMRES with the current network leaves), its
  gradient s gather(2 A^T (A M(r) - r)) / |r|^2 through the library's
  operator and transpose;
* supervised: exact solutions of solved sources and their combinations.

Media are seeded value-noise fBm extinction fields with albedo and g drawn
per medium.  The discrete P_N system in cell units depends only on
sigma_t h, albedo and g, so media for a grid of R cells are drawn with
sigma_t in [lo, hi] * R / 64 to match the optical thickness per cell of the
64^3 workload; the network (fully convolutional, fed log(sigma_t h)) is
trained on small grids and applied to 64^3 ones.  `compare` times flexible
GMRES with the network against plain GMRES, both inside FP64 refinement, on
held-out media.

Usage:
    python -m paper_1807_00410_gb300.learned train --out weights.npy
    python -m paper_1807_00410_gb300.learned eval --weights weights.npy
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ORDER = 3       # P3, K = 16
SIG_LO, SIG_HI = 0.5, 80.0   # sigma_t range of the 64^3 media


def medium(seed: int, R: int, tiny: bool = False):
    """Seeded fBm medium for an R^3 grid with the optical thickness per cell of
    the 64^3 workload (sigma_t in [0.5, 80] on 64^3)."""
    import pn_inputs
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    albedo = float(rng.uniform(0.8, 0.99))
    g = float(rng.uniform(0.0, 0.6))
    scale = R / 64.0
    st = (SIG_LO + (SIG_HI - SIG_LO) * pn_inputs.value_noise_fbm(R, seed)) * scale
    return st, albedo, g


def sources(seed: int, R: int, count: int):
    """Seeded source specifications: ('point', voxel) or ('beam', axis, sign, radius, centre)."""
    rng = np.random.Generator(np.random.PCG64(seed * 7 + 3))
    out = []
    for i in range(count):
        if i % 2 == 0:
            out.append(("point", tuple(int(v) for v in rng.integers(R // 8, R - R // 8, size=3))))
        else:
            out.append(("beam", int(rng.integers(3)), int(rng.choice([-1, 1])), float(rng.uniform(0.05, 0.2)),
                        (float(rng.uniform(0.3, 0.7)), float(rng.uniform(0.3, 0.7)))))
    return out


def solve_pairs(seed: int, R: int, n_src: int, torch, tol: float = 1e-6):
    """[(r32, u32, System)] for the seeded medium and sources (padded vectors)."""
    from paper_1807_00410_gb300 import System
    from paper_1807_00410_gb300 import pn as ppn
    st, albedo, g = medium(seed, R)
    st_d = torch.tensor(st, dtype=torch.float64, device="cuda")
    pairs = []
    for spec in sources(seed, R, n_src):
        if spec[0] == "point":
            Q = np.zeros((R, R, R))
            Q[spec[1]] = float(R ** 3)  # unit total strength
            sysm = System(N_ORDER, R, st_d, albedo, g, torch.tensor(Q, dtype=torch.float64, device="cuda"))
        else:
            _, axis, sign, radius, centre = spec
            Qm = ppn.single_scatter_beam(N_ORDER, st_d, albedo, g, axis, sign, radius, centre)
            sysm = System(N_ORDER, R, st_d, albedo, g, Qm)
        u = sysm.zeros(torch.float64)
        sysm.solve(u, solver="ir", tol=tol, restart=15, ortho="cgs1", max_iter=50000)
        r32 = sysm.zeros(torch.float32)
        sysm.residual(sysm.zeros(torch.float32), r32)  # r = Q - A 0 = Q in the padded layout
        pairs.append((r32, u.float(), sysm))
    return pairs


def hard_pairs(seed: int, R: int, n_src: int, torch, cycles=(0, 1, 3, 6, 10, 20), restart: int = 15):
    """Supervised pairs (r_k, e_k) for one medium: for each source, the
    residual r_k = Q - A x_k that plain GMRES(restart) leaves after k restart
    cycles from zero and its exact error e_k = x* - x_k (x* solved to 1e-8).
    The late residuals are dominated by the components restarted GMRES
    converges slowly on, the ones a preconditioner must supply."""
    out = []
    for r0, sq in source_vectors(seed, R, n_src, torch):
        xs = sq.zeros(torch.float64)
        sq.solve(xs, solver="ir", tol=1e-8, restart=restart, ortho="cgs1", max_iter=100000, raise_on_error=False)
        x = sq.zeros(torch.float32)
        done = 0
        for k in sorted(cycles):
            if k > done:
                sq.solve(x, solver="gmres", tol=1e-12, restart=restart, ortho="cgs1", max_iter=(k - done) * restart,
                         raise_on_error=False)
                done = k
            r = sq.zeros(torch.float32)
            sq.residual(x, r)
            out.append((r, (xs - x.double()).float(), sq))
        del r0
    return out


def make_hard_dataset(seeds, R: int, n_src: int, torch, log=print):
    """Features and supervised targets of hard_pairs over the media (GPU)."""
    feats, tgts = [], []
    t0 = time.time()
    for i, seed in enumerate(seeds):
        pairs = hard_pairs(seed, R, n_src, torch)
        n_act = pairs[0][2].layout.n_active
        for r, e, sq in pairs:
            rn = float(torch.linalg.vector_norm(r.double()))
            if not (rn > 0.0 and math.isfinite(rn)):
                continue
            rms = rn / math.sqrt(n_act)
            feats.append(sq.cnn_features(r, 1.0 / rms))
            tgts.append(sq.cnn_targets(e, r, 1.0 / rms))
        for sq in {id(p[2]): p[2] for p in pairs}.values():
            sq.close()
        if (i + 1) % 20 == 0:
            log(f"  data: {i + 1}/{len(seeds)} media, {len(feats)} samples, {time.time() - t0:.1f} s")
    return torch.stack(feats), torch.stack(tgts)


def make_dataset(seeds, R: int, n_src: int, n_mix: int, torch, log=print):
    """Features (S, R, R, R, K+3) and targets (S, R, R, R, K) on the GPU."""
    feats, tgts = [], []
    rng = np.random.Generator(np.random.PCG64(12345))
    t0 = time.time()
    for i, seed in enumerate(seeds):
        pairs = solve_pairs(seed, R, n_src, torch)
        sysm = pairs[0][2]
        combos = [(p[0], p[1]) for p in pairs]
        for _ in range(n_mix):
            w = rng.standard_normal(len(pairs))
            r = sum(float(wk) * p[0] for wk, p in zip(w, pairs))
            e = sum(float(wk) * p[1] for wk, p in zip(w, pairs))
            combos.append((r, e))
        n_unknowns = sysm.layout.n_active
        for r, e in combos:
            rms = float(torch.linalg.vector_norm(r.double())) / math.sqrt(n_unknowns)
            feats.append(sysm.cnn_features(r, 1.0 / rms))
            tgts.append(sysm.cnn_targets(e, r, 1.0 / rms))
        for p in pairs:
            p[2].close()
        if (i + 1) % 10 == 0:
            log(f"  data: {i + 1}/{len(seeds)} media, {len(feats)} samples, {time.time() - t0:.1f} s")
    return torch.stack(feats), torch.stack(tgts)


def source_vectors(seed: int, R: int, n_src: int, torch):
    """([r32 padded source vectors], System of the medium) for the seeded
    medium and sources."""
    from paper_1807_00410_gb300 import System
    from paper_1807_00410_gb300 import pn as ppn
    st, albedo, g = medium(seed, R)
    st_d = torch.tensor(st, dtype=torch.float64, device="cuda")
    vecs, keep = [], None
    for spec in sources(seed, R, n_src):
        if spec[0] == "point":
            Q = np.zeros((R, R, R))
            Q[spec[1]] = float(R ** 3)
            sysm = System(N_ORDER, R, st_d, albedo, g, torch.tensor(Q, dtype=torch.float64, device="cuda"))
        else:
            _, axis, sign, radius, centre = spec
            sysm = System(N_ORDER, R, st_d, albedo, g,
                          ppn.single_scatter_beam(N_ORDER, st_d, albedo, g, axis, sign, radius, centre))
        r = sysm.zeros(torch.float32)
        sysm.residual(sysm.zeros(torch.float32), r)  # r = Q
        vecs.append((r, sysm))
    return vecs


def residual_pool(seed: int, R: int, n_src: int, torch, partial=(5, 15, 45), powers=(1, 3), n_mix: int = 4,
                  rng=None):
    """(System, (n, n_elems) FP32 unit-RMS residual vectors) for one medium."""
    rng = rng or np.random.Generator(np.random.PCG64(seed))
    pairs = source_vectors(seed, R, n_src, torch)
    sysm = pairs[0][1]
    n_act = sysm.layout.n_active
    out = []

    def add(v):
        nv = float(torch.linalg.vector_norm(v.double()))
        if nv > 0.0 and math.isfinite(nv):
            out.append(v * (math.sqrt(n_act) / nv))

    for r, sq in pairs:
        add(r)
        for k in partial:
            x = sq.zeros(torch.float32)
            # stops after k iterations, unconverged: its residual is the sample
            sq.solve(x, solver="gmres", tol=1e-12, restart=15, ortho="cgs1", max_iter=k, raise_on_error=False)
            rk = sq.zeros(torch.float32)
            sq.residual(x, rk)
            add(rk)
        w = r
        for j in range(1, max(powers) + 1):
            w2 = sq.zeros(torch.float32)
            sq.apply(w, w2)
            w = w2 * (1.0 / max(float(torch.linalg.vector_norm(w2.double())), 1e-300))
            if j in powers:
                add(w)
    base = list(out)
    for _ in range(n_mix):
        c = rng.standard_normal(len(base))
        add(sum(float(ck) * v for ck, v in zip(c, base)))
    for _, sq in pairs[1:]:
        sq.close()
    return sysm, torch.stack(out)


def fgmres_residuals(net, seed: int, R: int, n_src: int, torch, cycles=(2, 5), restart: int = 15):
    """Residuals Q - A x_c that flexible GMRES with the current network leaves
    after c restart cycles, one per source and c (unit RMS, FP32): the
    components the network does not yet remove, which dominate the later
    Krylov vectors."""
    out = []
    for r, sq in source_vectors(seed, R, n_src, torch):
        n_act = sq.layout.n_active
        for c in cycles:
            u = sq.zeros(torch.float64)
            sq.solve(u, solver="ir_fgmres", tol=1e-12, restart=restart, ortho="cgs1", max_iter=c * restart,
                     max_outer=1, precond=net, raise_on_error=False)
            r64 = sq.zeros(torch.float64)
            sq.residual(u, r64)
            nv = float(torch.linalg.vector_norm(r64))
            if nv > 0.0 and math.isfinite(nv):
                out.append((r64 * (math.sqrt(n_act) / nv)).float())
        sq.close()
    return out


def residual_loss_step(net, sysm, rs, lr: float, torch):
    """One Adam step on mean_b |A M(r_b) - r_b|^2 / |r_b|^2 (rs: (B, n_elems)
    unit-RMS vectors of one medium).  Returns the loss before the step (a
    device tensor)."""
    B = rs.shape[0]
    n_act = sysm.layout.n_active
    X = torch.stack([sysm.cnn_features(rs[b], 1.0) for b in range(B)])
    out = net.forward(X)
    grads, loss = [], torch.zeros((), dtype=torch.float64, device=rs.device)
    Az = sysm.zeros(torch.float32)
    g = sysm.zeros(torch.float32)
    for b in range(B):
        z = sysm.cnn_output(out[b], 1.0, v=rs[b])
        sysm.apply(z, Az)
        q = Az - rs[b]
        loss = loss + torch.sum(q.double() ** 2) / n_act
        sysm.apply_t(q, g)
        grads.append(sysm.cnn_targets(g, None, 2.0 / n_act / B))
    net.backward(torch.stack(grads))
    net.adam_step(lr)
    return loss / B


def train_residual(net, pools, steps: int, batch: int, lr: float, torch, log=print, seed: int = 0):
    """Residual-loss training over [(System, vectors)] pools; one medium per step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    losses = []
    t0 = time.time()
    warm = max(1, steps // 20)
    pending = []
    for it in range(steps):
        sysm, vecs = pools[int(rng.integers(len(pools)))]
        idx = torch.as_tensor(rng.integers(0, vecs.shape[0], size=batch), device=vecs.device)
        lr_it = lr * min(1.0, (it + 1) / warm) * 0.5 * (1.0 + math.cos(math.pi * it / steps))
        pending.append(residual_loss_step(net, sysm, vecs[idx], lr_it, torch))
        if len(pending) >= 50:
            losses += [float(v) for v in torch.stack(pending).cpu()]
            pending = []
        if (it + 1) % max(1, steps // 10) == 0:
            if pending:
                losses += [float(v) for v in torch.stack(pending).cpu()]
                pending = []
            log(f"  train: step {it + 1}/{steps} residual loss {np.mean(losses[-50:]):.4f} ({time.time() - t0:.1f} s)")
    if pending:
        losses += [float(v) for v in torch.stack(pending).cpu()]
    return losses


def train(net, X, Y, steps: int, batch: int, lr: float, torch, log=print, seed: int = 0):
    gen = torch.Generator(device="cpu").manual_seed(seed)
    S = X.shape[0]
    losses = []
    t0 = time.time()
    warm = max(1, steps // 20)
    for it in range(steps):
        idx = torch.randint(0, S, (batch,), generator=gen).cuda()
        # linear warm-up, then cosine decay
        lr_it = lr * min(1.0, (it + 1) / warm) * 0.5 * (1.0 + math.cos(math.pi * it / steps))
        losses.append(net.train_step(X[idx], Y[idx], lr_it))
        if (it + 1) % max(1, steps // 10) == 0:
            log(f"  train: step {it + 1}/{steps} loss {np.mean(losses[-20:]):.4f} ({time.time() - t0:.1f} s)")
    return losses


def init_params(c_in: int, c_out: int, seed: int, widths=(16, 32, 48, 64)) -> np.ndarray:
    """He-style initial weights in the pn_cnn host parameter order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names_dims = [("e0a", c_in, widths[0]), ("e0b", widths[0], widths[0]), ("e1a", widths[0], widths[1]),
                  ("e1b", widths[1], widths[1]), ("e2a", widths[1], widths[2]), ("e2b", widths[2], widths[2]),
                  ("e3a", widths[2], widths[3]), ("e3b", widths[3], widths[3]),
                  ("d2", widths[3] + widths[2], widths[2]), ("d1", widths[2] + widths[1], widths[1]),
                  ("d0", widths[1] + widths[0], widths[0]), ("out", widths[0], c_out)]
    parts = []
    for name, ci, co in names_dims:
        std = math.sqrt(2.0 / (27 * ci)) * (0.1 if name == "out" else 1.0)
        parts += [rng.standard_normal(co * ci * 27) * std, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def compare(net, seeds, R: int, torch, restart: int = 15, log=print):
    """Learned FGMRES vs plain GMRES (both inside FP64 refinement) to 1e-6 on
    held-out media: wall time (CUDA events), iterations, residuals."""
    from paper_1807_00410_gb300 import System
    rows = []
    for seed in seeds:
        st, albedo, g = medium(seed, R)
        src = sources(seed, R, 1)[0]
        Q = np.zeros((R, R, R))
        Q[src[1]] = float(R ** 3)
        sysm = System(N_ORDER, R, st, albedo, g, Q)
        res = {}
        for mode in ("plain", "learned"):
            times = []
            for rep in range(2):
                u = sysm.zeros(torch.float64)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if mode == "plain":
                    s = sysm.solve(u, solver="ir", tol=1e-6, restart=restart, ortho="cgs1", max_iter=100000)
                else:
                    s = sysm.solve(u, solver="ir_fgmres", tol=1e-6, restart=restart, ortho="cgs1", max_iter=100000,
                                   precond=net)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            res[mode] = {"ms": min(times), "iterations": s["iterations"], "rel_residual": s["rel_residual"],
                         "precond_applications": s["precond_applications"], "fallback": s["fallback"]}
        rows.append({"seed": seed, **res})
        log(f"  eval seed {seed}: plain {res['plain']['ms']:.1f} ms ({res['plain']['iterations']} it), learned "
            f"{res['learned']['ms']:.1f} ms ({res['learned']['iterations']} it, fallback {res['learned']['fallback']})")
        sysm.close()
    return rows


def main(argv=None):
    import torch

    from paper_1807_00410_gb300 import Net, build
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--weights", default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--train-r", type=int, default=32)
    ap.add_argument("--media", type=int, default=200)
    ap.add_argument("--sources", type=int, default=4)
    ap.add_argument("--mix", type=int, default=4)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--loss", choices=["residual", "supervised", "hard"], default="hard",
                    help="residual: |A M(r) - r|^2 on residual pools; supervised: exact errors of solved sources; "
                         "hard: exact errors of the residuals plain GMRES leaves after k restart cycles")
    ap.add_argument("--rounds", type=int, default=1,
                    help="residual loss: after each round, add the residuals FGMRES with the network leaves "
                         "to the pools and train again")
    ap.add_argument("--eval-r", type=int, default=64)
    ap.add_argument("--eval-media", type=int, default=8)
    args = ap.parse_args(argv)
    build.build()
    K = (N_ORDER + 1) ** 2
    net = Net(K + 3, K)
    report = {}
    if args.cmd == "train":
        net.set_params(init_params(K + 3, K, seed=1))
        t0 = time.time()
        media = list(range(1000, 1000 + args.media))
        if args.loss == "residual":
            pools = []
            for i, seed in enumerate(media):
                pools.append(residual_pool(seed, args.train_r, args.sources, torch, n_mix=args.mix))
                if (i + 1) % 25 == 0:
                    print(f"  data: {i + 1}/{len(media)} media ({time.time() - t0:.1f} s)", flush=True)
            report["samples"] = int(sum(p[1].shape[0] for p in pools))
        elif args.loss == "hard":
            X, Y = make_hard_dataset(media, args.train_r, args.sources, torch)
            report["samples"] = int(X.shape[0])
        else:
            X, Y = make_dataset(media, args.train_r, args.sources, args.mix, torch)
            report["samples"] = int(X.shape[0])
        report["data_seconds"] = time.time() - t0
        t0 = time.time()
        if args.loss == "residual":
            losses = train_residual(net, pools, args.steps, args.batch, args.lr, torch)
            for rnd in range(1, args.rounds):
                t1 = time.time()
                for i, seed in enumerate(media):
                    extra = fgmres_residuals(net, seed, args.train_r, args.sources, torch)
                    if extra:
                        sysm, vecs = pools[i]
                        pools[i] = (sysm, torch.cat([vecs, torch.stack(extra)]))
                print(f"  round {rnd}: added FGMRES residuals ({time.time() - t1:.1f} s)", flush=True)
                losses = train_residual(net, pools, args.steps, args.batch, args.lr * 0.5, torch, seed=rnd)
        else:
            losses = train(net, X, Y, args.steps, args.batch, args.lr, torch)
        torch.cuda.synchronize()
        report["loss"] = args.loss
        report["train_seconds"] = time.time() - t0
        report["loss_start"] = float(np.mean(losses[:20]))
        report["loss_end"] = float(np.mean(losses[-50:]))
        if args.out:
            np.save(args.out, net.get_params())
    else:
        net.set_params(np.load(args.weights))
    xe = torch.randn((1, args.eval_r, args.eval_r, args.eval_r, K + 3), device="cuda")
    for _ in range(3):
        net.forward(xe)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        net.forward(xe)
    e1.record()
    e1.synchronize()
    report["net_forward_ms"] = e0.elapsed_time(e1) / 10
    rows = compare(net, list(range(90000, 90000 + args.eval_media)), args.eval_r, torch)
    report["eval"] = rows
    report["plain_ms_mean"] = float(np.mean([r["plain"]["ms"] for r in rows]))
    report["learned_ms_mean"] = float(np.mean([r["learned"]["ms"] for r in rows]))
    print(json.dumps(report))
    net.close()


if __name__ == "__main__":
    main()
