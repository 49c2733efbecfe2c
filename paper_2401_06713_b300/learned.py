"""Learned (P/n, alpha): the parameter regressor of Sec. V on the GPU.

Sec. V sweeps the palette fraction P' = P/|V| and the list factor alpha on
each training graph, keeps the pair that minimises the objective of Eq. ml
(colors against conflict edges), and trains a regressor that maps graph
features to that pair.  Here:

* the objective is the memory-constrained form of Eq. ml: fewest colors
  C = sum_l P_l among the grid points whose conflict structure fits the
  instance's byte budget in every round (ties: fewer peak bytes); the
  library enforces the budget itself (``byte_budget``), so an infeasible
  point stops after its first over-budget count pass;
* the grid is P/n in {1/4, 1/8, 1/16, 1/32} x alpha in {1, 1.5, 2, 3};
* the features are computed on the GPU by ``picasso_features``;
* the regressor is a 5-64-64-2 GELU MLP with bf16 weights and fp32
  accumulation, trained full-batch with AdamW by the library's own forward,
  backward and optimizer kernels (``picasso_mlp_*``);
* its two outputs are log2(n/P) - 3.5 and alpha - 2, snapped to the grid;
  a non-finite or out-of-range output falls back to the paper's normal mode
  P/n = 1/8, alpha = 2 (Sec. VI).

A second network of the same shape takes Eq. ml as the paper states it: the
weight beta (an input in place of the budget term) trades colors against
conflict edges, min beta C / C_min + (1 - beta) B / B_min over the grid,
where B is the largest round's conflict CSR bytes (8 per row + 4 per entry,
the size |E_c| sets) and each term is divided by its smallest value on the
instance's grid, so that beta weighs relative excesses of two quantities of
very different scale.  Labels for beta in {0.1, ..., 0.9} come from the
same unconstrained grid runs.

Every arithmetic step of the path (features, MLP, optimizer, the runs) is a
library kernel; the host loop only orders the calls and keeps the records.
"""
from __future__ import annotations

import math
import os

import numpy as np
import torch

from . import picasso, synth

GRID_DEN = (4, 8, 16, 32)
GRID_ALPHA = (1.0, 1.5, 2.0, 3.0)
DEFAULT = (8, 2.0)
T_SHIFT = (3.5, 2.0)  # targets: log2(den) - 3.5, alpha - 2
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "regressor_weights.npz")
BETA_WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "regressor_beta_weights.npz")
BETAS = tuple(round(0.1 * k, 1) for k in range(1, 10))


def targets(den: int, alpha: float):
    return (math.log2(den) - T_SHIFT[0], alpha - T_SHIFT[1])


def snap(y0: float, y1: float):
    """Grid point nearest to the regressor's output, or the default when the
    output is not finite or far outside the grid; returns (den, alpha, fell_back)."""
    if not (math.isfinite(y0) and math.isfinite(y1)):
        return DEFAULT[0], DEFAULT[1], True
    lg, a = y0 + T_SHIFT[0], y1 + T_SHIFT[1]
    if not (1.0 <= lg <= 6.0 and 0.0 <= a <= 4.5):
        return DEFAULT[0], DEFAULT[1], True
    den = min(GRID_DEN, key=lambda d: abs(math.log2(d) - lg))
    alpha = min(GRID_ALPHA, key=lambda x: abs(x - a))
    return den, alpha, False


class Regressor:
    """Device state of the MLP: fp32 master weights, their bf16 copy, AdamW
    moments and a gradient buffer."""

    def __init__(self, init: np.ndarray | None = None, seed: int = 0, device="cuda"):
        n = picasso.mlp_param_count()
        w = synth.mlp_init(seed) if init is None else np.asarray(init, dtype=np.float32)
        assert w.shape == (n,)
        self.device = device
        self.master = torch.from_numpy(w.copy()).to(device)
        self.w = picasso.mlp_to_bf16(self.master)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.grad = torch.zeros(n, dtype=torch.float32, device=device)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=device)
        self.step_count = 0

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return picasso.mlp_forward(self.w, x)

    def loss_and_grad(self, x, t, weights=(1.0, 1.0)) -> torch.Tensor:
        picasso.mlp_backward(self.w, x, t, self.grad, self.loss_buf, weights)
        return self.loss_buf

    def step(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self.step_count += 1
        picasso.mlp_adamw(self.master, self.w, self.grad, self.m, self.v, self.step_count, lr, beta1, beta2, eps,
                          weight_decay)

    def fit(self, x: torch.Tensor, t: torch.Tensor, steps: int, lr: float = 3e-3, weight_decay: float = 1e-4,
            log_every: int = 0, lr_final: float | None = None):
        """Full-batch AdamW; the learning rate decays on a cosine to
        ``lr_final`` (default lr / 20).  Returns the loss history (host floats,
        read every ``log_every`` steps)."""
        lr_final = lr / 20 if lr_final is None else lr_final
        hist = []
        for k in range(steps):
            lr_k = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(steps - 1, 1)))
            loss = self.loss_and_grad(x, t)
            if log_every and (k % log_every == 0 or k == steps - 1):
                hist.append((k, float(loss.item())))
            self.step(lr_k, weight_decay=weight_decay)
        return hist

    def predict(self, feat: torch.Tensor):
        """feat [B, 5] -> list of (den, alpha, fell_back)."""
        y = self.forward(feat.reshape(-1, 5).contiguous()).cpu().numpy()
        return [snap(float(a), float(b)) for a, b in y]

    def save(self, path: str = WEIGHTS_PATH, **meta):
        np.savez(path, master=self.master.cpu().numpy(), **{k: np.asarray(v) for k, v in meta.items()})

    @classmethod
    def load(cls, path: str = WEIGHTS_PATH, device="cuda"):
        d = np.load(path)
        return cls(init=d["master"], device=device)


def run_config(xz: torch.Tensor, q: int, seed: int, den: int, alpha: float, budget: float | None):
    """One whole run with P/n = 1/den and alpha; returns (colors, peak
    conflict bytes, feasible).  With a budget the library stops at the first
    round whose conflict structure exceeds it (colors is then None)."""
    try:
        with picasso.Picasso(xz, q, seed=seed, palette=(1, den), alpha=alpha,
                             byte_budget=int(budget) if budget else 0) as p:
            p.run()
            c, b, _ = p.set_stats()
            return int(c[0]), int(b[0]), True
    except picasso.PicassoError as e:
        if e.status == picasso.ERR_BUDGET:
            return None, None, False
        raise


def grid_search(xz: torch.Tensor, q: int, seed: int, budget: float):
    """All grid points that can fit: a point is skipped as infeasible when a
    point with no more aggressive palette and no larger alpha already failed
    (conflict entries only grow as P shrinks or alpha grows).  Returns
    {(den, alpha): (colors, peak_bytes, feasible)}."""
    res = {}
    for den in GRID_DEN:
        for alpha in GRID_ALPHA:
            if any(not f and d <= den and a <= alpha for (d, a), (_, _, f) in res.items()):
                res[(den, alpha)] = (None, None, False)
                continue
            res[(den, alpha)] = run_config(xz, q, seed, den, alpha, budget)
    return res


def best_of(res):
    """Grid label: fewest colors among feasible points, ties to fewer peak
    bytes; the least aggressive point when none fits."""
    ok = [(c, b, k) for k, (c, b, f) in res.items() if f]
    if not ok:
        return (GRID_DEN[0], GRID_ALPHA[0])
    return min(ok, key=lambda r: (r[0], r[1], r[2]))[2]


def backoff_order(den: int, alpha: float):
    """Grid points no more aggressive than (den, alpha), most aggressive
    first: alpha is lowered before the palette grows, since colors grow with
    P/n much faster than with a shorter list."""
    pts = [(d, a) for d in GRID_DEN for a in GRID_ALPHA if d <= den and a <= alpha]
    return sorted(pts, key=lambda r: (-r[0], -r[1]))


def run_learned(reg: "Regressor", xz: torch.Tensor, q: int, seed: int, budget: float, samples: int = 1 << 16):
    """Predict (P/n, alpha) for one set and run it under its budget; if the
    library reports the budget exceeded (after the round's count pass, before
    any CSR memory is taken), step back along ``backoff_order``.  Returns
    (den, alpha, colors, peak_bytes, attempts); colors is None when not even
    the least aggressive point fits."""
    _, f = picasso.features(xz, q, seed, budget, samples)
    den, alpha, _ = reg.predict(f)[0]
    tries = 0
    for d, a in backoff_order(den, alpha):
        tries += 1
        c, b, ok = run_config(xz, q, seed, d, a, budget)
        if ok:
            return d, a, c, b, tries
    return den, alpha, None, None, tries


def grid_full(xz: torch.Tensor, q: int, seed: int):
    """Every grid point run without a budget: {(den, alpha): (colors, peak
    conflict bytes)}."""
    return {(d, a): run_config(xz, q, seed, d, a, None)[:2] for d in GRID_DEN for a in GRID_ALPHA}


def beta_objective(grid, beta: float):
    """Eq. ml on one instance's grid, each term over its smallest value:
    {(den, alpha): beta C / C_min + (1 - beta) B / B_min}."""
    cmin = min(c for c, _ in grid.values())
    bmin = min(b for _, b in grid.values())
    return {k: beta * c / cmin + (1.0 - beta) * b / bmin for k, (c, b) in grid.items()}


def beta_label(grid, beta: float):
    """Grid point minimising the weighted objective (ties: fewer colors)."""
    j = beta_objective(grid, beta)
    return min(j, key=lambda k: (j[k], grid[k][0], k))


def predict_beta(reg: "Regressor", xz: torch.Tensor, q: int, seed: int, beta: float, samples: int = 1 << 16):
    """The beta network's pick for one set: (den, alpha, fell_back)."""
    _, f = picasso.features_beta(xz, q, seed, beta, samples)
    return reg.predict(f)[0]


def instance(spec, device="cuda"):
    """(xz on the GPU, q, budget) of a ``synth.learned_specs`` entry."""
    n, q, p, budget, seed, stream = spec
    chars = synth.pauli_weighted(n, q, p, seed, stream=stream)
    codes = torch.from_numpy(chars).to(device)
    return picasso.pack(codes), q, budget


def label_set(specs, seed_base: int = 0, samples: int = 1 << 16, log=None):
    """Features [N, 5] (GPU) and grid results for every instance."""
    feats, results = [], []
    for i, spec in enumerate(specs):
        xz, q, budget = instance(spec)
        _, f = picasso.features(xz, q, seed_base + i, budget, samples)
        feats.append(f)
        results.append(grid_search(xz, q, seed_base + i, budget))
        if log and (i % 100 == 0 or i == len(specs) - 1):
            log(f"labelled {i + 1}/{len(specs)}")
        del xz
    return torch.stack(feats), results


def evaluate(reg: Regressor, specs, seed_base: int, samples: int = 1 << 16, log=None):
    """Per held-out instance: the regressor's pick, the default and the grid
    best, each with (colors, peak bytes, fits the budget)."""
    rows = []
    for i, spec in enumerate(specs):
        xz, q, budget = instance(spec)
        seed = seed_base + i
        _, f = picasso.features(xz, q, seed, budget, samples)
        den, alpha, fell_back = reg.predict(f)[0]
        grid = grid_search(xz, q, seed, budget)
        best = best_of(grid)
        row = {"n": spec[0], "q": spec[1], "p": spec[2], "budget": budget, "pick": (den, alpha),
               "fell_back": fell_back, "best": best, "best_colors": grid[best][0], "best_bytes": grid[best][1],
               "best_fits": grid[best][2], "grid": {f"{d},{a}": v for (d, a), v in grid.items()}}
        # the budget guard of run_learned, read off the grid (pruned points
        # are the ones the guard would see fail)
        row["guarded"] = next((k for k in backoff_order(den, alpha) if grid[k][2]), None)
        if row["guarded"] is not None:
            row["guarded_colors"], row["guarded_bytes"] = grid[row["guarded"]][:2]
            row["guarded_fits"] = True
        else:
            row["guarded_colors"], row["guarded_bytes"], row["guarded_fits"] = None, None, False
        for name, (d, a) in (("learned", (den, alpha)), ("default", DEFAULT)):
            c, b, _ = run_config(xz, q, seed, d, a, None)
            row[name + "_colors"], row[name + "_bytes"], row[name + "_fits"] = c, b, b <= budget
        rows.append(row)
        if log and (i % 10 == 0 or i == len(specs) - 1):
            log(f"evaluated {i + 1}/{len(specs)}: pick {den},{alpha} best {best}")
        del xz
    return rows


def label_set_beta(specs, seed_base: int = 0, samples: int = 1 << 16, log=None):
    """Features [N * len(BETAS), 5] (GPU, one row per instance and beta) and
    the matching grid labels."""
    feats, labels = [], []
    for i, spec in enumerate(specs):
        xz, q, _ = instance(spec)
        grid = grid_full(xz, q, seed_base + i)
        for beta in BETAS:
            _, f = picasso.features_beta(xz, q, seed_base + i, beta, samples)
            feats.append(f)
            labels.append(beta_label(grid, beta))
        if log and (i % 100 == 0 or i == len(specs) - 1):
            log(f"labelled {i + 1}/{len(specs)}")
        del xz
    return torch.stack(feats), labels


def evaluate_beta(reg: Regressor, specs, seed_base: int, samples: int = 1 << 16, log=None):
    """Per held-out instance and beta: the objective of the regressor's pick,
    of the default and of the grid's best (1 + its relative excess)."""
    rows = []
    for i, spec in enumerate(specs):
        xz, q, _ = instance(spec)
        seed = seed_base + i
        grid = grid_full(xz, q, seed)
        for beta in BETAS:
            den, alpha, fell_back = predict_beta(reg, xz, q, seed, beta, samples)
            j = beta_objective(grid, beta)
            best = beta_label(grid, beta)
            rows.append({"n": spec[0], "q": spec[1], "p": spec[2], "beta": beta, "pick": (den, alpha),
                         "fell_back": fell_back, "best": best, "j_pick": j[(den, alpha)], "j_best": j[best],
                         "j_default": j[DEFAULT]})
        if log and (i % 10 == 0 or i == len(specs) - 1):
            log(f"evaluated {i + 1}/{len(specs)}")
        del xz
    return rows


def summarize_beta(rows):
    r_pick = [r["j_pick"] / r["j_best"] for r in rows]
    r_def = [r["j_default"] / r["j_best"] for r in rows]
    return {"cases": len(rows),
            "learned": {"picked_best": sum(1 for r in rows if tuple(r["pick"]) == tuple(r["best"])),
                        "within_5pct_of_best": sum(1 for x in r_pick if x <= 1.05),
                        "mean_objective_over_best": float(np.mean(r_pick)),
                        "fallbacks": sum(1 for r in rows if r["fell_back"])},
            "default": {"within_5pct_of_best": sum(1 for x in r_def if x <= 1.05),
                        "mean_objective_over_best": float(np.mean(r_def))}}


def summarize(rows):
    out = {"instances": len(rows)}
    ok = [r for r in rows if r["best_fits"]]
    out["grid_best_fits"] = len(ok)
    for name in ("learned", "default"):
        fits = [r for r in ok if r[name + "_fits"]]
        ratio = [r[name + "_colors"] / r["best_colors"] for r in fits]
        out[name] = {
            "fits_budget": len(fits),
            "within_5pct_of_best_and_fits": sum(1 for x in ratio if x <= 1.05),
            "mean_colors_over_best_when_fits": float(np.mean(ratio)) if ratio else None,
            "mean_colors_over_best_all": float(np.mean([r[name + "_colors"] / r["best_colors"] for r in ok]))
            if ok else None,
            "mean_peak_bytes_over_budget": float(np.mean([r[name + "_bytes"] / r["budget"] for r in rows])),
        }
    fits = [r for r in ok if r["guarded_fits"]]
    ratio = [r["guarded_colors"] / r["best_colors"] for r in fits]
    out["learned_guarded"] = {
        "fits_budget": len(fits),
        "within_5pct_of_best_and_fits": sum(1 for x in ratio if x <= 1.05),
        "mean_colors_over_best_when_fits": float(np.mean(ratio)) if ratio else None,
    }
    out["learned"]["fallbacks"] = sum(1 for r in rows if r["fell_back"])
    out["learned"]["picked_best"] = sum(1 for r in rows if tuple(r["pick"]) == tuple(r["best"]))
    return out


def main(argv=None):
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description="Label, train and evaluate the (P/n, alpha) regressor on the GPU.")
    ap.add_argument("--train", type=int, default=2000, help="training instances (n log-uniform in [1e3, 5e4])")
    ap.add_argument("--eval", type=int, default=200, help="held-out instances")
    ap.add_argument("--eval-n", type=int, default=200000)
    ap.add_argument("--eval-q", type=int, default=56)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--report", default=None, help="JSON report path")
    ap.add_argument("--weights", default=None, help="evaluate these weights; no labelling or training")
    ap.add_argument("--objective", choices=("memory", "beta"), default="memory",
                    help="memory: fewest colors within the byte budget; beta: Eq. ml weighted by beta")
    args = ap.parse_args(argv)

    def log(msg):
        print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)

    if args.objective == "beta":
        return main_beta(args, log)
    if args.weights:
        reg = Regressor.load(args.weights)
        eval_specs = synth.learned_specs(args.eval, args.seed + 1, n_lo=args.eval_n, n_hi=args.eval_n,
                                         qs=(args.eval_q,))
        rows = evaluate(reg, eval_specs, seed_base=10 ** 6, log=log)
        summary = summarize(rows)
        log(json.dumps(summary))
        if args.report:
            with open(args.report, "w") as fh:
                json.dump({"summary": summary, "rows": rows}, fh, indent=1, default=str)
        return

    t0 = time.time()
    train_specs = synth.learned_specs(args.train, args.seed)
    feats, results = label_set(train_specs, seed_base=0, log=log)
    labels = [best_of(r) for r in results]
    t = torch.tensor([targets(d, a) for d, a in labels], dtype=torch.float32, device="cuda")
    t_label = time.time() - t0
    log(f"labels done in {t_label:.1f} s: " + json.dumps({f"{d},{a}": labels.count((d, a)) for d, a in set(labels)}))

    reg = Regressor(seed=args.seed)
    t1 = time.time()
    hist = reg.fit(feats, t, args.steps, lr=args.lr, log_every=max(1, args.steps // 20))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    picks = reg.predict(feats)
    train_acc = sum(1 for (d, a, _), lab in zip(picks, labels) if (d, a) == lab) / len(labels)
    log(f"trained {args.steps} steps in {t_train:.2f} s; loss {hist[0][1]:.4f} -> {hist[-1][1]:.4f}; "
        f"train pick accuracy {train_acc:.3f}")
    reg.save(args.out, train=args.train, steps=args.steps, seed=args.seed)

    eval_specs = synth.learned_specs(args.eval, args.seed + 1, n_lo=args.eval_n, n_hi=args.eval_n,
                                     qs=(args.eval_q,))
    t2 = time.time()
    rows = evaluate(reg, eval_specs, seed_base=10 ** 6, log=log)
    summary = summarize(rows)
    summary.update({"train_instances": args.train, "label_s": t_label, "train_s": t_train,
                    "eval_s": time.time() - t2, "loss_history": hist, "train_pick_accuracy": train_acc,
                    "eval_workload": f"n={args.eval_n} q={args.eval_q} p~U[0.1,0.5] budget n*2^U[9,15]"})
    log(json.dumps({k: v for k, v in summary.items() if k != "loss_history"}))
    if args.report:
        with open(args.report, "w") as fh:
            json.dump({"summary": summary, "rows": rows}, fh, indent=1, default=str)


def main_beta(args, log):
    """Label, train and evaluate the beta network (Eq. ml as stated)."""
    import json
    import time

    out = args.out if args.out != WEIGHTS_PATH else BETA_WEIGHTS_PATH
    eval_specs = synth.learned_specs(args.eval, args.seed + 1, n_lo=args.eval_n, n_hi=args.eval_n, qs=(args.eval_q,))
    if args.weights:
        reg = Regressor.load(args.weights)
        summary = summarize_beta(evaluate_beta(reg, eval_specs, seed_base=10 ** 6, log=log))
        log(json.dumps(summary))
        return
    t0 = time.time()
    feats, labels = label_set_beta(synth.learned_specs(args.train, args.seed), seed_base=0, log=log)
    t = torch.tensor([targets(d, a) for d, a in labels], dtype=torch.float32, device="cuda")
    t_label = time.time() - t0
    log(f"labels done in {t_label:.1f} s: " + json.dumps({f"{d},{a}": labels.count((d, a)) for d, a in set(labels)}))
    reg = Regressor(seed=args.seed)
    t1 = time.time()
    hist = reg.fit(feats, t, args.steps, lr=args.lr, log_every=max(1, args.steps // 20))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    picks = reg.predict(feats)
    train_acc = sum(1 for (d, a, _), lab in zip(picks, labels) if (d, a) == lab) / len(labels)
    log(f"trained {args.steps} steps in {t_train:.2f} s; loss {hist[0][1]:.4f} -> {hist[-1][1]:.4f}; "
        f"train pick accuracy {train_acc:.3f}")
    reg.save(out, train=args.train, steps=args.steps, seed=args.seed, objective="beta")
    t2 = time.time()
    rows = evaluate_beta(reg, eval_specs, seed_base=10 ** 6, log=log)
    summary = summarize_beta(rows)
    summary.update({"train_instances": args.train, "label_s": t_label, "train_s": t_train,
                    "eval_s": time.time() - t2, "train_pick_accuracy": train_acc,
                    "eval_workload": f"n={args.eval_n} q={args.eval_q} p~U[0.1,0.5], beta in {list(BETAS)}"})
    log(json.dumps(summary))
    if args.report:
        with open(args.report, "w") as fh:
            json.dump({"summary": summary, "rows": rows}, fh, indent=1, default=str)


if __name__ == "__main__":
    main()
