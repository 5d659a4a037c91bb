"""Learned k ladder: training data from runs of the plain method, training
of the predictor on the GPU, and the learned-versus-plain comparison.

The paper tunes no ladder (its k values are uniform, its thermalisation
test is the tempering dynamics); this module adds a predictor on top of the
unchanged sampler.  Every run below is the plain method through the C ABI
(sweeps, tempering, measurements); the judge (qsg_judge) decides when a
sample is thermalised, so only the k positions and the schedule change.

A run is log-binned: bin m holds sweeps (2^m, 2^(m+1)]; after every
`sweeps_per_swap` sweeps one tempering step and one measurement; per bin, the
energy per site of every configuration (mean over the bin's tempering steps)
and q^2 of every replica pair (from the per-pair overlap sums).

Labels of a training sample, from its plain run on the uniform ladder:
  - ladder: equal acceptance between neighbours needs dk proportional to
    1/sigma_E(k) (sigma_E = standard deviation of the action at k), so the
    target k positions are the quantiles (j+1)/K of the density sigma_E(k)
    interpolated linearly between the ladder points; the targets are their
    spacings as fractions of k_max - k_min;
  - budget: log2(sweeps at which the judge passed) / 16 (the cap if never).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import qsg as Q
from . import workloads as W


def fractions_ladder(fr, k_min, k_max):
    """k_j = k_min + (k_max - k_min) sum_{i<=j} fr_i."""
    return k_min + (k_max - k_min) * np.cumsum(np.asarray(fr, dtype=np.float64))


def uniform_fractions(K):
    return np.full(K, 1.0 / K)


def softmax(a):
    a = np.asarray(a, dtype=np.float64)
    e = np.exp(a - a.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


@dataclass
class RunResult:
    first_pass_bin: np.ndarray   # [n] first thermalised bin (-1: never)
    sweeps_to_pass: np.ndarray   # [n] 2^(m+1), or the cap 2^max_bin if never
    sigma_E: np.ndarray          # [n][K] standard deviation of the action at each ladder point (late bins)
    step_seconds: float          # GPU seconds of one step (sweeps + tempering + measurement) of the whole run
    n_samples: int
    sweeps_per_swap: int

    def gpu_seconds_per_sample(self):
        """GPU seconds spent until each sample passed (cap if never), per sample
        of the batch: steps to pass x seconds per step / samples in the run."""
        return self.sweeps_to_pass / self.sweeps_per_swap * self.step_seconds / self.n_samples


def run(groups, L, Ltau, R, seed, sweeps_per_swap, max_bin, with_sigma=True):
    """Log-binned plain-method run of several groups (each: couplings [n][2][L][L]
    and its ladder) of one size; returns a RunResult over all samples in order."""
    import torch

    shapes = [Q.Shape(L, Ltau, len(J), R, len(lad), Q.HEATBATH, Q.PBC) for J, lad in groups]
    ctx = Q.Context(shapes)
    ctx.qsg_init_samples(seed, [lad for _, lad in groups])
    for gi, (J, _) in enumerate(groups):
        ctx.qsg_set_couplings(gi, J)
    try:
        ctx.qsg_set_option(Q.OPT_GRAPH, sweeps_per_swap)
    except Q.QSGError:
        pass
    N = L * L * Ltau
    K = len(groups[0][1])
    npair = R * (R - 1) // 2
    m0 = int(math.log2(sweeps_per_swap))
    ctx.qsg_sweep(2 ** m0)  # sweeps (0, 2^m0] before the first bin
    nb = max_bin - m0
    ns = [len(J) for J, _ in groups]
    Eb = [np.zeros((nb, n, R, K)) for n in ns]
    qb = [np.zeros((nb, n, K, npair)) for n in ns]
    sE = [np.zeros((n, R, K)) for n in ns]
    sE2 = [np.zeros((n, R, K)) for n in ns]
    nsig = 0
    for bi, m in enumerate(range(m0, max_bin)):
        steps = 2 ** m // sweeps_per_swap
        pp0 = [ctx.qsg_read_pair_overlaps(g) for g in range(len(groups))]
        for _ in range(steps):
            ctx.qsg_sweep(sweeps_per_swap)
            ctx.qsg_tempering_swap()
            ctx.qsg_measure_correlators()
            for g in range(len(groups)):
                E = ctx.qsg_read_energies(g).astype(np.float64)
                Eb[g][bi] += E / N
                if with_sigma and m >= max_bin - 2:
                    sE[g] += E
                    sE2[g] += E * E
            if with_sigma and m >= max_bin - 2:
                nsig += 1
        for g in range(len(groups)):
            Eb[g][bi] /= steps
            pp1 = ctx.qsg_read_pair_overlaps(g)
            qb[g][bi] = (pp1 - pp0[g]) / (steps * Ltau * float(L * L) ** 2)
    # GPU time of one step, without host reads in between
    st = ctx.stream
    with torch.cuda.stream(st):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(32):
            ctx.qsg_sweep(sweeps_per_swap)
            ctx.qsg_tempering_swap()
            ctx.qsg_measure_correlators()
        b.record(st)
        b.synchronize()
        step_s = a.elapsed_time(b) / 32 / 1e3
    fp, sig = [], []
    for g in range(len(groups)):
        first = Q.qsg_judge(Eb[g], qb[g])
        fp.append(np.where(first >= 0, first + m0, -1))
        if with_sigma and nsig:
            mean = sE[g].sum(axis=1) / (nsig * R)
            var = sE2[g].sum(axis=1) / (nsig * R) - mean ** 2
            sig.append(np.sqrt(np.maximum(var, 0.0)))
        else:
            sig.append(np.zeros((ns[g], K)))
    fp = np.concatenate(fp)
    sweeps = np.where(fp >= 0, 2.0 ** (fp + 1), 2.0 ** max_bin)
    ctx.close()
    return RunResult(fp, sweeps, np.concatenate(sig), step_s, int(sum(ns)), sweeps_per_swap)


def ladder_targets(sigma_E, ladder, k_min, k_max, fine=4096):
    """Target spacing fractions for equal acceptance: quantiles (j+1)/K of the
    density sigma_E(k), linear between the ladder points, constant outside."""
    K = len(ladder)
    kk = np.linspace(k_min, k_max, fine)
    out = np.zeros((sigma_E.shape[0], K))
    for i, s in enumerate(sigma_E):
        rho = np.interp(kk, ladder, np.maximum(s, 1e-12))
        cum = np.concatenate([[0.0], np.cumsum(0.5 * (rho[1:] + rho[:-1]) * np.diff(kk))])
        cum /= cum[-1]
        kq = np.interp((np.arange(K) + 1) / K, cum, kk)
        kq[-1] = k_max
        out[i] = np.diff(np.concatenate([[k_min], kq])) / (k_max - k_min)
    return out


SIZE_FEATURE = 63  # model input replaced by the lattice size (the coupling feature at offset (0, 8))


def features_of(J, L, Ltau):
    """Model inputs of every sample: the 64 coupling features (computed on the
    GPU), with input SIZE_FEATURE replaced by log2(L^2 L_tau) / 16 so that one
    predictor serves several lattice sizes (the sweep budget grows steeply
    with the size, which the coupling statistics alone do not carry)."""
    ctx = Q.Context([Q.Shape(L, Ltau, len(J), 1, 1)])
    ctx.qsg_init_samples(1, [np.array([0.3])])
    ctx.qsg_set_couplings(0, J)
    X = ctx.qsg_sample_features(0)
    ctx.close()
    X[:, SIZE_FEATURE] = math.log2(L * L * Ltau) / 16.0
    return X


def training_set(study, log=print):
    """Features and labels from plain runs on the uniform ladder."""
    Xs, Ts = [], []
    lad = fractions_ladder(uniform_fractions(study.n_k), study.k_min, study.k_max)
    for si, (L, Lt) in enumerate(study.train_sizes):
        J = W.bimodal_couplings(study.n_train_per_size, L, study.seed + 100 * si)
        X = features_of(J, L, Lt)
        res = run([(J, lad)], L, Lt, study.replicas, study.seed + si, study.sweeps_per_swap, study.max_bin)
        fr = ladder_targets(res.sigma_E, lad, study.k_min, study.k_max)
        T = np.zeros((len(J), 33), dtype=np.float32)
        T[:, :32] = fr
        T[:, 32] = np.log2(res.sweeps_to_pass) / 16.0
        Xs.append(X)
        Ts.append(T)
        log(f"  training runs L={L} L_tau={Lt}: {len(J)} samples, passed {np.mean(res.first_pass_bin >= 0):.2f}, "
            f"median sweeps {np.median(res.sweeps_to_pass):.0f}")
    return np.concatenate(Xs), np.concatenate(Ts)


def he_uniform(seed):
    """He-uniform weights, zero biases, in the parameter order of qsg.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in [(128, 64), (128,), (128, 128), (128,), (33, 128), (33,)]:
        if len(shape) == 2:
            lim = math.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


def train_predictor(X, T, seed, epochs=150, batch=128, lr=2e-3):
    """Train the predictor on the GPU (qsg_mlp_train); returns (MLP, losses)."""
    n = X.shape[0]
    m = Q.MLP(max(n, 1024), batch)
    m.set_params(he_uniform(seed))
    m.set_data(X, T)
    rng = np.random.default_rng(seed)
    per = n // batch
    idx = np.concatenate([rng.permutation(n)[:per * batch].reshape(per, batch) for _ in range(epochs)])
    losses = m.train(idx.astype(np.int32), lr)
    return m, losses


def grouped_ladders(Y, k_min, k_max, group=64):
    """Predicted ladders of the samples, grouped: samples sorted by their mean
    predicted k, cut into groups of `group`, each group on the mean of its
    members' ladders (64 samples share one multispin word and one ladder)."""
    lads = np.stack([fractions_ladder(softmax(y[:32]), k_min, k_max) for y in Y])
    order = np.argsort(lads.mean(axis=1), kind="stable")
    groups = [order[i:i + group] for i in range(0, len(order), group)]
    return [(g, lads[g].mean(axis=0)) for g in groups], lads


def compare(study, mlp, log=print):
    """Plain uniform ladder against the learned ladders on fresh samples."""
    L, Lt = study.eval_size
    J = W.bimodal_couplings(study.n_eval, L, study.seed + 7777)
    lad = fractions_ladder(uniform_fractions(study.n_k), study.k_min, study.k_max)
    plain = run([(J[i:i + 64], lad) for i in range(0, len(J), 64)], L, Lt, study.replicas, study.seed + 1,
                study.sweeps_per_swap, study.max_bin, with_sigma=False)
    X = features_of(J, L, Lt)
    Y = mlp.predict(X, bf16=True)
    groups, _ = grouped_ladders(Y, study.k_min, study.k_max)
    learned = run([(J[g], gl) for g, gl in groups], L, Lt, study.replicas, study.seed + 1, study.sweeps_per_swap,
                  study.max_bin, with_sigma=False)
    order = np.concatenate([g for g, _ in groups])
    # back to the sample order of the plain arm
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    sw_l = learned.sweeps_to_pass[inv]
    out = {
        "eval_size": {"L": L, "Ltau": Lt, "samples": study.n_eval, "k": [study.k_min, study.k_max],
                      "n_k": study.n_k, "replicas": study.replicas},
        "plain": {"passed": float(np.mean(plain.first_pass_bin >= 0)),
                  "mean_sweeps": float(plain.sweeps_to_pass.mean()),
                  "gpu_s_per_sample": float(plain.gpu_seconds_per_sample().mean())},
        "learned": {"passed": float(np.mean(learned.first_pass_bin >= 0)),
                    "mean_sweeps": float(sw_l.mean()),
                    "gpu_s_per_sample": float(learned.gpu_seconds_per_sample().mean())},
        "predicted_log2_budget_vs_actual_corr": float(np.corrcoef(16.0 * Y[:, 32], np.log2(plain.sweeps_to_pass))[0, 1])
        if plain.sweeps_to_pass.std() > 0 else None,
    }
    out["gain"] = out["plain"]["gpu_s_per_sample"] / max(out["learned"]["gpu_s_per_sample"], 1e-30)
    log(f"  plain:   passed {out['plain']['passed']:.2f}, mean sweeps {out['plain']['mean_sweeps']:.0f}")
    log(f"  learned: passed {out['learned']['passed']:.2f}, mean sweeps {out['learned']['mean_sweeps']:.0f}")
    # per-sample costs in the plain arm's sample order, for paired statistics
    out["_per_sample"] = {"plain": plain.gpu_seconds_per_sample(), "learned": learned.gpu_seconds_per_sample()[inv],
                          "plain_passed": plain.first_pass_bin >= 0,
                          "learned_passed": learned.first_pass_bin[inv] >= 0,
                          "pred_log2_budget": 16.0 * Y[:, 32].astype(np.float64),
                          "log2_sweeps_plain": np.log2(plain.sweeps_to_pass)}
    return out


def per_passed(cost, passed):
    """GPU-seconds spent on the samples (each until it passed, or to the cap)
    per sample that passed the judge: the cost of one thermalised sample when
    the runs are capped (the mean of the capped costs when every sample
    passes)."""
    n = np.sum(passed, axis=-1)
    return np.sum(cost, axis=-1) / np.maximum(n, 1) + np.where(n > 0, 0.0, np.inf)


def paired_bootstrap(plain, learned, plain_passed=None, learned_passed=None, n_boot=4000, seed=0, level=0.95):
    """Gain of the learned ladders (plain cost over learned cost) and its
    percentile interval from resampling the samples, both arms together so
    that each sample keeps its own pair of outcomes.  Without pass flags the
    cost is the mean GPU-seconds per sample (capped); with them, the
    GPU-seconds per sample that passed (per_passed)."""
    plain = np.asarray(plain, dtype=np.float64)
    learned = np.asarray(learned, dtype=np.float64)
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(plain), size=(n_boot, len(plain)))
    if plain_passed is None:
        ratios = plain[idx].mean(axis=1) / learned[idx].mean(axis=1)
        point = plain.mean() / learned.mean()
    else:
        pp = np.asarray(plain_passed, dtype=bool)
        lp = np.asarray(learned_passed, dtype=bool)
        ratios = per_passed(plain[idx], pp[idx]) / per_passed(learned[idx], lp[idx])
        point = per_passed(plain, pp) / per_passed(learned, lp)
    lo, hi = np.quantile(ratios, [(1 - level) / 2, (1 + level) / 2])
    return float(point), float(lo), float(hi)


def _rank(a):
    r = np.empty(len(a))
    r[np.argsort(a, kind="stable")] = np.arange(len(a))
    return r


def study_one(study, log=print):
    """One seed of the study: training runs, training, comparison."""
    import time
    t0 = time.time()
    X, T = training_set(study, log)
    t1 = time.time()
    mlp, losses = train_predictor(X, T, study.seed)
    t2 = time.time()
    log(f"  trained on {len(X)} samples: loss {losses[:10].mean():.4f} -> {losses[-10:].mean():.4f}")
    out = compare(study, mlp, log)
    # the budget head across the training sizes: predicted against actual
    # mean log2 sweeps per size
    sizes = []
    n = study.n_train_per_size
    Yt = mlp.predict(X, bf16=True)
    for si, (L, Lt) in enumerate(study.train_sizes):
        sl = slice(si * n, (si + 1) * n)
        sizes.append({"L": L, "Ltau": Lt, "pred_mean_log2_budget": float(16.0 * Yt[sl, 32].mean()),
                      "actual_mean_log2_sweeps": float(16.0 * T[sl, 32].mean())})
    out["budget_by_training_size"] = sizes
    out["train_samples"] = int(len(X))
    out["train_loss_first_last"] = [float(losses[:10].mean()), float(losses[-10:].mean())]
    out["wall_s"] = {"training_runs": t1 - t0, "training": t2 - t1, "comparison": time.time() - t2}
    return out


def study_main(study=None, seeds=None, log=print):
    """The learned-ladder study over several seeds (training samples,
    predictor initialisation and evaluation samples all change with the
    seed): per seed, the gain in GPU-seconds per sample; pooled over every
    evaluation sample, the gain with a paired bootstrap interval; and how the
    budget head's predictions track the sweeps the judge needed."""
    from dataclasses import replace
    study = study or W.ladder_study()
    seeds = list(seeds) if seeds is not None else list(study.seeds)
    per_seed, plain_c, learned_c, plain_p, learned_p, pred, actual = [], [], [], [], [], [], []
    for sd in seeds:
        log(f" seed {sd}")
        o = study_one(replace(study, seed=sd), log)
        ps = o.pop("_per_sample")
        plain_c.append(ps["plain"])
        learned_c.append(ps["learned"])
        plain_p.append(ps["plain_passed"])
        learned_p.append(ps["learned_passed"])
        pred.append(ps["pred_log2_budget"])
        actual.append(ps["log2_sweeps_plain"])
        o["gain_per_passed_sample"] = float(per_passed(ps["plain"], ps["plain_passed"])
                                            / per_passed(ps["learned"], ps["learned_passed"]))
        per_seed.append(o)
    plain_c, learned_c = np.concatenate(plain_c), np.concatenate(learned_c)
    plain_p, learned_p = np.concatenate(plain_p), np.concatenate(learned_p)
    pred, actual = np.concatenate(pred), np.concatenate(actual)
    gain, lo, hi = paired_bootstrap(plain_c, learned_c, plain_p, learned_p)
    gain_m, lo_m, hi_m = paired_bootstrap(plain_c, learned_c)
    L, Lt = study.eval_size
    out = {
        "metric": "GPU-s/sample to pass the judge, learned vs plain ladder",
        "eval_size": {"L": L, "Ltau": Lt, "samples_per_seed": study.n_eval, "k": [study.k_min, study.k_max],
                      "n_k": study.n_k, "replicas": study.replicas, "cap_sweeps": 2 ** study.max_bin},
        "train_sizes": [list(x) for x in study.train_sizes], "train_samples_per_size": study.n_train_per_size,
        "seeds": seeds,
        "gain": gain, "gain_interval95": [lo, hi],
        "gain_is": "plain over learned GPU-seconds per sample that passed the judge (the samples' costs until "
                   "they passed or hit the cap, summed, per passing sample)",
        "interval": "paired bootstrap over the pooled evaluation samples",
        "gain_per_seed": [o["gain_per_passed_sample"] for o in per_seed],
        "gain_capped_mean": gain_m, "gain_capped_mean_interval95": [lo_m, hi_m],
        "plain_gpu_s_per_passed_sample": float(per_passed(plain_c, plain_p)),
        "learned_gpu_s_per_passed_sample": float(per_passed(learned_c, learned_p)),
        "plain_gpu_s_per_sample_capped": float(plain_c.mean()),
        "learned_gpu_s_per_sample_capped": float(learned_c.mean()),
        "plain_passed": float(np.mean([o["plain"]["passed"] for o in per_seed])),
        "learned_passed": float(np.mean([o["learned"]["passed"] for o in per_seed])),
        "budget_within_eval_size": {
            "pearson": float(np.corrcoef(pred, actual)[0, 1]) if actual.std() > 0 else None,
            "spearman": float(np.corrcoef(_rank(pred), _rank(actual))[0, 1]) if actual.std() > 0 else None,
            "pred_mean_log2": float(pred.mean()), "actual_mean_log2": float(actual.mean())},
        "budget_by_training_size": per_seed[0]["budget_by_training_size"],
        "per_seed": per_seed,
    }
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--train-per-size", type=int, default=None)
    ap.add_argument("--eval", type=int, default=None)
    ap.add_argument("--max-bin", type=int, default=None)
    ap.add_argument("--seeds", type=int, default=None, help="number of seeds (default: the study's)")
    a = ap.parse_args()
    st = W.ladder_study()
    if a.train_per_size:
        st.n_train_per_size = a.train_per_size
    if a.eval:
        st.n_eval = a.eval
    if a.max_bin:
        st.max_bin = a.max_bin
    seeds = list(st.seeds)[:a.seeds] if a.seeds else None
    print(json.dumps(study_main(st, seeds=seeds)), flush=True)
