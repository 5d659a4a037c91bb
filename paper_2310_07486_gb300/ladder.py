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


def features_of(J, L, Ltau):
    """The 64 coupling features of every sample (computed on the GPU)."""
    ctx = Q.Context([Q.Shape(L, Ltau, len(J), 1, 1)])
    ctx.qsg_init_samples(1, [np.array([0.3])])
    ctx.qsg_set_couplings(0, J)
    X = ctx.qsg_sample_features(0)
    ctx.close()
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
    return out


def study_main(study=None, log=print):
    """The whole learned-ladder study: training runs, training, comparison."""
    import time
    study = study or W.ladder_study()
    t0 = time.time()
    X, T = training_set(study, log)
    t1 = time.time()
    mlp, losses = train_predictor(X, T, study.seed)
    t2 = time.time()
    log(f"  trained on {len(X)} samples: loss {losses[:10].mean():.4f} -> {losses[-10:].mean():.4f}")
    out = compare(study, mlp, log)
    out["train_samples"] = int(len(X))
    out["train_loss_first_last"] = [float(losses[:10].mean()), float(losses[-10:].mean())]
    out["wall_s"] = {"training_runs": t1 - t0, "training": t2 - t1, "comparison": time.time() - t2}
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--train-per-size", type=int, default=None)
    ap.add_argument("--eval", type=int, default=None)
    ap.add_argument("--max-bin", type=int, default=None)
    a = ap.parse_args()
    st = W.ladder_study()
    if a.train_per_size:
        st.n_train_per_size = a.train_per_size
    if a.eval:
        st.n_eval = a.eval
    if a.max_bin:
        st.max_bin = a.max_bin
    print(json.dumps(study_main(st)), flush=True)
