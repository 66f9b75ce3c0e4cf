"""Benchmark: agent-steps/s of the batched tracking-environment step on GB300.

Workload (default): 4096 envs x 5 agents x 5 targets, 2048 particles per
(agent, target) filter, dt = 30 s, targets at U[0.5, 1.5] m/s with N(0, 10 deg)
heading drift; actions from the random-init transformer agent when the
library has one, else uniform random actions.  One step = actions ->
kinematics -> targets -> pings -> communication -> particle filter
(predict/weight/estimate/resample) -> observation tokens -> reward.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The timed region replays one CUDA graph of K steps (rollout(K), captured and
uploaded before timing).  Particle state (3.4 GB) is far larger than L2
(129 MB), so no L2 flush is needed between steps.  Under torchrun the job is
one batch of N x 4096 envs and rank r steps envs [4096 r, 4096 (r+1)) with
global random-draw ids (weak scaling, no data-path collective; only the
timings and counts are reduced); rank 0 prints one JSON line.  --impl reference times the FP64 oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
METRIC = "agent-steps/s at 1 GB300 (PF vs learned estimator, RMSE within 10%); % HBM roofline"
BYTES_PER_PARTICLE = 32  # 16 B state read + 16 B written per particle-step


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


_ENVS = None


def _workload(name: str):
    from synth import preset
    return preset(name, n_envs=_ENVS)


def cpu_baseline(workload: str, budget_s: float = 12.0, n_envs: int = 64):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    n_envs environments of the same workload, as many steps as fit in the
    budget (policy forward included when the workload has one)."""
    import numpy as np

    import oracle
    import synth
    from synth import preset
    p = preset(workload, n_envs=n_envs)
    o = oracle.OracleEnv(p, 0)
    o.reset(0)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    use_policy = p.d_model > 0
    if use_policy:
        dims = synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions)
        params = synth.policy_params(dims)
        h = np.zeros((o.NA, p.d_model))
        tokens = None
    steps = 0
    t0 = time.perf_counter()
    while True:
        g = o.step_count + 1
        if use_policy and tokens is not None:
            logits, h = oracle.policy_forward(params, p.d_model, p.n_layers, p.n_heads, tokens, o.n_entities(), h,
                                              p.n_actions)
            act, _ = oracle.gumbel_actions(0, g, logits)
        else:
            act = o.random_actions(g)
        out = o.step(act, want=("tokens",) if use_policy else ())
        if use_policy:
            tokens = out["tokens"]
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    value = steps * o.NA / dt
    return {"value": value, "unit": "agent-steps/s", "cores": cores, "kind": "oracle", "per_core": value / cores,
            "sample": f"{n_envs} envs of the {workload} workload x {steps} steps ({dt:.1f} s, FP64, OpenMP)"}


def cpu_baseline_one_thread(workload: str, budget_s: float = 5.0):
    """The same oracle sample on one host thread (a child process, so that
    OpenMP starts with one thread)."""
    import subprocess
    import sys

    code = ("import json, bench; print(json.dumps(bench.cpu_baseline(%r, budget_s=%r)))" % (workload, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.abspath(__file__)), timeout=600)
    try:
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (IndexError, ValueError):
        return {"error": (r.stderr or "no output").strip().splitlines()[-1:]}


def learned_form(args, p, K, W, rank):
    """The learned-estimator form of the same workload: record ~20M
    (feature, label) transitions from filter-form rollouts, train the MLP with
    the library's kernels, then time a learned-form rollout and compare mean
    tracking RMSE against the filter form on held-out seeds."""
    import torch

    import paper_2505_08222_gb300 as ut
    import synth

    pol = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions)) if p.d_model else None
    env = ut.Env(p, ring=True)
    if pol is not None:
        env.set_policy(pol)
    F = env.F
    steps_rec = max(1, args.train_rows // F)
    X = torch.empty((steps_rec * F, 96), dtype=torch.float32, device="cuda")
    Y = torch.empty((steps_rec * F, 2), dtype=torch.float32, device="cuda")
    T_eval = args.eval_steps
    LEARNED = 2  # est_set_mode: the network also moves the estimate on steps without a fresh ping

    def record(t0_step, n_rec, seed, learned):
        # n_rec rows spread over EPISODES episodes from reset, each spanning the
        # evaluation horizon with a row every k-th step
        per = [n_rec // EPISODES + (1 if k < n_rec % EPISODES else 0) for k in range(EPISODES)]
        t = t0_step
        for k, nr in enumerate(per):
            if nr == 0:
                continue
            every = max(1, -(-T_eval // nr))
            env.est_set_mode(learned)
            env.reset(seed + 17 * k)
            for _ in range(nr):
                for _ in range(every):
                    env.step()
                env.est_record(X[t * F:(t + 1) * F], Y[t * F:(t + 1) * F])
                t += 1
        env.est_set_mode(False)

    # DAgger-style schedule: half the rows from filter-driven rollouts (the
    # filter's estimates as the update's inputs), then ROUNDS rounds of rows
    # from rollouts driven by the network itself, retraining on everything
    # recorded so far after each round.  Closed-loop quality varies with the
    # training seed, so several candidates are trained and the one with the
    # lowest RMSE on a validation seed (distinct from the held-out evaluation
    # seeds) is kept.
    def eval_rmse(learned: int, seed: int, T: int) -> float:
        env.est_set_mode(learned)
        env.reset(seed)
        return env.rollout(T)["rmse"]

    ar = torch.arange(F, device="cuda")

    def eval_split(learned: int, seed: int, T: int):
        """Pooled RMSE of T eager steps from env_reset(seed) (the same steps
        as rollout(T)), and the same pooled over the filter-steps whose
        newest received ping is from that step (fresh) and the rest."""
        env.est_set_mode(learned)
        env.reset(seed)
        acc = torch.zeros(4, dtype=torch.float64, device="cuda")
        for _ in range(T):
            out = env.step()
            st = env.state()
            ring = st["ring"].view(F, 16, 4)
            newest = ring[ar, (st["ring_head"].long() - 1) & 15, 3]
            fresh = (st["ring_count"] > 0) & (newest == float(st["step"]))
            e2 = out["err"].double() ** 2
            acc += torch.stack([e2.sum(), torch.tensor(float(F), dtype=torch.float64, device="cuda"),
                                (e2 * fresh).sum(), fresh.double().sum()])
        sq, n, sq_f, n_f = acc.tolist()
        return {"rmse": (sq / n) ** 0.5, "fresh_rmse": (sq_f / max(n_f, 1.0)) ** 0.5,
                "stale_rmse": ((sq - sq_f) / max(n - n_f, 1.0)) ** 0.5, "fresh_frac": n_f / n}

    ROUNDS, EPISODES = 8, 4
    t0 = time.perf_counter()
    half = steps_rec // 2
    rest = steps_rec - half
    chunks = [rest // ROUNDS + (1 if k < rest % ROUNDS else 0) for k in range(ROUNDS)]
    record(0, half, 7000 + rank, False)
    train_ms = 0.0
    cands = []
    for c in range(args.est_candidates):
        env.est_set_weights(synth.mlp_params(seed=4321 + c))
        tr = env.est_train(X[:half * F], Y[:half * F], steps=args.train_steps, batch=16384, lr=1e-3,
                           seed=rank + 100 * c, huber=1.0)
        losses = [tr["loss_last"]]
        train_ms += tr["ms"]
        upto = half
        for r, n in enumerate(chunks):
            record(upto, n, 7100 + 10 * r + rank + 1000 * c, LEARNED)
            upto += n
            tr = env.est_train(X[:upto * F], Y[:upto * F], steps=args.round_steps, batch=16384,
                               lr=5e-4, seed=rank + 100 * c + r + 1, huber=1.0)
            losses.append(tr["loss_last"])
            train_ms += tr["ms"]
        val = eval_rmse(LEARNED, 8000 + rank, T_eval)
        cands.append((val, c, env.est_get_weights(), losses))
    val_best, c_best, w_best, losses = min(cands, key=lambda t: t[0])
    env.est_set_weights(w_best)
    torch.cuda.synchronize()
    rec_s = time.perf_counter() - t0
    del X, Y
    torch.cuda.empty_cache()

    seeds = [9000 + rank, 9100 + rank]
    pf_rmse = [eval_rmse(False, s, T_eval) for s in seeds]
    le_rmse = [eval_rmse(LEARNED, s, T_eval) for s in seeds]
    # seeds 0-4 (held out from training and validation): per-seed ratio, and
    # the ratio over the steps with a fresh ping alone
    split_pf = [eval_split(False, sd, T_eval) for sd in range(5)]
    split_le = [eval_split(LEARNED, sd, T_eval) for sd in range(5)]
    ratios = [b["rmse"] / a["rmse"] for a, b in zip(split_pf, split_le)]

    def _pool(parts, key, wkey):
        num = sum(x[key] ** 2 * (x[wkey] if wkey else 1.0) for x in parts)
        den = sum((x[wkey] if wkey else 1.0) for x in parts)
        return (num / den) ** 0.5
    fresh_pf = _pool(split_pf, "fresh_rmse", "fresh_frac")
    fresh_le = _pool(split_le, "fresh_rmse", "fresh_frac")
    stale_pf = (sum(x["stale_rmse"] ** 2 * (1 - x["fresh_frac"]) for x in split_pf)
                / max(sum(1 - x["fresh_frac"] for x in split_pf), 1e-12)) ** 0.5
    stale_le = (sum(x["stale_rmse"] ** 2 * (1 - x["fresh_frac"]) for x in split_le)
                / max(sum(1 - x["fresh_frac"] for x in split_le), 1e-12)) ** 0.5
    # timed learned-form rollout
    env.est_set_mode(LEARNED)
    env.reset(1000 + rank)
    for _ in range(W):
        env.step()
    env.rollout_prepare(K)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    st = env.rollout(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    env.profile(True)
    for _ in range(K):
        env.step()
    est_ms, est_n = env.stage_time()
    env.profile(False)

    # least-squares trilateration tracker (est_set_mode 4) on the same seeds,
    # and a timed rollout of that form
    ls_rmse = [eval_rmse(4, s, T_eval) for s in seeds]
    env.est_set_mode(4)
    env.reset(1000 + rank)
    for _ in range(W):
        env.step()
    env.rollout_prepare(K)
    torch.cuda.synchronize()
    ev0.record(stream)
    st_ls = env.rollout(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_ls = ev0.elapsed_time(ev1)
    env.est_set_mode(0)
    env.close()
    pf_mean = sum(pf_rmse) / len(pf_rmse)
    le_mean = sum(le_rmse) / len(le_rmse)
    ls_mean = sum(ls_rmse) / len(ls_rmse)
    return {"value": st["agent_steps"] / (ms / 1e3), "unit": "agent-steps/s", "ms_per_step": ms / K,
            "estimator_kernel_ms": est_ms / max(est_n, 1),
            "rmse_m": le_mean, "pf_rmse_m": pf_mean, "rmse_ratio": le_mean / pf_mean,
            "eval": f"{len(seeds)} held-out seeds x {T_eval} steps each form, pooled RMSE per run, mean over seeds",
            "seeds_0_4": {"rmse_ratio": ratios, "mean": sum(ratios) / 5, "min": min(ratios), "max": max(ratios),
                          "pf_rmse_m": [x["rmse"] for x in split_pf], "learned_rmse_m": [x["rmse"] for x in split_le],
                          "fresh_ping_steps": {"pf_rmse_m": fresh_pf, "learned_rmse_m": fresh_le,
                                               "rmse_ratio": fresh_le / fresh_pf if fresh_pf > 0 else None,
                                               "share_of_filter_steps": sum(x["fresh_frac"] for x in split_pf) / 5},
                          "stale_steps": {"pf_rmse_m": stale_pf, "learned_rmse_m": stale_le,
                                          "rmse_ratio": stale_le / stale_pf if stale_pf > 0 else None},
                          "note": (f"seeds 0-4 (neither trained nor validated on), {T_eval} eager steps each; a "
                                   "filter-step is fresh when the filter's newest received ping is from that step")},
            "stale_rule": "network applied on steps without a fresh ping too (est_set_mode 2)",
            "ls_form": {"value": st_ls["agent_steps"] / (ms_ls / 1e3), "unit": "agent-steps/s", "ms_per_step": ms_ls / K,
                        "rmse_m": ls_mean, "rmse_ratio": ls_mean / pf_mean,
                        "tracker": "least-squares trilateration over each filter's 16 newest pings (est_set_mode 4)"},
            "train": {"rows": steps_rec * F, "wall_s": rec_s,
                      "steps": args.train_steps + ROUNDS * args.round_steps, "batch": 16384,
                      "candidates": len(cands), "validation_rmse_m": [round(v, 1) for v, _, _, _ in cands],
                      "chosen": c_best, "validation": "seed 8000, same horizon; evaluation seeds 9000 and 9100",
                      "schedule": f"50% filter-driven rows, then {ROUNDS} rounds of network-driven rows (retrain "
                                  f"after each); every round's rows from {EPISODES} episodes over the evaluation "
                                  "horizon, a row every k-th step",
                      "loss_last_per_round": losses, "train_ms": train_ms, "loss": "Huber, delta = 1 L"}}


def fp32_simt_peak_tflops(sm_mhz: float) -> float:
    """FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def ppo_flops_per_sample(d: int, L: int, n_tok: int, n_out: int) -> float:
    """Algorithmic FLOPs of one sample's forward + backward: the block GEMMs
    (QKV 3d^2, O d^2, FFN 8d^2 per token) three times (forward, input and
    weight gradients), attention (QK^T and PV, 2 n_tok^2 d each) three times,
    embedding and head."""
    gemm = 3 * 2 * n_tok * L * 12 * d * d
    attn = 3 * 2 * 2 * n_tok * n_tok * d * L
    return float(gemm + attn + 3 * 2 * (n_tok - 1) * 8 * d + 3 * 2 * d * n_out)


def ppo_update(args, p, rank):
    """TransfMAPPO update (Sec. II-B) on one batch collected by the env with
    the transformer agent acting: T steps, the batch split into 4 minibatches
    for the actor (agent-steps) and the critic (env-steps), one epoch, each
    minibatch one PPO gradient + Adam step of both networks, then the copy of
    the actor's weights into the env's agent."""
    import torch

    import paper_2505_08222_gb300 as ut
    import synth
    from paper_2505_08222_gb300 import ppo

    T = args.ppo_steps
    env = ut.Env(p)
    dims = synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions)
    prm = synth.policy_params(dims, seed=1234)
    crit = synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, 1), seed=4321)
    env.set_policy(prm)
    env.reset(1000)
    env.autotune(5)  # the filter launch variant, as in the timed rollout
    tr = ppo.Trainer(env, prm, crit, ppo.PPOConfig(T=T, epochs=1, minibatches=4))
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    e0, e1 = ev(), ev()
    e0.record(stream)
    tr.collect(1000)
    e1.record(stream)
    torch.cuda.synchronize()
    collect_ms = e0.elapsed_time(e1)
    for w in range(2):  # warm-up updates on the batch
        tr.update(w)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = tr.update(7)
    e1.record(stream)
    torch.cuda.synchronize()
    update_ms = e0.elapsed_time(e1)
    # the actor's gradient step alone, K minibatches of the same size
    NA, NS, d = tr.NA, tr.NS, tr.d
    tok, ne, h = tr.tok.view(T * NA, NS, 8), tr.ne.view(T * NA), tr.h.view(T * NA, d)
    sel = torch.randperm(T * NA, device="cuda")[:tr.mb_actor].to(torch.int32)
    act, logp, adv = tr.act.view(-1), tr.logp.view(-1), tr.adv_a.view(-1)
    reps = 6
    for _ in range(2):
        tr.actor.actor_grad(tok, ne, h, act, logp, adv, sel=sel, stats=False)
    e0.record(stream)
    for _ in range(reps):
        torch.cuda.nvtx.range_push("ppo_actor_step")
        tr.actor.actor_grad(tok, ne, h, act, logp, adv, sel=sel, stats=False)
        torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / reps
    n_tok = 1 + NS
    fps = ppo_flops_per_sample(d, p.n_layers, n_tok, p.n_actions)
    achieved = fps * tr.mb_actor / (step_ms * 1e-3) / 1e12
    tc = bool(getattr(tr.actor, "tensor_cores", False))
    if tc:  # BF16 GEMM operands on the tensor cores: against the measured bf16 peak
        peaks, peak_kind = _peaks()
        peak = peaks["bf16_tflops"]
        roof_kind = ("tensor", f"{peak_kind} cuBLAS bf16 GEMM (burst); the step also holds FP32 attention, "
                               "LayerNorm, loss and reduction kernels")
    else:
        peak = fp32_simt_peak_tflops(2070.0)
        roof_kind = ("alu", "derived FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz")
    variant = env.pf_variant_name()
    env.close()
    return {
        "metric": "PPO update throughput", "value": T * NA / (update_ms * 1e-3), "unit": "agent-samples/s",
        "ms_per_update": update_ms, "collect_ms": collect_ms,
        "iteration_agent_steps_per_s": T * NA / ((collect_ms + update_ms) * 1e-3),
        "T": T, "epochs": 1, "minibatches": 4, "actor_minibatch": tr.mb_actor, "critic_minibatch": tr.mb_critic,
        "dtype": "bf16 GEMM operands, f32 accumulation and activations" if tc else "f32",
        "roofline": {"bound": roof_kind[0], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": None, "scope": "actor PPO gradient step (forward, loss, backward: all kernels)",
                     "avg_step_ms": step_ms, "flops_per_sample": fps, "peak_kind": roof_kind[1],
                     "timing": "CUDA events around 6 gradient calls on one minibatch"},
        "stats_last_minibatch": stats,
        "filter_variant": variant,
        "note": (("linear layers on the tensor cores (BF16 operands, FP32 accumulation), the rest FP32"
                  if tc else "FP32 transformer training path on CUDA cores")
                 + "; the batch is a real collection (env_reset(1000), T steps with the agent acting, one CUDA "
                   "graph), the critic fed the true state"),
    }


def variant_form(args, p, K, W, rank, env_main, tracker, **kw):
    """A tracker variant of the same workload (``kw`` replaces parameters:
    shared_filter=1, one filter per (env, target) fed every ping of the
    target; pf_ess_num=k, resampling only when the effective sample size
    falls below k/16 of P).  Timed like the main line (one graph of K steps
    after W warm-up steps); pooled RMSE against the main form on the
    held-out seeds."""
    import torch

    import paper_2505_08222_gb300 as ut
    import synth

    T_eval = args.eval_steps
    seeds = [9000 + rank, 9100 + rank]
    ps = p.replace(**kw)
    env = ut.Env(ps)
    if p.d_model:
        env.set_policy(synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions)))
    if env_main.pf_variant() in env.pf_variants():
        env.set_pf_variant(env_main.pf_variant())

    def rmse(e, seed):
        e.reset(seed)
        return e.rollout(T_eval)["rmse"]

    sh = [rmse(env, s) for s in seeds]
    pa = [rmse(env_main, s) for s in seeds]
    env.reset(1000 + rank)
    for _ in range(W):
        env.step()
    env.rollout_prepare(K)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st = env.rollout(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    F = env.F
    env.close()
    sh_mean, pa_mean = sum(sh) / len(sh), sum(pa) / len(pa)
    return {"value": st["agent_steps"] / (ms / 1e3), "unit": "agent-steps/s", "ms_per_step": ms / K,
            "filters_per_gpu": F, "rmse_m": sh_mean, "main_form_rmse_m": pa_mean, "rmse_ratio": sh_mean / pa_mean,
            "eval": f"{len(seeds)} held-out seeds x {T_eval} steps, pooled RMSE per run, mean over seeds",
            "tracker": tracker}


def run_reference(args):
    world, rank, _ = _dist_env()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    budget = max(2.0, min(20.0, 4.0 * args.steps))
    cb = cpu_baseline(args.workload, budget_s=budget)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "agent-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "note": "FP64 CPU oracle on a bounded sample"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "agent-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


PF_SOURCES = ("pf_kernel.cuh", "pf_kernel.cu", "pf_inst_a.cu", "pf_inst_b.cu", "pf_variants.h", "common.cuh",
              "env.cuh", "f32x2.cuh")
TRAFFIC_NOTE = os.path.join(ROOT, "profiles", "pf_step_kernel_fleet5.json")


def pf_source_hash() -> str:
    """SHA-256 (first 16 hex digits) over the filter kernel's sources."""
    import hashlib

    h = hashlib.sha256()
    for name in PF_SOURCES:
        with open(os.path.join(ROOT, "paper_2505_08222_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _pf_traffic(variant: str, particles: int):
    """DRAM bytes per launch from the committed ncu figure
    (profiles/pf_step_kernel_fleet5.json: {"variant", "sources",
    "bytes_per_particle", ...}); it applies only while the kernel sources
    still hash to "sources" and the launch variant is "variant"; the
    capture's bytes per particle are scaled to this launch's particles."""
    try:
        with open(TRAFFIC_NOTE) as f:
            t = json.load(f)
        if t.get("variant") == variant and t.get("sources") == pf_source_hash():
            return float(t["bytes_per_particle"]) * particles
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return None


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2505_08222_gb300 as ut
    import synth

    from paper_2505_08222_gb300 import shard

    p = _workload(args.workload)
    if args.ppo_only:
        # the TransfMAPPO update measurement alone (profiling case)
        if rank == 0:
            print(json.dumps({"workload": args.workload, "n_envs": p.n_envs, "ppo": ppo_update(args, p, rank)}),
                  flush=True)
        return 0
    if world > 1:
        # weak scaling: the job is one batch of world x n_envs envs; rank r
        # steps its contiguous shard, random draws keyed by global ids
        p = shard.shard_params(p.replace(n_envs=p.n_envs * world), rank, world)
    env = ut.Env(p)
    if p.d_model > 0 and hasattr(env, "set_policy"):
        env.set_policy(synth.policy_params(synth.PolicyDims(p.d_model, p.n_layers, p.n_heads, p.n_actions)))
    env.reset(1000)
    if args.pf_variant:
        names = {ut.lib.pf_variant_label(v).decode(): v for v in env.pf_variants()}
        if args.pf_variant not in names:
            raise SystemExit(f"--pf-variant: {args.pf_variant!r} not usable here; choose from {sorted(names)}")
        env.set_pf_variant(names[args.pf_variant])
    elif not args.no_autotune:
        env.autotune(5)  # picks the filter launch variant, then the episode restarts
        env.reset(1000)
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup
    policy_on = bool(getattr(env, "policy_ready", False))

    # warm-up: W eager steps, then capture + upload the K-step graph (untimed)
    for _ in range(W):
        env.step()
    env.rollout_prepare(K)
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_index = int(vis[local]) if local < len(vis) and vis[local].strip().isdigit() else local
    clocks = ClockSampler(gpu_index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = env.rollout(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    agent_steps = float(shard.reduce_sums([stats["agent_steps"]])[0])

    # the same timed rollout (same graph, W warm-up steps) from seeds 0..4
    sweep, sweep_rmse = [], []
    for sd in range(5):
        env.reset(sd)
        for _ in range(W):
            env.step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev0.record(stream)
        st_sd = env.rollout(K)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_sd = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms_sd], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms_sd = float(t.item())
        sweep.append(float(shard.reduce_sums([st_sd["agent_steps"]])[0]) / (ms_sd / 1e3))
        sq = shard.reduce_sums([st_sd["sum_sq_err"], st_sd["n_err"]])
        sweep_rmse.append(float((sq[0] / max(sq[1], 1.0)) ** 0.5))
    # dominant-kernel duration: CUDA events around each particle-filter launch
    # on its stream (events recorded by graph nodes cannot be timed), over an
    # eager replay of the timed steps: same seed, W untimed steps, then the
    # same K steps the graph ran
    env.reset(1000)
    for _ in range(W):
        env.step()
    env.profile(True)
    for _ in range(K):
        env.step()
    pf_ms, pf_launches = env.stage_time()
    env.profile(False)
    value = agent_steps / (ms / 1e3)

    # roofline of the dominant kernel (particle filter step)
    peaks, peak_kind = _peaks()
    bytes_per_launch = env.F * env.P * BYTES_PER_PARTICLE
    pf_avg_ms = pf_ms / max(pf_launches, 1)
    achieved = bytes_per_launch / (pf_avg_ms / 1e3) / 1e9
    traffic = _pf_traffic(env.pf_variant_name(), env.F * env.P)

    # end to end through the C ABI, eager steps from the timed region's start,
    # every step's reward + done read back into pinned host memory: (1) the
    # step as timed above (the on-device policy, or the device's random
    # actions, picks the actions: the step has no host input); (2) a host
    # controller's actions (pinned) copied in every step in place of the policy
    NA, E = env.NA, env.E
    rew_host = torch.empty((K, E), dtype=torch.float32).pin_memory()
    done_host = torch.empty((K, E), dtype=torch.int32).pin_memory()

    def _e2e_loop(step_fn):
        # the same episode steps as the timed region: same seed, W warm-up steps
        env.reset(1000)
        for _ in range(W):
            step_fn(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(K):
            out = step_fn(k)
            rew_host[k].copy_(out["reward"], non_blocking=True)
            done_host[k].copy_(out["done"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([t_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_ms = float(t.item())
        return K * float(shard.reduce_sums([NA])[0]) / (t_ms / 1e3)

    e2e_policy = _e2e_loop(lambda k: env.step(None))
    act_host = torch.from_numpy(np.random.default_rng(rank).integers(0, p.n_actions, (K, NA)).astype(np.int32))
    act_host = act_host.pin_memory()
    act_dev = torch.zeros(NA, dtype=torch.int32, device="cuda")

    def _host_actions(k):
        act_dev.copy_(act_host[k], non_blocking=True)
        return env.step(act_dev)

    e2e_host = _e2e_loop(_host_actions)

    # roofline of the transformer agent (it dominates the large workload): its
    # forward over this batch's tokens through the stand-alone entry (the same
    # device code as the step's), CUDA events over K launches on the stream;
    # algorithmic FLOPs of the real tokens (below)
    pol_roof = None
    if policy_on:
        tok = env.step(None)["obs"].view(torch.bfloat16)
        a_cnt, t_cnt = p.counts()
        n_ent = torch.from_numpy(np.repeat(a_cnt + t_cnt, a_cnt).astype(np.int32)).cuda()
        h_tmp = torch.zeros((NA, p.d_model), dtype=torch.bfloat16, device="cuda")
        for _ in range(3):
            env.policy_forward(tok, n_ent, h_tmp)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            env.policy_forward(tok, n_ent, h_tmp)
        e1.record(stream)
        torch.cuda.synchronize()
        pol_ms = e0.elapsed_time(e1) / K
        apt = 128 // (1 + p.max_agents + p.max_targets)
        tiles = -(-NA // apt)
        # algorithmic FLOPs of the real tokens (an agent of env e has 1 + A_e + T_e):
        # the block GEMMs 2 * 12 d^2 per token per layer, attention 4 n_tok^2 d per
        # agent per layer (QK^T and PV); the padded rows of the 128-row tiles are
        # not counted.  With 17-token agents the kernel skips the last block's
        # entity queries (only the recurrent row reaches the head): that block's
        # attention counts 4 n_tok d per agent
        n_tok = (1 + a_cnt + t_cnt).astype(np.int64)
        tok_rows = int((a_cnt * n_tok).sum())
        split = 1 + p.max_agents + p.max_targets > 16
        attn = int((a_cnt * n_tok * n_tok).sum()) * 4 * p.d_model * (p.n_layers - 1 if split else p.n_layers)
        if split:
            attn += int((a_cnt * n_tok).sum()) * 4 * p.d_model
        flops = tok_rows * 2 * 12 * p.d_model ** 2 * p.n_layers + attn
        pol_tf = flops / (pol_ms / 1e3) / 1e12
        pol_roof = {"bound": "tensor", "achieved": pol_tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": pol_tf / peaks["bf16_tflops"], "traffic": None, "kernel": "policy_fwd_kernel",
                    "avg_launch_ms": pol_ms, "launches": K, "tiles": tiles, "flops_per_launch": flops,
                    "flops": ("real tokens only: 24 d^2 L per token + 4 n_tok^2 d per agent and block "
                              "(attention; the last block's recurrent query alone with 17-token agents)"),
                    "peak_kind": f"{peak_kind} cuBLAS bf16 GEMM (burst)",
                    "timing": "CUDA events over K stand-alone launches on the batch's tokens"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "agent-steps/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n_envs_per_gpu": p.n_envs, "agents": p.max_agents,
                       "targets": p.max_targets, "particles": p.n_particles, "filters_per_gpu": env.F,
                       "policy": (f"transformer d={p.d_model} L={p.n_layers} H={p.n_heads} bf16" if policy_on
                                  else "uniform random actions"),
                       "pf_variant": env.pf_variant_name(),
                       "l2": "inputs larger than L2 (3.4 GB particle state per GPU), no flush",
                       "timed": "one CUDA graph of K steps (rollout)", "parallelism": f"env-sharded x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": "pf_step_kernel", "avg_launch_ms": pf_avg_ms, "launches": pf_launches,
                         "timing": "CUDA events around each launch on its stream, eager replay of the K timed steps (same seed and warm-up)",
                         "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "e2e": {"value": e2e_host, "unit": "agent-steps/s", "h2d_bytes_per_step": NA * 4,
                    "d2h_bytes_per_step": E * 8,
                    "note": ("eager env_step calls through the C ABI from the timed region's start state: every "
                             "step a host controller's actions [NA] int32 are copied in from pinned host memory "
                             "and the step's reward and done [E] are read back into pinned host memory"),
                    "device_actions": {"value": e2e_policy, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": E * 8,
                                       "note": ("the same, with the actions picked on the device as in the timed "
                                                "step (no host input)")}},
            "gpu_launches": stats["kernel_launches"],
            "seeds_0_4": {"values": sweep, "mean": sum(sweep) / len(sweep), "min": min(sweep), "max": max(sweep),
                          "median": sorted(sweep)[len(sweep) // 2],
                          "rmse_m": sweep_rmse, "rmse_mean_m": sum(sweep_rmse) / len(sweep_rmse),
                          "note": "the timed rollout repeated from env_reset(seed), seeds 0..4 (pooled RMSE over "
                                  "the K steps per seed)"},
            "policy_roofline": pol_roof,
            "clocks": clock_info,
            "rmse_m": stats["rmse"],
        }
        if not args.no_learned:
            line["learned"] = learned_form(args, p, K, W, rank)
        if not args.no_shared:
            line["shared_filter"] = variant_form(
                args, p, K, W, rank, env, "one particle filter per (env, target), every ping of the target "
                "(shared_filter 1)", shared_filter=1)
            line["ess_resampling"] = variant_form(
                args, p, K, W, rank, env, "per-agent filters, weights carried across steps, resampling when "
                "the effective sample size < P/2 (pf_ess_num 8)", pf_ess_num=8)
        if not args.no_ppo and getattr(p, "d_model", 0):
            line["ppo"] = ppo_update(args, p, rank)
        if world == 1 and not args.no_cpu_baseline:
            os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
            line["cpu_baseline"] = cpu_baseline(args.workload)
            line["cpu_baseline"]["one_thread"] = cpu_baseline_one_thread(args.workload)
        print(json.dumps(line), flush=True)
    env.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="fleet5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--pf-variant", default=None, help="fixed filter launch variant (e.g. nt512x4m3), no autotune")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-estimator form")
    ap.add_argument("--no-shared", action="store_true", help="skip the shared-filter and ESS-resampling forms")
    ap.add_argument("--no-ppo", action="store_true", help="skip the TransfMAPPO update measurement")
    ap.add_argument("--ppo-steps", type=int, default=32, help="steps collected for the PPO batch")
    ap.add_argument("--ppo-only", action="store_true", help="only the TransfMAPPO update measurement")
    ap.add_argument("--train-rows", type=int, default=None,
                    help="recorded estimator rows (default 20M; 64M for the large workload, whose 4.2M filters "
                         "per step would otherwise give too few recorded episodes)")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps on the filter-driven rows")
    ap.add_argument("--round-steps", type=int, default=800, help="Adam steps after each DAgger round")
    ap.add_argument("--eval-steps", type=int, default=100)
    ap.add_argument("--est-candidates", type=int, default=3, help="estimator trainings to choose from")
    ap.add_argument("--envs", type=int, default=None, help="override the env count (profiling cases)")
    args = ap.parse_args()
    if args.train_rows is None:
        args.train_rows = 64_000_000 if args.workload == "large" else 20_000_000
    global _ENVS
    _ENVS = args.envs
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
