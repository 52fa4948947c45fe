"""Learned warm start for SQNGD: training data from the method's own
converged designs, training and proposals through the warm-start network's
C ABI, and the time-to-PSL-target experiment.

The paper feeds the initial phase configuration y0 to its generator network
(Section II-B, Eq. 17).  Here the network's seed channel carries the random
initial code b0 and it is trained (cross-entropy) to output the design that
SQNGD converges to from b0; its argmax proposal then replaces b0 as the
starting point of the optimiser.

    python -m paper_2604_25728_gb300.warmstart train --out <file.npz>

generates the designs on the GPU, trains the network and writes its FP32
parameter vector with the training record.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import api
from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PARAMS = os.path.join(HERE, "data", "warmstart_params.npz")

# problem family the network is trained on (the learned workload's grid and
# delay window with two problem sizes and two waveform counts)
TRAIN_CONFIGS = [(2, 256), (4, 256), (2, 512), (4, 512)]
TRAIN_B, TRAIN_WINDOW, TRAIN_L, TRAIN_KMAX = 16, 0.1, 128, 50


def _ctx(M, N, B, window, L, kmax, path, w=None):
    nu = wl.window_grid(window, L)
    kw = {} if w is None else dict(eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c, n_h=w.n_h, n_x=w.n_x,
                                   lr_h=w.lr_h, lr_x=w.lr_x)
    return api.Context(M, N, B, nu, -kmax, kmax, path=path, **kw)


def converge(ctx, b0: np.ndarray, n_outer: int) -> np.ndarray:
    """Run SQNGD for n_outer outer iterations from the code b0 ([M, N]) and
    return the phase indices of the best hard design it found."""
    dev = ctx.device
    u, h = ctx.sqngd_init(torch.from_numpy(np.ascontiguousarray(b0, dtype=np.int32)).to(dev))
    st = api.SqngdState.create(u, h)
    ctx.sqngd_step(st, n_outer, log=False)
    ctx.af_sync()
    return (st.best_q.cpu().numpy() % ctx.B).astype(np.int32)


def generate(n_per_config: int, n_outer: int, seed0: int = 10_000, path=api.AF_PATH_SPLIT_BF16, configs=None):
    """Converged designs of the training family (or of `configs`, a list of
    (M, N)): list of (M, N, b0, b_star)."""
    data = []
    for (M, N) in (configs or TRAIN_CONFIGS):
        ctx = _ctx(M, N, TRAIN_B, TRAIN_WINDOW, TRAIN_L, TRAIN_KMAX, path)
        for i in range(n_per_config):
            b0 = wl.phase_indices(seed0 + 1000 * M + N + i, M, N, TRAIN_B)
            data.append((M, N, b0, converge(ctx, b0, n_outer)))
        ctx.close()
    return data


def cond_of(M: int, N: int, B: int, window: float, kmax: int):
    return api.ws_cond(M, N, B, window, kmax)


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded starting parameters in the ABI's packed order: W ~ N(0, 1/(cin*5)), biases 0."""
    rng = np.random.default_rng(seed)
    out = []
    for cin in (32, 64, 64, 64):
        w = rng.standard_normal((64, cin, 5)) / np.sqrt(cin * 5)
        out.append(w.astype(np.float16).astype(np.float32).ravel())
        out.append(np.zeros(64, np.float32))
    return np.concatenate(out)


def train(data, epochs: int = 30, lr: float = 2e-3, batch: int = 32, seed: int = 0, net=None, log=None):
    """Train on (M, N, b0, b_star) designs; batches are drawn within one (M, N)."""
    n_max = max(N for _, N, _, _ in data)
    net = net or api.WarmStart(batch, n_max)
    net.set_params(init_params(seed))
    groups = {}
    for M, N, b0, bs in data:
        groups.setdefault((M, N), []).append((b0, bs))
    rng = np.random.default_rng(seed)
    dev = net.device
    history = []
    for ep in range(epochs):
        losses = []
        keys = list(groups)
        rng.shuffle(keys)
        for key in keys:
            M, N = key
            items = groups[key]
            order = rng.permutation(len(items))
            cond = cond_of(M, N, TRAIN_B, TRAIN_WINDOW, TRAIN_KMAX)
            for s in range(0, len(order), batch):
                idx = order[s:s + batch]
                b0 = torch.from_numpy(np.stack([items[i][0] for i in idx]).astype(np.int32)).to(dev)
                tg = torch.from_numpy(np.stack([items[i][1] for i in idx]).astype(np.int32)).to(dev)
                losses.append(net.train_step(b0, tg, TRAIN_B, cond, lr))
        history.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f}")
    return net, history


def propose(net, b0: np.ndarray, B: int, window: float, kmax: int) -> np.ndarray:
    """The network's starting code for a design whose random initial code is b0 ([M, N])."""
    M, N = b0.shape
    t = torch.from_numpy(np.ascontiguousarray(b0[None], dtype=np.int32)).to(net.device)
    _, b = net.forward(t, B, cond_of(M, N, B, window, kmax), logits=False)
    return b[0].cpu().numpy()


def save(path: str, params: np.ndarray, record: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=params.astype(np.float32), record=json.dumps(record))


def load(path: str = DEFAULT_PARAMS):
    z = np.load(path, allow_pickle=False)
    return z["params"], json.loads(str(z["record"]))


# ------------------------------------------------------------ time to target
def _trajectory(ctx, b0, t_max, chunk, stream, stop=None, init_s=0.0):
    """SQNGD from the code b0 in chunks of `chunk` outer iterations.  The
    starting design and, after each chunk, the current hard design are scored
    in FP64 (af_eval_hard, not timed).  Returns [(outer iterations, device
    seconds of the optimiser so far, PSLR dB, max SNRL dB)] from iteration 0,
    stopping early once stop(pslr, snrl) holds."""
    dev = ctx.device
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, h = ctx.sqngd_init(torch.from_numpy(np.ascontiguousarray(b0, dtype=np.int32)).to(dev))
    st = api.SqngdState.create(u, h)
    e1.record(stream)
    e1.synchronize()
    t = init_s + e0.elapsed_time(e1) / 1e3
    it = 0
    acc = ctx.af_eval_hard(st.u, st.h)
    out = [(0, t, float(acc[2]), float(acc[3]))]
    if stop is not None and stop(acc[2], acc[3]):
        ctx.af_sync()
        return out
    while it < t_max:
        e0.record(stream)
        ctx.sqngd_step(st, chunk, log=False)
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        it += chunk
        acc = ctx.af_eval_hard(st.u, st.h)
        out.append((it, t, float(acc[2]), float(acc[3])))
        if stop is not None and stop(acc[2], acc[3]):
            break
    ctx.af_sync()
    return out


def time_to_target(params=None, seeds=(0, 1, 2, 3, 4), t_max: int = 2000, chunk: int = 5, log=None, nets=None):
    """Time to a PSL target at equal SNRL on the learned workload (M=4,
    N=1024, B=16, 128 bins on |nu| <= 0.1, |k| <= 50).

    The plain FP32 GPU form (the SIMT DFT path on this grid) runs t_max
    outer iterations from random codes; the SNRL budget is the worst final
    max SNRL of those runs and the PSL target their worst final hard PSLR.
    An arm reaches the target at the first checkpoint (every `chunk` outer
    iterations) where its current hard design meets both; its time is the
    device time (CUDA events) of the optimiser (and of the warm-start
    proposal) up to that checkpoint.  `nets` maps arm names to further
    parameter vectors (each becomes a split-BF16 warm-start arm); the record
    holds every arm's starting PSLR (iteration 0) and, for the networks, the
    share of the random code's indices their proposals change."""
    w = wl.learned()
    kmax = w.k_hi
    window = float(np.max(np.abs(w.nu)))
    stream = torch.cuda.current_stream()
    starts = {s: wl.phase_indices(20_000 + s, w.M, w.N, w.B) for s in seeds}
    out = {"workload": w.name, "t_max": t_max, "chunk": chunk, "seeds": list(seeds),
           "target_rule": "worst final hard PSLR and worst final max SNRL of the FP32 arm at t_max"}

    ctx = _ctx(w.M, w.N, w.B, window, w.L, kmax, api.AF_PATH_DFT, w)
    traj_a = {s: _trajectory(ctx, starts[s], t_max, chunk, stream) for s in seeds}
    ctx.close()
    snrl_budget = max(tr[-1][3] for tr in traj_a.values())
    target = max(tr[-1][2] for tr in traj_a.values())
    out["snrl_budget_db"] = snrl_budget
    out["target_pslr_db"] = target
    out["start_pslr_db"] = {"random": [traj_a[s][0][2] for s in seeds]}

    def ok(pslr, snrl):
        return pslr <= target and snrl <= snrl_budget

    def reached(tr):
        for it, t, pslr, snrl in tr:
            if ok(pslr, snrl):
                return it, t
        return None, None

    arms = {"fp32_random": {s: reached(traj_a[s]) for s in seeds}}
    if log:
        log(f"target {target:.2f} dB at max SNRL <= {snrl_budget:.3f} dB")
    ctx = _ctx(w.M, w.N, w.B, window, w.L, kmax, api.AF_PATH_SPLIT_BF16, w)
    arms["split_random"] = {s: reached(_trajectory(ctx, starts[s], t_max, chunk, stream, ok)) for s in seeds}
    all_nets = dict(nets or {})
    if params is not None:
        all_nets = {"split_warmstart": params, **all_nets}
    out["changed_fraction"] = {}
    for name, prm in all_nets.items():
        net = api.WarmStart(1, w.N)
        net.set_params(prm)
        res, starts_db, changed = {}, [], []
        for s in seeds:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b_ws = propose(net, starts[s], w.B, window, kmax)
            e1.record(stream)
            e1.synchronize()
            changed.append(float(np.mean(b_ws != starts[s])))
            tr = _trajectory(ctx, b_ws, t_max, chunk, stream, ok, e0.elapsed_time(e1) / 1e3)
            starts_db.append(tr[0][2])
            res[s] = reached(tr)
        arms[name] = res
        out["start_pslr_db"][name] = starts_db
        out["changed_fraction"][name] = float(np.mean(changed))
        net.close()
    ctx.close()
    for name, res in arms.items():
        times = [t for it, t in res.values() if t is not None]
        its = [it for it, t in res.values() if it is not None]
        out[name] = {"reached": len(times), "median_s": float(np.median(times)) if len(times) == len(res) else None,
                     "median_outer": float(np.median(its)) if len(its) == len(res) else None,
                     "per_seed_s": [None if t is None else float(t) for _, t in res.values()],
                     "per_seed_outer": [it for it, _ in res.values()]}
    base = out["fp32_random"]["median_s"]
    for name in arms:
        if name != "fp32_random" and out[name]["median_s"] and base:
            out[name]["speedup_vs_fp32_random"] = base / out[name]["median_s"]
    return out


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = p.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train", help="generate converged designs on the GPU and train the warm-start network")
    t.add_argument("--per-config", type=int, default=128)
    t.add_argument("--outer", type=int, default=400)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--out", default=DEFAULT_PARAMS)
    r = sub.add_parser("ttt", help="time to PSL target with the saved network")
    r.add_argument("--params", default=DEFAULT_PARAMS)
    r.add_argument("--t-max", type=int, default=2000)
    st = sub.add_parser("study", help="time to PSL target over more seeds with a check every outer iteration, "
                                      "optionally with a second network trained at the evaluated size")
    st.add_argument("--params", default=DEFAULT_PARAMS)
    st.add_argument("--seeds", type=int, default=10)
    st.add_argument("--chunk", type=int, default=1)
    st.add_argument("--t-max", type=int, default=2000)
    st.add_argument("--train-at-size", type=int, default=0,
                    help="designs to generate at the evaluated size (M=4, N=1024) for a second network (0: none)")
    st.add_argument("--outer", type=int, default=800)
    st.add_argument("--out", default="")
    a = p.parse_args(argv)
    torch.cuda.set_device(0)
    if a.cmd == "train":
        t0 = time.time()
        data = generate(a.per_config, a.outer)
        t1 = time.time()
        net, hist = train(data, epochs=a.epochs, lr=a.lr, log=print)
        params = net.get_params()
        # how far the proposals are from the converged designs (held-out seeds)
        held = generate(4, a.outer, seed0=90_000)
        acc = []
        for M, N, b0, bs in held:
            bp = propose(net, b0, TRAIN_B, TRAIN_WINDOW, TRAIN_KMAX)
            acc.append(float(np.mean(bp == bs)))
        rec = {"configs": TRAIN_CONFIGS, "B": TRAIN_B, "window": TRAIN_WINDOW, "L": TRAIN_L, "kmax": TRAIN_KMAX,
               "designs": len(data), "outer_iterations": a.outer, "epochs": a.epochs, "lr": a.lr,
               "loss_history": hist, "held_out_index_agreement": float(np.mean(acc)),
               "generate_s": t1 - t0, "train_s": time.time() - t1}
        save(a.out, params, rec)
        print(json.dumps({k: v for k, v in rec.items() if k != "loss_history"}))
    elif a.cmd == "study":
        params, rec = load(a.params)
        nets, extra = {}, {}
        if a.train_at_size > 0:
            w = wl.learned()
            t0 = time.time()
            data = generate(a.train_at_size, a.outer, seed0=50_000, configs=[(w.M, w.N)])
            t1 = time.time()
            net, hist = train(data, epochs=30, lr=2e-3, log=print)
            nets["split_warmstart_at_size"] = net.get_params()
            extra = {"designs": len(data), "outer_iterations": a.outer, "generate_s": t1 - t0,
                     "train_s": time.time() - t1, "final_loss": hist[-1]}
            net.close()
        res = time_to_target(params, seeds=tuple(range(a.seeds)), t_max=a.t_max, chunk=a.chunk, log=print, nets=nets)
        res["network_at_size"] = extra
        txt = json.dumps(res)
        if a.out:
            with open(a.out, "w") as f:
                f.write(txt)
        print(txt)
    else:
        params, rec = load(a.params)
        print(json.dumps(time_to_target(params, t_max=a.t_max, log=print)))


if __name__ == "__main__":
    main()
