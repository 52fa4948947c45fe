"""The transmit-side ResNet generator (Eq. 17) as a user-facing mode, and the
convergence comparison against the direct-logit form.

    python -m paper_2604_25728_gb300.generator compare --workload mid --outer 2000 --seeds 3

runs SQNGD twice from the same random phases per seed -- once with the
logits u trained directly (the default transmit parameterisation) and once
with the ResNet generator producing u from y0 (learning rate 1e-5, Section IV)
-- and prints the final hard PSLR, the max SNRL (FP64, af_eval_hard) and the
optimiser time of each arm.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import api
from . import workloads as wl

WIDTH = 128
BLOCKS = 5


def init_params(P: int, z0, seed: int) -> np.ndarray:
    """Flat parameters (include/resnet.h order): hidden-layer weights
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from the seeded uniform stream, zero
    biases, W_out = 0 and b_out = logit(z0), so that the generator starts at
    the phases z0 (the direct-logit form's starting design)."""
    n_total = api.ResNetGenerator.param_count(P)
    th = np.zeros(n_total, dtype=np.float64)
    o = 0
    th[o:o + WIDTH * P] = (2.0 * wl.uniform(seed, WIDTH * P, 31) - 1.0) / np.sqrt(P)
    o += WIDTH * P + WIDTH
    for k in range(BLOCKS):
        for j in range(2):
            th[o:o + WIDTH * WIDTH] = (2.0 * wl.uniform(seed, WIDTH * WIDTH, 32 + 2 * k + j) - 1.0) / np.sqrt(WIDTH)
            o += WIDTH * WIDTH + WIDTH
    o += P * WIDTH                                   # W_out = 0
    z = np.asarray(z0, dtype=np.float64).ravel()
    th[o:o + P] = np.log(z / (1.0 - z))
    assert o + P == n_total
    return th.astype(np.float32)


def _run(w, seed: int, outer: int, generator: bool, lr_net: float):
    dev = torch.device("cuda", torch.cuda.current_device())
    b = wl.phase_indices(seed, w.M, w.N, w.B)
    ctx = api.Context(w.M, w.N, w.B, w.nu, w.k_lo, w.k_hi, eps=w.eps, snrl_db=w.snrl_db, r_n=w.r_n, c=w.c,
                      n_h=w.n_h, n_x=w.n_x, lr_h=w.lr_h, lr_x=lr_net if generator else w.lr_x)
    u, h = ctx.sqngd_init(torch.from_numpy(b).to(dev))
    rn = None
    if generator:
        P = w.M * w.N
        z0 = ((w.r_n // 2) * w.B + b.astype(np.float64)) / (w.B * w.r_n)
        rn = api.ResNetGenerator(P)
        rn.set_params(init_params(P, z0, seed))
        y0 = torch.from_numpy((b.astype(np.float32) / w.B).ravel()).to(dev)
        u = rn.forward(y0).reshape(w.M, w.N).contiguous()
        ctx.attach_generator(rn, y0)
    st = api.SqngdState.create(u, h)
    start = ctx.af_eval_hard(st.u, st.h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.sqngd_step(st, outer, log=False)
    e1.record()
    e1.synchronize()
    ctx.af_sync()
    out = ctx.af_eval_hard(st.u, st.h)
    ctx.close()
    if rn is not None:
        rn.close()
    return dict(start_pslr_db=float(start[2]), final_pslr_db=float(out[2]), final_max_snrl_db=float(out[3]),
                seconds=e0.elapsed_time(e1) / 1e3)


def compare(which: str = "mid", outer: int = 2000, seeds: int = 3, lr_net: float = 1e-5):
    w = getattr(wl, which)()
    res = {"workload": w.name, "outer_iterations": outer, "lr_generator": lr_net, "lr_logits": w.lr_x}
    for arm, gen in (("direct_logits", False), ("resnet_generator", True)):
        runs = [_run(w, s, outer, gen, lr_net) for s in range(seeds)]
        res[arm] = {k: float(np.median([r[k] for r in runs])) for k in runs[0]}
        res[arm]["runs"] = runs
    return res


def main():
    p = argparse.ArgumentParser()
    p.add_argument("cmd", choices=["compare"])
    p.add_argument("--workload", default="mid")
    p.add_argument("--outer", type=int, default=2000)
    p.add_argument("--seeds", type=int, default=3)
    p.add_argument("--lr", type=float, default=1e-5)
    a = p.parse_args()
    t0 = time.time()
    r = compare(a.workload, a.outer, a.seeds, a.lr)
    r["wall_seconds"] = time.time() - t0
    print(json.dumps(r))


if __name__ == "__main__":
    main()
