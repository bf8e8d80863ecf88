"""Learned planner pipeline: timings -> cost-model training on the GPU -> plan choice.

1. ``collect``: for each shape, every candidate plan (depth 0..4 x leaf tile
   {128, 256, 512}) is timed on the device by the library's exhaustive autotuner
   (``fmm_autotune``); each (shape, candidate, milliseconds) is one record.
2. ``train``: the 6-64-64-1 network predicts log(ms) from the standardised
   features; it is trained with the library's own forward/backward/Adam
   kernels (``fmm_mlp_train_step``), full batch, on the device.
3. ``register``: the trained weights go to ``fmm_set_cost_model``; plans made
   with planner="mlp" then score their candidates with the inference kernel.
4. ``evaluate``: on unseen shapes, the time of the plan each planner picks,
   against the exhaustive best (regret) and the fixed-threshold planner.

Weights are stored as a small versioned little-endian file (``save``/``load``).
"""
from __future__ import annotations

import math
import struct

import numpy as np

from . import fmm

MAGIC = b"FMMCOST1"


def collect(shapes, reps=1, precision="fp32", seed=0, device="cuda"):
    """Time every candidate of every (M, K, N) shape.  Returns a list of dicts."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    recs = []
    for (M, K, N) in shapes:
        A = torch.rand((M, K), generator=g, device=device) * 2 - 1
        B = torch.rand((K, N), generator=g, device=device) * 2 - 1
        Cm = torch.empty((M, N), device=device)
        for d, t, ms in fmm.fmm_autotune(M, N, K, A, B, Cm, reps=reps, precision=precision):
            recs.append(dict(M=M, K=K, N=N, depth=d, tile=t, ms=float(ms), precision=precision))
        del A, B, Cm
    return recs


def features(recs):
    prec_id = {"fp32": 0, "tf32": 1, "bf16x3": 2, "fp16x3": 3}
    X = np.array([fmm.fmm_plan_features(r["M"], r["N"], r["K"], r["depth"], r["tile"], prec_id[r["precision"]])
                  for r in recs], dtype=np.float32)
    y = np.log(np.array([max(r["ms"], 1e-4) for r in recs], dtype=np.float32))
    return X, y


def init_params(seed=0):
    """He-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 6)) * math.sqrt(2 / 6)
    W2 = rng.standard_normal((64, 64)) * math.sqrt(2 / 64)
    W3 = rng.standard_normal((1, 64)) * math.sqrt(1 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(1)]).astype(
        np.float32)


def train(X, y, steps=2000, lr=3e-3, seed=0, device="cuda", log_every=0):
    """Full-batch Adam on the device.  Returns (params, mean, std, losses)."""
    import torch
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std < 1e-6] = 1.0
    Xs = ((X - mean) / std).astype(np.float32)
    dX = torch.from_numpy(Xs).to(device)
    dT = torch.from_numpy(y.astype(np.float32)).to(device)
    p = torch.from_numpy(init_params(seed)).to(device)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    ws = torch.empty(fmm.mlp_workspace_bytes(len(Xs)), dtype=torch.uint8, device=device)
    loss = torch.zeros(1, device=device)
    losses = []
    for step in range(1, steps + 1):
        fmm.fmm_mlp_train_step(p, m, v, step, lr, dX, dT, ws, loss_out=loss)
        if log_every and (step % log_every == 0 or step == 1):
            losses.append((step, float(loss.item())))
    losses.append((steps, float(loss.item())))
    return p.cpu().numpy(), mean.astype(np.float32), std.astype(np.float32), losses


def predict(params, mean, std, X, device="cuda"):
    import torch
    dX = torch.from_numpy(((X - mean) / std).astype(np.float32)).to(device)
    dP = torch.from_numpy(np.asarray(params, np.float32)).to(device)
    dY = torch.empty(len(X), device=device)
    fmm.fmm_mlp_forward(dP, dX, dY)
    return dY.cpu().numpy()


def register(params, mean, std):
    fmm.fmm_set_cost_model(params, mean, std)


def choice(M, N, K, planner, precision="fp32", cutoff=None):
    """(depth, tile) the library's planner picks for a shape (no timing);
    cutoff None = the library's default."""
    import torch
    q = fmm.options(planner=planner, precision=precision)
    if cutoff is not None:
        q.cutoff = int(cutoff)
    _, need = fmm.fmm_plan(M, N, K, K, N, N, q, query_only=True)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h, _ = fmm.fmm_plan(M, N, K, K, N, N, q, ws.data_ptr(), ws.numel())
    info = fmm.fmm_plan_info(h)
    fmm.fmm_free(h)
    return info["depth"], info["leaf_tile"]


def evaluate(recs, precision="fp32", cutoff=None):
    """For every shape in `recs` (all candidates timed): time of the MLP's pick,
    of the fixed planner's pick (at the library's default cut-off unless given)
    and of the best candidate."""
    by_shape = {}
    for r in recs:
        by_shape.setdefault((r["M"], r["K"], r["N"]), {})[(r["depth"], r["tile"])] = r["ms"]
    out = []
    for (M, K, N), table in by_shape.items():
        best = min(table.values())
        pm = choice(M, N, K, "mlp", precision, cutoff)
        pf = choice(M, N, K, "fixed", precision, cutoff)
        out.append(dict(M=M, K=K, N=N, best=best, mlp=table.get(pm, float("nan")), fixed=table.get(pf, float("nan")),
                        mlp_plan=pm, fixed_plan=pf, flops=2.0 * M * N * K))
    return out


def summary(ev):
    t_best = sum(e["best"] for e in ev)
    t_mlp = sum(e["mlp"] for e in ev)
    t_fixed = sum(e["fixed"] for e in ev)
    fl = sum(e["flops"] for e in ev)
    return dict(shapes=len(ev), total_ms_best=t_best, total_ms_mlp=t_mlp, total_ms_fixed=t_fixed,
                regret_mlp=t_mlp / t_best - 1, regret_fixed=t_fixed / t_best - 1,
                gain_over_fixed=t_fixed / t_mlp - 1,
                gflops_best=fl / t_best / 1e6, gflops_mlp=fl / t_mlp / 1e6, gflops_fixed=fl / t_fixed / 1e6,
                exact_pick_rate=float(np.mean([e["mlp"] == e["best"] for e in ev])))


def save(path, params, mean, std):
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<II", 1, len(params)))
        f.write(np.asarray(params, "<f4").tobytes())
        f.write(np.asarray(mean, "<f4").tobytes())
        f.write(np.asarray(std, "<f4").tobytes())


def load(path):
    with open(path, "rb") as f:
        assert f.read(8) == MAGIC, "not a cost-model file"
        ver, n = struct.unpack("<II", f.read(8))
        assert ver == 1 and n == fmm.NPARAM
        params = np.frombuffer(f.read(4 * n), "<f4").copy()
        mean = np.frombuffer(f.read(24), "<f4").copy()
        std = np.frombuffer(f.read(24), "<f4").copy()
    return params, mean, std
