"""Training and use of the learned spreading kernel (width 4).

The model (an MLP that maps per-source-tile features to a tabulated kernel,
plus a learned deconvolution correction; see include/asfd.h) lives inside a
plan of kind "learned" and is trained on the GPU by asfd_learned_train_step,
whose forward, adjoint, gradient and optimiser kernels are the library's
own.  Training pairs are seeded (surface, field) inputs of one geometry; the
target of each pair is the transform with the ES kernel at width 12, the
reference for the learned kernel's error.

    model, losses = train_model(train_set())
    model.save("learned_w4.npz"); LearnedModel.load(path).apply_to(plan)
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import capi, workloads as W
from .fresnel import FresnelPlan

REFERENCE_WIDTH = 12


def train_set(name="smooth_random2048", scale=1, surfaces=2, fields=1, seed=100):
    """Seeded (geometry, u1, d1) pairs of one geometry: `surfaces` smooth random
    height maps (the workload's recipe, other seeds) x `fields` random fields.
    The default is the full-size geometry, so that the samples' spacing on the
    fine grid (and every tile feature) is the one the model is used at."""
    out = []
    for s in range(surfaces):
        g, _, d1 = W.make(name, seed=seed + s, scale=scale)
        rng = np.random.default_rng(seed + 1000 + s)
        for _ in range(fields):
            out.append((g, W.field_random_amp_phase(g, rng), d1))
    return out


def reference_fields(pairs, width=REFERENCE_WIDTH):
    """Forward transforms with the ES kernel at `width` (device tensors)."""
    refs = []
    for g, u1, d1 in pairs:
        with FresnelPlan(g, d1, kernel_width=width) as p:
            refs.append(p.execute(torch.as_tensor(u1, device="cuda")))
    torch.cuda.synchronize()
    return refs


class LearnedModel:
    """A learned-kernel model: the flat parameter vector plus training metadata."""

    def __init__(self, params: np.ndarray, meta: dict | None = None):
        self.params = np.ascontiguousarray(params, np.float32)
        self.meta = dict(meta or {})

    def apply_to(self, plan: FresnelPlan) -> None:
        capi.asfd_learned_set_params(plan.handle, self.params)

    def save(self, path: str) -> None:
        np.savez(path, params=self.params, **{k: np.asarray(v) for k, v in self.meta.items()})

    @classmethod
    def load(cls, path: str) -> "LearnedModel":
        z = np.load(path)
        meta = {k: z[k].tolist() for k in z.files if k != "params"}
        return cls(z["params"], meta)


def train_model(pairs, refs=None, steps=10000, lr=3e-3, lr_final=1e-5, plan=None, log=None,
                loss_every=100):
    """Adam on the relative squared error against the reference fields,
    cycling over the pairs (the plan is rebuilt when the surface changes).
    lr decays geometrically from `lr` to `lr_final`; the loss is read back
    (a stream synchronisation) every `loss_every` steps and at the last one.
    Returns (model, losses) with losses[i] the loss at the i-th readback."""
    if refs is None:
        refs = reference_fields(pairs)
    g0, _, d10 = pairs[0]
    own = plan is None
    if own:
        plan = FresnelPlan(g0, d10, kind="learned")
    losses = []
    current = id(pairs[0][2])
    u1s = [torch.as_tensor(u1, device="cuda") for _, u1, _ in pairs]
    try:
        for it in range(steps):
            k = it % len(pairs)
            g, _, d1 = pairs[k]
            if id(d1) != current:
                plan.update_d1(d1)
                current = id(d1)
            frac = it / max(1, steps - 1)
            rate = lr * math.exp(frac * math.log(lr_final / lr))
            want = it % max(1, loss_every) == 0 or it == steps - 1
            loss = capi.asfd_learned_train_step(plan.handle, u1s[k], refs[k], rate, plan.shape1,
                                                plan.shape2, want_loss=want)
            if want:
                losses.append(loss)
            if log and want and (it % max(1, steps // 10) < max(1, loss_every) or it == steps - 1):
                log(f"step {it:5d}  lr {rate:.2e}  rel-L2 {math.sqrt(loss):.3e}")
        params = capi.asfd_learned_get_params(plan.handle)
    finally:
        if own:
            plan.close()
    meta = {"steps": steps, "lr": lr, "lr_final": lr_final, "pairs": len(pairs),
            "final_rel_l2": math.sqrt(losses[-1]) if losses else float("nan")}
    return LearnedModel(params, meta), losses


def rel_l2_vs(plan: FresnelPlan, u1, ref) -> float:
    out = plan.execute(torch.as_tensor(u1, device="cuda"))
    return float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
