"""Learned initial guess for the iterative solver: training data from the
solver itself, training, inference, and the uniform-start fallback.

The paper starts each solve from a uniform state and observes that the
iteration needs many steps at small Knudsen number (Section 4.1).  Here a
solve of a cavity starts instead from a guess: the converged solution of the
same problem on a grid twice as coarse, upsampled trilinearly, plus a
correction predicted by a 3D convolutional network (about one million
parameters, channels 11-48-112-112-112-48-8) from (log Kn, lid speed, solid
flag, upsampled coarse fields).  A guess that is not a physical state (a
non-finite value, rho <= 0 or T <= 0 anywhere) is rejected and the solve
starts from the uniform state.

Every numeric step runs in libkgs's CUDA kernels (kgs_batch_* for the
solves, kgs_surrogate_* for the feature and guess maps, kgs_net_* for the
network); this module orders those calls and keeps the device buffers
(torch tensors) between them.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import inputs, kgs

DEFAULT_CHANNELS = (11, 48, 112, 112, 112, 48, 8)
N_FEATURES = 11
N_FIELDS = 8


def lid_speed(prob: inputs.Problem) -> float:
    """Largest wall speed of the problem (the lid of a cavity)."""
    return max(math.sqrt(sum(u * u for u in uw)) for uw in prob.U_w)


def coarse_problem(prob: inputs.Problem, factor: int = 2) -> inputs.Problem:
    """The same problem on cells `factor` times wider in each direction (the
    velocity grid, gas and boundaries unchanged).  Needs equal-width cells,
    extents divisible by `factor` and no solid cells."""
    if prob.solid is not None:
        raise ValueError("coarse_problem: problems with solid cells are not supported")
    dims = (prob.nx, prob.ny, prob.nz)
    if any(n % factor for n in dims):
        raise ValueError("coarse_problem: extents %s not divisible by %d" % (dims, factor))
    for d in (prob.dx, prob.dy, prob.dz):
        if not np.allclose(d, d[0], rtol=1e-12, atol=0.0):
            raise ValueError("coarse_problem: cells must have equal widths")
    nx, ny, nz = (n // factor for n in dims)
    return dataclasses.replace(prob, nx=nx, ny=ny, nz=nz, dx=np.full(nx, prob.dx[0] * factor),
                               dy=np.full(ny, prob.dy[0] * factor), dz=np.full(nz, prob.dz[0] * factor),
                               name=prob.name + " (coarse /%d)" % factor)


def solve(probs: Sequence[inputs.Problem], precision=kgs.KGS_MIXED, tol=1e-6, max_iters=5000,
          initial: Optional[Sequence[Optional[np.ndarray]]] = None):
    """Solve a batch of problems to `tol` in one kgs_batch.  Returns (list of
    macroscopic fields [8, nz, ny, nx], iterations per problem, residuals,
    status code)."""
    b = kgs.kgs_batch_setup(list(probs), precision=precision, tol=tol, max_iters=max_iters)
    if initial is not None:
        for i, m in enumerate(initial):
            if m is not None:
                kgs.kgs_batch_set_initial(b, i, m)
    rc, done, res = kgs.kgs_batch_iterate(b, 0)
    out = [kgs.kgs_batch_moments(b, i) for i in range(len(probs))]
    kgs.kgs_batch_destroy(b)
    return out, done, res, rc


def upsample(prob: inputs.Problem, coarse: np.ndarray, kn: Optional[float] = None):
    """Features x [nz, ny, nx, 11] (float32) and the upsampled coarse fields
    up [8, nz, ny, nx] (float64), both device tensors."""
    cz, cy, cx = coarse.shape[1:]
    x = torch.empty((prob.nz, prob.ny, prob.nx, N_FEATURES), dtype=torch.float32, device="cuda")
    up = torch.empty((N_FIELDS, prob.nz, prob.ny, prob.nx), dtype=torch.float64, device="cuda")
    cd = torch.as_tensor(np.ascontiguousarray(coarse), dtype=torch.float64, device="cuda")
    sd = None
    if prob.solid is not None:
        sd = torch.as_tensor(np.ascontiguousarray(prob.solid), dtype=torch.uint8, device="cuda")
    kgs.kgs_surrogate_features((prob.nx, prob.ny, prob.nz), (cx, cy, cz), cd.data_ptr(),
                               sd.data_ptr() if sd is not None else None, prob.Kn if kn is None else kn,
                               lid_speed(prob), x.data_ptr(), up.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    return x, up


def coarse_solution(prob: inputs.Problem, factor: int = 2, tol: float = 1e-4, max_iters: int = 1000) -> np.ndarray:
    """Macroscopic fields of `prob` on the grid `factor` times coarser, from
    the mixed-precision iteration stopped at residual `tol` (the network's
    input needs no tighter solution; 1e-4 lies above the mixed path's noise
    floor).  Returns [8, nz/f, ny/f, nx/f]."""
    c = kgs.kgs_setup(coarse_problem(prob, factor), precision=kgs.KGS_MIXED, tol=tol, max_iters=max_iters)
    kgs.kgs_iterate(c, 0)
    m = kgs.kgs_moments(c)
    kgs.kgs_destroy(c)
    return m


@dataclasses.dataclass
class Sample:
    prob: inputs.Problem
    coarse: np.ndarray       # converged coarse-grid fields [8, nz/2, ny/2, nx/2]
    fine: np.ndarray         # converged fields [8, nz, ny, nx]
    iters_coarse: int
    iters_fine: int


def draw_cavities(n: int, seed: int, cells: int, vels: int, kn_range=(0.05, 0.5), lid_range=(0.05, 0.3),
                  L_v: float = 4.0) -> List[inputs.Problem]:
    """Cavities of one size: Kn log-uniform and lid speed uniform on the given
    ranges, drawn from splitmix64(seed)."""
    g = inputs.SplitMix64(seed)
    out = []
    for _ in range(n):
        kn = kn_range[0] * (kn_range[1] / kn_range[0]) ** g.uniform()
        lid = lid_range[0] + (lid_range[1] - lid_range[0]) * g.uniform()
        out.append(inputs.cavity(cells, vels, Kn=kn, lid=lid, L_v=L_v))
    return out


def make_samples(probs: Sequence[inputs.Problem], precision=kgs.KGS_MIXED, tol=1e-6, max_iters=5000,
                 factor: int = 2) -> List[Sample]:
    """Converged coarse and fine solutions of each problem; the fine solves
    start from the upsampled coarse solutions (only the converged fields are
    kept, so the start changes nothing but the time taken)."""
    coarse_probs = [coarse_problem(p, factor) for p in probs]
    coarse, it_c, _, _ = solve(coarse_probs, precision, tol, max_iters)
    starts = []
    for p, c in zip(probs, coarse):
        _, up = upsample(p, c)
        starts.append(up.cpu().numpy())
    fine, it_f, _, _ = solve(probs, precision, tol, max_iters, initial=starts)
    return [Sample(p, c, f, ic, jf) for p, c, f, ic, jf in zip(probs, coarse, fine, it_c, it_f)]


class Surrogate:
    """A kgs_net with the feature and guess maps around it."""

    def __init__(self, channels=DEFAULT_CHANNELS, seed: int = 0):
        if channels[0] != N_FEATURES or channels[-1] != N_FIELDS:
            raise ValueError("the network maps %d features to %d fields" % (N_FEATURES, N_FIELDS))
        self.channels = tuple(channels)
        self.net = kgs.kgs_net_create(self.channels, seed=seed,
                                      stream=torch.cuda.current_stream().cuda_stream)

    def num_params(self) -> int:
        return kgs.kgs_net_num_params(self.net)[0]

    def train(self, samples: Sequence[Sample], steps: int, batch: int = 8, lr: float = 1e-3, seed: int = 0,
              lr_final: Optional[float] = None) -> List[float]:
        """Adam on the mean squared error of the normalised correction, on
        mini-batches drawn without replacement from a seeded permutation;
        the step size decays by cosine to lr_final (default lr / 20).
        All samples must share one grid.  Returns the loss per step."""
        shape = (samples[0].prob.nz, samples[0].prob.ny, samples[0].prob.nx)
        if any((s.prob.nz, s.prob.ny, s.prob.nx) != shape for s in samples):
            raise ValueError("train: samples must share one grid")
        ncell = int(np.prod(shape))
        X = torch.empty((len(samples),) + shape + (N_FEATURES,), dtype=torch.float32, device="cuda")
        T = torch.empty((len(samples), ncell, N_FIELDS), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for i, s in enumerate(samples):
            x, up = upsample(s.prob, s.coarse)
            X[i].copy_(x)
            fd = torch.as_tensor(np.ascontiguousarray(s.fine), dtype=torch.float64, device="cuda")
            kgs.kgs_surrogate_target(ncell, fd.data_ptr(), up.data_ptr(), T[i].data_ptr(), stream)
        batch = min(batch, len(samples))
        xb = torch.empty((batch,) + X.shape[1:], dtype=X.dtype, device="cuda")
        tb = torch.empty((batch,) + T.shape[1:], dtype=T.dtype, device="cuda")
        rng = np.random.default_rng(seed)
        lr_final = lr / 20 if lr_final is None else lr_final
        order, pos, losses = rng.permutation(len(samples)), 0, []
        for step in range(steps):
            if pos + batch > len(order):
                order, pos = rng.permutation(len(samples)), 0
            idx = torch.as_tensor(order[pos:pos + batch], device="cuda")
            pos += batch
            torch.index_select(X, 0, idx, out=xb)
            torch.index_select(T, 0, idx, out=tb)
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / max(steps, 1)))
            losses.append(kgs.kgs_net_train_step(self.net, xb.data_ptr(), tb.data_ptr(), None, (batch,) + shape,
                                                 lr_t))
        return losses

    def guess(self, prob: inputs.Problem, coarse: np.ndarray):
        """Initial fields [8, nz, ny, nx] (host) for `prob` from its coarse
        solution, or None when the guess is rejected (the caller then starts
        from the uniform state), and the number of cells that failed the check."""
        x, up = upsample(prob, coarse)
        y = torch.empty((prob.ncell, N_FIELDS), dtype=torch.float32, device="cuda")
        kgs.kgs_net_forward(self.net, x.data_ptr(), (1, prob.nz, prob.ny, prob.nx), y.data_ptr())
        m = torch.empty_like(up)
        n_bad = kgs.kgs_surrogate_apply(prob.ncell, up.data_ptr(), y.data_ptr(), m.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        if n_bad:
            return None, n_bad
        return m.cpu().numpy(), 0

    def predict(self, prob: inputs.Problem, coarse: np.ndarray) -> np.ndarray:
        """Raw network output for prob: normalised correction [nz, ny, nx, 8]."""
        x, _ = upsample(prob, coarse)
        y = torch.empty((prob.ncell, N_FIELDS), dtype=torch.float32, device="cuda")
        kgs.kgs_net_forward(self.net, x.data_ptr(), (1, prob.nz, prob.ny, prob.nx), y.data_ptr())
        return y.cpu().numpy().reshape(prob.nz, prob.ny, prob.nx, N_FIELDS)


def iterations_to(prob: inputs.Problem, initial: Optional[np.ndarray], precision=kgs.KGS_MIXED, tol=1e-6,
                  max_iters=5000):
    """(iterations, seconds, residual, status) of one solve from `initial`
    (None = uniform state), timed around kgs_iterate."""
    ctx = kgs.kgs_setup(prob, precision=precision, tol=tol, max_iters=max_iters)
    kgs.kgs_set_initial(ctx, initial)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, n, res = kgs.kgs_iterate(ctx, 0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    kgs.kgs_destroy(ctx)
    return n, dt, res, rc


def main(argv=None):
    """Train the network on solver-generated cavities and report the
    iterations and time to a residual of 1e-6 on held-out cavities, from the
    uniform state (plain FP64; mixed then FP64) and from the guess.

        python -m paper_1810_00348_gb300.surrogate --samples 512 --steps 3000
    """
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=512, help="training cavities (seed 1)")
    ap.add_argument("--cells", type=int, default=16)
    ap.add_argument("--vels", type=int, default=16)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--kn", default="0.05,0.2,0.5", help="held-out Knudsen numbers")
    ap.add_argument("--lids", default="0.1,0.25", help="held-out lid speeds")
    ap.add_argument("--save", default="", help="write the trained parameters (float32) to this file")
    ap.add_argument("--eval-cells", type=int, default=0,
                    help="also evaluate on held-out cavities of this size (cells per side; 0 = training size)")
    ap.add_argument("--eval-vels", type=int, default=0, help="velocities per side of the extra evaluation")
    ap.add_argument("--eval-kn", default="0.5", help="Knudsen numbers of the extra evaluation")
    ap.add_argument("--forward-only", type=int, default=0,
                    help="only time forward passes of the untrained network on one N^3 volume and exit")
    ap.add_argument("--train-only", type=int, default=0,
                    help="only time training steps of the network on a batch of 4 random N^3 volumes and exit")
    args = ap.parse_args(argv)
    kgs.load()
    if args.forward_only:
        n = args.forward_only
        s = Surrogate(seed=0)
        shape = (1, n, n, n)
        x = torch.randn(shape + (N_FEATURES,), device="cuda")
        y = torch.empty(shape + (N_FIELDS,), device="cuda")
        ms = []
        for _ in range(4):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            kgs.kgs_net_forward(s.net, x.data_ptr(), shape, y.data_ptr())
            ms.append((time.perf_counter() - t1) * 1e3)
        print(json.dumps({"forward_ms": ms[1:], "voxels": n ** 3}))
        return
    if args.train_only:
        n = args.train_only
        s = Surrogate(seed=0)
        shape = (4, n, n, n)
        x = torch.randn(shape + (N_FEATURES,), device="cuda")
        t = torch.randn(shape + (N_FIELDS,), device="cuda")
        ms = []
        for _ in range(4):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            kgs.kgs_net_train_step(s.net, x.data_ptr(), t.data_ptr(), None, shape, 1e-5)
            ms.append((time.perf_counter() - t1) * 1e3)
        print(json.dumps({"train_step_ms": ms[1:], "voxels": 4 * n ** 3}))
        return
    t0 = time.perf_counter()
    samples = make_samples(draw_cavities(args.samples, seed=1, cells=args.cells, vels=args.vels),
                           precision=kgs.KGS_FP64, tol=1e-6, max_iters=5000)
    t_data = time.perf_counter() - t0
    s = Surrogate(seed=0)
    t0 = time.perf_counter()
    losses = s.train(samples, steps=args.steps, batch=args.batch, lr=args.lr, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if args.save:
        kgs.kgs_net_get(s.net, 0).tofile(args.save)
    cases = []
    for kn in [float(v) for v in args.kn.split(",")]:
        for lid in [float(v) for v in args.lids.split(",")]:
            p = inputs.cavity(args.cells, args.vels, Kn=kn, lid=lid)
            n_fp64, t_fp64, _, _ = iterations_to(p, None, kgs.KGS_FP64, 1e-6, 5000)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, _, nm, nd, _ = kgs.kgs_solve(p, None, 1e-6, 5000)
            t_mixed = time.perf_counter() - t1
            t1 = time.perf_counter()
            coarse = coarse_solution(p)
            guess, n_bad = s.guess(p, coarse)
            _, _, sm, sd, _ = kgs.kgs_solve(p, guess, 1e-6, 5000)
            torch.cuda.synchronize()
            t_sur = time.perf_counter() - t1
            _, up = upsample(p, coarse)
            n_up, _, _, _ = iterations_to(p, up.cpu().numpy(), kgs.KGS_FP64, 1e-6, 5000)
            n_nn, _, _, _ = iterations_to(p, guess, kgs.KGS_FP64, 1e-6, 5000) if guess is not None else (None,) * 4
            cases.append({"Kn": kn, "lid": lid,
                          "fp64_iterations": {"uniform": n_fp64, "upsampled_coarse": n_up, "surrogate": n_nn},
                          "seconds": {"fp64_uniform": t_fp64, "mixed_fp64_uniform": t_mixed,
                                      "mixed_fp64_surrogate_incl_coarse": t_sur},
                          "mixed_fp64_iterations": {"uniform": [nm, nd], "surrogate": [sm, sd]},
                          "guess_rejected": guess is None})
    extra = []
    if args.eval_cells:
        # a larger grid than the training one: the network was trained at
        # another cell size, so the guess may help less (or be rejected)
        for kn in [float(v) for v in args.eval_kn.split(",")]:
            p = inputs.cavity(args.eval_cells, args.eval_vels or args.vels, Kn=kn, lid=0.16)
            n_fp64, t_fp64, _, rc_f = iterations_to(p, None, kgs.KGS_FP64, 1e-6, 400)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rc_m, _, nm, nd, _ = kgs.kgs_solve(p, None, 1e-6, 400)
            t_mixed = time.perf_counter() - t1
            t1 = time.perf_counter()
            coarse = coarse_solution(p)
            guess, n_bad = s.guess(p, coarse)
            rc_s, _, sm, sd, _ = kgs.kgs_solve(p, guess, 1e-6, 400)
            torch.cuda.synchronize()
            t_sur = time.perf_counter() - t1
            extra.append({"cells": args.eval_cells, "vels": args.eval_vels or args.vels, "Kn": kn, "lid": 0.16,
                          "fp64_uniform": {"iterations": n_fp64, "s": t_fp64, "rc": rc_f},
                          "mixed_fp64_uniform": {"iterations": [nm, nd], "s": t_mixed, "rc": rc_m},
                          "mixed_fp64_surrogate": {"iterations": [sm, sd], "s": t_sur, "rc": rc_s,
                                                   "guess_rejected": guess is None}})
    print(json.dumps({"samples": len(samples), "cells": args.cells, "vels": args.vels, "data_s": t_data,
                      "train_s": t_train, "steps": args.steps, "loss_first": float(np.mean(losses[:20])),
                      "loss_last": float(np.mean(losses[-20:])), "params": s.num_params(), "cases": cases,
                      "larger_grid": extra},
                     indent=1))


if __name__ == "__main__":
    main()
