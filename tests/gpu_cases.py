"""Shared set-up for the GPU parity tests: one seeded case = inputs + the oracle's results.

Inputs come only from `synth` (seeded generators); expected values only from `oracle`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import oracle
from oracle import wproj
import synth

ARCMIN = math.pi / (180 * 60)

# Tolerances (peak-relative max error against the float64 oracle): float32 tables and
# float32 accumulation must reach 1e-5 on the dirty image; float16 tables 1e-3; bfloat16
# tables (8-bit mantissa) are reported against 3e-3.
TOL_IMAGE = {"f32": 1e-5, "f16": 1e-3, "bf16": 3e-3}


def inner(a):
    """The inner half of an image, |l|, |m| < L/4, where the taper is far from zero."""
    n = a.shape[0]
    return a[n // 4: 3 * n // 4, n // 4: 3 * n // 4]


def peak_rel(a, ref):
    a = np.asarray(a)
    ref = np.asarray(ref)
    scale = np.abs(ref).max()
    return float(np.abs(a - ref).max() / scale), float(np.sqrt(np.mean(np.abs(a - ref) ** 2)) / scale)


@dataclass
class Case:
    prm: oracle.Params
    uvw: np.ndarray
    freqs: np.ndarray
    vis: np.ndarray
    weight: np.ndarray | None
    pairs: bool
    tables: list
    nu: float


def parity_case(pairs=False, weights=True, rows=None) -> Case:
    """The 27-antenna parity workload (21,060 visibilities, 256^2, 16 planes, support 7)."""
    cfg = synth.config("parity")
    ob = synth.observe(cfg, rows=rows)
    prm = oracle.Params(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=ob.w_max, s_min=cfg.s_min, s_max=cfg.s_max,
                        os=cfg.oversample)
    tabs, nu = oracle.wkernels(prm)
    wt = (0.5 + np.random.default_rng(77).random(ob.weight.shape)).astype(np.float32) if weights else None
    return Case(prm, ob.uvw, ob.freqs, ob.vis, wt, pairs, tabs, nu)


def random_case(n=64, nrow=700, nchan=3, n_w=6, s_min=6, s_max=10, os_=8, pairs=False, seed=5,
                off_grid=0.1, cell=2.0 * ARCMIN) -> Case:
    """Random uvw over the grid (a fraction beyond it), several channels, w both signs."""
    rng = np.random.default_rng(seed)
    field = n * cell
    freqs = np.linspace(1.0e9, 1.3e9, nchan)
    lam_max = oracle.C_LIGHT / freqs.max()
    umax = (n / 2) / field * lam_max * (1 + off_grid)         # metres
    uvw = np.stack([rng.uniform(-umax, umax, nrow), rng.uniform(-umax, umax, nrow),
                    rng.uniform(-1, 1, nrow) * 3000 * lam_max], axis=1)
    w_max = float(np.abs(uvw[:, 2]).max() * freqs.max() / oracle.C_LIGHT)
    vis, wt = synth.random_visibilities(nrow, nchan, seed + 1)
    prm = oracle.Params(n=n, cell=cell, n_w=n_w, w_max=w_max, s_min=s_min, s_max=s_max, os=os_)
    tabs, nu = oracle.wkernels(prm)
    return Case(prm, uvw, freqs, vis, wt, pairs, tabs, nu)


def oracle_results(case: Case):
    crd = oracle.coords(case.uvw, case.freqs, case.prm, hermitian_pairs=case.pairs)
    c = wproj.gridded_values(case.vis, case.weight, crd)
    g = oracle.grid(crd, c, case.tables, case.prm, threads=4)
    sw = oracle.sum_weights(case.weight, crd)
    return crd, g, sw


def make_wproj(case: Case, table="f32", tile=(0, 0), units_per_cta=0):
    import paper_1905_03213_b300 as W
    p = case.prm
    w = W.WProj(n=p.n, cell=p.cell, n_w=p.n_w, w_max=p.w_max, support_min=p.s_min, support_max=p.s_max,
                oversample=p.os, screen_m=p.m, table=table, tile=tile, units_per_cta=units_per_cta)
    w.make_wkernels()
    return w


def to_dev(case: Case):
    import torch
    d = torch.device("cuda")
    uvw = torch.from_numpy(np.ascontiguousarray(case.uvw)).to(d)
    f = torch.from_numpy(np.ascontiguousarray(case.freqs)).to(d)
    vis = torch.from_numpy(np.ascontiguousarray(case.vis)).to(d)
    wt = None if case.weight is None else torch.from_numpy(np.ascontiguousarray(case.weight)).to(d)
    return uvw, f, vis, wt
