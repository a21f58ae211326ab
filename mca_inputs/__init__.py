"""Seeded synthetic crossbar inputs shared by the oracle, the tests and the bench.

This module draws random numbers and fills parameter records; it holds none of the
method's arithmetic (no residual, Jacobian, preconditioner or solver).  Both the CPU
oracle and the CUDA path consume exactly the arrays it returns.

Circuit recipe (Section 2 of the paper describes the topology; the values follow the
workloads this library is measured on):

* top layer: one wire per row (word line), segment conductance ``g_wire_top``;
  the left end of row i is driven by ``V_in[i]`` through ``g_src`` (10 ohm), the right
  end goes to ground through ``g_term_top_right`` (1 kohm);
* bottom layer: one wire per column (bit line), segment conductance ``g_wire_bot``;
  the top end (row 0) goes to ground through ``g_term_bot_top`` (1 kohm), the bottom
  end (row m-1) is sensed at virtual ground through ``g_sense`` (10 ohm);
* memristor at each (i, j): i = (g_ij / b) * sinh(b * dV), b = 2 1/V.

Draw order for one crossbar: the conductance map (row-major) first, then the input
vectors, all from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, field

import numpy as np


@dataclass
class CrossbarParams:
    rows: int
    cols: int
    g_wire_top: float = 1.0
    g_wire_bot: float = 1.0
    g_src: float = 0.1
    g_term_top_right: float = 1e-3
    g_term_bot_top: float = 1e-3
    g_sense: float = 0.1
    b: float = 2.0
    # device model: a2/a1 of the Yakopcic-form I-V curve (current scale for dV < 0 over the
    # one for dV >= 0); 1 gives the symmetric sinh device
    neg_ratio: float = 1.0

    def as_dict(self):
        return asdict(self)


@dataclass
class Crossbar:
    params: CrossbarParams
    gmap: np.ndarray          # (rows, cols) float64, siemens, row-major
    vin: np.ndarray           # (nvec, rows) float64, volts
    seed: int = 0
    tags: dict = field(default_factory=dict)


def log_uniform(rng, shape, lo=1e-6, hi=1e-4):
    """g = 10**U(log10 lo, log10 hi)."""
    return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=shape)


def bimodal(rng, shape, p_on=0.1, g_on=1e-4, g_off=1e-6, sigma=0.1):
    """Bernoulli(p_on) picks g_on else g_off, then a median-preserving lognormal factor."""
    on = rng.random(shape) < p_on
    g = np.where(on, g_on, g_off)
    return g * np.exp(sigma * rng.standard_normal(shape))


def make_crossbar(rows, cols, seed, nvec=1, gdist="loguniform", sigma=0.0,
                  vmax=0.3, vmin=0.0, **wiring) -> Crossbar:
    """One crossbar: conductance map then ``nvec`` input vectors V_in ~ U[vmin, vmax]."""
    rng = np.random.default_rng(seed)
    shape = (rows, cols)
    if gdist == "loguniform":
        g = log_uniform(rng, shape)
        if sigma > 0:
            g = g * np.exp(sigma * rng.standard_normal(shape))
    elif gdist == "bimodal":
        g = bimodal(rng, shape)
    elif gdist == "uniform_paper":
        # normalised regime of the paper's experiments: wire g = 1, devices up to 0.4
        g = rng.uniform(0.0, 0.4, size=shape)
    else:
        raise ValueError(gdist)
    vin = rng.uniform(vmin, vmax, size=(nvec, rows))
    p = CrossbarParams(rows=rows, cols=cols, **wiring)
    return Crossbar(params=p, gmap=np.ascontiguousarray(g, dtype=np.float64),
                    vin=np.ascontiguousarray(vin, dtype=np.float64), seed=seed)


# ---- the five workloads -------------------------------------------------------------

def config_small(seed=0):
    """32x32, log-uniform g in [1e-6, 1e-4] S, one input vector, Newton to 1e-10."""
    return make_crossbar(32, 32, seed)


def config_bimodal(seed):
    """256x256, bimodal g (10% 1e-4 S, 90% 1e-6 S, x lognormal 0.1); map s and V_in s."""
    return make_crossbar(256, 256, seed, gdist="bimodal")


def config_large(n, seed, nvec=1):
    """n x n (1024 or 2048), log-uniform g, top wire 1 S, bottom wire 0.5 S."""
    return make_crossbar(n, n, seed, nvec=nvec, g_wire_bot=0.5)


@dataclass
class CrossbarSet:
    """Several crossbars of one shape and wiring with their input vectors interleaved:
    vector v belongs to crossbar map_index[v]."""
    params: CrossbarParams
    gmaps: np.ndarray       # (k, m, n)
    vin: np.ndarray         # (nvec, m)
    map_index: np.ndarray   # (nvec,) int32
    seeds: tuple


def config_large_set(n, seeds=(0, 1, 2, 3), nvec=4):
    """The n x n workload over several crossbars (seeds 0-3 by default): crossbar k is
    config_large(n, seeds[k]); vector v is crossbar v % k's own vector v // k."""
    k = len(seeds)
    per = (nvec + k - 1) // k
    cbs = [config_large(n, s, nvec=per) for s in seeds]
    idx = np.arange(nvec)
    vin = np.stack([cbs[v % k].vin[v // k] for v in idx])
    return CrossbarSet(params=cbs[0].params, gmaps=np.stack([c.gmap for c in cbs]),
                       vin=np.ascontiguousarray(vin), map_index=(idx % k).astype(np.int32),
                       seeds=tuple(seeds))


BATCH_SIZES = (64, 128, 256, 512)


def config_batched(count=128, nvec=16, base_seed=1000, sizes=BATCH_SIZES):
    """Statistical characterisation: ``count`` crossbars, rows and cols each drawn
    from ``sizes`` ({64,128,256,512}; by a size rng seeded with base_seed), log-uniform g
    with lognormal sigma 0.1 variation, ``nvec`` input vectors each; crossbar c uses seed
    base_seed + c for its own draws."""
    srng = np.random.default_rng(base_seed)
    dims = srng.choice(sizes, size=(count, 2))
    out = []
    for c in range(count):
        out.append(make_crossbar(int(dims[c, 0]), int(dims[c, 1]), base_seed + c,
                                 nvec=nvec, sigma=0.1))
    return out


def config_paper_regime(n, seed):
    """Normalised regime of the paper's Table 1 runs: wire g = 1, terminations = g,
    linear-conductance devices drawn in [0, 0.4] (the paper's device model parameters
    are not given, so the devices are linear: b = 0)."""
    return make_crossbar(n, n, seed, gdist="uniform_paper", g_src=1.0,
                         g_term_top_right=1.0, g_term_bot_top=1.0, g_sense=1.0, b=0.0)
