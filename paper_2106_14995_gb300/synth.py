"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path's tests/benchmark and by the oracle's tests.  It
draws random numbers and lays them out in the packed formats of the C-ABI; it contains
none of the solver's or the ADMM's arithmetic.  The paper's MATPOWER/PGLIB cases
(Table 4, Sec. 6.1) are not available, so power-network-shaped random data stands in.

Seeds are ``SEED_BASE + workload index`` with numpy's ``default_rng``.

Packed layouts (shared contract with ``include/tron.h``):

* branch record, 36 doubles: ``[0:8]`` gc_ij, bc_ij, g_ij, b_ij, gc_ji, bc_ji, g_ji,
  b_ji (eqs. pij-qji); ``[8:16]`` multipliers, ``[16:24]`` targets and ``[24:32]``
  penalties of the pairs (p_ij, q_ij, p_ji, q_ji, w_i, w_j, theta_i, theta_j);
  ``[32]`` squared line limit; ``[33]`` line penalty; ``[34:36]`` zero.
* dense quartic record, n^2 + 2n doubles: Q (row-major), c, d with
  f = 1/2 x'Qx + c'x + sum d_i x_i^4.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2106149950
TWO_PI = 2.0 * math.pi
BRANCH_RECORD = 36


def rng_for(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + index + 1000003 * salt)


# --------------------------------------------------------------------- line data

def line_coefficients(r, x, bc):
    """Eight coefficients of eqs. pij-qji for a pi-model line with series impedance
    r + jx and total charging susceptance bc (no tap, no phase shift).

    With y = 1/(r + jx) = gs + j bs: g_ij = g_ji = gs, b_ij = b_ji = -bs,
    gc_ij = gc_ji = gs, bc_ij = bc_ji = -(bs + bc/2)."""
    r = np.asarray(r, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    bc = np.asarray(bc, dtype=np.float64)
    z2 = r * r + x * x
    gs = r / z2
    bs = -x / z2
    coef = np.stack([gs, -(bs + bc / 2), gs, -bs, gs, -(bs + bc / 2), gs, -bs], axis=-1)
    return coef


def random_lines(rng: np.random.Generator, m: int):
    r = rng.uniform(0.001, 0.05, m)
    x = rng.uniform(0.01, 0.3, m)
    bc = rng.uniform(0.0, 0.1, m)
    smax = rng.uniform(0.5, 2.0, m)
    return r, x, bc, smax


# ------------------------------------------------- 256 branch subproblems (n = 4)

def branch_batch(B: int = 256, seed_index: int = 0, rho: float = 400.0,
                 target_sd: float = 0.5):
    """B branch subproblems of eq. exp-branch with the line-limit penalty.

    lambda ~ N(0, 1) and targets ~ N(0, target_sd^2) for all eight pairs; rho for every
    pair and for the line term; bounds v in [0.9, 1.1], theta in [-2 pi, 2 pi]; x0 is
    the box midpoint (1, 1, 0, 0); delta0 = 1."""
    rng = rng_for(seed_index)
    r, x, bc, smax = random_lines(rng, B)
    rec = np.zeros((B, BRANCH_RECORD))
    rec[:, 0:8] = line_coefficients(r, x, bc)
    rec[:, 8:16] = rng.normal(0.0, 1.0, (B, 8))
    rec[:, 16:24] = rng.normal(0.0, target_sd, (B, 8))
    rec[:, 24:32] = rho
    rec[:, 32] = smax * smax
    rec[:, 33] = rho
    lo = np.tile(np.array([0.9, 0.9, -TWO_PI, -TWO_PI]), (B, 1))
    hi = np.tile(np.array([1.1, 1.1, TWO_PI, TWO_PI]), (B, 1))
    x0 = 0.5 * (lo + hi)
    delta0 = np.ones(B)
    return dict(kind=1, n=4, params=rec, l=lo, u=hi, x0=x0, delta0=delta0)


# ------------------------------------------------------- dense quartic problems

def haar_orthogonal(rng: np.random.Generator, B: int, n: int) -> np.ndarray:
    """B random orthogonal n x n matrices (QR of a Gaussian with the sign fix)."""
    G = rng.standard_normal((B, n, n))
    Qm, R = np.linalg.qr(G)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return Qm * d[:, None, :]


def dense_records(rng: np.random.Generator, B: int, n: int, cond: float = 1e3,
                  c_sd: float = 4.0, quartic: float = 0.1, diag_only: bool = False,
                  neg_frac: float = 0.0):
    """Q = U diag(lam) U' with U Haar, lam log-uniform in [1, cond]; c ~ N(0, c_sd^2);
    d = quartic; l ~ U[-2, -0.5]; u ~ U[0.5, 2]; x0 = 0.  neg_frac > 0: that fraction of
    each problem's eigenvalues (rounded up) is -U[0.5, 50] instead, an indefinite Q (the
    box and the quartic keep f bounded; the Hessian's shifted factorization and the
    PCG's negative-curvature exit come into play)."""
    lam = np.exp(rng.uniform(0.0, math.log(cond), (B, n)))
    if neg_frac > 0.0:
        k = int(math.ceil(neg_frac * n))
        lam[:, :k] = -rng.uniform(0.5, 50.0, (B, k))
    if diag_only:
        Q = np.zeros((B, n, n))
        idx = np.arange(n)
        Q[:, idx, idx] = lam
    else:
        U = haar_orthogonal(rng, B, n)
        Q = np.einsum("bij,bj,bkj->bik", U, lam, U)
        Q = 0.5 * (Q + np.transpose(Q, (0, 2, 1)))
    c = rng.normal(0.0, c_sd, (B, n))
    d = np.full((B, n), float(quartic))
    rec = np.concatenate([Q.reshape(B, n * n), c, d], axis=1)
    lo = rng.uniform(-2.0, -0.5, (B, n))
    hi = rng.uniform(0.5, 2.0, (B, n))
    x0 = np.zeros((B, n))
    return rec, lo, hi, x0


def dense_batch(B: int = 10000, n: int = 32, seed_index: int = 1, **kw):
    """Generic dense problems: f = 1/2 x'Qx + c'x + 0.1 sum x^4 (n = 32, B = 10,000)."""
    rng = rng_for(seed_index)
    rec, lo, hi, x0 = dense_records(rng, B, n, **kw)
    return dict(kind=2, n=n, params=rec, l=lo, u=hi, x0=x0, delta0=np.ones(B))


UNEVEN_SIZES = (4, 6, 8, 16, 32, 64, 128)
UNEVEN_PROBS = (0.4, 0.2, 0.15, 0.1, 0.08, 0.05, 0.02)


def uneven_batch(B: int = 100000, seed_index: int = 3, sizes=UNEVEN_SIZES,
                 probs=UNEVEN_PROBS):
    """Dense problems with n drawn from ``sizes`` with ``probs``; flat concatenated
    layout (params of problem p at its own offset, vectors concatenated)."""
    rng = rng_for(seed_index)
    nvec = rng.choice(np.asarray(sizes), size=B, p=np.asarray(probs)).astype(np.int32)
    params = [None] * B
    lo = [None] * B
    hi = [None] * B
    for n in sizes:
        idx = np.nonzero(nvec == n)[0]
        if idx.size == 0:
            continue
        sub = rng_for(seed_index, salt=int(n))
        rec, l_, u_, _ = dense_records(sub, idx.size, int(n))
        for t, p in enumerate(idx):
            params[p] = rec[t]
            lo[p] = l_[t]
            hi[p] = u_[t]
    params = np.concatenate(params)
    lo = np.concatenate(lo)
    hi = np.concatenate(hi)
    x0 = np.zeros_like(lo)
    return dict(kind=2, nvec=nvec, params=params, l=lo, u=hi, x0=x0, delta0=np.ones(B))


def hs45_batch(B: int, n: int):
    """hs45 variant of Sec. 4.2: f = 120 - prod x_i, 0 <= x_i <= i, x0 = midpoint."""
    hi = np.tile(np.arange(1, n + 1, dtype=np.float64), (B, 1))
    lo = np.zeros((B, n))
    x0 = 0.5 * hi
    return dict(kind=3, n=n, params=np.zeros((B, 0)), l=lo, u=hi, x0=x0, delta0=np.ones(B))


# -------------------------------------------------------------- power networks

def network(nbus: int = 10000, nchord: int = 3000, ngen: int = 3000, seed_index: int = 2,
            load_scale: float = 1.0, rng: np.random.Generator | None = None) -> dict:
    """Synthetic power network: random spanning tree (after a random permutation, bus k
    attaches to a uniformly chosen earlier bus) plus ``nchord`` distinct extra edges;
    generators on distinct random buses; line data as in ``random_lines``; loads
    p ~ U[0, 1], q ~ U[-0.2, 0.5] (times ``load_scale``); costs c2 ~ U[0.001, 0.05],
    c1 ~ U[5, 40]; p_min = 0, p_max = U[0.5, 1.5] * 2 * sum(p_d) / ngen,
    q_max = p_max / 2, q_min = -q_max; no shunts."""
    rng = rng or rng_for(seed_index)
    perm = rng.permutation(nbus)
    parent_pos = (rng.random(nbus) * np.arange(nbus)).astype(np.int64)
    frm = perm[parent_pos[1:]]
    to = perm[1:]
    edges = set()
    for a, b in zip(frm.tolist(), to.tolist()):
        edges.add((min(a, b), max(a, b)))
    cf, ct = [], []
    nchord = min(nchord, nbus * (nbus - 1) // 2 - (nbus - 1))
    while len(cf) < nchord:
        a, b = rng.integers(0, nbus, 2).tolist()
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in edges:
            continue
        edges.add(key)
        cf.append(a)
        ct.append(b)
    br_from = np.concatenate([frm, np.asarray(cf, dtype=np.int64)]).astype(np.int32)
    br_to = np.concatenate([to, np.asarray(ct, dtype=np.int64)]).astype(np.int32)
    nl = br_from.size
    r, x, bc, smax = random_lines(rng, nl)
    ngen = min(ngen, nbus)
    gen_bus = rng.choice(nbus, size=ngen, replace=False).astype(np.int32)
    pd = rng.uniform(0.0, 1.0, nbus) * load_scale
    qd = rng.uniform(-0.2, 0.5, nbus) * load_scale
    pmax = rng.uniform(0.5, 1.5, ngen) * 2.0 * pd.sum() / max(ngen, 1)
    return dict(
        nbus=int(nbus), br_from=br_from, br_to=br_to, br_r=r, br_x=x, br_bc=bc,
        br_coef=line_coefficients(r, x, bc), br_smax2=smax * smax, gen_bus=gen_bus,
        gen_c2=rng.uniform(0.001, 0.05, ngen), gen_c1=rng.uniform(5.0, 40.0, ngen),
        gen_pmin=np.zeros(ngen), gen_pmax=pmax, gen_qmin=-0.5 * pmax, gen_qmax=0.5 * pmax,
        bus_pd=pd, bus_qd=qd, bus_gsh=np.zeros(nbus), bus_bsh=np.zeros(nbus))


def load_profile(T: int = 24, swing: float = 0.2) -> np.ndarray:
    """Per-period load scale of a synthetic day: 1 + swing sin(2 pi (t - 6) / 24), so the
    load rises through the morning, peaks at hour 12 and falls through the evening."""
    t = np.arange(T, dtype=np.float64)
    return 1.0 + swing * np.sin(2.0 * math.pi * (t - 6.0) / 24.0)


def genramp_batch(B: int = 3000, T: int = 24, seed_index: int = 8, rho: float = 400.0,
                  rho_ramp: float = 1.0e4) -> dict:
    """Multi-period generator problems (record [c2 c1 rho rho_r R 0 0 0 | lambda | target]):
    c2 ~ U[0.001, 0.05], c1 ~ U[5, 40], p in [0, p_max] with p_max ~ U[0.5, 1.5], ramp
    R ~ U[0.02, 0.2] p_max, multipliers ~ N(0, 20^2), targets ~ U[0, p_max] per period
    (so that ramps bind), x0 = the targets."""
    rng = rng_for(seed_index)
    c2 = rng.uniform(0.001, 0.05, B)
    c1 = rng.uniform(5.0, 40.0, B)
    pmax = rng.uniform(0.5, 1.5, B)
    ramp = rng.uniform(0.02, 0.2, B) * pmax
    lam = rng.normal(0.0, 20.0, (B, T))
    tgt = rng.uniform(0.0, 1.0, (B, T)) * pmax[:, None]
    rec = np.zeros((B, 8 + 2 * T))
    rec[:, 0] = c2
    rec[:, 1] = c1
    rec[:, 2] = rho
    rec[:, 3] = rho_ramp
    rec[:, 4] = ramp
    rec[:, 8:8 + T] = lam
    rec[:, 8 + T:] = tgt
    lo = np.zeros((B, T))
    hi = np.repeat(pmax[:, None], T, axis=1)
    return dict(kind=4, n=T, params=rec, l=lo, u=hi, x0=tgt.copy(), delta0=np.ones(B))


def serving_stream(duration_s: float = 60.0, rate_hz: float = 200.0, seed_index: int = 4,
                   bus_lo: int = 500, bus_hi: int = 20000, load_lo: float = 0.8,
                   load_hi: float = 1.2):
    """Poisson arrivals of independent ADMM instances: arrival times, bus counts
    log-uniform in [bus_lo, bus_hi] (branches 1.3x, generators 0.3x), load scaling
    U[load_lo, load_hi] and a per-instance seed."""
    rng = rng_for(seed_index)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        nb = int(round(math.exp(rng.uniform(math.log(bus_lo), math.log(bus_hi)))))
        out.append(dict(t=t, nbus=nb, nchord=int(round(0.3 * nb)),
                        ngen=max(1, int(round(0.3 * nb))),
                        load_scale=float(rng.uniform(load_lo, load_hi)),
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out


def instance_network(spec: dict) -> dict:
    return network(spec["nbus"], spec["nchord"], spec["ngen"], load_scale=spec["load_scale"],
                   rng=np.random.default_rng(spec["seed"]))
