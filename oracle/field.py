"""Spatially correlated random fields in FP64 (Section 5 of arXiv 2212.04415).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What is computed, step by step:

1. Random numbers.  The KL coefficients xi_k ~ N(0, 1) of sample ``sample_id``
   on MLMC level ``level`` come from the Philox4x32-10 counter-based generator
   (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed low word, seed high word),
   counter = (block j, sample_id low, sample_id high, level). Each block gives
   four 32-bit words; words (0, 1) and (2, 3) form two 53-bit uniforms
   u = ((w_a << 32 | w_b) >> 11 + 1/2) 2^-53 in (0, 1), and the Box-Muller
   transform turns them into xi_{2j} = r cos(2 pi u2), xi_{2j+1} = r sin(2 pi u2),
   r = sqrt(-2 ln u1). Pinned by the published known-answer vectors.
2. Covariance.  Squared exponential C(r) = exp(-r^2 / l^2) (the measured
   workloads) or the paper's exponential C(r) = exp(-r / l_c)
   (Eq. exponential_correlation_function), variance 1.
3. Truncated KL expansion (Section 5).  For the separable squared-exponential
   kernel on a regular grid the covariance matrix is the Kronecker product of
   three 1D matrices, so each 3D mode is a product of 1D eigenvectors with
   eigenvalue lambda_a lambda_b lambda_c; the K largest products are kept.
   1D eigenpairs come from ``numpy.linalg.eigh`` (a library primitive).
   Readings: 1D eigenvalues sorted descending; each 1D eigenvector signed so
   its largest-magnitude entry is positive (lowest index among entries within
   1e-9 relative of the largest); products sorted descending, and each run of
   products within 1e-10 relative of the run's first is ordered by (a, b, c)
   ascending. For the exponential kernel (not separable) the
   dense covariance is decomposed directly (small meshes only), same sign rule.
   Pinned by: the Kronecker modes agree with the dense decomposition; the
   truncated covariance Phi Lambda Phi^T tends to the full matrix as K -> N.
4. Gaussian field g = Phi diag(sqrt(lambda)) xi.
5. Level coupling (Section 4.2, "a coarsened version of the random sample"):
   the coarse-level field is the mean of the fine field over the 2x2x2 fine
   children of each coarse node (2x2 for a plane hierarchy of one-layer
   grids), before the marginal transform.
6. Marginal transform (copula, Section 5.2): lognormal
   s0 = exp(mu + sigma g), sigma^2 = ln(1 + COV^2), mu = ln(mean) - sigma^2/2;
   Weibull s0 = F_W^-1(Phi(g)) with modulus m and scale mean / Gamma(1 + 1/m).
7. Chain rule back to the coefficients (for gradients of a quantity J with
   respect to xi, given dJ/ds0 per node): dJ/dg_i = dJ/ds0_i ds0/dg_i with
   ds0/dg = sigma s0 (lognormal) or, for the Weibull copula with
   q = 1 - Phi(g), ds0/dg = (scale / m) (-ln q)^(1/m - 1) phi(g) / q; then
   dJ/dxi_k = sum_i dJ/dg_i sqrt(lambda_k) Phi_ik. Pinned by central
   differences of the whole chain xi -> s0 -> run -> J.
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on arrays: ctr (..., 4) uint32, key (..., 2) uint32."""
    c = [np.asarray(ctr[..., i], np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], np.uint64)
    k1 = np.asarray(key[..., 1], np.uint64)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def draw_xi(seed: int, level: int, sample_ids, n_modes: int) -> np.ndarray:
    """KL coefficients xi [B, K] (FP64) for the given samples of one level."""
    sid = np.asarray(sample_ids, np.uint64).reshape(-1)
    B = sid.size
    nblk = (n_modes + 1) // 2
    j = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((B, nblk, 4), np.uint32)
    ctr[..., 0] = j[None, :]
    ctr[..., 1] = (sid & _MASK)[:, None]
    ctr[..., 2] = (sid >> np.uint64(32))[:, None]
    ctr[..., 3] = level
    key = np.zeros((B, nblk, 2), np.uint32)
    key[..., 0] = seed & 0xFFFFFFFF
    key[..., 1] = (seed >> 32) & 0xFFFFFFFF
    w = philox4x32_10(ctr, key).astype(np.uint64)
    a = ((w[..., 0] << np.uint64(32)) | w[..., 1]) >> np.uint64(11)
    b = ((w[..., 2] << np.uint64(32)) | w[..., 3]) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (b.astype(np.float64) + 0.5) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    z0 = r * np.cos(2.0 * np.pi * u2)
    z1 = r * np.sin(2.0 * np.pi * u2)
    xi = np.empty((B, 2 * nblk))
    xi[:, 0::2] = z0
    xi[:, 1::2] = z1
    return xi[:, :n_modes]


def _sign_fix(vecs: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of each column positive (lowest index on a near-tie)."""
    out = vecs.copy()
    for k in range(vecs.shape[1]):
        a = np.abs(vecs[:, k])
        top = a.max()
        idx = int(np.nonzero(a >= top * (1.0 - 1e-9))[0][0])
        if vecs[idx, k] < 0:
            out[:, k] = -vecs[:, k]
    return out


def cov1d(n: int, dx: float, length: float, kernel: int = 0) -> np.ndarray:
    """1D covariance of n cell-centred nodes (squared exponential: exact factor of 3D)."""
    x = (np.arange(n) + 0.5) * dx
    r = np.abs(x[:, None] - x[None, :])
    if kernel == 0:
        return np.exp(-(r * r) / (length * length))
    return np.exp(-r / length)


def eig1d(n: int, dx: float, length: float):
    """1D eigenpairs of the squared-exponential covariance, descending, sign-fixed."""
    lam, vec = np.linalg.eigh(cov1d(n, dx, length, 0))
    order = np.argsort(-lam, kind="stable")
    return lam[order], _sign_fix(vec[:, order])


def select_modes(lx, ly, lz, K):
    """Indices (a, b, c) of the K largest products lx[a] ly[b] lz[c].

    Products are sorted descending; each run of products lying within 1e-10
    relative of the run's first product counts as tied and is taken in
    ascending (a, b, c) order."""
    cand = []
    for a in range(len(lx)):
        for b in range(len(ly)):
            for c in range(len(lz)):
                cand.append((lx[a] * ly[b] * lz[c], a, b, c))
    cand.sort(key=lambda t: (-t[0], t[1], t[2], t[3]))
    out = []
    g0 = 0
    while g0 < len(cand):
        g1 = g0 + 1
        while g1 < len(cand) and cand[g0][0] - cand[g1][0] <= 1e-10 * abs(cand[g0][0]):
            g1 += 1
        out.extend(sorted(cand[g0:g1], key=lambda t: t[1:]))
        g0 = g1
    return [(a, b, c) for _, a, b, c in out[:K]]


def kl_separable(grid, length: float, K: int):
    """Phi [N, K] (x fastest node order) and lambda [K] for exp(-r^2/l^2)."""
    lx, vx = eig1d(grid.nx, grid.dx, length)
    ly, vy = eig1d(grid.ny, grid.dx, length)
    lz, vz = eig1d(grid.nz, grid.dx, length)
    # keep enough 1D modes to contain the top K products
    kx, ky, kz = min(grid.nx, K), min(grid.ny, K), min(grid.nz, K)
    sel = select_modes(lx[:kx], ly[:ky], lz[:kz], K)
    N = grid.nx * grid.ny * grid.nz
    Phi = np.empty((N, len(sel)))
    lam = np.empty(len(sel))
    for k, (a, b, c) in enumerate(sel):
        m = vz[:, c][:, None, None] * vy[:, b][None, :, None] * vx[:, a][None, None, :]
        Phi[:, k] = m.reshape(-1)
        lam[k] = lx[a] * ly[b] * lz[c]
    return Phi, lam


def node_coords(grid) -> np.ndarray:
    n = np.arange(grid.nx * grid.ny * grid.nz)
    ix = n % grid.nx
    iy = (n // grid.nx) % grid.ny
    iz = n // (grid.nx * grid.ny)
    return np.stack([(ix + 0.5) * grid.dx, (iy + 0.5) * grid.dx, (iz + 0.5) * grid.dx], 1)


def dense_cov(grid, length: float, kernel: int) -> np.ndarray:
    x = node_coords(grid)
    r2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    if kernel == 0:
        return np.exp(-r2 / (length * length))
    return np.exp(-np.sqrt(r2) / length)


def kl_dense(grid, length: float, K: int, kernel: int):
    """Truncated KL from the dense covariance matrix (small meshes only)."""
    lam, vec = np.linalg.eigh(dense_cov(grid, length, kernel))
    order = np.argsort(-lam, kind="stable")[:K]
    return _sign_fix(vec[:, order]), lam[order]


def gaussian(Phi, lam, xi) -> np.ndarray:
    """g = Phi diag(sqrt(lambda)) xi, for xi [B, K]: returns [B, N]."""
    return (Phi @ (np.sqrt(lam)[:, None] * np.asarray(xi, np.float64).T)).T


def restrict(g: np.ndarray, grid) -> np.ndarray:
    """Mean over the fine children of each coarse node; g is [B, N_fine]: 2x2x2
    children in 3D, 2x2 on a one-layer grid (a plane hierarchy keeps nz = 1)."""
    B = g.shape[0]
    a = g.reshape(B, grid.nz, grid.ny, grid.nx)
    if grid.nz == 1:
        a = a.reshape(B, grid.ny // 2, 2, grid.nx // 2, 2)
        a = a[..., 0] + a[..., 1]
        a = a[:, :, 0, :] + a[:, :, 1, :]
        return (a * 0.25).reshape(B, -1)
    a = a.reshape(B, grid.nz // 2, 2, grid.ny // 2, 2, grid.nx // 2, 2)
    # sum in a fixed order: x pairs, then y pairs, then z pairs
    a = a[..., 0] + a[..., 1]
    a = a[:, :, :, :, 0, :] + a[:, :, :, :, 1, :]
    a = a[:, :, 0] + a[:, :, 1]
    return (a * 0.125).reshape(B, -1)


def lognormal(g, mean: float, cov: float):
    s2 = math.log(1.0 + cov * cov)
    mu = math.log(mean) - 0.5 * s2
    return np.exp(mu + math.sqrt(s2) * np.asarray(g))


def weibull(g, mean: float, m: float):
    from scipy.special import ndtr
    scale = mean / math.gamma(1.0 + 1.0 / m)
    p = ndtr(np.asarray(g))
    return scale * (-np.log1p(-p)) ** (1.0 / m)


def grad_xi(fcfg, Phi, lam, xi, dJ_ds0):
    """dJ/dxi [B, K] from dJ/ds0 [B, N] through the marginal transform and the
    truncated KL expansion (step 7 above)."""
    g = gaussian(Phi, lam, xi)
    dJ = np.asarray(dJ_ds0, np.float64)
    if fcfg.marginal == 0:
        s2 = math.log(1.0 + fcfg.cov * fcfg.cov)
        dg = dJ * math.sqrt(s2) * lognormal(g, fcfg.mean, fcfg.cov)
    else:
        from scipy.special import ndtr
        m = fcfg.weibull_m
        scale = fcfg.mean / math.gamma(1.0 + 1.0 / m)
        q = 1.0 - ndtr(g)
        pdf = np.exp(-0.5 * g * g) / math.sqrt(2.0 * math.pi)
        dg = dJ * (scale / m) * (-np.log(q)) ** (1.0 / m - 1.0) * pdf / q
    return (dg @ Phi) * np.sqrt(lam)[None, :]


def sample_field(w, Phi, lam, seed, level, sample_ids):
    """s0 per node [B, N] for a workload's field settings (FP64)."""
    f = w.field
    xi = draw_xi(seed, level, sample_ids, f.n_modes)
    g = gaussian(Phi, lam, xi)
    if f.marginal == 0:
        return lognormal(g, f.mean, f.cov)
    return weibull(g, f.mean, f.weibull_m)
