"""Seeded synthetic Tucker tensors: the generator of Section 8.2 of the
TuckerMPI paper (arXiv 1901.06043), which the paper ships "for testing and
debugging".

Recipe (draw order: core, then the factors of modes 0..N-1, then noise):

* core G of size R_0 x ... x R_{N-1} with N(0,1) entries, each scaled by
  10^(-decay * (r_0 + ... + r_{N-1})) (zero-based core indices; decay = 0
  is the paper's plain Gaussian core), or a superdiagonal core
  G[k,...,k] = sigma_k when ``superdiag`` is given;
* factors U_n (I_n x R_n): the Q factor of the reduced QR of an N(0,1)
  matrix, i.e. orthonormal columns;
* M = G x_0 U_0 ... x_{N-1} U_{N-1};
* X = M + eta * ||M|| / sqrt(I^*) * Nz with Nz of N(0,1) entries (the
  paper's ||Nz|| ~ sqrt(I^*) approximation), so ||X - M|| / ||X|| ~ eta.

Tensors are returned flat, in natural-descending order (first index
fastest, Section 4.1).  This module only builds inputs: it uses library
contractions (numpy / torch) for M and holds none of the decomposition's
arithmetic; both the oracle and the CUDA path read what it produces.
"""
from __future__ import annotations

import numpy as np


def _core_scale(core_dims, decay):
    """10^(-decay * sum of zero-based indices), natural-descending flat."""
    s = np.zeros(int(np.prod(core_dims)), dtype=np.float64)
    lin = np.arange(s.shape[0], dtype=np.int64)
    for d in core_dims:
        s += (lin % int(d)).astype(np.float64)
        lin //= int(d)
    return np.power(10.0, -float(decay) * s)


def tucker_numpy(dims, core_dims, decay=0.0, eta=0.0, seed=0, superdiag=None):
    """Small inputs on the host, numpy PCG64 stream ``default_rng(seed)``.

    Returns (x, parts): x is the flat float64 tensor, parts holds the core,
    the factors and M's norm for tests that need the generating model."""
    dims = tuple(int(d) for d in dims)
    core_dims = tuple(int(r) for r in core_dims)
    rng = np.random.default_rng(seed)
    if superdiag is not None:
        sig = np.asarray(superdiag, dtype=np.float64)
        g = np.zeros(int(np.prod(core_dims)), dtype=np.float64)
        step = sum(int(np.prod(core_dims[:k])) for k in range(len(core_dims)))
        for k, s in enumerate(sig):
            g[k * step] = s
    else:
        g = rng.standard_normal(int(np.prod(core_dims))) * _core_scale(core_dims, decay)
    factors = []
    for I, R in zip(dims, core_dims):
        q, _ = np.linalg.qr(rng.standard_normal((I, R)), mode="reduced")
        factors.append(q)
    # M = G x_0 U_0 ... : natural-descending == Fortran order for numpy.
    m = g.reshape(core_dims, order="F")
    for n, U in enumerate(factors):
        m = np.moveaxis(np.tensordot(U, m, axes=(1, n)), 0, n)
    x = np.asarray(m, dtype=np.float64).reshape(-1, order="F").copy()
    mnorm = float(np.sqrt(np.dot(x, x)))
    if eta:
        x += eta * mnorm / np.sqrt(x.shape[0]) * rng.standard_normal(x.shape[0])
    return x, {"core": g, "core_dims": core_dims, "factors": factors, "m_norm": mnorm}


def tucker_torch(dims, core_dims, decay=0.0, eta=0.0, seed=0, dtype=None,
                 device="cuda", chunk=1 << 27):
    """Large inputs built on the device with ``torch.Generator(device)``
    seeded by ``seed``; same recipe as :func:`tucker_numpy` (but a different
    random stream).  Returns the flat tensor (natural-descending) in
    ``dtype`` (default float32) on ``device``."""
    import torch

    dims = tuple(int(d) for d in dims)
    core_dims = tuple(int(r) for r in core_dims)
    dtype = torch.float32 if dtype is None else dtype
    N = len(dims)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    ncore = int(np.prod(core_dims))
    g = torch.randn(ncore, generator=gen, device=device, dtype=torch.float64)
    g *= torch.from_numpy(_core_scale(core_dims, decay)).to(device)
    factors = []
    for I, R in zip(dims, core_dims):
        a = torch.randn(I, R, generator=gen, device=device, dtype=torch.float64)
        # small QR on the host (numpy LAPACK): keeps the generator free of
        # torch's lazily loaded linear-algebra library
        q, _ = np.linalg.qr(a.cpu().numpy(), mode="reduced")
        factors.append(torch.from_numpy(q).to(device))
    # torch C-order shape (J_{N-1}, ..., J_0) == natural-descending.
    t = g.reshape(tuple(reversed(core_dims)))
    cur = list(core_dims)
    # Expand the modes that grow the least first to bound intermediates.
    order = sorted(range(N), key=lambda n: dims[n] / core_dims[n])
    for n in order:
        A = int(np.prod(cur[n + 1:]))
        B = int(np.prod(cur[:n]))
        last = n == order[-1]
        U = factors[n].to(dtype if last else torch.float64)
        src = t.reshape(A, cur[n], B).to(U.dtype)
        t = torch.matmul(U, src)          # (A, I_n, B)
        del src
        cur[n] = dims[n]
    x = t.reshape(-1)
    if x.dtype != dtype:
        x = x.to(dtype)
    del t
    total = x.numel()
    ss = torch.zeros((), dtype=torch.float64, device=device)
    for s in range(0, total, chunk):
        v = x[s:s + chunk].to(torch.float64)
        ss += torch.dot(v, v)
    mnorm = float(torch.sqrt(ss))
    if eta:
        scale = eta * mnorm / float(np.sqrt(total))
        for s in range(0, total, chunk):
            e = min(s + chunk, total)
            nz = torch.randn(e - s, generator=gen, device=device, dtype=x.dtype)
            x[s:e].add_(nz, alpha=scale)
    return x
