"""RBF-FD sub-domain solver (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY: the plain reference that the library's RBF-FD
kernels are checked against.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It imports
nothing from the CUDA library's package.

Sec. 3.2 of arXiv:1603.09311: once the interface values are known, each
sub-domain is solved on its own nodes by radial-basis-function finite
differences.  At node x_0 with stencil x_1 .. x_n (the node itself and its
n - 1 nearest neighbours, n = 9), the weights w of an operator L solve
    A w = b,  A_ij = phi(|x_i - x_j|),  b_j = L phi(|x - x_j|) at x = x_0,
with the multiquadric phi(r) = sqrt(1 + (eps r)^2).  The operator here is
the Laplacian (the sum of the paper's separate d^2/dx^2 and d^2/dz^2
matrices: the weights are linear in b), for which
    Lap phi(r) = (2 eps^2 + eps^4 r^2) / phi(r)^3   in two dimensions.
The sub-domain equation is Lap u = i kappa u (TE; a TM strip of diffusion D
is the same with kappa / D), with Dirichlet values at the boundary nodes:
for every unknown node i,
    sum_{j in stencil(i)} w_ij u_j - i kappa_i u_i = 0,
the boundary nodes' terms moved to the right-hand side.

Readings where the paper is silent: ties in the nearest-neighbour order go
to the lower node index (distance squared dx*dx + dz*dz compared exactly);
boundary nodes get no equation and keep their values.
"""
from __future__ import annotations

import numpy as np


def mq(r, eps):
    return np.sqrt(1.0 + (eps * r) ** 2)


def mq_lap(r, eps):
    """Laplacian of phi(|x - x_j|) in two dimensions, as a function of r."""
    p = mq(r, eps)
    return (2.0 * eps ** 2 + eps ** 4 * r ** 2) / p ** 3


def stencils(nodes, ns: int) -> np.ndarray:
    """[n][ns] indices: each node's ns nearest nodes (itself first), ordered
    by squared distance, ties by index."""
    p = np.asarray(nodes, dtype=np.float64)
    n = len(p)
    out = np.zeros((n, ns), dtype=np.int64)
    idx = np.arange(n)
    for i in range(n):
        dx = p[:, 0] - p[i, 0]
        dz = p[:, 1] - p[i, 1]
        d2 = dx * dx + dz * dz
        order = np.lexsort((idx, d2))
        out[i] = order[:ns]
    return out


def weights(nodes, ns: int, eps: float):
    """(stencil [n][ns], Laplacian weights [n][ns])."""
    p = np.asarray(nodes, dtype=np.float64)
    st = stencils(p, ns)
    w = np.zeros(st.shape)
    for i in range(len(p)):
        q = p[st[i]]
        r = np.hypot(q[:, None, 0] - q[None, :, 0], q[:, None, 1] - q[None, :, 1])
        A = mq(r, eps)
        b = mq_lap(np.hypot(q[:, 0] - p[i, 0], q[:, 1] - p[i, 1]), eps)
        w[i] = np.linalg.solve(A, b)
    return st, w


def solve(nodes, dirichlet, values, kappa, ns: int, eps: float):
    """u [n] complex: the RBF-FD solution of Lap u = i kappa u with u = values
    at the Dirichlet nodes (a direct sparse solve)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.linalg import spsolve

    p = np.asarray(nodes, dtype=np.float64)
    n = len(p)
    bnd = np.asarray(dirichlet, dtype=bool)
    vals = np.asarray(values, dtype=np.complex128)
    kap = np.asarray(kappa, dtype=np.float64)
    st, w = weights(p, ns, eps)
    unk = np.flatnonzero(~bnd)
    pos = -np.ones(n, dtype=np.int64)
    pos[unk] = np.arange(len(unk))
    rows, cols, data = [], [], []
    rhs = np.zeros(len(unk), dtype=np.complex128)
    for r, i in enumerate(unk):
        for j, wij in zip(st[i], w[i]):
            if bnd[j]:
                rhs[r] -= wij * vals[j]
            else:
                rows.append(r)
                cols.append(pos[j])
                data.append(wij + (-1j * kap[i] if j == i else 0.0))
    K = csr_matrix((np.asarray(data, dtype=np.complex128), (rows, cols)), shape=(len(unk), len(unk)))
    u = vals.copy()
    if len(unk):
        u[unk] = spsolve(K.tocsc(), rhs)
    return u
