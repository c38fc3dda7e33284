"""Sub-meshes cut around one element of a structured mesh, for checking
element quantities of a large workload with the oracle (test helpers).

An element's residual depends on the states of the elements within two face
steps (through the neighbours' LDG gradients), so on the 5^D elements
around it the oracle reproduces it exactly; its diagonal Jacobian block
depends only on the elements one step away (3^D)."""
import itertools

import numpy as np

from oracle.residual import full_residual

H_CS = 1e-30


def submesh(m, center, r):
    """Elements within r index steps of `center` on a structured mesh (no
    wrap: the centre lies at least r elements from the periodic seam), as a
    non-periodic mesh with Dirichlet faces on its outside. Returns the mesh,
    the global element ids and the position of the centre among them."""
    n, D = m["shape"], m["D"]
    rng = [range(center[d] - r, center[d] + r + 1) for d in range(D)]
    ids, tags = [], []
    for t in itertools.product(*[rng[d] for d in reversed(range(D))]):
        t = t[::-1]
        ids.append(sum(t[d] * int(np.prod(n[:d])) for d in range(D)))
        tag = -np.ones(2 * D, dtype=np.int32)
        for d in range(D):
            if t[d] == center[d] - r:
                tag[2 * d] = 0
            if t[d] == center[d] + r:
                tag[2 * d + 1] = 0
        tags.append(tag)
    ids = np.array(ids)
    k = int(np.nonzero(ids == sum(center[d] * int(np.prod(n[:d])) for d in range(D)))[0][0])
    sub = {"D": D, "p": m["p"], "s": m["s"], "nodes": m["nodes"][ids], "vertices": m["vertices"][ids],
           "btag": np.array(tags)}
    return sub, ids, k


def oracle_eq(eq):
    return dict(eq, bc={0: "dirichlet"})


def diag_block(disc, U, k, batch=48):
    """Dense d R_k / d U_k of the element at position k (complex step per
    column), rows and columns ordered (c, node)."""
    nc, npe = U.shape[1], U.shape[2]
    ncol = nc * npe
    blk = np.zeros((ncol, ncol))
    for c0 in range(0, ncol, batch):
        cols = range(c0, min(ncol, c0 + batch))
        X = np.repeat(U[None].astype(np.complex128), len(cols), axis=0)
        for j, col in enumerate(cols):
            X[j, k, col // npe, col % npe] += 1j * H_CS
        Y = np.imag(full_residual(disc, X, U)) / H_CS
        for j, col in enumerate(cols):
            blk[:, col] = Y[j, k].reshape(ncol)
    return blk
