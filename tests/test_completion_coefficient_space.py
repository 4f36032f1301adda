"""Basis completion by Gram-Schmidt in coefficient space (the form the CUDA path runs for
mutually orthogonal candidate families) equals R11's one-by-one definition in the oracle.

For orthonormal columns Q0 and mutually orthogonal candidates c_j, each accepted column is
q = C a + Q0 b, and the projections of a new candidate on the earlier accepted ones follow
from w_j = Q0^T c_j / |c_j| alone (g_k = b_k^T w_j); its residual norm is
(1 - |w_j|^2 - |g|^2)^1/2.  Restated here from that derivation (not from the kernels) and
compared with oracle.dd_dlra.complete_basis on the spatial cosine family (with Q0 holding
low-frequency cosines, so that candidates are rejected) and on the angular family of a
product quadrature."""
import itertools
import math

import numpy as np

from oracle import dd_dlra
from paper_2602_14854_gb300 import inputs


def coefficient_space_complete(Q0, C, r_out, accept=0.5):
    """Q0: rows x cur0 orthonormal; C: b x rows, mutually orthogonal candidates in order."""
    cur0 = Q0.shape[1]
    W = Q0.T @ C.T                                  # cur0 x b
    nrm2 = np.sum(C * C, axis=1)
    A, B, picked = [], [], []
    for j in range(C.shape[0]):
        if cur0 + len(A) == r_out:
            break
        if nrm2[j] == 0.0:
            continue
        inv = 1.0 / math.sqrt(nrm2[j])
        wt = W[:, j] * inv
        g = np.array([b @ wt for b in B])
        rn2 = 1.0 - wt @ wt - (g @ g if len(g) else 0.0)
        if rn2 < accept * accept:
            continue
        ir = 1.0 / math.sqrt(rn2)
        a = np.zeros(C.shape[0])
        a[j] = inv
        b = -wt.copy()
        for k in range(len(A)):
            a -= g[k] * A[k]
            b -= g[k] * B[k]
        A.append(a * ir)
        B.append(b * ir)
        picked.append(j)
    Qn = C.T @ np.array(A).T + Q0 @ np.array(B).T if A else np.zeros((Q0.shape[0], 0))
    return np.concatenate([Q0, Qn], axis=1), picked


class _Sub:
    def __init__(self, nx, ny):
        self.nxk, self.nyk = nx, ny


def _orthonormal(M):
    q, _ = np.linalg.qr(M)
    return q


def test_spatial_family_with_rejections():
    rng = np.random.default_rng(5)
    nx, ny = 12, 10
    cands = np.array(list(itertools.islice(dd_dlra.spatial_candidates(_Sub(nx, ny)), 60)))
    # Q0: two low-frequency cosines mixed with random data (several early candidates lie
    # mostly in its span and are rejected) plus random columns
    low = cands[[0, 1, 2, 4]].T / np.linalg.norm(cands[[0, 1, 2, 4]], axis=1)
    Q0 = _orthonormal(np.concatenate([low + 0.05 * rng.standard_normal(low.shape),
                                      rng.standard_normal((nx * ny, 3))], axis=1))
    r_out = 20
    ref = dd_dlra.complete_basis(Q0, np.ones(nx * ny), r_out, iter(cands))
    got, picked = coefficient_space_complete(Q0, cands, r_out)
    assert got.shape == ref.shape == (nx * ny, r_out)
    assert len(picked) + Q0.shape[1] == r_out and picked != list(range(len(picked)))  # rejections
    np.testing.assert_allclose(got, ref, atol=1e-13)
    np.testing.assert_allclose(got.T @ got, np.eye(r_out), atol=1e-13)


def test_angular_family_of_a_product_quadrature():
    rng = np.random.default_rng(6)
    wl = inputs.config_c0()                               # 8 mu x 16 phi
    sw = np.sqrt(wl.w)
    cands = np.array(list(itertools.islice(dd_dlra.angular_candidates(wl), 40)))
    Cw = cands * sw[None, :]                              # the weighted (Euclidean) family
    Q0 = _orthonormal(rng.standard_normal((wl.n, 6)))
    r_out = 18
    ref = dd_dlra.complete_basis(Q0, sw, r_out, iter(cands))
    got, _ = coefficient_space_complete(Q0, Cw, r_out)
    np.testing.assert_allclose(got, ref, atol=1e-13)
