"""Pins of the DD-DLRA oracle by independent restatements (no GPU).

Nothing here calls a helper of oracle/dd_dlra.py; each restatement is written from
the paper and compared with the oracle:

* Brute force on tiny grids: Algorithm 6 carried out on the full distribution f of
  every subdomain (an N_k x n matrix), the projectors of the projector-splitting
  integrator (Section 2: K-step df/dt = P_V F, S-step df/dt = -P_U P_V F, L-step
  df/dt = P_U F) applied literally, the augmented basis of Algorithm 4 taken from the
  eigenvectors of the summed angular Gram matrices of the subdomain and its
  neighbours, the boundary data of Eq. (generate_Kboundary) formed as a ghost row of
  f (inflow directions from the neighbour, outflow from the own projected face), the
  upwind rule of Appendix A as a loop over the eigen-directions of C, each a scalar
  field advected with speed lambda_j, and the truncation of Algorithm 5 as the
  weighted SVD of f itself.
* Classic DLRA: a one-domain projector-splitting integrator (Section 2, Algorithms
  1-3) in factored form with explicit difference matrices and Householder QR; the
  oracle on a 1x1 tiling must reproduce it (Algorithm 4 then degenerates to a
  rotation of V).
* Collision at full rank: the K-step is the S_N collision sub-step, and the S- and
  L-steps obey a closed-form identity (Euler) or their dense restatement (RK4).
* The tolerance rule of Algorithm 4 on a constructed spectrum.
* Planted mistakes: each plausible error, planted in a copy of an oracle method,
  fails a named pin.
"""
import inspect
import math

import numpy as np
import pytest

from oracle import dd_dlra
from paper_2602_14854_gb300 import inputs


# ---------------------------------------------------------------------------------
# shared, oracle-independent helpers
# ---------------------------------------------------------------------------------
def rk(y, rhs, dt, method):
    """Explicit Euler or classic RK4 (Section 4 introduction)."""
    if method == "euler":
        return y + dt * rhs(y)
    a = rhs(y)
    b = rhs(y + 0.5 * dt * a)
    c = rhs(y + 0.5 * dt * b)
    d = rhs(y + dt * c)
    return y + dt * (a + 2.0 * b + 2.0 * c + d) / 6.0


def tail_count(sig, tol):
    """Smallest r with (sum_{j >= r} sigma_j^2)^1/2 <= tol (sigma descending)."""
    for r in range(len(sig) + 1):
        if math.sqrt(float(np.sum(np.asarray(sig[r:]) ** 2))) <= tol:
            return r
    return len(sig)


class Tiling:
    """Subdomains of a block tiling; cells x-fastest inside a subdomain."""

    def __init__(self, wl):
        self.wl = wl
        self.TX, self.TY = len(wl.xcuts) - 1, len(wl.ycuts) - 1
        self.subs = []
        for J in range(self.TY):
            for I in range(self.TX):
                x0, x1, y0, y1 = wl.xcuts[I], wl.xcuts[I + 1], wl.ycuts[J], wl.ycuts[J + 1]
                ii, jj = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1))
                self.subs.append(dict(I=I, J=J, nx=x1 - x0, ny=y1 - y0,
                                      cells=(jj * wl.nx + ii).reshape(-1)))

    def neighbours(self, k, axis):
        s = self.subs[k]
        if axis == "x":
            return (k - 1 if s["I"] > 0 else None, k + 1 if s["I"] < self.TX - 1 else None)
        return (k - self.TX if s["J"] > 0 else None, k + self.TX if s["J"] < self.TY - 1 else None)

    def lines(self, k, axis):
        """Cell indices (local) as an array [line, position] along the axis."""
        s = self.subs[k]
        grid = np.arange(s["nx"] * s["ny"]).reshape(s["ny"], s["nx"])
        return grid if axis == "x" else grid.T

    def diff_matrices(self, k, axis, h):
        """Backward and forward difference matrices with ghost injection:
        D- a + E- g = (a_c - a_{c-1}) / h with a_{-1} = g(line),
        D+ a + E+ g = (a_{c+1} - a_c) / h with a_len = g(line)."""
        L = self.lines(k, axis)
        nl, ln = L.shape
        N = nl * ln
        Dm, Dp = np.zeros((N, N)), np.zeros((N, N))
        Em, Ep = np.zeros((N, nl)), np.zeros((N, nl))
        for l in range(nl):
            for p in range(ln):
                c = L[l, p]
                Dm[c, c] += 1.0 / h
                Dp[c, c] -= 1.0 / h
                if p > 0:
                    Dm[c, L[l, p - 1]] -= 1.0 / h
                else:
                    Em[c, l] = -1.0 / h
                if p < ln - 1:
                    Dp[c, L[l, p + 1]] += 1.0 / h
                else:
                    Ep[c, l] = 1.0 / h
        return Dm, Dp, Em, Ep


def random_factor_state(wl, rank, seed):
    """Seeded random rank-`rank` factors per subdomain (U weighted-orthonormal in
    hx hy sum, V in sum w), as in the oracle's own tests."""
    t = Tiling(wl)
    return [inputs.random_factors(seed + k, len(s["cells"]), wl.n, rank, wl.hx, wl.hy, wl.w)
            for k, s in enumerate(t.subs)]


# ---------------------------------------------------------------------------------
# brute force: Algorithm 6 on the full f of every subdomain
# ---------------------------------------------------------------------------------
class BruteForce:
    def __init__(self, wl, factors, tau=1e-5):
        self.wl, self.tau = wl, tau
        self.t = Tiling(wl)
        self.hxy = wl.hx * wl.hy
        self.w = np.asarray(wl.w, dtype=np.float64)
        self.floor = wl.rank if wl.rank_mode == "fixed" else wl.r_min
        self.f = [U @ S @ V.T for (U, S, V) in factors]
        self.rank = [S.shape[0] for (_, S, _) in factors]
        self.ssum = float(np.sum(self.w))

    # weighted SVD of f: sqrt(hx hy) f W^1/2 = A diag(s) B^T
    def wsvd(self, f):
        M = math.sqrt(self.hxy) * f * np.sqrt(self.w)[None, :]
        A, s, Bt = np.linalg.svd(M, full_matrices=False)
        return A, s, Bt

    def significant(self, s):
        return int(np.sum(s > self.tau * s[0])) if s.size and s[0] > 0 else 0

    def col_basis(self, f, r):
        """Weighted-orthonormal basis of the r-dimensional column span of f."""
        A, s, _ = self.wsvd(f)
        assert self.significant(s) == r, "the brute force covers no basis completion"
        return A[:, :r] / math.sqrt(self.hxy)

    def PU(self, U, g):
        return U @ (self.hxy * (U.T @ g))

    def PV(self, V, g):
        return (g * self.w[None, :]) @ V @ V.T

    def face(self, f, k, axis, side):
        L = self.t.lines(k, axis)
        return f[L[:, 0 if side == 0 else -1], :]

    def inflow(self, k, axis, side):
        """Physical inflow f = g(s) h(Omega) on a boundary side as a virtual neighbour:
        (its data extended across a subdomain-sized block, every cell taking the value
        of its line; the ghost row g(line) m_in h), or None."""
        key = axis + ("_lo" if side == 0 else "_hi")
        if key not in self.wl.inflow:
            return None
        g, hq = self.wl.inflow[key]
        s = self.t.subs[k]
        om = self.wl.omega_x if axis == "x" else self.wl.omega_y
        m_in = (om >= 0) if side == 0 else (om < 0)
        lo = self.wl.ycuts[s["J"]] if axis == "x" else self.wl.xcuts[s["I"]]
        L = self.t.lines(k, axis)
        g_face = np.asarray(g, dtype=np.float64)[lo:lo + L.shape[0]]
        prof = np.asarray(hq, dtype=np.float64) * m_in
        ext = np.zeros((L.size, self.wl.n))
        for l in range(L.shape[0]):
            ext[L[l]] = g_face[l] * prof
        return ext, np.outer(g_face, prof)

    def advection_phase(self, axis):
        wl, t = self.wl, self.t
        om = wl.omega_x if axis == "x" else wl.omega_y
        h = wl.hx if axis == "x" else wl.hy
        snap, snap_rank = self.f, self.rank
        new_f, new_rank = [], []
        for k, s in enumerate(t.subs):
            nbs = t.neighbours(k, axis)
            # Algorithm 4: eigenvectors of sum_i (W^1/2 <f_i, f_i>_x W^1/2) over the
            # subdomain and its neighbours = left singular vectors of L0 (weighted)
            G = np.zeros((wl.n, wl.n))
            blocks = [snap[i] for i in (k,) + tuple(nb for nb in nbs if nb is not None)]
            blocks += [self.inflow(k, axis, side)[0] for side, nb in enumerate(nbs)
                       if nb is None and self.inflow(k, axis, side) is not None]
            for fb in blocks:
                M = math.sqrt(self.hxy) * fb * np.sqrt(self.w)[None, :]
                G += M.T @ M
            lam, E = np.linalg.eigh(G)
            lam, E = lam[::-1], E[:, ::-1]
            sig = np.sqrt(np.maximum(lam, 0.0))
            p = self.significant(sig)
            r_tail = tail_count(sig, wl.tol) if wl.rank_mode == "tol" else p
            cap = min(wl.r_aug_max, wl.n, len(s["cells"]))
            r_t = min(max(min(r_tail, p), snap_rank[k], self.floor), cap)
            assert r_t <= p, "the brute force covers no basis completion"
            Vh = E[:, :r_t] / np.sqrt(self.w)[:, None]
            f0 = self.PV(Vh, snap[k])
            # Eq. (generate_Kboundary): ghost row of f, inflow directions from the
            # neighbour's adjacent face, outflow directions from the own projected face
            m_in = [(om >= 0).astype(float), (om < 0).astype(float)]
            ghosts = []
            for side, nb in enumerate(nbs):
                g = self.face(f0, k, axis, side) * m_in[1 - side][None, :]
                if nb is not None:
                    g = g + self.face(snap[nb], nb, axis, 1 - side) * m_in[side][None, :]
                elif self.inflow(k, axis, side) is not None:
                    g = g + self.inflow(k, axis, side)[1]
                ghosts.append(self.PV(Vh, g))                     # K^b V_hat^T
            Dm, Dp, Em, Ep = t.diff_matrices(k, axis, h)
            # Appendix A: every eigen-direction v_j of C is a scalar field <f, v_j>
            # advected with speed lambda_j, upwinded by its sign
            C = Vh.T @ ((self.w * om)[:, None] * Vh)
            lc, Pc = np.linalg.eigh(C)

            def FA(f):
                out = np.zeros_like(f)
                for j in range(r_t):
                    v = Vh @ Pc[:, j]
                    a = f @ (self.w * v)
                    if lc[j] > 0:
                        d = Dm @ a + Em @ (ghosts[0] @ (self.w * v))
                    elif lc[j] < 0:
                        d = Dp @ a + Ep @ (ghosts[1] @ (self.w * v))
                    else:
                        continue
                    out += -wl.c_adv * lc[j] * np.outer(d, v)
                return out

            def Fdir(f):                                           # per-direction upwind
                out = np.zeros_like(f)
                for q in range(wl.n):
                    if om[q] > 0:
                        out[:, q] = -wl.c_adv * om[q] * (Dm @ f[:, q] + Em @ ghosts[0][:, q])
                    elif om[q] < 0:
                        out[:, q] = -wl.c_adv * om[q] * (Dp @ f[:, q] + Ep @ ghosts[1][:, q])
                return out

            f1 = rk(f0, lambda f: self.PV(Vh, FA(f)), wl.dt, wl.integrator)        # K-step
            U1 = self.col_basis(f1, r_t)
            f2 = rk(f1, lambda f: -self.PU(U1, self.PV(Vh, FA(f))), wl.dt, wl.integrator)
            f3 = rk(f2, lambda f: self.PU(U1, Fdir(f)), wl.dt, wl.integrator)        # L-step
            # Algorithm 5 on f itself
            A, sg, Bt = self.wsvd(f3)
            p3 = self.significant(sg)
            if wl.rank_mode == "tol":
                r1 = min(max(tail_count(sg, wl.tol), wl.r_min), wl.r_max)
            else:
                r1 = wl.rank
            r1 = min(r1, p3)
            new_f.append(((A[:, :r1] * sg[:r1]) @ Bt[:r1]) / math.sqrt(self.hxy)
                         / np.sqrt(self.w)[None, :])
            new_rank.append(r1)
        self.f, self.rank = new_f, new_rank

    def collision_phase(self):
        wl = self.wl
        new_f = []
        for k, s in enumerate(self.t.subs):
            r = self.rank[k]
            assert min(max(r, self.floor), wl.n, len(s["cells"])) == r, "no completion here"
            _, sg, Bt = self.wsvd(self.f[k])
            V = Bt[:r].T / np.sqrt(self.w)[:, None]
            c = s["cells"]
            ss, st, Q = wl.sigma_s[c], wl.sigma_s[c] + wl.sigma_a[c], wl.source[c]

            def F(f):                                              # Eq. (rt), collision part
                rho = f @ self.w
                return (ss * rho / self.ssum)[:, None] - st[:, None] * f + Q[:, None]

            f1 = rk(self.f[k], lambda f: self.PV(V, F(f)), wl.dt, wl.integrator)
            U1 = self.col_basis(f1, r)
            f2 = rk(f1, lambda f: -self.PU(U1, self.PV(V, F(f))), wl.dt, wl.integrator)
            new_f.append(rk(f2, lambda f: self.PU(U1, F(f)), wl.dt, wl.integrator))
        self.f = new_f

    def step(self):
        self.advection_phase("x")
        self.advection_phase("y")
        self.collision_phase()

    def full_f(self):
        out = np.zeros((self.wl.ncells, self.wl.n))
        for f, s in zip(self.f, self.t.subs):
            out[s["cells"]] = f
        return out.reshape(self.wl.ny, self.wl.nx, self.wl.n)


def tiny_problem(integrator, ragged, tol_mode=False, seed=5):
    cuts = dict(xcuts=[0, 3, 5, 8], ycuts=[0, 5, 8]) if ragged else {}
    wl = inputs.random_small_problem(seed, nx=8, ny=8, tiles_x=2, tiles_y=2, n_mu=2, n_phi=4,
                                     rank=2, r_aug_max=6, integrator=integrator, **cuts)
    if tol_mode:
        wl = wl.with_(rank_mode="tol", tol=0.08, r_min=2, r_max=4)   # ranks 2..4, r_t 4..6
    return wl


def pin_brute_force(cls, wl, nsteps=3, seed=50):
    """Max |f_oracle - f_brute| / max |f| after nsteps full steps, and whether the ranks
    agree after every step."""
    facs = random_factor_state(wl, 2, seed)
    o = cls(wl)
    o.set_state(facs)
    b = BruteForce(wl, facs)
    ranks_ok = True
    for _ in range(nsteps):
        o.step()
        b.step()
        ranks_ok &= o.ranks() == b.rank
    fo, fb = o.full_f(), b.full_f()
    return float(np.max(np.abs(fo - fb)) / np.max(np.abs(fb))), ranks_ok


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
@pytest.mark.parametrize("ragged", [False, True])
def test_brute_force_tiny_grid(integrator, ragged):
    """The oracle's Algorithm 6 equals the dense restatement to roundoff (8 x 8
    cells, 8 directions, rank 2, r_t <= 6; a 2 x 2 tiling and a ragged 3 x 2 one)."""
    err, ranks_ok = pin_brute_force(dd_dlra.DDDLRA, tiny_problem(integrator, ragged))
    assert ranks_ok
    assert err < 1e-13, err


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_brute_force_tolerance_mode(integrator):
    """Brute force with the tolerance rules of Algorithms 4 and 5 (tol 0.08, ranks 2..4)."""
    wl = tiny_problem(integrator, True, tol_mode=True)
    err, ranks_ok = pin_brute_force(dd_dlra.DDDLRA, wl)
    assert ranks_ok
    assert err < 1e-13, err


def test_brute_force_with_inflow_tolerance_mode():
    """Brute force with inflow in tolerance mode, where the augmentation column's norm
    |g|_x = (hx hy len sum g^2)^1/2 (R22) enters the rank decisions."""
    err, ranks_ok = pin_brute_force(dd_dlra.DDDLRA, inflow_tol_problem())
    assert ranks_ok
    assert err < 1e-13, err


def test_brute_force_with_inflow():
    """Brute force with physical inflow on all four sides (random g, h; R22): the inflow acts
    as a neighbour in the ghost rows and in Algorithm 4."""
    wl = tiny_problem("rk4", False)
    rng = np.random.default_rng(12)
    wl = wl.with_(inflow={key: (rng.uniform(0.5, 1.5, 8), rng.uniform(0.0, 1.0, wl.n))
                          for key in ("x_lo", "x_hi", "y_lo", "y_hi")})
    err, ranks_ok = pin_brute_force(dd_dlra.DDDLRA, wl)
    assert ranks_ok
    assert err < 1e-13, err


# ---------------------------------------------------------------------------------
# classic (one-domain) DLRA, factored form
# ---------------------------------------------------------------------------------
class ClassicDLRA:
    """Projector-splitting integrator on the whole domain (Section 2; Algorithms 1-3
    without neighbours), fixed rank, zero inflow, Appendix A's C+-, QR by Householder."""

    def __init__(self, wl, U, S, V):
        self.wl = wl
        self.U, self.S, self.V = U.copy(), S.copy(), V.copy()
        self.t = Tiling(wl)
        assert len(self.t.subs) == 1
        self.hxy = wl.hx * wl.hy
        self.w = np.asarray(wl.w, dtype=np.float64)
        self.mats = {ax: self.t.diff_matrices(0, ax, wl.hx if ax == "x" else wl.hy)
                     for ax in ("x", "y")}

    def wqr_space(self, K):
        Q, R = np.linalg.qr(math.sqrt(self.hxy) * K)
        return Q / math.sqrt(self.hxy), R

    def wqr_angle(self, L):
        Q, R = np.linalg.qr(np.sqrt(self.w)[:, None] * L)
        return Q / np.sqrt(self.w)[:, None], R

    def advection(self, axis):
        wl = self.wl
        om = wl.omega_x if axis == "x" else wl.omega_y
        Dm, Dp, Em, Ep = self.mats[axis]
        L = self.t.lines(0, axis)
        U, S, V = self.U, self.S, self.V
        Wv = self.w[:, None] * V
        C = V.T @ (om[:, None] * Wv)
        lam, P = np.linalg.eigh(C)
        Cp = P @ np.diag(np.maximum(lam, 0.0)) @ P.T
        Cm = P @ np.diag(np.minimum(lam, 0.0)) @ P.T
        K = U @ S
        # boundary data: zero inflow, own outflow values on the boundary faces
        Kb_lo = K[L[:, 0]] @ (V.T @ ((om < 0)[:, None] * Wv))
        Kb_hi = K[L[:, -1]] @ (V.T @ ((om >= 0)[:, None] * Wv))
        RK = lambda K_: -wl.c_adv * ((Dm @ K_ + Em @ Kb_lo) @ Cp + (Dp @ K_ + Ep @ Kb_hi) @ Cm)
        K1 = rk(K, RK, wl.dt, wl.integrator)
        U1, S1 = self.wqr_space(K1)
        S2 = rk(S1, lambda S_: -self.hxy * U1.T @ RK(U1 @ S_), wl.dt, wl.integrator)
        # L-step in Galerkin form: per direction an r x r linear ODE
        Tm, Tp = self.hxy * U1.T @ Dm @ U1, self.hxy * U1.T @ Dp @ U1
        Gm, Gp = self.hxy * U1.T @ Em, self.hxy * U1.T @ Ep
        fb_lo, fb_hi = Kb_lo @ V.T, Kb_hi @ V.T          # (lines, n) ghost values of f
        pos, neg = np.where(om > 0, om, 0.0), np.where(om < 0, om, 0.0)

        def Lrhs(L_):
            up = L_ @ Tm.T + fb_lo.T @ Gm.T
            dn = L_ @ Tp.T + fb_hi.T @ Gp.T
            return -wl.c_adv * (pos[:, None] * up + neg[:, None] * dn)

        L1 = rk(V @ S2.T, Lrhs, wl.dt, wl.integrator)
        V1, R = self.wqr_angle(L1)
        self.U, self.S, self.V = U1, R.T, V1

    def collision(self):
        wl = self.wl
        ss, st, Q = wl.sigma_s, wl.sigma_s + wl.sigma_a, wl.source
        ssum = float(np.sum(self.w))
        U, S, V = self.U, self.S, self.V
        a = V.T @ self.w

        def F(f):
            return (ss * (f @ self.w) / ssum)[:, None] - st[:, None] * f + Q[:, None]

        Kr = lambda K_: (ss / ssum * (K_ @ a))[:, None] * a[None, :] - st[:, None] * K_ \
            + Q[:, None] * a[None, :]
        K1 = rk(U @ S, Kr, wl.dt, wl.integrator)
        U1, S1 = self.wqr_space(K1)
        S2 = rk(S1, lambda S_: -self.hxy * U1.T @ F(U1 @ S_ @ V.T) @ (self.w[:, None] * V),
                wl.dt, wl.integrator)
        L1 = rk(V @ S2.T, lambda L_: (self.hxy * U1.T @ F(U1 @ L_.T)).T, wl.dt, wl.integrator)
        V1, R = self.wqr_angle(L1)
        self.U, self.S, self.V = U1, R.T, V1

    def step(self):
        self.advection("x")
        self.advection("y")
        self.collision()

    def full_f(self):
        f = np.zeros((self.wl.ncells, self.wl.n))
        f[self.t.subs[0]["cells"]] = self.U @ self.S @ self.V.T
        return f.reshape(self.wl.ny, self.wl.nx, self.wl.n)


def pin_one_by_one(cls, integrator, nsteps=3):
    wl = inputs.random_small_problem(17, nx=10, ny=8, tiles_x=1, tiles_y=1, n_mu=2, n_phi=8,
                                     rank=3, r_aug_max=6, integrator=integrator)
    facs = random_factor_state(wl, 3, 70)
    o = cls(wl)
    o.set_state(facs)
    c = ClassicDLRA(wl, *facs[0])
    for _ in range(nsteps):
        o.step()
        c.step()
    fo, fc = o.full_f(), c.full_f()
    return float(np.max(np.abs(fo - fc)) / np.max(np.abs(fc))), o.ranks() == [3]


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_one_by_one_tiling_is_classic_dlra(integrator):
    """A 1 x 1 tiling reduces Algorithm 6 to the classic projector-splitting DLRA
    (Algorithm 4 only rotates V; the fixed rank keeps r_t = r; the truncation only
    rotates the factors)."""
    err, ranks_ok = pin_one_by_one(dd_dlra.DDDLRA, integrator)
    assert ranks_ok
    assert err < 1e-12, err


# ---------------------------------------------------------------------------------
# collision (Algorithm 3) at full rank
# ---------------------------------------------------------------------------------
def collision_F(wl):
    """sigma_s/|S| rho - sigma_t f + Q (the collision part of Eq. (rt)); and its linear part."""
    w = np.asarray(wl.w, dtype=np.float64)
    ssum = float(np.sum(w))

    def make(cells, with_source):
        ss, st = wl.sigma_s[cells], wl.sigma_s[cells] + wl.sigma_a[cells]
        Q = wl.source[cells] if with_source else np.zeros(len(cells))
        return lambda f: (ss * (f @ w) / ssum)[:, None] - st[:, None] * f + Q[:, None]

    return make


def pin_collision_full_rank(cls, integrator):
    """Max over subdomains of |f3 - expect| / max |f|, f3 the oracle's Algorithm 3 at full
    rank from anisotropic random factors with heterogeneous sigma and Q."""
    wl = inputs.random_small_problem(23, nx=6, ny=6, tiles_x=2, tiles_y=1, n_mu=0, n_phi=8,
                                     rank=8, r_aug_max=8, integrator=integrator)
    o = cls(wl, tau=1e-12)
    facs = random_factor_state(wl, wl.n, 90)
    o.set_state(facs)
    make = collision_F(wl)
    hxy = wl.hx * wl.hy
    worst = 0.0
    for k, (U, S, V) in enumerate(facs):
        cells = dd_dlra.cell_index(wl, o.subs[k])
        F, A = make(cells, True), make(cells, False)
        f0 = U @ S @ V.T
        f1 = rk(f0, F, wl.dt, integrator)                 # the S_N collision sub-step
        U1, S3, V1, _ = o.psi_collision(k, U, S, V)
        f3 = U1 @ S3 @ V1.T
        Uq = np.linalg.qr(math.sqrt(hxy) * f1)[0] / math.sqrt(hxy)   # span of f1's columns
        P = lambda g: Uq @ (hxy * (Uq.T @ g))
        if integrator == "euler":
            expect = f1 - wl.dt ** 2 * P(A(P(F(f1))))
        else:
            f2 = rk(f1, lambda g: -P(F(g)), wl.dt, integrator)
            expect = rk(f2, lambda g: P(F(g)), wl.dt, integrator)
        worst = max(worst, float(np.max(np.abs(f3 - expect)) / np.max(np.abs(f1))))
    return worst


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_collision_full_rank(integrator):
    """At full rank (V square) the collision K-step is the S_N collision sub-step, and
    with explicit Euler the S- and L-steps give f3 = f1 - dt^2 P_U A P_U F(f1) (A the
    linear part of the collision operator); with RK4 they are the backward and forward
    RK4 flows of P_U F on span(U1) x R^n (Eqs. (coll_evolK), (coll_evolS), (coll_evolL))."""
    assert pin_collision_full_rank(dd_dlra.DDDLRA, integrator) < 1e-12


# ---------------------------------------------------------------------------------
# Algorithm 4 in tolerance mode
# ---------------------------------------------------------------------------------
def constructed_augmentation(tol, r_min=1, r_aug_max=9):
    """Three subdomains in a row; the middle one sees both neighbours.  The angular
    bases of the three are mutually orthogonal blocks of one orthonormal basis, so the
    singular values of L0 are the union of the three cores' singular values."""
    n = 16
    wl = inputs.random_small_problem(31, nx=12, ny=4, tiles_x=3, tiles_y=1, n_mu=2, n_phi=8,
                                     rank=3, r_aug_max=r_aug_max)
    wl = wl.with_(rank_mode="tol", tol=tol, r_min=r_min, r_max=3)
    assert wl.n == n
    rng = np.random.default_rng(4)
    Qb = np.linalg.qr(rng.standard_normal((n, 9)))[0] / np.sqrt(wl.w)[:, None]
    svals = [[1.0, 0.3, 0.02], [0.5, 0.04, 0.001], [0.2, 0.01, 0.0005]]   # own, lo, hi
    order = [1, 0, 2]                                       # subdomain k -> block
    facs = []
    for k in range(3):
        b = order[k]
        U = np.linalg.qr(rng.standard_normal((16, 3)))[0] / math.sqrt(wl.hx * wl.hy)
        P = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        Qm = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        facs.append((U, P @ np.diag(svals[b]) @ Qm.T, Qb[:, 3 * b:3 * b + 3]))
    o = dd_dlra.DDDLRA(wl)
    o.set_state(facs)
    return o, sorted(sum(svals, []), reverse=True)


@pytest.mark.parametrize("tol,r_min,cap,expect", [
    (0.025, 1, 9, 5),      # tail after 5: |(.02,.01,.001,.0005)| = 0.0224 <= tol < 0.0458
    (0.05, 1, 9, 4),       # tail after 4 = 0.0458
    (0.5, 1, 9, 3),        # tail rule says 2; the own rank 3 is the floor
    (0.0004, 1, 9, 9),     # even the smallest singular value (5e-4) is above tol
    (0.025, 6, 9, 6),      # the rank floor r_min raises it
    (0.0004, 1, 7, 7),     # the cap r_aug_max lowers it
])
def test_augmentation_tolerance_rule(tol, r_min, cap, expect):
    """Algorithm 4 in tolerance mode: r_t is the smallest rank whose discarded tail of
    L0's singular values is <= tol, at least max(r, r_min), at most r_aug_max; the
    augmented basis holds exactly the leading r_t singular directions."""
    o, sig = constructed_augmentation(tol, r_min, cap)
    K0, Vh, info = o.augment(1, "x", o.state)
    assert info["r_t"] == expect
    # the span of V_hat: the leading `expect` left singular directions of W^1/2 L0
    w = o.w
    blocks = [V @ S.T for (_, S, V) in o.state]
    L0 = np.concatenate([blocks[1], blocks[0], blocks[2]], axis=1)
    A = np.linalg.svd(np.sqrt(w)[:, None] * L0, full_matrices=False)[0][:, :expect]
    Q = np.sqrt(w)[:, None] * Vh
    assert np.max(np.abs(Q @ Q.T - A @ A.T)) < 1e-12


# ---------------------------------------------------------------------------------
# planted mistakes: each must fail a named pin
# ---------------------------------------------------------------------------------
MUTANTS = {
    # name: (method, original text, planted text, pins that must fail)
    "s_step_sign": ("psi_advection", "lambda S: -self._ip_x(U1, rk(U1 @ S))",
                    "lambda S: self._ip_x(U1, rk(U1 @ S))", ["brute_force"]),
    "swapped_masks": ("boundary", "in_lo = (om >= 0).astype(np.float64)",
                      "in_lo = (om < 0).astype(np.float64)", ["brute_force"]),
    "untransposed_s3": ("psi_advection", "S3 = self._ip_phi(V1, L1).T",
                        "S3 = self._ip_phi(V1, L1)", ["brute_force", "one_by_one"]),
    "upwind_direction": ("kstep_rhs_adv", "D = np.where(lam[None, :] > 0, Dm,",
                         "D = np.where(lam[None, :] < 0, Dm,", ["brute_force", "one_by_one"]),
    "neighbour_face": ("boundary", "Kn_face = self._face(Kn, self.subs[nb], axis, 1 - side)",
                       "Kn_face = self._face(Kn, self.subs[nb], axis, side)", ["brute_force"]),
    "collision_s_sign": ("psi_collision", "return -((1.0 / ss) * Ms @ Sm @ np.outer(a, a)",
                         "return ((1.0 / ss) * Ms @ Sm @ np.outer(a, a)",
                         ["collision_full_rank", "brute_force"]),
    "sigma_t_to_s": ("psi_collision", "- sig_t[:, None] * K \\",
                     "- sig_s[:, None] * K \\", ["collision_full_rank", "brute_force"]),
    "l_step_ghost": ("psi_advection", "fb_lo = Kb_lo @ Vhat.T",
                     "fb_lo = 0.0 * Kb_lo @ Vhat.T", ["brute_force"]),
    "inflow_norm": ("_inflow_column", "math.sqrt(self.hx * self.hy * ln * float(np.sum(g_face ** 2)))",
                    "math.sqrt(self.hx * self.hy * float(np.sum(g_face ** 2)))",
                    ["brute_force_inflow"]),
    "inflow_mask": ("_inflow_face", "return g_face, np.asarray(hq, dtype=np.float64)",
                    "return g_face, np.asarray(hq, dtype=np.float64)[::-1]",
                    ["brute_force_inflow"]),
}

PINS = {
    "brute_force": lambda cls: pin_brute_force(cls, tiny_problem("rk4", True), nsteps=2)[0] > 1e-8,
    "one_by_one": lambda cls: pin_one_by_one(cls, "rk4", nsteps=2)[0] > 1e-8,
    "collision_full_rank": lambda cls: pin_collision_full_rank(cls, "euler") > 1e-8,
    "brute_force_inflow": lambda cls: pin_brute_force(cls, inflow_tol_problem(), nsteps=2)[0] > 1e-8,
}


def inflow_tol_problem():
    """Inflow on two sides in tolerance mode: the scale of the inflow's augmentation
    column decides ranks here (in fixed mode only its span matters)."""
    return tiny_problem("rk4", False, tol_mode=True).with_(
        tol=0.08, inflow={"x_lo": (np.linspace(0.5, 1.5, 8), np.linspace(0.1, 1.0, 8)),
                          "y_hi": (np.linspace(1.5, 0.5, 8), np.linspace(1.0, 0.2, 8))})


def mutant(method, old, new):
    src = inspect.getsource(getattr(dd_dlra.DDDLRA, method))
    assert src.count(old) == 1, (method, old)
    lines = src.replace(old, new).splitlines()
    indent = len(lines[0]) - len(lines[0].lstrip())
    ns = dict(vars(dd_dlra))
    exec("\n".join(l[indent:] for l in lines), ns)
    return type("Mutant", (dd_dlra.DDDLRA,), {method: ns[method]})


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_its_pins(name):
    method, old, new, pins = MUTANTS[name]
    cls = mutant(method, old, new)
    for pin in pins:
        assert PINS[pin](cls), f"planted mistake {name} passes pin {pin}"


def test_pins_pass_on_the_oracle_itself():
    for pin, fails in PINS.items():
        assert not fails(dd_dlra.DDDLRA), pin
