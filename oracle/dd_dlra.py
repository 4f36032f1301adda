"""Domain-decomposition dynamical low-rank (DD-DLRA) oracle — TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatement of Algorithm 6 of arXiv 2602.14854 ("Domain
decomposition dynamical low-rank for multi-dimensional radiative transfer
equations"), following the paper's order and notation:

  per time step, on every subdomain
    1. augmentation with the x-neighbours' bases (Algorithm 4),
    2. projector-splitting integrator for x-advection (Algorithm 1) with the
       inflow/outflow boundary data K^b of Eq. (generate_Kboundary) and the
       upwind rule of Appendix A for the K-step,
    3. truncation (Algorithm 5),
    4.-6. the same in y (Algorithm 2, Eq. (generate_Kboundary_yadvection)),
    7. projector-splitting integrator for absorption, scattering and source
       (Algorithm 3, Eqs. (coll_evolK), (coll_evolS), (coll_evolL)).

Factors are kept in the paper's form f = U S V^T with U orthonormal in
<u,v>_{x,y} = hx*hy*sum_c u_c v_c and V orthonormal in <a,b>_phi = sum_q w_q a_q b_q
(Section 2, orthonormality conditions; Section 3.4 matrix form).  Library
primitives used as single steps: numpy SVD, symmetric eigendecomposition and
matrix products.  No blocking, fusion or reordering beyond the paper's steps.

Optional, not part of the paper's scheme: the conserved-moment correction (R18 below).
Optional, the second-order splitting Section 3 points to: Strang splitting of the step
(R20 below).  Optional, not the paper's Appendix A: C+/C- of the advection K-step from
the direction split instead of the eigen-split (R21 below).  Physical inflow data
(R22 below).

Readings where the paper is silent or ambiguous:
  R1  general quadrature: scattering is sigma_s/|S| * sum_q w_q f_q, |S| = sum_q w_q.
  R2  inflow masks are the paper's inclusive ones: at the low side of an axis a
      direction is inflow when its velocity component is >= 0 (Section 3.1,
      "phi <= pi/2 or phi >= 3 pi/2"); at the high side when it is < 0.
  R3  explicit Euler (default) or RK4 for every sub-step ODE; the S-step is the
      minus-sign ODE of Eq. (Sstep_general) integrated forward with the same scheme.
  R4  S-step of an advection = the K-step operator of Appendix A projected on U
      (consistent with the K-step); L-step = per-direction upwind of f = U L^T
      with ghost value f^b = K^b V^T (V the basis the K-step used).
  R5  "evaluating the low-rank representation at x_L" = cell-centred ghost: the
      neighbour term uses the neighbour's cells adjacent to the interface, the own
      outflow term the own first/last cells.
  R6  boundary data frozen over a sub-step: computed once after augmentation and
      used for every stage of the K-, S- and L-steps (Section 4.2 remark).
  R7  all subdomains read neighbour data from one snapshot: start of step for
      the x-phase, the post-x state for the y-phase.
  R8  Appendix A's C for x-advection uses cos(phi) (the printed sin is the
      y-case); Eq. (generate_Kboundary_yadvection)'s V_j^B inside the sum is V_l^B.
  R9  Algorithm 4's random U_rand never reaches the result (the K-step starts
      from K = U_hat S_hat whose extra rows are zero), so K^0 = U^0 S^0 <V^0, V_hat>.
  R10 rank rules.  tau = relative numerical-rank threshold (default 1e-5): a
      singular value sigma_j <= tau*sigma_1 is treated as zero.  (Keeping
      directions with smaller singular values makes the projector-splitting step
      ill-conditioned: a 1e-15 perturbation of the start data then changes the
      scalar flux by ~1e-7 within two steps.)  Augmentation: r_t = minimal
      number whose tail is <= tol (tolerance mode) or all significant ones (fixed
      mode), never more than the significant count, at least max(r, r_floor),
      at most r_aug_max.  Truncation: minimal tail <= tol clamped to [r_min, r_max]
      (tolerance mode) or r (fixed mode), never more than the significant count.
  R11 deterministic basis completion: whenever an orthonormal basis needs more
      columns than the significant span provides (rank-deficient K or L, an
      augmentation floor above the significant rank, a collision step started
      below the rank floor), the missing columns are taken in order from a fixed
      exactly-orthogonal candidate family, each Gram-Schmidt'd twice against the
      columns so far and accepted when its residual norm is >= 1/2:
        space: products of DCT-II cosines cos(pi a (i+1/2)/nx_k) cos(pi b (j+1/2)/ny_k),
               ordered by a+b, then a descending;
        angle: even Legendre P_2l(mu) (GL-orthogonal) times cos(m phi) / sin(m phi),
               ordered by m + 2l, then m descending, cos before sin.
  R12 the isotropic initial state is stored at rank 1: U = g/|g|, V = 1/sqrt(|S|),
      S = |g| sqrt(|S|) (zero rank where g vanishes on a subdomain).
  R13 the collision step (Algorithm 3) starts from the truncated state padded to
      the rank floor by angular completion (zero rows/columns of S), so a source
      can enter a subdomain whose stored rank is below the floor.

Pins: tests/test_oracle_dd_dlra.py (full-rank identities, closed forms,
invariances) and tests/test_oracle_pins.py (a dense brute-force restatement of
Algorithm 6 on tiny grids, with and without physical inflow, fixed and tolerance
ranks; an independently written one-domain classic DLRA that a 1x1 tiling must
reproduce; the collision step at full rank; the tolerance rule of Algorithm 4 on a
constructed spectrum; planted mistakes that each fail a named pin).
  R18 conserved-moment correction (off unless the workload asks for it): the
      K-steps move the scalar flux rho = sum_q w_q f_q conservatively, the S- and
      L-steps and the truncation do not.  Over a step, delta = sum over its three
      phases of [rho(K^1 V^T) - rho(end of the phase)] is the mass the
      non-conservative parts changed; at the end of the step the isotropic
      rank-one term delta(x) (x) 1/|S| is added to f and the result truncated by
      Algorithm 5's rule.  Without truncation loss the step's rho is then the one
      of the conservative K-step chain.
  R20 Strang splitting (off unless the workload asks for it): a step is x(dt/2),
      y(dt/2), collision(dt), y(dt/2), x(dt/2), each advection phase a full
      Algorithm 1/2 (augmentation, K-, S-, L-step, truncation) with the half step;
      neighbour data come from the start of each phase (R7).  The Lie order of
      Algorithm 6 is the default.
  R21 flux-split K-step (off unless the workload asks for it): C+ = <V, Omega+ V>,
      C- = <V, Omega- V> with Omega+- = max/min(Omega, 0), i.e. the per-direction
      upwind flux of the L-step projected on the augmented angular basis, in place of
      Appendix A's C+- = P Lambda+- P^T.  Both split C = C+ + C-; at full rank they
      coincide (the eigenvectors of C are then the directions themselves); at low rank
      the flux split needs no eigendecomposition.
  R22 physical inflow f(s, Omega) = g(s) h(Omega) on a side, for the directions that
      enter through it (the masks of R2), acts as a virtual neighbour: its ghost term
      is g(line) <m_in h, V_hat>_phi (as a neighbour's face row times M_in), and the
      augmentation input L0 gets the column m_in h |g|_x with
      |g|_x^2 = hx hy len sum_{face lines} g^2, the norm of the data extended across a
      subdomain of the same size (Algorithm 4 takes a neighbour's whole V S^T), so that
      V_hat can represent the inflow.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
@dataclass
class Sub:
    k: int
    I: int
    J: int
    ix0: int
    ix1: int
    jy0: int
    jy1: int

    @property
    def nxk(self):
        return self.ix1 - self.ix0

    @property
    def nyk(self):
        return self.jy1 - self.jy0

    @property
    def N(self):
        return self.nxk * self.nyk


def make_subdomains(wl):
    subs = []
    TX = len(wl.xcuts) - 1
    TY = len(wl.ycuts) - 1
    for J in range(TY):
        for I in range(TX):
            subs.append(Sub(J * TX + I, I, J, wl.xcuts[I], wl.xcuts[I + 1],
                            wl.ycuts[J], wl.ycuts[J + 1]))
    return subs


def cell_index(wl, sub):
    """Global flat cell indices of a subdomain, x fastest."""
    i = np.arange(sub.ix0, sub.ix1)
    j = np.arange(sub.jy0, sub.jy1)
    return (j[:, None] * wl.nx + i[None, :]).reshape(-1)


# ----------------------------------------------------------------------------
# helpers in the paper's weighted inner products
# ----------------------------------------------------------------------------
def integrate(y, rhs, dt, method):
    """One step of explicit Euler or classic RK4 (Section 4 introduction)."""
    if method == "euler":
        return y + dt * rhs(y)
    if method == "rk4":
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * dt * k1)
        k3 = rhs(y + 0.5 * dt * k2)
        k4 = rhs(y + dt * k3)
        return y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    raise ValueError(method)


def _legendre(l, x):
    p0 = np.ones_like(x)
    if l == 0:
        return p0
    p1 = x.copy()
    for k in range(1, l):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return p1


def spatial_candidates(sub):
    """Fixed completion family on a subdomain (R11): DCT-II cosine products
    cos(pi a (i+1/2)/nx_k) * cos(pi b (j+1/2)/ny_k), ordered by a+b, then a descending.
    The family is exactly orthogonal on the cell grid."""
    nxk, nyk = sub.nxk, sub.nyk
    i = np.arange(nxk)
    j = np.arange(nyk)
    for d in range(nxk + nyk - 1):
        for a in range(min(d, nxk - 1), -1, -1):
            b = d - a
            if b >= nyk:
                break
            cx = np.cos(math.pi * a * (i + 0.5) / nxk)
            cy = np.cos(math.pi * b * (j + 0.5) / nyk)
            yield (cy[:, None] * cx[None, :]).reshape(-1)


def angular_candidates(wl):
    """Fixed completion family in angle (R11), defined from the direction table.

    phi = atan2(Omega_y, Omega_x), mu^2 = 1 - Omega_x^2 - Omega_y^2.  Candidates are
    P_{2l}(mu) * cos(m phi) and P_{2l}(mu) * sin(m phi) (even Legendre polynomials
    only: planar transport never distinguishes mu from -mu), with m <= n_phi/2 and
    2l < n_mu (l = 0 only on the circle).  Order: degree m + 2l ascending, then m
    descending, cos before sin.  Candidates whose weighted norm^2 is below
    1e-12 |S| (e.g. cos at the Nyquist azimuth of an offset grid) are skipped.
    The unit vectors e_q follow as a last resort.
    """
    ox, oy, w = wl.omega_x, wl.omega_y, wl.w
    phi = np.arctan2(oy, ox)
    mu2 = np.maximum(0.0, 1.0 - (ox * ox + oy * oy))
    circle = wl.n_mu == 0
    l_count = 1 if circle else (wl.n_mu + 1) // 2
    m_max = wl.n_phi // 2
    ssum = float(np.sum(w))
    for deg in range(0, m_max + 2 * (l_count - 1) + 1):
        for m in range(min(deg, m_max), -1, -1):
            if (deg - m) % 2:
                continue
            l = (deg - m) // 2
            if l >= l_count:
                continue
            p2l = _legendre_even(l, mu2)
            for trig in (np.cos, np.sin):
                if trig is np.sin and m == 0:
                    continue
                c = p2l * trig(m * phi)
                if float(np.sum(w * c * c)) < 1e-12 * ssum:
                    continue
                yield c
    # last resort (only reached when more than the even family is needed): unit vectors
    for q in range(ox.shape[0]):
        e = np.zeros(ox.shape[0])
        e[q] = 1.0
        yield e


def _legendre_even(l, mu2):
    """P_{2l}(mu) evaluated from mu^2 through the three-term recurrence in mu."""
    mu = np.sqrt(mu2)
    return _legendre(2 * l, mu)


def complete_basis(Qw, sw, r_out, candidates, accept=0.5):
    """Append candidates to the Euclidean-orthonormal columns Qw (already scaled by
    the square-root weights sw) until r_out columns (R11): each candidate is
    normalised, Gram-Schmidt'd twice against the current columns and accepted
    when its residual norm is >= accept."""
    Q = Qw
    if Q.shape[1] >= r_out:
        return Q[:, :r_out]
    for c in candidates:
        cw = sw * c
        nrm = np.linalg.norm(cw)
        if nrm == 0.0:
            continue
        cw = cw / nrm
        res = cw - Q @ (Q.T @ cw)
        res = res - Q @ (Q.T @ res)
        rn = np.linalg.norm(res)
        if rn >= accept:
            Q = np.concatenate([Q, (res / rn)[:, None]], axis=1)
            if Q.shape[1] == r_out:
                return Q
    raise RuntimeError("completion family exhausted")


def orthonormal_basis(A, sw, r_out, candidates, tau, accept=0.5):
    """Weighted-orthonormal basis with r_out columns of the significant span of A.

    sw are the square roots of the inner-product weights (<u,v> = sum sw^2 u v).
    Significant span: left singular vectors with sigma_j > tau*sigma_1 (at most
    r_out of them); the remaining columns come from the candidate family (R11).
    Returns (Q, p), p = number of significant columns.
    """
    Aw = sw[:, None] * A
    if Aw.size and np.max(np.abs(Aw)) > 0.0:
        Ue, s, _ = np.linalg.svd(Aw, full_matrices=False)
        p = min(int(np.sum(s > tau * s[0])), r_out)
        Qe = Ue[:, :p]
    else:
        p = 0
        Qe = np.zeros((A.shape[0], 0))
    Qe = complete_basis(Qe, sw, r_out, candidates, accept)
    return Qe / sw[:, None], p


def tail_rank(sig, tol):
    """Minimal r with (sum_{j>r} sigma_j^2)^{1/2} <= tol (Algorithms 4 and 5)."""
    m = sig.shape[0]
    for r in range(m + 1):
        if math.sqrt(float(np.sum(sig[r:] ** 2))) <= tol:
            return r
    return m


# ----------------------------------------------------------------------------
# the scheme
# ----------------------------------------------------------------------------
class DDDLRA:
    """DD-DLRA solver on one problem (Algorithm 6), FP64."""

    def __init__(self, wl, tau=1e-5, accept=0.5):
        self.wl = wl
        self.dt_scale = 1.0          # fraction of dt the current phase advances (R20)
        self.tau = float(tau)
        self.accept = float(accept)
        self.subs = make_subdomains(wl)
        self.TX = len(wl.xcuts) - 1
        self.TY = len(wl.ycuts) - 1
        self.hx = wl.hx
        self.hy = wl.hy
        self.sw_x = math.sqrt(self.hx * self.hy)
        self.w = np.asarray(wl.w, dtype=np.float64)
        self.sw_phi = np.sqrt(self.w)
        self.ssum = float(np.sum(self.w))
        self.cells = [cell_index(wl, s) for s in self.subs]
        self.sig_s = [wl.sigma_s[c] for c in self.cells]
        self.sig_t = [wl.sigma_s[c] + wl.sigma_a[c] for c in self.cells]
        self.Q = [wl.source[c] for c in self.cells]
        if wl.rank_mode == "fixed":
            self.r_floor = wl.rank
        else:
            self.r_floor = wl.r_min
        self.state = None
        self.log = []
        self.init_isotropic()

    # -- state -----------------------------------------------------------------
    def init_isotropic(self):
        """Rank-1 factors of the isotropic initial data (R12)."""
        st = []
        for s, c in zip(self.subs, self.cells):
            g = self.wl.g0[c]
            gn = self.sw_x * np.linalg.norm(g)
            if gn == 0.0:
                st.append((np.zeros((s.N, 0)), np.zeros((0, 0)), np.zeros((self.wl.n, 0))))
                continue
            U = (g / gn)[:, None]
            V = np.full((self.wl.n, 1), 1.0 / math.sqrt(self.ssum))
            S = np.array([[gn * math.sqrt(self.ssum)]])
            st.append((U, S, V))
        self.state = st

    def set_state(self, factors):
        self.state = [(np.array(U, dtype=np.float64), np.array(S, dtype=np.float64),
                       np.array(V, dtype=np.float64)) for (U, S, V) in factors]

    def ranks(self):
        return [S.shape[0] for (_, S, _) in self.state]

    def _ip_x(self, A, B):
        return (self.hx * self.hy) * (A.T @ B)

    def _ip_phi(self, A, B):
        return A.T @ (self.w[:, None] * B)

    # -- geometry along an axis ------------------------------------------------
    def _neighbours(self, sub, axis):
        if axis == "x":
            lo = sub.k - 1 if sub.I > 0 else None
            hi = sub.k + 1 if sub.I < self.TX - 1 else None
        else:
            lo = sub.k - self.TX if sub.J > 0 else None
            hi = sub.k + self.TX if sub.J < self.TY - 1 else None
        return lo, hi

    @staticmethod
    def _lines(A, sub, axis):
        """View a (N_k, r) array as (n_lines, line_len, r) along the axis."""
        A3 = A.reshape(sub.nyk, sub.nxk, -1)
        return A3 if axis == "x" else A3.transpose(1, 0, 2)

    def _face(self, A, sub, axis, side):
        """Rows of A on the cells of the subdomain face (side 0 = low, 1 = high)."""
        L = self._lines(A, sub, axis)
        return L[:, 0, :] if side == 0 else L[:, -1, :]

    def _diff(self, A, sub, axis, ghost, kind):
        """Upwind difference along the axis of every column of A with ghost cells.

        kind 'minus': (u_c - u_{c-1})/h with u_{-1} = ghost;
        kind 'plus' : (u_{c+1} - u_c)/h with u_{len} = ghost.
        """
        h = self.hx if axis == "x" else self.hy
        L = self._lines(A, sub, axis)
        g = ghost[:, None, :]
        if kind == "minus":
            prev = np.concatenate([g, L[:, :-1, :]], axis=1)
            D = (L - prev) / h
        else:
            nxt = np.concatenate([L[:, 1:, :], g], axis=1)
            D = (nxt - L) / h
        if axis == "x":
            return D.reshape(sub.N, -1)
        return D.transpose(1, 0, 2).reshape(sub.N, -1)

    def _omega(self, axis):
        return self.wl.omega_x if axis == "x" else self.wl.omega_y

    # -- Algorithm 4: augmentation ---------------------------------------------
    def augment(self, k, axis, snap):
        U, S, V = snap[k]
        sub = self.subs[k]
        wl = self.wl
        blocks = [V @ S.T]
        for side, nb in enumerate(self._neighbours(sub, axis)):
            if nb is not None:
                _, Sn, Vn = snap[nb]
                blocks.append(Vn @ Sn.T)
            else:
                col = self._inflow_column(sub, axis, side)        # R22
                if col is not None:
                    blocks.append(col[:, None])
        L0 = np.concatenate(blocks, axis=1)
        Lw = self.sw_phi[:, None] * L0
        if Lw.size and np.max(np.abs(Lw)) > 0.0:
            Ue, sig, _ = np.linalg.svd(Lw, full_matrices=False)
            p = int(np.sum(sig > self.tau * sig[0]))
        else:
            Ue, sig, p = np.zeros((wl.n, 0)), np.zeros(0), 0
        r_tail = tail_rank(sig, wl.tol) if wl.rank_mode == "tol" else p
        r_sig = min(r_tail, p)
        r_cap = min(wl.r_aug_max, wl.n, sub.N)
        r_t = min(max(r_sig, S.shape[0], self.r_floor), r_cap)
        keep = min(r_t, p)
        # V_hat: leading left singular vectors (weighted), completed if needed (R11)
        Vw = complete_basis(Ue[:, :keep], self.sw_phi, r_t, angular_candidates(wl), self.accept)
        Vhat = Vw / self.sw_phi[:, None]
        K0 = U @ S @ self._ip_phi(V, Vhat)            # R9
        return K0, Vhat, dict(m=L0.shape[1], p=p, r_t=r_t)

    # -- boundary data, Eq. (generate_Kboundary) -------------------------------
    def boundary(self, k, axis, snap, K0, Vhat):
        sub = self.subs[k]
        om = self._omega(axis)
        in_lo = (om >= 0).astype(np.float64)       # R2
        in_hi = (om < 0).astype(np.float64)
        Kb = []
        for side, nb, m_in, m_out in ((0, self._neighbours(sub, axis)[0], in_lo, in_hi),
                                      (1, self._neighbours(sub, axis)[1], in_hi, in_lo)):
            own = self._face(K0, sub, axis, side) @ self._ip_phi(m_out[:, None] * Vhat, Vhat)
            if nb is not None:
                Un, Sn, Vn = snap[nb]
                Kn = Un @ Sn
                # the neighbour's cells adjacent to this face: its opposite face (R5)
                Kn_face = self._face(Kn, self.subs[nb], axis, 1 - side)
                own = own + Kn_face @ self._ip_phi(m_in[:, None] * Vn, Vhat)
            else:
                gh = self._inflow_face(sub, axis, side)           # R22
                if gh is not None:
                    g_face, hq = gh
                    own = own + g_face[:, None] * self._ip_phi((m_in * hq)[:, None], Vhat)
            Kb.append(own)
        return Kb[0], Kb[1]

    def _inflow_face(self, sub, axis, side):
        """Physical inflow on the face of a boundary subdomain (R22): the values of g
        on the face's lines and h, or None."""
        key = axis + ("_lo" if side == 0 else "_hi")
        if key not in self.wl.inflow:
            return None
        g, hq = self.wl.inflow[key]
        g = np.asarray(g, dtype=np.float64)
        g_face = g[sub.jy0:sub.jy1] if axis == "x" else g[sub.ix0:sub.ix1]
        return g_face, np.asarray(hq, dtype=np.float64)

    def _inflow_column(self, sub, axis, side):
        """The augmentation column of a physical inflow side (R22), or None."""
        gh = self._inflow_face(sub, axis, side)
        if gh is None:
            return None
        g_face, hq = gh
        om = self._omega(axis)
        m_in = (om >= 0) if side == 0 else (om < 0)
        ln = sub.nxk if axis == "x" else sub.nyk
        return (m_in * hq) * math.sqrt(self.hx * self.hy * ln * float(np.sum(g_face ** 2)))

    # -- Appendix A: K-step right-hand side ------------------------------------
    def kstep_rhs_adv(self, K, C, Kb_lo, Kb_hi, sub, axis):
        """-c_adv D K C with D upwinded per eigenvector of C (Appendix A)."""
        lam, P = np.linalg.eigh(C)
        KP = K @ P
        glo = Kb_lo @ P
        ghi = Kb_hi @ P
        Dm = self._diff(KP, sub, axis, glo, "minus")
        Dp = self._diff(KP, sub, axis, ghi, "plus")
        D = np.where(lam[None, :] > 0, Dm, np.where(lam[None, :] < 0, Dp, 0.0))
        return -self.wl.c_adv * (D * lam[None, :]) @ P.T

    def kstep_rhs_flux(self, K, Cp, Cm, Kb_lo, Kb_hi, sub, axis):
        """-c_adv (D- K C+ + D+ K C-) with the direction split C+- (R21): backward
        differences carry the part of the flux moving towards higher coordinates,
        forward differences the rest."""
        Dm = self._diff(K, sub, axis, Kb_lo, "minus")
        Dp = self._diff(K, sub, axis, Kb_hi, "plus")
        return -self.wl.c_adv * (Dm @ Cp + Dp @ Cm)

    # -- Algorithms 1 / 2 -------------------------------------------------------
    def psi_advection(self, k, axis, K0, Vhat, Kb_lo, Kb_hi):
        wl = self.wl
        sub = self.subs[k]
        om = self._omega(axis)
        dt = wl.dt * self.dt_scale
        m = wl.integrator
        C = self._ip_phi(Vhat, om[:, None] * Vhat)       # <V_j, Omega V_k>_phi
        if wl.kstep_split == "flux":                     # R21
            Cp = self._ip_phi(Vhat, np.maximum(om, 0.0)[:, None] * Vhat)
            Cm = self._ip_phi(Vhat, np.minimum(om, 0.0)[:, None] * Vhat)
            rk = lambda K: self.kstep_rhs_flux(K, Cp, Cm, Kb_lo, Kb_hi, sub, axis)
        else:
            rk = lambda K: self.kstep_rhs_adv(K, C, Kb_lo, Kb_hi, sub, axis)
        # 1: K-step, Eq. (advx_evolK)
        K1 = integrate(K0, rk, dt, m)
        # 2: QR of K
        r_t = K0.shape[1]
        U1, pK = orthonormal_basis(K1, np.full(sub.N, self.sw_x), r_t,
                                   spatial_candidates(sub), self.tau, self.accept)
        S1 = self._ip_x(U1, K1)
        # 3: S-step, Eq. (advx_evolS): dS/dt = -<U1, R_K(U1 S)> (R4)
        S2 = integrate(S1, lambda S: -self._ip_x(U1, rk(U1 @ S)), dt, m)
        # 4: L-step, Eq. (advx_evolL), per-direction upwind, ghost f^b = K^b V^T (R4)
        fb_lo = Kb_lo @ Vhat.T
        fb_hi = Kb_hi @ Vhat.T
        pos = om > 0
        neg = om < 0

        def lrhs(L):
            f = U1 @ L.T
            Fm = self._diff(f, sub, axis, fb_lo, "minus")
            Fp = self._diff(f, sub, axis, fb_hi, "plus")
            F = np.zeros_like(f)
            F[:, pos] = -wl.c_adv * om[pos][None, :] * Fm[:, pos]
            F[:, neg] = -wl.c_adv * om[neg][None, :] * Fp[:, neg]
            return self._ip_x(U1, F).T

        L1 = integrate(Vhat @ S2.T, lrhs, dt, m)
        # 5: QR of L
        V1, pL = orthonormal_basis(L1, self.sw_phi, r_t, angular_candidates(wl),
                                   self.tau, self.accept)
        S3 = self._ip_phi(V1, L1).T
        rho_k = K1 @ (Vhat.T @ self.w)                       # mass of the K-step (R18)
        return U1, S3, V1, dict(pK=pK, pL=pL, rho_k=rho_k)

    # -- Algorithm 5 ------------------------------------------------------------
    def truncate(self, U, S, V):
        wl = self.wl
        if S.size and np.max(np.abs(S)) > 0.0:
            Ub, sig, Vbt = np.linalg.svd(S)
            p = int(np.sum(sig > self.tau * sig[0]))
        else:
            Ub = np.eye(S.shape[0])
            Vbt = np.eye(S.shape[0])
            sig = np.zeros(S.shape[0])
            p = 0
        if wl.rank_mode == "tol":
            r1 = min(max(tail_rank(sig, wl.tol), wl.r_min), wl.r_max)
        else:
            r1 = wl.rank
        r1 = min(r1, p)
        return U @ Ub[:, :r1], np.diag(sig[:r1]), V @ Vbt.T[:, :r1]

    # -- Algorithm 3 ------------------------------------------------------------
    def psi_collision(self, k, U, S, V):
        wl = self.wl
        sub = self.subs[k]
        dt = wl.dt * self.dt_scale
        m = wl.integrator
        r = S.shape[0]
        r_c = min(max(r, self.r_floor), wl.n, sub.N)
        K0 = np.zeros((sub.N, r_c))
        K0[:, :r] = U @ S
        if r < r_c:                                          # R13
            Vw = complete_basis(self.sw_phi[:, None] * V, self.sw_phi, r_c,
                                angular_candidates(wl), self.accept)
            V = Vw / self.sw_phi[:, None]
        sig_s, sig_t, Q = self.sig_s[k], self.sig_t[k], self.Q[k]
        a = V.T @ self.w                                     # <V_j>_phi
        ss = self.ssum

        def krhs(K):                                         # Eq. (coll_evolK)
            return ((sig_s / ss) * (K @ a))[:, None] * a[None, :] - sig_t[:, None] * K \
                + Q[:, None] * a[None, :]

        K1 = integrate(K0, krhs, dt, m)
        U1, pK = orthonormal_basis(K1, np.full(sub.N, self.sw_x), r_c,
                                   spatial_candidates(sub), self.tau, self.accept)
        S1 = self._ip_x(U1, K1)
        Ms = self._ip_x(U1, sig_s[:, None] * U1)
        Mt = self._ip_x(U1, sig_t[:, None] * U1)
        q = self._ip_x(U1, Q[:, None])[:, 0]

        def srhs(Sm):                                        # Eq. (coll_evolS)
            return -((1.0 / ss) * Ms @ Sm @ np.outer(a, a) - Mt @ Sm + np.outer(q, a))

        S2 = integrate(S1, srhs, dt, m)

        def lrhs(L):                                         # Eq. (coll_evolL)
            mean = L.T @ self.w
            return np.ones(wl.n)[:, None] * ((1.0 / ss) * (Ms @ mean) + q)[None, :] \
                - L @ Mt.T

        L1 = integrate(V @ S2.T, lrhs, dt, m)
        V1, pL = orthonormal_basis(L1, self.sw_phi, r_c, angular_candidates(wl), self.tau,
                                   self.accept)
        S3 = self._ip_phi(V1, L1).T
        rho_k = K1 @ a                                       # mass of the K-step (R18)
        return U1, S3, V1, dict(r_c=r_c, pK=pK, pL=pL, rho_k=rho_k)

    # -- Algorithm 6 ------------------------------------------------------------
    def advection_phase(self, axis):
        snap = self.state                                     # R7
        new = []
        info = []
        for k in range(len(self.subs)):
            K0, Vhat, ia = self.augment(k, axis, snap)
            Kb_lo, Kb_hi = self.boundary(k, axis, snap, K0, Vhat)
            U1, S3, V1, ip = self.psi_advection(k, axis, K0, Vhat, Kb_lo, Kb_hi)
            Ut, St, Vt = self.truncate(U1, S3, V1)
            new.append((Ut, St, Vt))
            ip["dmass"] = ip.pop("rho_k") - self._mass(Ut, St, Vt, k)
            info.append(dict(ia, **ip, r=St.shape[0]))
        self.state = new
        return info

    def collision_phase(self):
        new = []
        info = []
        for k in range(len(self.subs)):
            U, S, V = self.state[k]
            U1, S3, V1, ic = self.psi_collision(k, U, S, V)
            new.append((U1, S3, V1))
            ic["dmass"] = ic.pop("rho_k") - self._mass(U1, S3, V1, k)
            info.append(ic)
        self.state = new
        return info

    def _mass(self, U, S, V, k):
        """Per-cell scalar flux of one subdomain's factors."""
        if S.shape[0] == 0:
            return np.zeros(self.subs[k].N)
        return U @ (S @ (V.T @ self.w))

    def mass_correction(self, deltas):
        """R18: add delta (x) 1/|S| to f on every subdomain and truncate (Algorithm 5's
        rule).  The augmented factors are orthonormalised by weighted QR."""
        new = []
        for k, ((U, S, V), d) in enumerate(zip(self.state, deltas)):
            if not np.any(d):
                new.append((U, S, V))
                continue
            Ua = np.concatenate([U, d[:, None]], axis=1)
            Va = np.concatenate([V, np.full((self.wl.n, 1), 1.0 / self.ssum)], axis=1)
            Sa = np.zeros((S.shape[0] + 1, S.shape[0] + 1))
            Sa[:S.shape[0], :S.shape[0]] = S
            Sa[-1, -1] = 1.0
            Qu, Ru = np.linalg.qr(self.sw_x * Ua)
            Qv, Rv = np.linalg.qr(self.sw_phi[:, None] * Va)
            new.append(self.truncate(Qu / self.sw_x, Ru @ Sa @ Rv.T, Qv / self.sw_phi[:, None]))
        self.state = new

    def _phase(self, kind, scale):
        self.dt_scale = scale
        try:
            return self.collision_phase() if kind == "c" else self.advection_phase(kind)
        finally:
            self.dt_scale = 1.0

    def step(self):
        if self.wl.splitting == "strang":                    # R20
            order = [("x", 0.5), ("y", 0.5), ("c", 1.0), ("y", 0.5), ("x", 0.5)]
        else:
            order = [("x", 1.0), ("y", 1.0), ("c", 1.0)]
        infos = [self._phase(kind, scale) for kind, scale in order]
        if self.wl.mass_fix:
            self.mass_correction([sum(ph[k]["dmass"] for ph in infos)
                                  for k in range(len(self.subs))])
        entry = {"phases": [(kind, inf) for (kind, _), inf in zip(order, infos)]}
        for (kind, _), inf in zip(order, infos):
            entry.setdefault(kind, inf)                      # first phase of each kind
        self.log.append(entry)

    def run(self, nsteps=None):
        for _ in range(self.wl.nsteps if nsteps is None else nsteps):
            self.step()
        return self

    # -- observables -------------------------------------------------------------
    def scalar_flux(self):
        """rho = U S <V, 1>_phi on every subdomain, global x-fastest order (Section 2)."""
        rho = np.zeros(self.wl.ncells)
        for (U, S, V), c in zip(self.state, self.cells):
            if S.shape[0]:
                rho[c] = U @ (S @ (V.T @ self.w))
        return rho

    def full_f(self):
        """The full distribution f (ny, nx, n); small problems only."""
        f = np.zeros((self.wl.ncells, self.wl.n))
        for (U, S, V), c in zip(self.state, self.cells):
            if S.shape[0]:
                f[c] = U @ S @ V.T
        return f.reshape(self.wl.ny, self.wl.nx, self.wl.n)
