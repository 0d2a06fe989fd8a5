"""O1: the tensor jump method on matrix product states, plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring): the slow, readable
reference the CUDA path is compared with.  Every function follows a passage of
arXiv:2501.17913 (TJM); where the paper leaves a choice open, the reading taken
is stated in the function's docstring and is the one the CUDA path implements.

Conventions
-----------
* Site tensor  M_l  has shape (chi_l, d, chi_{l+1})  (left bond, physical, right
  bond); bonds are numbered b = 0..L with chi_0 = chi_L = 1 (Methods, Eq. MPS).
* MPO site  W_l[w, v, t, s]: left MPO bond w, right MPO bond v, output (bra)
  physical index t, input (ket) index s, so H = sum prod_l W_l^{t_l s_l}
  |t><s| (Methods, Sec. "Matrix product (density) operators").
* Left environment  Lenv[b][x, w, a]  covers sites 0..b-1 (bra x, MPO w, ket a);
  right environment Renv[b][v, b, y] covers sites b..L-1 (MPO v, ket b, bra y)
  (Sec. "Hybrid strategy": environments reused through the sweep).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import expm as _scipy_expm

from .philox import uniforms


# --------------------------------------------------------------------------
# problem description (Sec. "Initialization": Psi(0), H0 as MPO, {L_m, gamma_m},
# dt, T, chi_max, N)
# --------------------------------------------------------------------------
@dataclass
class Problem:
    W: list                     # L arrays (Dl, Dr, d, d)
    jumps: list                 # [(site, 2x2 op, gamma)] in the user's order
    dt: float
    chi_max: int
    trunc_eps: float = 1e-10
    krylov_tol: float = 1e-12
    krylov_max: int = 30
    exact: bool = False         # full bond dimension, no truncation at all
    L: int = field(init=False)
    d: int = field(init=False)

    def __post_init__(self):
        self.W = [np.asarray(w, dtype=np.complex128) for w in self.W]
        self.L = len(self.W)
        self.d = self.W[0].shape[2]
        self.jumps = [(int(s), np.asarray(op, dtype=np.complex128), float(g))
                      for (s, op, g) in self.jumps]
        # Reading: jumps are ordered site-major (site 0..L-1), then by the
        # user's order among the jumps acting on the same site.
        self.jump_order = sorted(range(len(self.jumps)),
                                 key=lambda m: (self.jumps[m][0], m))


def dissipator_site(prob: Problem, site: int, tau: float) -> np.ndarray:
    """D_l[tau] = exp(-tau/2 * sum_{j in S(l)} gamma_j L_j^dag L_j)  (Eq. DissipativeMPO)."""
    A = np.zeros((prob.d, prob.d), dtype=np.complex128)
    for (s, op, g) in prob.jumps:
        if s == site:
            A += g * (op.conj().T @ op)
    return _scipy_expm(-0.5 * tau * A)


# --------------------------------------------------------------------------
# elementary MPS operations (Methods, Sec. "Matrix product states": canonical
# forms, moving the orthogonality centre by QR)
# --------------------------------------------------------------------------
def apply_site_op(op, M):
    """Contract a d x d operator into the physical index of a site tensor."""
    return np.einsum('ts,asb->atb', op, M)


def qr_move_right(mps, l):
    """M_l = Q R (Q left-orthonormal); M_l <- Q, M_{l+1} <- R M_{l+1}."""
    chl, d, chr_ = mps[l].shape
    Q, R = np.linalg.qr(mps[l].reshape(chl * d, chr_))
    k = Q.shape[1]
    mps[l] = Q.reshape(chl, d, k)
    mps[l + 1] = np.einsum('kb,bsc->ksc', R, mps[l + 1])
    return R


def rq_move_left(mps, l):
    """M_l = C Q (Q right-orthonormal, from the QR of M_l^dag); M_l <- Q, M_{l-1} <- M_{l-1} C."""
    chl, d, chr_ = mps[l].shape
    Qh, Rh = np.linalg.qr(mps[l].reshape(chl, d * chr_).conj().T)
    k = Qh.shape[1]
    mps[l] = Qh.conj().T.reshape(k, d, chr_)
    C = Rh.conj().T
    mps[l - 1] = np.einsum('asb,bk->ask', mps[l - 1], C)
    return C


def trunc_rank(S, prob: Problem, rec=None) -> int:
    """Number of singular values kept after a two-site update or a jump.

    Reading of the unspecified cut-off of Sec. 1TDVP and 2TDVP as tensor
    networks: keep the smallest r >= 1 with sum_{i>=r} S_i^2 <= trunc_eps *
    sum_i S_i^2 (relative discarded weight), capped at chi_max.  In exact mode
    every singular value is kept, zeros included.
    """
    n = len(S)
    if prob.exact:
        return n
    w = np.asarray(S, dtype=np.float64) ** 2
    total = float(np.sum(w))
    tail = 0.0
    r = n
    # walk from the smallest value upwards while the discarded tail stays small
    for i in range(n - 1, 0, -1):
        if tail + w[i] <= prob.trunc_eps * total:
            tail += w[i]
            r = i
        else:
            break
    r = max(1, min(r, prob.chi_max))
    if rec is not None and n > 1:
        # how close this decision was to going the other way (diagnostics only):
        # the discarded tail against the threshold on both sides of the cut
        thr = prob.trunc_eps * total
        kept_tail = float(np.sum(w[r:]))
        m = abs(thr - kept_tail) / total
        if r - 1 >= 1:
            m = min(m, abs(kept_tail + w[r - 1] - thr) / total)
        rec['trunc_margin'] = min(rec.get('trunc_margin', math.inf), m)
        if r < n:
            rec['cut_gap'] = min(rec.get('cut_gap', math.inf), float((S[r - 1] - S[r]) / S[0]))
    return r


def local_expectations(mps, ops):
    """<psi|O_i|psi> for local operators [(site, op)], by the plain definition.

    op is 2 x 2 (acting on `site`) or 4 x 4 (acting on sites `site`, `site`+1,
    row index (t1 t2), column index (s1 s2), the first site most significant;
    the two-site correlators of Fig. 4b, e.g. X (x) X).  Left and right transfer
    matrices are built once with no canonical-form assumption; the values are
    NOT divided by <psi|psi>.  Also returns <psi|psi>.
    """
    L = len(mps)
    Lt = [np.ones((1, 1), dtype=np.complex128)]
    for l in range(L):
        Lt.append(np.einsum('ab,asc,bsd->cd', Lt[l], mps[l].conj(), mps[l], optimize=True))
    Rt = [None] * (L + 1)
    Rt[L] = np.ones((1, 1), dtype=np.complex128)
    for l in range(L - 1, -1, -1):
        Rt[l] = np.einsum('asc,bsd,cd->ab', mps[l].conj(), mps[l], Rt[l + 1], optimize=True)
    norm2 = Lt[L][0, 0].real
    vals = []
    for (site, op) in ops:
        op = np.asarray(op)
        M = mps[site]
        if op.shape == (2, 2):
            vals.append(np.einsum('ab,atc,ts,bsd,cd->', Lt[site], M.conj(), op, M, Rt[site + 1], optimize=True))
        else:
            N = mps[site + 1]
            O4 = op.reshape(2, 2, 2, 2)       # [t1, t2, s1, s2]
            vals.append(np.einsum('ab,atc,cue,tusv,bsd,dvf,ef->', Lt[site], M.conj(), N.conj(), O4, M, N,
                                  Rt[site + 2], optimize=True))
    return np.array(vals), norm2


def tangent_projector(mps):
    """The projector P onto the tangent space of the fixed-bond-dimension manifold at the state of `mps`
    (dense, small L), and the normalised state vector psi:
        P = sum_{l=0}^{L-1} P_L(<l) (x) 1_l (x) P_R(>l)  -  sum_{l=0}^{L-2} P_L(<=l) (x) P_R(>l),
    P_L(<l) the projector onto the span of the left block states of sites 0..l-1 and P_R(>l) onto the
    right block states of sites l+1..L-1, both from a left- and a right-canonical copy of the MPS
    (Sec. "Error measures"; the 1TDVP projector of Sec. "1TDVP and 2TDVP as tensor networks")."""
    L = len(mps)
    d = mps[0].shape[1]
    left = [np.array(m) for m in mps]
    for l in range(L - 1):
        qr_move_right(left, l)
    right = [np.array(m) for m in mps]
    for l in range(L - 1, 0, -1):
        rq_move_left(right, l)
    # psi from the right-canonical copy (centre at site 0), normalised
    psi = right[0]
    for M in right[1:]:
        psi = np.tensordot(psi, M, ([psi.ndim - 1], [0]))
    psi = psi.reshape(-1)
    psi = psi / np.linalg.norm(psi)
    # left block states: the columns of BL[l] (d^(l+1), chi_{l+1}); right block states: the rows of
    # BR[l] (chi_l, d^(L-l))
    BL = []
    acc = np.ones((1, 1), dtype=np.complex128)
    for l in range(L):
        acc = np.tensordot(acc, left[l], ([1], [0])).reshape(-1, left[l].shape[2])
        BL.append(acc)
    BR = [None] * L
    acc = np.ones((1, 1), dtype=np.complex128)
    for l in range(L - 1, -1, -1):
        acc = np.tensordot(right[l], acc.reshape(right[l].shape[2], -1), ([2], [0])).reshape(right[l].shape[0], -1)
        BR[l] = acc

    def PL(n):        # sum_a |a><a| over the left block states of sites 0..n-1
        if n == 0:
            return np.ones((1, 1))
        B = BL[n - 1]
        return B @ B.conj().T

    def PR(n):        # sum_b |b><b| over the right block states of sites n..L-1
        if n == L:
            return np.ones((1, 1))
        B = BR[n]
        return B.T @ B.conj()

    P = np.zeros((d ** L, d ** L), dtype=np.complex128)
    for l in range(L):
        P += np.kron(np.kron(PL(l), np.eye(d)), PR(l + 1))
    for l in range(L - 1):
        P -= np.kron(PL(l + 1), PR(l + 1))
    return P, psi


def projection_error(mps, W):
    """Projection error of 1TDVP at the state of `mps` (Sec. "Error measures"):
    eps = || (I - P) H |psi> ||_2 for the normalised |psi>, P = tangent_projector(mps); H from the MPO.
    Written out densely (small L only)."""
    from .dense import mpo_to_dense
    P, psi = tangent_projector(mps)
    v = mpo_to_dense(W) @ psi
    return float(np.linalg.norm(v - P @ v))


def measure(mps, observables):
    """Re <O_i> = Re <psi|O_i|psi> / <psi|psi>  (Eq. TJMExpVal, one trajectory)."""
    vals, norm2 = local_expectations(mps, observables)
    return (vals / norm2).real


# --------------------------------------------------------------------------
# environments and effective Hamiltonians (Fig. 2; Sec. "Hybrid strategy")
# --------------------------------------------------------------------------
def env_left_update(Lenv, A, W):
    """Lenv[b+1][y, v, b'] = sum conj(A[x,t,y]) Lenv[b][x,w,a] W[w,v,t,s] A[a,s,b']."""
    T1 = np.tensordot(Lenv, A, ([2], [0]))            # x w s b
    T2 = np.tensordot(T1, W, ([1, 2], [0, 3]))        # x b v t
    out = np.tensordot(A.conj(), T2, ([0, 1], [0, 3]))  # y b v
    return out.transpose(0, 2, 1)


def env_right_update(Renv, B, W):
    """Renv[b][w, a, x] = sum B[a,s,b] W[w,v,t,s] Renv[b+1][v,b,y] conj(B[x,t,y])."""
    T1 = np.tensordot(B, Renv, ([2], [1]))            # a s v y
    T2 = np.tensordot(T1, W, ([1, 2], [3, 1]))        # a y w t
    out = np.tensordot(T2, B.conj(), ([1, 3], [2, 1]))  # a w x
    return out.transpose(1, 0, 2)


def heff1(Lenv, W, Renv, M):
    """One-site H^eff_l M (degree-6 network of Fig. 2, top):
    y[x,t,y] = sum Lenv[x,w,a] W[w,v,t,s] M[a,s,b] Renv[v,b,y]."""
    T1 = np.tensordot(Lenv, M, ([2], [0]))            # x w s b
    T2 = np.tensordot(T1, W, ([1, 2], [0, 3]))        # x b v t
    return np.tensordot(T2, Renv, ([1, 2], [1, 0]))   # x t y


def heff2(Lenv, W1, W2, Renv, th):
    """Two-site H^eff_{l,l+1} theta (degree-8 network of Fig. 2, bottom):
    y[x,t,q,y] = sum Lenv[x,w,a] W1[w,u,t,p] W2[u,v,q,s] th[a,p,s,b] Renv[v,b,y]."""
    T1 = np.tensordot(Lenv, th, ([2], [0]))           # x w p s b
    T2 = np.tensordot(T1, W1, ([1, 2], [0, 3]))       # x s b u t
    T3 = np.tensordot(T2, W2, ([1, 3], [3, 0]))       # x b t v q
    return np.tensordot(T3, Renv, ([1, 3], [1, 0]))   # x t q y


def heff0(Lenv, Renv, C):
    """Bond H~^eff_l C (degree-4 network of Fig. 2, middle):
    y[x,y] = sum Lenv[x,w,a] C[a,b] Renv[w,b,y]."""
    T1 = np.tensordot(Lenv, C, ([2], [0]))            # x w b
    return np.tensordot(T1, Renv, ([1, 2], [0, 1]))   # x y


# --------------------------------------------------------------------------
# Lanczos exponential (Sec. 1TDVP: "matricize and exponentiate it using the
# Lanczos method"; Sec. "Hybrid strategy": a limited number of iterations)
# --------------------------------------------------------------------------
def expm_tridiag(alpha, beta, coef):
    """First column of exp(coef * T) for the Lanczos tridiagonal T (scipy expm)."""
    n = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    if n > 1:
        off = np.asarray(beta[:n - 1], dtype=np.float64)
        T = T + np.diag(off, 1) + np.diag(off, -1)
    return _scipy_expm(coef * T)[:, 0]


def expm_lanczos(apply_H, v, coef, tol, kmax):
    """exp(coef * H) v for Hermitian H given as a matvec, coef = -i tau or +i tau.

    Reading of the stopping rule: after building the k-th Lanczos vector,
    stop when |beta_k * [exp(coef T_k) e_1]_k| < tol (the a-posteriori
    Krylov error estimate) or when k reaches kmax.  Full re-orthogonalisation
    (classical Gram-Schmidt, two passes) against all previous vectors.
    Returns (result, number of matvecs).
    """
    beta0 = float(np.linalg.norm(v))
    if beta0 == 0.0:
        return v.copy(), 0
    V = [v / beta0]
    alpha, beta = [], []
    c = None
    for k in range(kmax):
        w = apply_H(V[k])
        a = float(np.vdot(V[k], w).real)
        alpha.append(a)
        w = w - a * V[k]
        if k > 0:
            w = w - beta[k - 1] * V[k - 1]
        for _ in range(2):
            h = [np.vdot(u, w) for u in V]
            for hi, u in zip(h, V):
                w = w - hi * u
        b = float(np.linalg.norm(w))
        c = expm_tridiag(alpha, beta, coef)
        if b * abs(c[-1]) < tol or k == kmax - 1:
            break
        beta.append(b)
        V.append(w / b)
    y = np.zeros_like(v)
    for ci, u in zip(c, V):
        y = y + ci * u
    return beta0 * y, len(alpha)


# --------------------------------------------------------------------------
# dynamic TDVP  U[dt]  (Sec. "Dynamic TDVP"; Eq. 1TDVP_ForwardEvolving,
# 1TDVP_BackwardEvolving, 2TDVP_ForwardEvolving; the piecewise U of Sec.
# "Hybrid strategy")
# --------------------------------------------------------------------------
class Sweeper:
    """Holds the environments of one trajectory and counts the work done."""

    def __init__(self, prob: Problem):
        self.prob = prob
        L = prob.L
        self.Lenv = [None] * (L + 1)
        self.Renv = [None] * (L + 1)
        one = np.ones((1, 1, 1), dtype=np.complex128)
        self.Lenv[0] = one
        self.Renv[L] = one
        self.matvecs = {'heff1': 0, 'heff2': 0, 'heff0': 0, 'env': 0}
        self.updates = {'one_site': 0, 'two_site': 0}
        self.rec = {}

    def build_right_envs(self, mps):
        """Renv[b] for b = L-1..1 from a right-canonical MPS (centre at site 0)."""
        W = self.prob.W
        for l in range(self.prob.L - 1, 0, -1):
            self.Renv[l] = env_right_update(self.Renv[l + 1], mps[l], W[l])
            self.matvecs['env'] += 1

    def _exp(self, kind, f, x, coef):
        y, k = expm_lanczos(f, x, coef, self.prob.krylov_tol, self.prob.krylov_max)
        self.matvecs[kind] += k
        return y

    def sweep(self, mps, tau):
        """One TDVP time step: left-to-right then right-to-left half sweep, each of tau = dt/2.

        Readings: a sweep is two half sweeps of dt/2 (Sec. Dynamic TDVP); the
        switch is local per bond -- when the sweep reaches a bond of dimension
        chi < chi_max a two-site update is used, otherwise a one-site update
        (Sec. Dynamic TDVP).  Forward updates use exp(-i H tau), backward
        updates exp(+i H tau).  Precondition: centre at site 0, sites 1..L-1
        right-canonical, Renv[1..L] valid.  Postcondition: the same, for the
        evolved state.
        """
        p = self.prob
        L, W, chi_max = p.L, p.W, p.chi_max
        Le, Re = self.Lenv, self.Renv
        mi, pi = -1j * tau, +1j * tau
        # ---- left to right ----
        last_two = False
        for l in range(L - 1):
            chl, d, _ = mps[l].shape
            chr_ = mps[l + 1].shape[2]
            if mps[l].shape[2] < chi_max:
                self.updates['two_site'] += 1
                th = np.einsum('asb,bpc->aspc', mps[l], mps[l + 1])
                th = self._exp('heff2', lambda x, l=l: heff2(Le[l], W[l], W[l + 1], Re[l + 2], x), th, mi)
                U, S, Vh = np.linalg.svd(th.reshape(chl * d, d * chr_), full_matrices=False)
                r = trunc_rank(S, p, self.rec)
                mps[l] = U[:, :r].reshape(chl, d, r)
                mps[l + 1] = (S[:r, None] * Vh[:r]).reshape(r, d, chr_)
                Le[l + 1] = env_left_update(Le[l], mps[l], W[l])
                self.matvecs['env'] += 1
                if l + 1 < L - 1:
                    mps[l + 1] = self._exp('heff1', lambda x, l=l: heff1(Le[l + 1], W[l + 1], Re[l + 2], x),
                                           mps[l + 1], pi)
                last_two = True
            else:
                self.updates['one_site'] += 1
                mps[l] = self._exp('heff1', lambda x, l=l: heff1(Le[l], W[l], Re[l + 1], x), mps[l], mi)
                chb = mps[l].shape[2]
                Q, R = np.linalg.qr(mps[l].reshape(chl * d, chb))
                k = Q.shape[1]
                mps[l] = Q.reshape(chl, d, k)
                Le[l + 1] = env_left_update(Le[l], mps[l], W[l])
                self.matvecs['env'] += 1
                C = self._exp('heff0', lambda x, l=l: heff0(Le[l + 1], Re[l + 1], x), R, pi)
                mps[l + 1] = np.einsum('kb,bsc->ksc', C, mps[l + 1])
                last_two = False
        if not last_two:
            self.updates['one_site'] += 1
            mps[L - 1] = self._exp('heff1', lambda x: heff1(Le[L - 1], W[L - 1], Re[L], x), mps[L - 1], mi)
        # ---- right to left ----
        last_two = False
        for l in range(L - 1, 0, -1):
            chl = mps[l - 1].shape[0]
            _, d, chr_ = mps[l].shape
            if mps[l].shape[0] < chi_max:
                self.updates['two_site'] += 1
                th = np.einsum('asb,bpc->aspc', mps[l - 1], mps[l])
                th = self._exp('heff2', lambda x, l=l: heff2(Le[l - 1], W[l - 1], W[l], Re[l + 1], x), th, mi)
                U, S, Vh = np.linalg.svd(th.reshape(chl * d, d * chr_), full_matrices=False)
                r = trunc_rank(S, p, self.rec)
                mps[l] = Vh[:r].reshape(r, d, chr_)
                mps[l - 1] = (U[:, :r] * S[None, :r]).reshape(chl, d, r)
                Re[l] = env_right_update(Re[l + 1], mps[l], W[l])
                self.matvecs['env'] += 1
                if l - 1 > 0:
                    mps[l - 1] = self._exp('heff1', lambda x, l=l: heff1(Le[l - 1], W[l - 1], Re[l], x),
                                           mps[l - 1], pi)
                last_two = True
            else:
                self.updates['one_site'] += 1
                mps[l] = self._exp('heff1', lambda x, l=l: heff1(Le[l], W[l], Re[l + 1], x), mps[l], mi)
                cha = mps[l].shape[0]
                Qh, Rh = np.linalg.qr(mps[l].reshape(cha, d * chr_).conj().T)
                k = Qh.shape[1]
                mps[l] = Qh.conj().T.reshape(k, d, chr_)
                C = Rh.conj().T
                Re[l] = env_right_update(Re[l + 1], mps[l], W[l])
                self.matvecs['env'] += 1
                C = self._exp('heff0', lambda x, l=l: heff0(Le[l], Re[l], x), C, pi)
                mps[l - 1] = np.einsum('asb,bk->ask', mps[l - 1], C)
                last_two = False
        if not last_two:
            self.updates['one_site'] += 1
            mps[0] = self._exp('heff1', lambda x: heff1(Le[0], W[0], Re[1], x), mps[0], mi)


# --------------------------------------------------------------------------
# dissipative contraction D[tau] and stochastic jump J_eps
# (Sec. "Dissipative contraction", Sec. "Stochastic jump process")
# --------------------------------------------------------------------------
def dissipate_and_jump(mps, prob: Problem, Dops, u1, u2, trec=None):
    """Phi <- J_eps( D[tau] Phi ), in place.  Returns a record of the decisions.

    Readings:
    * D is contracted site by site during a right-to-left sweep that moves the
      orthogonality centre by RQ, so the centre ends at site 0 and
      dp = 1 - ||M_0||^2 is exact (Eq. for dp; no first-order expansion).
    * A jump happens iff u1 < dp (Sec. "A jump occurs").
    * Weights w_m = gamma_m <Phi|L_m^dag L_m|Phi> for all m (Eq.
      ProbabilityCalc...), normalised by their sum (the paper's Pi_m uses the
      first-order dt*gamma/dp, which does not sum to one); the chosen m is the
      smallest index, in site-major order, with u2 * sum(w) < cumsum_m.
    * sqrt(gamma_m) L_m is contracted into its site; the state is then brought
      to left-canonical form by a QR sweep and "normalised through successive
      SVDs": a right-to-left SVD sweep truncating every bond by trunc_rank,
      then scaled to unit norm.
    Postcondition in both branches: centre at site 0, sites 1..L-1
    right-canonical, unit norm.
    """
    L = prob.L
    for l in range(L - 1, -1, -1):
        mps[l] = apply_site_op(Dops[l], mps[l])
        if l > 0:
            rq_move_left(mps, l)
    norm2 = float(np.vdot(mps[0], mps[0]).real)
    dp = 1.0 - norm2
    rec = {'dp': dp, 'margin1': abs(u1 - dp), 'jump': -1, 'margin2': math.inf}
    if not (u1 < dp):
        mps[0] = mps[0] / math.sqrt(norm2)
        return rec
    ops = [(prob.jumps[m][0], prob.jumps[m][1].conj().T @ prob.jumps[m][1]) for m in prob.jump_order]
    vals, _ = local_expectations(mps, ops)
    w = np.array([prob.jumps[m][2] * vals[i].real for i, m in enumerate(prob.jump_order)])
    total = 0.0
    csum = []
    for x in w:
        total += x
        csum.append(total)
    target = u2 * total
    pick = len(w) - 1
    for i, c in enumerate(csum):
        if target < c:
            pick = i
            break
    rec['margin2'] = min(abs(target - c) for c in csum) / total
    m = prob.jump_order[pick]
    site, op, g = prob.jumps[m]
    rec['jump'] = m
    mps[site] = math.sqrt(g) * apply_site_op(op, mps[site])
    for l in range(L - 1):
        qr_move_right(mps, l)
    for l in range(L - 1, 0, -1):
        chl, d, chr_ = mps[l].shape
        U, S, Vh = np.linalg.svd(mps[l].reshape(chl, d * chr_), full_matrices=False)
        r = trunc_rank(S, prob, trec)
        mps[l] = Vh[:r].reshape(r, d, chr_)
        mps[l - 1] = np.einsum('asb,bk->ask', mps[l - 1], U[:, :r] * S[None, :r])
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    return rec


# --------------------------------------------------------------------------
# initial states
# --------------------------------------------------------------------------
def product_mps(phis):
    """Product state as an MPS of bond dimension 1, each site normalised."""
    out = []
    for v in phis:
        v = np.asarray(v, dtype=np.complex128)
        out.append((v / np.linalg.norm(v)).reshape(1, -1, 1))
    return out


def padded_product_mps(phis, rng=None):
    """The same product state with every bond at its full dimension min(d^b, d^(L-b)).

    Used by exact mode (Thm. 1's "MPS format of full bond dimension").  The
    extra basis vectors have zero weight; they are an arbitrary orthonormal
    completion (random, then QR), sites 1..L-1 right-canonical.
    """
    rng = np.random.default_rng(12345) if rng is None else rng
    L = len(phis)
    d = len(phis[0])
    chi = [min(d ** b, d ** (L - b)) for b in range(L + 1)]
    mps = [None] * L
    for l in range(L - 1, -1, -1):
        phi = np.asarray(phis[l], dtype=np.complex128)
        phi = phi / np.linalg.norm(phi)
        e0 = np.zeros(chi[l + 1], dtype=np.complex128)
        e0[0] = 1.0
        v = np.kron(phi, e0)                     # index (s, b)
        n = d * chi[l + 1]
        X = rng.standard_normal((n, chi[l])) + 1j * rng.standard_normal((n, chi[l]))
        X[:, 0] = v
        Q, _ = np.linalg.qr(X)
        Q[:, 0] *= np.vdot(Q[:, 0], v) / abs(np.vdot(Q[:, 0], v))
        mps[l] = Q.T.reshape(chi[l], d, chi[l + 1])
    return mps


# --------------------------------------------------------------------------
# one trajectory (Sec. "Algorithm": sampling MPS Phi, F_0, F_j, F_n)
# --------------------------------------------------------------------------
def run_trajectory(prob: Problem, psi0, traj_id, seed, observables, n_steps, sample_steps, order=2, on_sample=None):
    """Observables of one TJM trajectory at the sampled steps.

    Reading of the sampling-MPS indexing (Eqs. TimeEvolutionFunctions,
    MPSTimeEvolution, SimulationStep): Psi(0) is measured directly;
    Phi_0 = J(D[dt/2] Psi(0)); for j = 1..n: X = U[dt] Phi_{j-1};
    Psi(j dt) = J'(D[dt/2] X) on a copy (own uniforms, branch 1);
    Phi_j = J(D[dt] X) if j < n (branch 0).
    order=1 is the first-order baseline of Fig. 4a (dotted lines), read as the
    plain Lie-Trotter product with the same U, D and J: for j = 1..n
    Psi(j dt) = J(D[dt] U[dt] Psi((j-1) dt)) (branch 0), measured directly.
    on_sample(j, state), if given, sees every measured state (e.g. for the projection error).
    Returns (values[n_sample, n_obs], stats).
    """
    mps = [np.array(m, dtype=np.complex128) for m in psi0]
    nrm = math.sqrt(local_expectations(mps, [])[1])
    mps[0] = mps[0] / nrm
    D_half = [dissipator_site(prob, l, 0.5 * prob.dt) for l in range(prob.L)]
    D_full = [dissipator_site(prob, l, prob.dt) for l in range(prob.L)]
    sample_steps = list(sample_steps)
    want = set(sample_steps)
    vals = {}
    stats = {'jumps': 0, 'min_margin1': math.inf, 'min_margin2': math.inf, 'records': []}

    def note(rec, step):
        rec['step'] = step
        stats['records'].append(rec)
        stats['min_margin1'] = min(stats['min_margin1'], rec['margin1'])
        if rec['jump'] >= 0:
            stats['jumps'] += 1
            stats['min_margin2'] = min(stats['min_margin2'], rec['margin2'])

    sw = Sweeper(prob)
    if 0 in want:
        vals[0] = measure(mps, observables)
        if on_sample:
            on_sample(0, mps)
    if order == 1:
        for j in range(1, n_steps + 1):
            sw.build_right_envs(mps)
            sw.sweep(mps, 0.5 * prob.dt)
            u1, u2 = uniforms(seed, traj_id, j, 0)
            note(dissipate_and_jump(mps, prob, D_full, u1, u2, sw.rec), j)
            if j in want:
                vals[j] = measure(mps, observables)
                if on_sample:
                    on_sample(j, mps)
    if order == 2 and n_steps > 0:
        u1, u2 = uniforms(seed, traj_id, 0, 0)
        note(dissipate_and_jump(mps, prob, D_half, u1, u2, sw.rec), 0)
    for j in range(1, n_steps + 1 if order == 2 else 1):
        sw.build_right_envs(mps)
        sw.sweep(mps, 0.5 * prob.dt)
        if j in want:
            X = [m.copy() for m in mps]
            u1, u2 = uniforms(seed, traj_id, j, 1)
            note(dissipate_and_jump(X, prob, D_half, u1, u2, sw.rec), j)
            vals[j] = measure(X, observables)
            if on_sample:
                on_sample(j, X)
        if j < n_steps:
            u1, u2 = uniforms(seed, traj_id, j, 0)
            note(dissipate_and_jump(mps, prob, D_full, u1, u2, sw.rec), j)
    stats['matvecs'] = dict(sw.matvecs)
    stats['updates'] = dict(sw.updates)
    stats['final_bonds'] = [m.shape[2] for m in mps[:-1]]
    stats['trunc_margin'] = sw.rec.get('trunc_margin', math.inf)
    stats['cut_gap'] = sw.rec.get('cut_gap', math.inf)
    out = np.array([vals[s] for s in sample_steps]) if sample_steps else np.zeros((0, len(observables)))
    return out, stats


def ensemble(values):
    """Mean and standard error over trajectories (Eq. TJMExpVal); values [N, ...]."""
    v = np.asarray(values, dtype=np.float64)
    n = v.shape[0]
    mean = v.mean(axis=0)
    sem = v.std(axis=0, ddof=1) / math.sqrt(n) if n > 1 else np.zeros_like(mean)
    return mean, sem
