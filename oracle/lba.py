"""Linear analysis and linearized buckling analysis (exact and multilevel).

  linear_analysis       Algorithm 1 step 2 (LA): u = K[x]^{-1} f, compliance J = f^T u.
  buckling_pencil       Algorithm 1 step 4 (EA) / Sec. 2.1 step 1: the q lowest positive load factors
                        of (K + lambda G) phi = 0 (eq. eigenvalueProblem0), modes normalised as
                        phi_i^T K phi_j = delta_ij (Sec. 2).
  exact_lba             Algorithm 1 on the fine grid.
  multilevel_lba        Sec. 2.1 steps 1-4 (Algorithm 2 without the optional per-level smoothing):
                        Galerkin K^l, G^l; coarse eigenpairs; prolongation Psi^j = I^j_{j+1} Psi^{j+1};
                        fine solve K Phi~ = G Psi (eq. FineScaleBVP); Rayleigh quotients (eq. FineScaleRQ).

All vectors returned on the full DOF set (zeros at fixed DOFs).  Readings of the paper used here:
only positive load factors are kept (negative ones belong to the reversed load); modes are scaled
to phi^T K phi = 1 and signed so that their entry of largest magnitude is positive; the fine-grid
load factors are per-column Rayleigh quotients, re-sorted ascending.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assembly, grid, transfer


class Problem:
    """Oracle view of a synthetic.Problem: assembled operators on the free DOFs."""

    def __init__(self, prob):
        self.p = prob
        self.dim = prob.dim
        self.nel = prob.nel
        self.fixed = np.asarray(prob.fixed, dtype=np.uint8)
        self.free = np.flatnonzero(self.fixed == 0)
        self.n = prob.num_dofs
        self.K = assembly.assemble_K(prob.nel, prob.dim, prob.x, prob.nu, prob.penal, prob.E0, prob.Emin)
        self.Kf = assembly.restrict_free(self.K, self.fixed)
        self._lu = None

    def solve(self, B: np.ndarray) -> np.ndarray:
        """K_ff^{-1} B on free DOFs by sparse LU (SuperLU)."""
        if self._lu is None:
            self._lu = spla.splu(self.Kf.tocsc())
        return self._lu.solve(np.asarray(B, dtype=np.float64))

    def to_full(self, vf: np.ndarray) -> np.ndarray:
        shape = (self.n,) + vf.shape[1:]
        out = np.zeros(shape)
        out[self.free] = vf
        return out

    def G(self, u: np.ndarray) -> sp.csr_matrix:
        p = self.p
        return assembly.assemble_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin)


def linear_analysis(op: Problem):
    """Algorithm 1 step 2: u = K^{-1} f (direct), J = f^T u."""
    f = np.asarray(op.p.f, dtype=np.float64)
    u = op.to_full(op.solve(f[op.free]))
    return u, float(f @ u)


def _normalise_modes(Kf, Phi):
    """Scale to phi^T K phi = 1 (Sec. 2) and fix the sign (largest-magnitude entry positive)."""
    Phi = np.array(Phi, dtype=np.float64, copy=True)
    for i in range(Phi.shape[1]):
        c = Phi[:, i]
        c /= np.sqrt(c @ (Kf @ c))
        if c[np.argmax(np.abs(c))] < 0:
            c *= -1.0
        Phi[:, i] = c
    return Phi


def buckling_pencil(Kf, Gf, q: int, dense_limit: int = 4000):
    """q lowest positive lambda of (K + lambda G) phi = 0 on free DOFs.

    With mu = 1/lambda the pencil is -G phi = mu K phi (K SPD); the q largest positive mu give the q
    smallest positive lambda.  Dense generalized eigh for small systems, otherwise ARPACK Lanczos
    on the same pencil (which='LA', tight tolerance).  Returns (lambda [q] ascending, Phi [nf, q])."""
    n = Kf.shape[0]
    if n <= dense_limit:
        mu, V = sla.eigh(-Gf.toarray(), Kf.toarray())
    else:
        k = min(n - 2, q + 10)
        mu, V = spla.eigsh(-Gf.tocsc(), k=k, M=Kf.tocsc(), which="LA", tol=1e-14,
                           ncv=min(n - 1, max(4 * k, 60)))
    pos = np.flatnonzero(mu > 0)
    order = pos[np.argsort(-mu[pos])][:q]
    if order.size < q:
        raise RuntimeError("fewer than q positive buckling load factors found")
    lam = 1.0 / mu[order]
    return lam, _normalise_modes(Kf, V[:, order])


def exact_lba(op: Problem, u: np.ndarray, q: int, dense_limit: int = 4000):
    """Algorithm 1 on the fine grid: (lambda_i, phi_i), i = 1..q, phi full-length."""
    G = op.G(u)
    Gf = assembly.restrict_free(G, op.fixed)
    lam, Phi = buckling_pencil(op.Kf, Gf, q, dense_limit)
    return lam, op.to_full(Phi), Gf


def galerkin_levels(op: Problem, Gf, eig_level: int):
    """K^l = P^T ... K ... P and G^l likewise (Sec. 2.1 step 1; Algorithm 2 'restrict'), with the
    chain of free interpolations from level eig_level up to level 1."""
    nels, fixeds, Ps = transfer.hierarchy(op.nel, op.dim, op.fixed, eig_level)
    Kl, Gl = op.Kf, Gf
    for P in Ps:
        Kl = (P.T @ Kl @ P).tocsr()
        Gl = (P.T @ Gl @ P).tocsr()
    return Kl, Gl, Ps, nels, fixeds


def multilevel_lba(op: Problem, u: np.ndarray, q: int, eig_level: int, dense_limit: int = 4000):
    """Sec. 2.1 steps 1-4.  Returns dict with the fine pairs (lam, Phi), the coarse eigenpairs
    (lam_coarse, Psi_coarse on level eig_level free DOFs) and the prolongated Psi (fine, full)."""
    G = op.G(u)
    Gf = assembly.restrict_free(G, op.fixed)
    Kl, Gl, Ps, nels, fixeds = galerkin_levels(op, Gf, eig_level)
    lam_c, Psi_c = buckling_pencil(Kl, Gl, q, dense_limit)          # step 1
    Psi = Psi_c
    for P in reversed(Ps):                                           # step 2
        Psi = P @ Psi
    Phi = op.solve(Gf @ Psi)                                         # step 3
    num = np.einsum("ij,ij->j", Phi, op.Kf @ Phi)
    den = np.einsum("ij,ij->j", Phi, Gf @ Phi)
    lam = -num / den                                                 # step 4
    order = np.argsort(lam)
    lam = lam[order]
    Phi = _normalise_modes(op.Kf, Phi[:, order])
    return dict(lam=lam, Phi=op.to_full(Phi), lam_coarse=lam_c, Psi_coarse=Psi_c,
                Psi=op.to_full(Psi), Gf=Gf, Kl=Kl, Gl=Gl, fixed_levels=fixeds, nels=nels)


def eig_residual(Kf, Gf, lam, phi_free):
    """||(K + lambda G) phi|| / ||K phi||, the residual measure of eq. eigResidual."""
    Kp = Kf @ phi_free
    return float(np.linalg.norm(Kp + lam * (Gf @ phi_free)) / np.linalg.norm(Kp))


# ------------------------------------------------------------------------------------------------
# Algorithm 2 with its per-level steps (the optional refinement of Sec. 2.1, Appendix A)
# ------------------------------------------------------------------------------------------------
def multicolour_rows(nel, dim, fixed) -> np.ndarray:
    """A row order for Kaczmarz sweeps on a level (the paper gives none): the free rows grouped by the
    colour (i mod 3) + 3 (j mod 3) + 9 (k mod 3) of their node (i, j, k), colours ascending, nodes in
    increasing index within a colour, the d rows of a node in turn.  Returned as indices into the
    free-DOF numbering.  Rows of different nodes of one colour share no unknown (their nodes are
    three or more apart along some axis, each row touches only the 3^d surrounding nodes), so their
    relative order does not change the result."""
    nd = grid.node_dims(nel, dim)
    fixed = np.asarray(fixed, dtype=np.uint8)
    free_index = np.full(fixed.size, -1, dtype=np.int64)
    free_index[fixed == 0] = np.arange(int((fixed == 0).sum()))
    nodes = np.arange(int(np.prod(nd[:dim])))
    i = nodes % nd[0]
    j = (nodes // nd[0]) % nd[1]
    k = nodes // (nd[0] * nd[1]) if dim == 3 else np.zeros_like(nodes)
    colour = i % 3 + 3 * (j % 3) + 9 * (k % 3)
    order = []
    for col in range(27 if dim == 3 else 9):
        for a in nodes[colour == col]:
            for c in range(dim):
                r = free_index[dim * a + c]
                if r >= 0:
                    order.append(r)
    return np.asarray(order, dtype=np.int64)


def kaczmarz(A: sp.spmatrix, Psi: np.ndarray, sweeps: int, order=None) -> np.ndarray:
    """Kaczmarz sweeps for A psi = 0 on every column of Psi (Appendix A: Gauss-Seidel on A^T A):
    for the rows i in turn (`order`, default 0, 1, 2, ...), psi <- psi - (a_i . psi / |a_i|^2) a_i."""
    A = A.tocsr()
    rn = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    Psi = np.array(Psi, dtype=np.float64, copy=True)
    rows = range(A.shape[0]) if order is None else order
    for _ in range(sweeps):
        for i in rows:
            if rn[i] == 0.0:
                continue
            s, e = A.indptr[i], A.indptr[i + 1]
            cols, vals = A.indices[s:e], A.data[s:e]
            r = vals @ Psi[cols]
            Psi[cols] -= np.outer(vals, r / rn[i])
    return Psi


def ritz(Kl, Gl, Psi: np.ndarray):
    """Rayleigh-Ritz of the pencil (K + lambda G) on span(Psi) (Algorithm 2 'R[Psi]'): the positive
    load factors in ascending order and their K-normalised Ritz vectors."""
    Kq = Psi.T @ (Kl @ Psi)
    Gq = Psi.T @ (Gl @ Psi)
    mu, Y = sla.eigh(-0.5 * (Gq + Gq.T), 0.5 * (Kq + Kq.T))
    pos = np.flatnonzero(mu > 0)
    order = pos[np.argsort(-mu[pos])]
    return 1.0 / mu[order], _normalise_modes(Kl, Psi @ Y[:, order])


def multilevel_lba_refined(op: Problem, u: np.ndarray, q: int, eig_level: int, sweeps: int = 1,
                           ritz_projection: bool = True, dense_limit: int = 4000, order: str = "natural",
                           fine_steps: int = 1):
    """Algorithm 2: the coarse eigenpairs of level eig_level, then on every level j = eig_level-1 down
    to 1 (the fine grid; the printed loop index is garbled): prolongate Psi^j = I^j_{j+1} Psi^{j+1},
    shift by the smallest load factor of the level above, `sweeps` Kaczmarz sweeps on
    (K^j + shift G^j) psi = 0 for every mode (rows in increasing order, or order = "multicolour":
    multicolour_rows), Rayleigh-Ritz on span Psi^j; finally the fine solve K Phi~ = G Psi and the
    per-column Rayleigh quotients, normalised and sorted.  fine_steps > 1 repeats the fine solve
    from the previous step's modes: inverse iteration on Omega_1, eq. PInvIt-GeneralInteration with
    the preconditioner P = K (then phi - K^{-1}(K + s G) phi = -s K^{-1} G phi, a multiple of the
    inverse-iteration step whatever the shift s).  With sweeps = 0, no Ritz projection and one fine
    step this is Sec. 2.1 steps 1-4 (multilevel_lba)."""
    G = op.G(u)
    Gf = assembly.restrict_free(G, op.fixed)
    nels, fixeds, Ps = transfer.hierarchy(op.nel, op.dim, op.fixed, eig_level)
    Ks, Gs = [op.Kf], [Gf]
    for P in Ps:
        Ks.append((P.T @ Ks[-1] @ P).tocsr())
        Gs.append((P.T @ Gs[-1] @ P).tocsr())
    lam_c, Psi = buckling_pencil(Ks[-1], Gs[-1], q, dense_limit)
    Lam = lam_c
    levels = []
    for j in reversed(range(len(Ps))):                               # level j + 1 (1-based) = Omega_{j+1}
        Psi = Ps[j] @ Psi
        if sweeps > 0:
            rows = multicolour_rows(nels[j], op.dim, fixeds[j]) if order == "multicolour" else None
            Psi = kaczmarz(Ks[j] + Lam.min() * Gs[j], Psi, sweeps, rows)
        if ritz_projection:
            Lam, Psi = ritz(Ks[j], Gs[j], Psi)
            if Lam.size < q:
                raise RuntimeError("Rayleigh-Ritz lost a positive load factor on level %d" % (j + 1))
        levels.append(dict(level=j + 1, lam=Lam.copy(), K=Ks[j], G=Gs[j]))
    for _ in range(max(1, fine_steps)):
        Phi = op.solve(Gf @ Psi)
        num = np.einsum("ij,ij->j", Phi, op.Kf @ Phi)
        den = np.einsum("ij,ij->j", Phi, Gf @ Phi)
        lam = -num / den
        srt = np.argsort(lam)
        lam, Psi = lam[srt], _normalise_modes(op.Kf, Phi[:, srt])
    return dict(lam=lam, Phi=op.to_full(Psi), lam_coarse=lam_c, levels=levels, Gf=Gf)
