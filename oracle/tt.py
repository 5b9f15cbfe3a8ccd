"""L1 oracle: plain tensor-train (QTT / MPS-MPO) algebra in NumPy, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg do.

Conventions (arXiv:2507.05222, Sec. II):
* an MPS core A[k] has shape (r_{k-1}, d, r_k) (eq:simpleMPS), an MPO core
  M[k] has shape (w_{k-1}, d_out, d_in, w_k) (eq:simpleMatrix);
* the first core carries the most significant bit (App. D's worked example);
* outputs of every rounding are right-canonical (cores 2..n right-orthonormal,
  the norm in core 1), the gauge the paper keeps (Sec. II).

Operations and the passage each follows:
* ``tt_svd``                 -- right-to-left successive truncated SVDs of a dense tensor (Fig. 1);
* ``round_tt``               -- TT-rounding (Sec. II.A intro): QR left-to-right, truncated SVD
                                right-to-left; equal to ``tt_svd`` of the represented tensor;
* ``direct_sum``             -- vector-vector addition by block cores (Sec. II.A.1);
* ``mpo_mps``                -- mat-vec by core-wise contraction over r_k (Sec. II.A.2);
* ``hadamard_exact``         -- copy tensor turns a into diag(a), then mat-vec (Sec. II.A.3);
* ``fit``                    -- variational (fit) evaluation of sums of products at fixed
                                bond dimension (Sec. II.B, Table I right column);
* ``als``                    -- single-site DMRG / ALS for SPD systems (Sec. II.A.4, Fig. 5)
                                with local CG on the "fast matvec" (App. G), swept until the
                                true relative residual (``residual``) meets a tolerance or
                                stops falling (stop rule above ``als``).
The truncation rule (keep min(chi, #sigma > eps*sigma_1, structural bound)) is the
reading of Sec. II ("first chi values" / "below a threshold").
"""
from __future__ import annotations

import numpy as np

# Multi-operand contractions go pairwise (greedy order, BLAS where possible); numpy's default
# path search refuses intermediates larger than the inputs and would fall back to one nested
# loop over all indices.  The order of a sum changes only the rounding, not the result.
OPT = ("greedy", 1e12)

# --------------------------------------------------------------------------------------
# dense <-> TT
# --------------------------------------------------------------------------------------


def full(cores) -> np.ndarray:
    """Dense vector of an MPS, index q = sum_k s_k d^(n-k) (first core = most significant)."""
    t = np.ones((1, 1))
    for c in cores:
        t = np.einsum("xa,asb->xsb", t, c).reshape(-1, c.shape[2])
    return t.reshape(-1)


def full_mpo(cores) -> np.ndarray:
    """Dense matrix of an MPO (rows = output index, columns = input index)."""
    t = np.ones((1, 1, 1))
    for c in cores:
        t = np.einsum("xya,asrb->xsyrb", t, c)
        t = t.reshape(t.shape[0] * t.shape[1], t.shape[2] * t.shape[3], c.shape[3])
    return t[:, :, 0]


def bonds(cores) -> list[int]:
    return [cores[0].shape[0]] + [c.shape[-1] for c in cores]


def nvps(cores) -> int:
    """Number of stored values 2 * sum alpha_{k-1} alpha_k (Sec. IV, NVPS_TT)."""
    return int(sum(c.size for c in cores))


def _cap(d: int, k: int) -> int:
    return d ** min(k, 62)


def kept_rank(sig, chi: int, eps: float, struct: int) -> int:
    """Number of singular values kept: min(chi, struct) and, if eps > 0, only sigma > eps*sigma_1."""
    b = min(chi, struct, len(sig))
    if eps > 0.0 and len(sig) > 0:
        b = min(b, int(np.count_nonzero(sig > eps * sig[0])))
    return max(b, 1)


def left_struct(pre_bonds, d: int) -> list[int]:
    """m_k = min(R_k, d m_{k-1}): rank bound at each cut from the left (m_0 = 1)."""
    m = [1]
    for k in range(1, len(pre_bonds)):
        m.append(min(pre_bonds[k], d * m[-1]))
    return m


def tt_svd(t, n: int, d: int, chi: int, eps: float = 0.0, pre_bonds=None):
    """Right-to-left TT-SVD of a dense tensor with d^n entries (Fig. 1, reversed sweep).

    At the cut after core k-1 (k = n..2) the current tensor (d^(k-1) x d r_k) is split by
    an SVD; the top b_{k-1} right singular vectors become core k, U S is carried left.
    ``pre_bonds`` (if given) are the bonds of an exact TT of t: they bound the kept ranks
    (rank at cut k <= min(R_k, d m_{k-1})), which fixes the bond profile when eps = 0.
    """
    pre = pre_bonds if pre_bonds is not None else [1] + [_cap(d, min(k, n - k)) for k in range(1, n)] + [1]
    m = left_struct(pre, d)
    cores = [None] * n
    cur = np.asarray(t, dtype=np.float64).reshape(-1, 1)      # (d^n, r_n=1)
    rk = 1
    for k in range(n, 1, -1):
        mat = cur.reshape(_cap(d, k - 1), d * rk)
        U, S, Vt = np.linalg.svd(mat, full_matrices=False)
        b = kept_rank(S, chi, eps, min(m[k - 1], d * rk))
        cores[k - 1] = Vt[:b].reshape(b, d, rk)
        cur = U[:, :b] * S[:b]
        rk = b
    cores[0] = cur.reshape(1, d, rk)
    return cores


def qr_pos(a):
    """Reduced QR (Householder via LAPACK)."""
    return np.linalg.qr(a, mode="reduced")


def round_tt(cores, chi: int, eps: float = 0.0, info: dict | None = None):
    """TT-rounding (Sec. II.A): left-to-right QR, then right-to-left truncated SVD.

    Equals ``tt_svd`` of the represented tensor with pre_bonds = bonds(cores).  ``info`` (a dict,
    optional) receives ``discarded_norm`` = sqrt(sum over cuts of the discarded sigma^2).
    """
    d = cores[0].shape[1]
    n = len(cores)
    pre = bonds(cores)
    m = left_struct(pre, d)
    c = [x.copy() for x in cores]
    for k in range(n - 1):
        r0, _, r1 = c[k].shape
        Q, R = qr_pos(c[k].reshape(r0 * d, r1))
        c[k] = Q.reshape(r0, d, Q.shape[1])
        c[k + 1] = np.einsum("ab,bsc->asc", R, c[k + 1])
    disc = 0.0
    for k in range(n - 1, 0, -1):
        r0, _, r1 = c[k].shape
        U, S, Vt = np.linalg.svd(c[k].reshape(r0, d * r1), full_matrices=False)
        b = kept_rank(S, chi, eps, min(m[k], d * r1))
        disc += float(np.sum(S[b:] ** 2))
        c[k] = Vt[:b].reshape(b, d, r1)
        c[k - 1] = np.einsum("asb,bc->asc", c[k - 1], U[:, :b] * S[:b])
    if info is not None:
        info["discarded_norm"] = float(np.sqrt(disc))
    return c


def right_orth(cores):
    """Right-canonical form without truncation (LQ sweep right to left)."""
    c = [x.copy() for x in cores]
    d = c[0].shape[1]
    for k in range(len(c) - 1, 0, -1):
        r0, _, r1 = c[k].shape
        Q, R = qr_pos(c[k].reshape(r0, d * r1).T)
        c[k] = Q.T.reshape(Q.shape[1], d, r1)
        c[k - 1] = np.einsum("asb,cb->asc", c[k - 1], R)
    return c


# --------------------------------------------------------------------------------------
# exact (unrounded) algebra
# --------------------------------------------------------------------------------------


def direct_sum(alpha, x, beta, y):
    """Cores of alpha x + beta y by the block construction of Sec. II.A.1."""
    n = len(x)
    out = []
    for k in range(n):
        a, b = x[k], y[k]
        if n == 1:
            out.append(alpha * a + beta * b)
            continue
        if k == 0:
            out.append(np.concatenate([alpha * a, beta * b], axis=2))
        elif k == n - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            c = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]))
            c[:a.shape[0], :, :a.shape[2]] = a
            c[a.shape[0]:, :, a.shape[2]:] = b
            out.append(c)
    return out


def mpo_mps(M, x):
    """B[k]_{(a w),(a' w')}^{s'} = sum_s M[k]^{s',s}_{w,w'} A[k]^s_{a,a'} (Sec. II.A.2)."""
    out = []
    for W, A in zip(M, x):
        c = np.einsum("wtsv,asb->awtbv", W, A)
        out.append(c.reshape(A.shape[0] * W.shape[0], W.shape[1], A.shape[2] * W.shape[3]))
    return out


def diag_mpo(a):
    """Copy tensor delta^{s'}_{s,s''} contracted into each core: diag(a) as an MPO (Sec. II.A.3)."""
    out = []
    for A in a:
        d = A.shape[1]
        W = np.zeros((A.shape[0], d, d, A.shape[2]))
        for s in range(d):
            W[:, s, s, :] = A[:, s, :]
        out.append(W)
    return out


def hadamard_exact(a, b):
    return mpo_mps(diag_mpo(a), b)


def mpo_mpo(M1, M2):
    """Cores of the product M1 M2 (contraction over the shared physical index)."""
    out = []
    for A, B in zip(M1, M2):
        c = np.einsum("asrb,crtd->acstbd", A, B)
        out.append(c.reshape(A.shape[0] * B.shape[0], A.shape[1], B.shape[2], A.shape[3] * B.shape[3]))
    return out


def mpo_direct_sum(alpha, A, beta, B):
    """alpha A + beta B for MPOs (block cores, Sec. II.A.1 applied to fused physical indices)."""
    fa = [c.reshape(c.shape[0], -1, c.shape[3]) for c in A]
    fb = [c.reshape(c.shape[0], -1, c.shape[3]) for c in B]
    s = direct_sum(alpha, fa, beta, fb)
    d_out, d_in = A[0].shape[1], A[0].shape[2]
    return [c.reshape(c.shape[0], d_out, d_in, c.shape[2]) for c in s]


def round_mpo(M, chi: int, eps: float):
    d_out, d_in = M[0].shape[1], M[0].shape[2]
    f = [c.reshape(c.shape[0], d_out * d_in, c.shape[3]) for c in M]
    r = round_tt(f, chi, eps)
    return [c.reshape(c.shape[0], d_out, d_in, c.shape[2]) for c in r]


def scale(x, s):
    return [x[0] * s] + [c.copy() for c in x[1:]]


def dot(a, b) -> float:
    """<a, b> by left-to-right transfer matrices."""
    E = np.ones((1, 1))
    for A, B in zip(a, b):
        E = np.einsum("ab,asc,bsd->cd", E, A, B, optimize=OPT)
    return float(E[0, 0])


def norm(a) -> float:
    return float(np.sqrt(max(dot(a, a), 0.0)))


# --------------------------------------------------------------------------------------
# variational fit (Table I, right column)
# --------------------------------------------------------------------------------------
# A target is a list of terms:
#   ("vec", coef, x)            coef * x
#   ("had", coef, a, b)         coef * (a (.) b)
#   ("mpo", coef, M, x)         coef * (M x)
# Environments: left L[k] contracts sites < k of (current c, term tensors); right R[k]
# contracts sites > k.  Index order of an environment: (c, term bonds...).

def _ones_env(term):
    kind = term[0]
    if kind == "vec":
        return np.ones((1, 1))
    if kind == "had":
        return np.ones((1, 1, 1))
    return np.ones((1, 1, 1))


def _left_update(term, L, C, k):
    kind = term[0]
    if kind == "vec":
        X = term[2][k]
        return np.einsum("ca,csd,asb->db", L, C, X, optimize=OPT)
    if kind == "had":
        A, B = term[2][k], term[3][k]
        return np.einsum("cab,csd,ase,bsf->def", L, C, A, B, optimize=OPT)
    W, X = term[2][k], term[3][k]
    return np.einsum("cwa,csd,wstv,atb->dvb", L, C, W, X, optimize=OPT)


def _right_update(term, R, C, k):
    kind = term[0]
    if kind == "vec":
        X = term[2][k]
        return np.einsum("db,csd,asb->ca", R, C, X, optimize=OPT)
    if kind == "had":
        A, B = term[2][k], term[3][k]
        return np.einsum("def,csd,ase,bsf->cab", R, C, A, B, optimize=OPT)
    W, X = term[2][k], term[3][k]
    return np.einsum("dvb,csd,wstv,atb->cwa", R, C, W, X, optimize=OPT)


def _local(term, L, R, k):
    """Projection of one term onto the frames of sites != k: a core (r_{k-1}, d, r_k)."""
    kind = term[0]
    coef = term[1]
    if kind == "vec":
        X = term[2][k]
        return coef * np.einsum("ca,asb,db->csd", L, X, R, optimize=OPT)
    if kind == "had":
        A, B = term[2][k], term[3][k]
        return coef * np.einsum("cab,ase,bsf,def->csd", L, A, B, R, optimize=OPT)
    W, X = term[2][k], term[3][k]
    return coef * np.einsum("cwa,wstv,atb,dvb->csd", L, W, X, R, optimize=OPT)


def fit(terms, init, sweeps: int = 1):
    """Fixed-bond variational fit of sum(terms), started from ``init``.

    ``init`` is taken to the right-canonical form first (no truncation).  One sweep is a
    left-to-right half-sweep followed by a right-to-left half-sweep; at every site the
    core is replaced by the projection of the target onto the current frames and,
    except at the last site of the half-sweep, by an orthonormal basis of its range
    (QR).  The result is right-canonical.
    """
    c = right_orth(init)
    n = len(c)
    d = c[0].shape[1]
    Rs = [[None] * (n + 1) for _ in terms]
    Ls = [[None] * (n + 1) for _ in terms]
    for t, term in enumerate(terms):
        Rs[t][n] = _ones_env(term)
        for k in range(n - 1, 0, -1):
            Rs[t][k] = _right_update(term, Rs[t][k + 1], c[k], k)
        Ls[t][0] = _ones_env(term)
    for _ in range(sweeps):
        for k in range(n):
            T = sum(_local(term, Ls[t][k], Rs[t][k + 1], k) for t, term in enumerate(terms))
            if k < n - 1:
                r0, _, r1 = T.shape
                Q, _ = qr_pos(T.reshape(r0 * d, r1))
                c[k] = Q.reshape(r0, d, r1)
                for t, term in enumerate(terms):
                    Ls[t][k + 1] = _left_update(term, Ls[t][k], c[k], k)
            else:
                c[k] = T
        for k in range(n - 1, -1, -1):
            T = sum(_local(term, Ls[t][k], Rs[t][k + 1], k) for t, term in enumerate(terms))
            if k > 0:
                r0, _, r1 = T.shape
                Q, _ = qr_pos(T.reshape(r0, d * r1).T)
                c[k] = Q.T.reshape(r0, d, r1)
                for t, term in enumerate(terms):
                    Rs[t][k] = _right_update(term, Rs[t][k + 1], c[k], k)
            else:
                c[k] = T
    return c


def zipup_hadamard(a, b, chi: int):
    """Right-to-left zip-up of a (.) b: contract one site, truncated SVD, carry U S left.

    Used as the starting point of the Hadamard fit.  Kept rank at each cut:
    min(chi, m_{k-1}, d b_k) with m from the exact product bonds r_a r_b.
    """
    n = len(a)
    d = a[0].shape[1]
    pre = [x * y for x, y in zip(bonds(a), bonds(b))]
    m = left_struct(pre, d)
    cores = [None] * n
    C = np.ones((1, 1, 1))          # (c, a', b') carry
    for k in range(n - 1, 0, -1):
        T = np.einsum("ase,bsf,cef->absc", a[k], b[k], C, optimize=OPT)
        ra, rb, _, rc = T.shape
        U, S, Vt = np.linalg.svd(T.reshape(ra * rb, d * rc), full_matrices=False)
        bk = kept_rank(S, chi, 0.0, min(m[k], d * rc))
        cores[k] = Vt[:bk].reshape(bk, d, rc)
        C = (U[:, :bk] * S[:bk]).T.reshape(bk, ra, rb)
    T = np.einsum("ase,bsf,cef->absc", a[0], b[0], C, optimize=OPT)
    cores[0] = T.reshape(1, d, T.shape[3])
    return cores


def hadamard_round(a, b, chi: int, sweeps: int = 2, init=None):
    """c = a (.) b at bond profile min(chi, ...) by the variational fit (Table I)."""
    c0 = zipup_hadamard(a, b, chi) if init is None else init
    return fit([("had", 1.0, a, b)], c0, sweeps)


# --------------------------------------------------------------------------------------
# ALS / single-site DMRG (Sec. II.A.4)
# --------------------------------------------------------------------------------------

def _op_left(L, X, W):
    return np.einsum("cwa,csd,wstv,atb->dvb", L, X, W, X, optimize=OPT)


def _op_right(R, X, W):
    return np.einsum("dvb,csd,wstv,atb->cwa", R, X, W, X, optimize=OPT)


def _op_local(L, W, R, x):
    """Fast matvec (App. G): successive contractions L . x . W . R, never the assembled matrix."""
    return np.einsum("cwa,wstv,atb,dvb->csd", L, W, x, R, optimize=OPT)


def cg(matvec, b, x0, iters: int, tol: float, dinv=None):
    """Conjugate gradients (preconditioned by the diagonal scaling ``dinv`` when given) with an
    iteration budget; stops early when ||r|| <= tol ||b|| (or r = 0, or p.Ap <= 0)."""
    x = x0.copy()
    r = b - matvec(x)
    z = r * dinv if dinv is not None else r
    p = z.copy()
    rr = float(np.vdot(r, r))
    rz = float(np.vdot(r, z))
    bb = float(np.vdot(b, b))
    it = 0
    while it < iters and rr > tol * tol * bb and rr > 0.0:
        Ap = matvec(p)
        pAp = float(np.vdot(p, Ap))
        if pAp <= 0.0:
            break
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = r * dinv if dinv is not None else r
        rz_new = float(np.vdot(r, z))
        rr = float(np.vdot(r, r))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def local_diag(L, W, R):
    """Diagonal of the local ALS matrix L . W . R (Fig. 5): d[c, s, e] = sum_{w, v} L[c, w, c]
    W[w, s, s, v] R[e, v, e]."""
    return np.einsum("cwc,wssv,eve->cse", L, W, R)


# Stop rule of the ALS solver (the paper leaves it open; Sec. II.A.4 only says "sweeps").
# After every full sweep the true relative residual ||A x - b|| / ||b|| of the un-truncated
# TT A x (+) (-b) is evaluated entry by entry (``residual``), and the solve stops with
#   CONVERGED   once it is <= rel_tol;
#   STALLED     once a sweep after the first reduced it by less than the fraction ``stall`` (> 0;
#               0 disables the test; the first sweep from a poor start may raise the residual,
#               since the sweeps minimise the energy, not the residual): at a fixed bond the
#               ALS converges to a stationary point of the energy on the rank-chi manifold, whose
#               residual is bounded below by the truncation, so further sweeps cannot reach rel_tol;
#   MAX_SWEEPS  after max_sweeps sweeps.
# Each local CG solve of a sweep stops once ||r_loc|| <= cg_tol * res ||b_loc||, res being the
# true relative residual before the sweep (inexact local solves tied to the global error), or
# after cg_max_iter iterations.
CONVERGED, STALLED, MAX_SWEEPS = 0, 1, 2


def dense_terms(terms) -> np.ndarray:
    """Dense value of a sum of fit/ALS terms, each product formed as a TT first (no dense matrix)."""
    out = 0.0
    for term in terms:
        if term[0] == "vec":
            out = out + term[1] * full(term[2])
        elif term[0] == "had":
            out = out + term[1] * full(term[2]) * full(term[3])
        else:
            out = out + term[1] * full(mpo_mps(term[2], term[3]))
    return out


def residual(A, x, b_dense, b_norm) -> float:
    """||A x - b|| / ||b||: the exact TT A x is reconstructed and b subtracted entry by entry, so
    the difference carries only the rounding of each entry (no cancellation of squared norms)."""
    r = full(mpo_mps(A, x)) - b_dense
    return float(np.linalg.norm(r) / b_norm)


def als(A, terms, x0, max_sweeps: int, cg_max_iter: int, cg_tol: float, rel_tol: float = 0.0,
        stall: float = 0.1):
    """Single-site ALS for A x = sum(terms) with A symmetric positive definite.

    Minimises 1/2 <x, A x> - <x, b> core by core (Sec. II.A.4): the local system
    M_eff x_k = b_eff (size r_{k-1} d r_k) is solved by CG on the fast matvec, preconditioned
    by the inverse of M_eff's diagonal (the paper preconditions the local updates but does not
    say how, App. G; where a diagonal entry is not positive it is left unscaled), warm-started
    from the current core; the core is then split by QR and the R factor pushed into the
    neighbour (gauge move).  A sweep is a left-to-right half-sweep followed by a right-to-left
    one; the result is right-canonical.  Sweeps continue under the stop rule above.  Returns (x, info) with info = dict(sweeps, cg_iters, rel_residual, status, history).
    """
    b_dense = dense_terms(terms)
    nb = float(np.linalg.norm(b_dense))
    nb = nb if nb > 0.0 else 1.0
    x = right_orth(x0)
    n = len(x)
    d = x[0].shape[1]
    LA = [None] * (n + 1); RA = [None] * (n + 1)
    LA[0] = np.ones((1, 1, 1)); RA[n] = np.ones((1, 1, 1))
    Rs = [[None] * (n + 1) for _ in terms]
    Ls = [[None] * (n + 1) for _ in terms]
    for t, term in enumerate(terms):
        Rs[t][n] = _ones_env(term); Ls[t][0] = _ones_env(term)
    for k in range(n - 1, 0, -1):
        RA[k] = _op_right(RA[k + 1], x[k], A[k])
        for t, term in enumerate(terms):
            Rs[t][k] = _right_update(term, Rs[t][k + 1], x[k], k)
    total_cg = 0
    res = residual(A, x, b_dense, nb)
    history = [res]

    def solve_site(k, tol):
        nonlocal total_cg
        bk = sum(_local(term, Ls[t][k], Rs[t][k + 1], k) for t, term in enumerate(terms))
        mv = lambda v: _op_local(LA[k], A[k], RA[k + 1], v)
        dg = local_diag(LA[k], A[k], RA[k + 1])
        dinv = np.where(dg > 0.0, 1.0 / np.where(dg > 0.0, dg, 1.0), 1.0)
        xk, it = cg(mv, bk, x[k], cg_max_iter, tol, dinv)
        total_cg += it
        return xk

    status = MAX_SWEEPS
    if res <= rel_tol:
        status = CONVERGED
    sweep = 0
    while status != CONVERGED and sweep < max_sweeps:
        tol = cg_tol * res
        for k in range(n):
            xk = solve_site(k, tol)
            if k < n - 1:
                r0, _, r1 = xk.shape
                Q, R = qr_pos(xk.reshape(r0 * d, r1))
                x[k] = Q.reshape(r0, d, r1)
                x[k + 1] = np.einsum("ab,bsc->asc", R, x[k + 1])
                LA[k + 1] = _op_left(LA[k], x[k], A[k])
                for t, term in enumerate(terms):
                    Ls[t][k + 1] = _left_update(term, Ls[t][k], x[k], k)
            else:
                x[k] = xk
        for k in range(n - 1, -1, -1):
            xk = solve_site(k, tol)
            if k > 0:
                r0, _, r1 = xk.shape
                Q, R = qr_pos(xk.reshape(r0, d * r1).T)
                x[k] = Q.T.reshape(r0, d, r1)
                x[k - 1] = np.einsum("asb,cb->asc", x[k - 1], R)
                RA[k] = _op_right(RA[k + 1], x[k], A[k])
                for t, term in enumerate(terms):
                    Rs[t][k] = _right_update(term, Rs[t][k + 1], x[k], k)
            else:
                x[k] = xk
        sweep += 1
        new = residual(A, x, b_dense, nb)
        history.append(new)
        if new <= rel_tol:
            status = CONVERGED
        elif stall > 0.0 and sweep >= 2 and not (new <= (1.0 - stall) * res):
            status = STALLED
        res = new
        if status == STALLED:
            break
    info = dict(sweeps=sweep, cg_iters=total_cg, rel_residual=res, status=status, history=history)
    return x, info


def terms_full(terms) -> np.ndarray:
    """Dense value of a list of fit/ALS terms (for tests)."""
    return dense_terms(terms)
