"""FP64 CPU oracle for the alpha-circulant preconditioned Crank-Nicolson all-at-once solve
(arXiv 2401.16113).

TEST INFRASTRUCTURE ONLY. This module is the plain, slow, obviously-correct reference
that the CUDA path is checked against. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does. It shares no code
with the CUDA path: numpy/scipy calls (FFT, banded and dense solves, sparse products,
eigenvalues) serve as library primitives, and every step is written in the order the
paper states it.

Readings of points the paper leaves open (each one also listed in the design notes):
  * eigenvalues of the alpha-circulant blocks are obtained numerically from their
    definition D_l = diag(sqrt(Nt) F Lambda_alpha C_l(:,1)) (Sec. 3.1), with the unitary
    DFT of the paper (omega = exp(-2 pi i / Nt)); this fixes the pairing of each shifted
    system with its frequency bin.
  * Dirichlet data enter f^{k+1/2} through the CN average of the boundary values at
    t_k and t_{k+1}.
  * Black-Scholes in S: S_i = i h, h = s_max/(Nx+1), 3-point central differences.
  * time-dependent coefficients (local volatility): row k of the AaO system uses
    A(t_{k+1/2}) for both time levels (the form of Eq. 5.8); the preconditioner uses the
    time mean of those matrices, the direct generalisation of d-bar in Sec. 5.3.
  * Riesz operator: fractional centred difference with Dirichlet exterior values.
  * Heston operator (Sec. 5.1): central differences on a uniform (s, v) grid, the s = S_max
    Neumann condition through a ghost node, the v = 0 boundary equation with a one-sided
    second-order u_v.
  * SABR operator (Sec. 5.2, Eq. 5.7): the Heston grid and s- and V_max-boundary conditions, at
    v = 0 the boundary equation u_t = r s u_s - r u (u_t = 0 for r = 0, parameter Sets III and
    IV). For r != 0 (Set V) the operator is Eq. 5.7 itself, each term with its own power of
    D(t) = e^{-rt}, at t_{k+1/2} in block row k; the preconditioner uses its time mean, as for
    the local volatility. (Sec. 5.2 motivates the preconditioner with the form L(t) = d(t) L; the
    errors printed in Table 4 fit Eq. 5.7 and not that form.)
Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl
import scipy.special as sps

# ----------------------------------------------------------------------------------------
# Spatial discretisation A (Sec. 2.1: A ~ L by finite differences) and boundary data.
# ----------------------------------------------------------------------------------------


def spatial_grid(p):
    """Interior nodes: S_i = i h (Black-Scholes), or x_i = -s_max + i h (Riesz), i = 1..Nx."""
    nx = int(p["nx"])
    if p["op"] == "riesz":
        h = 2.0 * p["s_max"] / (nx + 1)
        return -p["s_max"] + h * np.arange(1, nx + 1), h
    h = p["s_max"] / (nx + 1)
    return h * np.arange(1, nx + 1), h


def is_2d(p):
    """The two-dimensional operators in (s, v): Heston (Sec. 5.1) and SABR (Sec. 5.2)."""
    return p["op"] in ("heston", "sabr")


def time_dependent(p):
    """Operators whose A depends on t: local volatility, and SABR with r != 0 (D(t) = e^{-rt})."""
    return p["op"] == "localvol" or (p["op"] == "sabr" and p["r"] != 0.0)


def n_space(p):
    """Spatial unknowns per time level: Nx, or Ns Nv for the two-dimensional operators."""
    return int(p["nx"]) * (int(p["nv"]) if is_2d(p) else 1)


def time_grid(p):
    """t_k = k tau, tau = T/Nt (Sec. 2.1)."""
    nt = int(p["nt"])
    tau = p["T"] / nt
    return tau * np.arange(nt + 1), tau


def local_sigma(p, S, t):
    """sigma(S, t) = sigma + lv_bump * g(S) * (1 + lv_tslope * t), t = time to maturity, with the
    bump shape g(S) = exp(-ln^2(S/K)) (the local-volatility workload), or g = 1 when
    p['lv_shape'] == 'flat' (a volatility that depends on time only, whose European price has a
    closed form); constant sigma for 'bs'."""
    if p["op"] == "localvol":
        if p.get("lv_shape", "gauss") == "flat":
            g = np.ones_like(S)
        else:
            g = np.exp(-np.log(S / p["K"]) ** 2)
        return p["sigma"] + p["lv_bump"] * g * (1.0 + p["lv_tslope"] * t)
    return p["sigma"] * np.ones_like(S)


def bs_matrix(p, t):
    """Black-Scholes operator u_t = 1/2 sigma^2 S^2 u_SS + r S u_S - r u at time t (sparse
    Nx x Nx), 3-point central differences on the S grid, Dirichlet nodes removed.
    Also returns the coefficients of the two Dirichlet nodes in rows 1 and Nx."""
    S, h = spatial_grid(p)
    sig = local_sigma(p, S, t)
    diff = 0.5 * sig ** 2 * S ** 2 / h ** 2
    conv = 0.5 * p["r"] * S / h
    lower = diff - conv
    diag = -2.0 * diff - p["r"]
    upper = diff + conv
    A = sp.diags([lower[1:], diag, upper[:-1]], [-1, 0, 1], format="csr")
    return A, lower[0], upper[-1]


def riesz_weights(beta, n):
    """Fractional centred difference weights g_k = (-1)^k G(b+1) / (G(b/2-k+1) G(b/2+k+1)),
    k = 0..n-1, from the Gamma-function definition. The Gamma ratios are evaluated as
    sign * exp(-log|G(a)| - log|G(b)|) so that large k does not overflow; 1/G vanishes at
    the poles a = 0, -1, -2, ..."""
    k = np.arange(n, dtype=np.float64)
    a = beta / 2 - k + 1
    b = beta / 2 + k + 1
    pole = (a <= 0) & (a == np.floor(a))
    a_safe = np.where(pole, 0.5, a)
    mag = np.exp(sps.gammaln(beta + 1.0) - sps.gammaln(a_safe) - sps.gammaln(b))
    g = (-1.0) ** k * sps.gammasgn(a_safe) * mag
    return np.where(pole, 0.0, g)


def riesz_matrix(p):
    """Riesz operator of Eq. 1.2 (second case) in log-price:
    u_t = kappa d^beta u/d|x|^beta + (r - kappa) u_x - r u, kappa = sigma^2/2, with
    d^beta/d|x|^beta u(x_i) ~ -h^-beta sum_k g_k u(x_{i-k}) and central u_x.
    Returns (A, left-exterior coefficient vector, left drift coefficient)."""
    x, h = spatial_grid(p)
    nx = x.size
    kappa = 0.5 * p["sigma"] ** 2
    g = riesz_weights(p["beta"], nx + 1)
    A = -kappa * h ** (-p["beta"]) * g[np.abs(np.subtract.outer(np.arange(nx), np.arange(nx)))]
    drift = (p["r"] - kappa) / (2.0 * h)
    A[np.arange(nx - 1), np.arange(1, nx)] += drift
    A[np.arange(1, nx), np.arange(nx - 1)] -= drift
    A[np.arange(nx), np.arange(nx)] -= p["r"]
    # exterior nodes j <= 0 all carry the left Dirichlet value: row i (1-based) collects
    # sum_{m >= i} g_m, with sum_{m >= 1} g_m = -g_0/2 (the weights sum to zero).
    tail = -0.5 * g[0] - np.concatenate(([0.0], np.cumsum(g[1:nx])))
    left_ext = -kappa * h ** (-p["beta"]) * tail
    return A, left_ext, -drift


def heston_grid(p):
    """Heston unknowns (Sec. 5.1): s_i = i h_s, i = 1..Ns (s = S_max included: Neumann), v_j = j h_v,
    j = 0..Nv-1 (v = 0 included: the degenerate boundary equation; v = V_max is Dirichlet),
    h_s = S_max / Ns, h_v = V_max / Nv; unknown (i, j) at position j Ns + (i - 1)."""
    ns, nv = int(p["nx"]), int(p["nv"])
    hs, hv = p["s_max"] / ns, p["v_max"] / nv
    return hs * np.arange(1, ns + 1), hv * np.arange(nv), hs, hv


def heston_matrix(p):
    """The Heston operator of Eq. 5.1 by second-order central differences on the uniform grid of
    heston_grid (u_ss, u_vv, u_s, u_v central; u_sv by the four-point cross stencil), with
    u(0, v) = 0, u(s, V_max) = s, u_s(S_max, v) = 1 through a ghost node u_{Ns+1} = u_{Ns-1} + 2 h_s,
    and at v = 0 the boundary equation u_t = kappa eta u_v + r s u_s - r u with the one-sided
    second-order u_v = (-3 u_0 + 4 u_1 - u_2) / (2 h_v). Returns the sparse A and the constant vector f
    through which the boundary data enter (u' = A u + f)."""
    ns, nv = int(p["nx"]), int(p["nv"])
    S, V, hs, hv = heston_grid(p)
    r, kap, eta, sig, rho = p["r"], p["kappa"], p["eta"], p["sigma"], p["rho"]
    rows, cols, vals = [], [], []
    f = np.zeros(ns * nv)

    def add(i, j, ii, jj, c):
        """coefficient c of u(ii, jj) in the equation of unknown (i, j), i, ii 1-based in s"""
        row = j * ns + (i - 1)
        if jj == nv:                       # v = V_max: u = s
            f[row] += c * ii * hs
        elif ii == 0:                      # s = 0: u = 0
            pass
        elif ii == ns + 1:                 # ghost beyond S_max
            add(i, j, ns - 1, jj, c)
            f[row] += c * 2.0 * hs
        else:
            rows.append(row)
            cols.append(jj * ns + (ii - 1))
            vals.append(c)

    for j in range(nv):
        v = V[j]
        for i in range(1, ns + 1):
            s_ = S[i - 1]
            if j == 0:
                add(i, j, i, 0, -3.0 * kap * eta / (2 * hv) - r)
                add(i, j, i, 1, 4.0 * kap * eta / (2 * hv))
                add(i, j, i, 2, -kap * eta / (2 * hv))
                add(i, j, i + 1, 0, r * s_ / (2 * hs))
                add(i, j, i - 1, 0, -r * s_ / (2 * hs))
                continue
            ass = 0.5 * v * s_ * s_ / hs ** 2
            avv = 0.5 * sig * sig * v / hv ** 2
            asv = sig * rho * s_ * v / (4 * hs * hv)
            bs = r * s_ / (2 * hs)
            bv = kap * (eta - v) / (2 * hv)
            add(i, j, i, j, -2 * ass - 2 * avv - r)
            add(i, j, i + 1, j, ass + bs)
            add(i, j, i - 1, j, ass - bs)
            add(i, j, i, j + 1, avv + bv)
            add(i, j, i, j - 1, avv - bv)
            add(i, j, i + 1, j + 1, asv)
            add(i, j, i - 1, j - 1, asv)
            add(i, j, i + 1, j - 1, -asv)
            add(i, j, i - 1, j + 1, -asv)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(ns * nv, ns * nv))
    A.sum_duplicates()
    return A, f


def sabr_matrix(p, t=0.0):
    """The SABR operator of Eq. 5.7 at time t (time to maturity), D = e^{-rt}:
    u_t = 1/2 v^2 s^(2 beta) D^(2(1-beta)) u_ss + rho sigma s^beta D^(1-beta) v^2 u_sv
          + 1/2 sigma^2 v^2 u_vv + r s u_s - r u,
    on the grid of heston_grid with the boundary conditions shared with Heston (Sec. 5.2):
    u(0, v) = 0, u(s, V_max) = s, u_s(S_max, v) = 1 through a ghost node u_{Ns+1} = u_{Ns-1} + 2 h_s;
    at v = 0 the boundary equation u_t = r s u_s - r u (central u_s), an all-zero row for r = 0.
    Central differences, u_sv by the four-point cross stencil. Returns the sparse A and f
    (u' = A u + f)."""
    ns, nv = int(p["nx"]), int(p["nv"])
    S, V, hs, hv = heston_grid(p)
    beta, sig, rho, r = p["beta"], p["sigma"], p["rho"], p["r"]
    D = math.exp(-r * t)
    gss, gsv = D ** (2.0 * (1.0 - beta)), D ** (1.0 - beta)
    rows, cols, vals = [], [], []
    f = np.zeros(ns * nv)

    def add(i, j, ii, jj, c):
        """coefficient c of u(ii, jj) in the equation of unknown (i, j), i, ii 1-based in s"""
        row = j * ns + (i - 1)
        if jj == nv:                       # v = V_max: u = s
            f[row] += c * ii * hs
        elif ii == 0:                      # s = 0: u = 0
            pass
        elif ii == ns + 1:                 # ghost beyond S_max
            add(i, j, ns - 1, jj, c)
            f[row] += c * 2.0 * hs
        else:
            rows.append(row)
            cols.append(jj * ns + (ii - 1))
            vals.append(c)

    for j in range(nv):
        v = V[j]
        for i in range(1, ns + 1):
            s_ = S[i - 1]
            bs = r * s_ / (2 * hs)
            if j == 0:                     # u_t = r s u_s - r u (nothing to add for r = 0)
                if r != 0.0:
                    add(i, j, i, j, -r)
                    add(i, j, i + 1, j, bs)
                    add(i, j, i - 1, j, -bs)
                continue
            ass = 0.5 * v * v * s_ ** (2 * beta) * gss / hs ** 2
            avv = 0.5 * sig * sig * v * v / hv ** 2
            asv = rho * sig * s_ ** beta * gsv * v * v / (4 * hs * hv)
            add(i, j, i, j, -2 * ass - 2 * avv - r)
            add(i, j, i + 1, j, ass + bs)
            add(i, j, i - 1, j, ass - bs)
            add(i, j, i, j + 1, avv)
            add(i, j, i, j - 1, avv)
            add(i, j, i + 1, j + 1, asv)
            add(i, j, i - 1, j - 1, asv)
            add(i, j, i + 1, j - 1, -asv)
            add(i, j, i - 1, j + 1, -asv)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(ns * nv, ns * nv))
    A.sum_duplicates()
    return A, f


def operator_at(p, t):
    """A(t) as a dense matrix, plus the coefficients through which the left/right Dirichlet
    values enter the first/last interior rows. op 'matrix' takes a user matrix p['A']
    (constant in time, no boundary data) for the spectral pins."""
    if p["op"] == "matrix":
        A = np.asarray(p["A"], dtype=np.float64)
        return A, np.zeros(A.shape[0]), np.zeros(A.shape[0])
    if is_2d(p):
        A, f = heston_matrix(p) if p["op"] == "heston" else sabr_matrix(p, t)
        return A, f, np.zeros(A.shape[0])
    if p["op"] == "riesz":
        A, left_ext, left_drift = riesz_matrix(p)
        cl = left_ext.copy()
        cl[0] += left_drift
        return A, cl, np.zeros(A.shape[0])
    A, lo, up = bs_matrix(p, t)
    nx = A.shape[0]
    cl = np.zeros(nx)
    cr = np.zeros(nx)
    cl[0] = lo
    cr[-1] = up
    return A, cl, cr


def boundary_values(p, t):
    """Dirichlet values (g_L(t), g_R(t)) in time-to-maturity t."""
    if p["op"] == "matrix":
        return 0.0, 0.0
    if is_2d(p):
        return 1.0, 0.0  # time-independent data, carried by the vector f of heston/sabr_matrix
    disc = p["K"] * math.exp(-p["r"] * t)
    if p["op"] == "riesz":
        return disc - math.exp(-p["s_max"]), 0.0
    if p["payoff"] == "put":
        return disc, 0.0
    return 0.0, p["s_max"] - disc


def payoff(p):
    """u_0: the option payoff at the interior nodes (Eq. 1.1, u(., 0) = u_0)."""
    if p["op"] == "matrix":
        return np.asarray(p.get("u0", np.ones(int(p["nx"]))), dtype=np.float64)
    if is_2d(p):
        S, _, _, _ = heston_grid(p)
        return np.tile(np.maximum(S - p["K"], 0.0), int(p["nv"]))  # call, Eq. 5.2 (both operators)
    x, _ = spatial_grid(p)
    if p["op"] == "riesz":
        return np.maximum(p["K"] - np.exp(x), 0.0)
    if p["payoff"] == "put":
        return np.maximum(p["K"] - x, 0.0)
    return np.maximum(x - p["K"], 0.0)


def step_operator(p, k):
    """A_k = A(t_{k+1/2}) used by CN step k -> k+1 (Eq. 2.1; Eq. 5.8 for time-dependent A)."""
    t, tau = time_grid(p)
    return operator_at(p, t[k] + 0.5 * tau)


def forcing(p, k):
    """f^{k+1/2}: Dirichlet contribution averaged over t_k and t_{k+1} (CN)."""
    t, _ = time_grid(p)
    _, cl, cr = step_operator(p, k)
    gl0, gr0 = boundary_values(p, t[k])
    gl1, gr1 = boundary_values(p, t[k + 1])
    return cl * 0.5 * (gl0 + gl1) + cr * 0.5 * (gr0 + gr1)


# ----------------------------------------------------------------------------------------
# Sequential CN (Eq. 2.1) and the all-at-once system M u = b (Eq. 2.2 / Eq. 5.8).
# ----------------------------------------------------------------------------------------


def _solve(Amat, rhs):
    """Direct solve of one spatial system: banded LAPACK for sparse tridiagonal matrices,
    dense LU otherwise."""
    if sp.issparse(Amat):
        n = Amat.shape[0]
        coo = Amat.tocoo()
        if coo.nnz and np.abs(coo.row - coo.col).max() > 1:
            # wider than tridiagonal (the two-dimensional Heston operator): sparse LU
            return spl.spsolve(sp.csc_matrix(Amat, dtype=np.result_type(Amat.dtype, rhs.dtype)), rhs)
        ab = np.zeros((3, n), dtype=np.result_type(Amat.dtype, rhs.dtype))
        ab[0, 1:] = Amat.diagonal(1)
        ab[1, :] = Amat.diagonal(0)
        ab[2, :-1] = Amat.diagonal(-1)
        return sla.solve_banded((1, 1), ab, rhs)
    return np.linalg.solve(Amat, rhs)


def _eye_like(A):
    return sp.identity(A.shape[0], format="csr") if sp.issparse(A) else np.eye(A.shape[0])


def _dense(A):
    return A.toarray() if sp.issparse(A) else np.asarray(A)


def sequential_cn(p):
    """Time stepping of Eq. 2.1: (I - tau/2 A_k) u^{k+1} = (I + tau/2 A_k) u^k + tau f^{k+1/2}.
    Returns U with U[k] = u^{k+1}, k = 0..Nt-1 (the AaO unknown ordering of Eq. 2.2)."""
    nt = int(p["nt"])
    _, tau = time_grid(p)
    u = payoff(p)
    out = np.empty((nt, u.size))
    lu = None
    for k in range(nt):
        A, _, _ = step_operator(p, k)
        I = _eye_like(A)
        rhs = (I + 0.5 * tau * A) @ u + tau * forcing(p, k)
        if not sp.issparse(A) and not time_dependent(p):
            # constant dense A: the same matrix I - tau/2 A at every step, factored once
            if lu is None:
                lu = sla.lu_factor(I - 0.5 * tau * A)
            u = sla.lu_solve(lu, rhs)
        else:
            u = _solve(I - 0.5 * tau * A, rhs)
        out[k] = u
    return out


def assemble_M(p):
    """M of Eq. 2.2 (B1 (x) I - B2 (x) A~, A~ = tau A) for constant A; for time-dependent A the
    form of Eq. 5.8 with A~_k = tau A(t_{k+1/2}) in block row k. Sparse CSR, time-major."""
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    I = sp.identity(nx, format="csr")
    if not time_dependent(p):
        At = sp.csr_matrix(tau * step_operator(p, 0)[0])
        B1 = sp.diags([np.ones(nt), -np.ones(nt - 1)], [0, -1], shape=(nt, nt))
        B2 = 0.5 * sp.diags([np.ones(nt), np.ones(nt - 1)], [0, -1], shape=(nt, nt))
        return (sp.kron(B1, I) - sp.kron(B2, At)).tocsr()
    blocks = [[None] * nt for _ in range(nt)]
    for k in range(nt):
        At = sp.csr_matrix(tau * step_operator(p, k)[0])
        blocks[k][k] = I - 0.5 * At
        if k > 0:
            blocks[k][k - 1] = -(I + 0.5 * At)
    return sp.bmat(blocks, format="csr")


def assemble_b(p):
    """b = xi + tau f (Eq. 2.2), xi = [(I + A~_0/2) u^0; 0; ...; 0]."""
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    b = np.empty((nt, nx))
    for k in range(nt):
        b[k] = tau * forcing(p, k)
    A0, _, _ = step_operator(p, 0)
    b[0] += payoff(p) + 0.5 * tau * (A0 @ payoff(p))
    return b.reshape(-1)


def matvec(p, x, M=None):
    """y = M x with the explicit sparse M."""
    if M is None:
        M = assemble_M(p)
    return M @ x


def matvec_blocks(p, x):
    """y = M x by the block rows of Eq. 2.2 for a constant A: y_t = Q1 x_t - Q2 x_{t-1},
    Q1 = I - A~/2, Q2 = I + A~/2 (dense A, all time levels in one matrix product)."""
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    A = _dense(step_operator(p, 0)[0])
    X = np.asarray(x, dtype=np.float64).reshape(nt, nx)
    Xm = np.vstack([np.zeros((1, nx)), X[:-1]])
    S = X + Xm
    return ((X - Xm) - 0.5 * tau * (S @ A.T)).reshape(-1)


# ----------------------------------------------------------------------------------------
# The preconditioner P_alpha (Eq. 3.1) and its three-step inverse (Eq. 3.2).
# ----------------------------------------------------------------------------------------


def alpha_circulants(nt, alpha):
    """C1^(alpha) and C2^(alpha) of Sec. 3.1: B1, B2 with corner entries -alpha and alpha/2."""
    C1 = np.eye(nt) - np.eye(nt, k=-1)
    C2 = 0.5 * (np.eye(nt) + np.eye(nt, k=-1))
    C1[0, nt - 1] += -alpha
    C2[0, nt - 1] += 0.5 * alpha
    if nt == 1:
        C1 = np.array([[1.0 - alpha]])
        C2 = np.array([[0.5 * (1.0 + alpha)]])
    return C1, C2


def mean_operator(p):
    """A-bar used by the preconditioner: A itself for constant coefficients; the mean of
    A(t_{k+1/2}) over k for time-dependent ones (generalising d-bar of Sec. 5.3)."""
    if not time_dependent(p):
        return step_operator(p, 0)[0]
    nt = int(p["nt"])
    acc = step_operator(p, 0)[0]
    for k in range(1, nt):
        acc = acc + step_operator(p, k)[0]
    return (acc / nt).tocsr()


def dense_P(p, alpha=None):
    """P_alpha = C1 (x) I_s - C2 (x) A~ (Eq. 3.1), A~ = tau A-bar. Dense; tiny sizes only."""
    alpha = p["alpha"] if alpha is None else alpha
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    C1, C2 = alpha_circulants(nt, alpha)
    return np.kron(C1, np.eye(nx)) - np.kron(C2, tau * _dense(mean_operator(p)))


def apply_P(p, z, alpha=None):
    """P_alpha z = (C1 (x) I_s - C2 (x) A~) z (Eq. 3.1) without forming P: C1 and C2 act along time
    as B1 and B2 (z_t - z_{t-1}, (z_t + z_{t-1})/2) with the alpha corner at t = 0 (Sec. 3.1),
    A~ = tau A-bar along space. Any size."""
    alpha = p["alpha"] if alpha is None else alpha
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    Z = np.asarray(z, dtype=np.float64).reshape(nt, nx)
    prev = np.roll(Z, 1, axis=0)  # z_{t-1}; row 0 holds z_{nt-1}
    prev[0] = alpha * prev[0]
    At = tau * mean_operator(p)
    return ((Z - prev) - (At @ (0.5 * (Z + prev)).T).T).reshape(-1)


def dense_M(p):
    return assemble_M(p).toarray()


def precond_dense(p, v, alpha=None):
    """z = P_alpha^{-1} v by a dense LU solve of Eq. 3.1 (brute force)."""
    return np.linalg.solve(dense_P(p, alpha), v)


def circulant_eigs(nt, alpha):
    """Lambda_alpha and D_l = diag(sqrt(Nt) F Lambda_alpha C_l(:,1)) (Sec. 3.1), F the unitary
    DFT with omega = exp(-2 pi i/Nt); sqrt(Nt) F y is numpy's unnormalised forward FFT."""
    lam = alpha ** (np.arange(nt) / nt)
    C1, C2 = alpha_circulants(nt, alpha)
    d1 = np.fft.fft(lam * C1[:, 0])
    d2 = np.fft.fft(lam * C2[:, 0])
    return lam, d1, d2


def precond_fft(p, v, alpha=None, return_spectrum=False):
    """z = P_alpha^{-1} v by the three steps of Eq. 3.2:
    (a) z1 = (V_alpha^{-1} (x) I) v with V_alpha^{-1} = F Lambda_alpha,
    (b) (lambda_{1,k} I - lambda_{2,k} A~) z2_k = z1_k for every k = 1..Nt,
    (c) z = (V_alpha (x) I) z2 with V_alpha = Lambda_alpha^{-1} F^*.
    All Nt shifted systems are solved (the conjugate-pair saving of Remark 1 is not used)."""
    alpha = p["alpha"] if alpha is None else alpha
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    lam, d1, d2 = circulant_eigs(nt, alpha)
    At = tau * mean_operator(p)
    V = np.asarray(v, dtype=np.float64).reshape(nt, nx)
    # step (a): unitary DFT along time of the Lambda-scaled blocks
    z1 = np.fft.fft(lam[:, None] * V, axis=0) / math.sqrt(nt)
    # step (b): Nt independent complex-shifted spatial solves
    z2 = np.empty_like(z1)
    I = _eye_like(At)
    for k in range(nt):
        z2[k] = _solve(d1[k] * I - d2[k] * At, z1[k])
    # step (c): inverse unitary DFT, then Lambda^{-1}
    z = (np.fft.ifft(z2, axis=0) * math.sqrt(nt)) / lam[:, None]
    if return_spectrum:
        return z, z1, z2
    return z.real.reshape(-1)


# ----------------------------------------------------------------------------------------
# Right-preconditioned flexible GMRES(m) (Sec. 5: right-preconditioned GMRES, zero initial
# guess, relative-residual stopping; Its = inner iterations = matrix-vector products).
# ----------------------------------------------------------------------------------------


def fgmres(apply_M, apply_Pinv, b, tol, m, maxit, x0=None):
    """Flexible right-preconditioned GMRES(m): Arnoldi with classical Gram-Schmidt applied
    twice, Givens rotations on the Hessenberg matrix, restart after m inner steps; the
    stopping test uses the true residual ||b - M x|| / ||b|| at every restart.
    Returns (x, info) with info = dict(its, restarts, rel_res, converged, history)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(its=0, restarts=0, rel_res=0.0, converged=True, history=[])
    r = b - apply_M(x)
    beta = np.linalg.norm(r)
    its = 0
    restarts = 0
    hist = [beta / bnorm]
    while True:
        if beta <= tol * bnorm:
            return x, dict(its=its, restarts=restarts, rel_res=beta / bnorm, converged=True, history=hist)
        if its >= maxit:
            return x, dict(its=its, restarts=restarts, rel_res=beta / bnorm, converged=False, history=hist)
        Vs = [r / beta]
        Zs = []
        H = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        g[0] = beta
        cs = np.zeros(m)
        sn = np.zeros(m)
        jd = 0
        for j in range(m):
            z = apply_Pinv(Vs[j])
            Zs.append(z)
            w = apply_M(z)
            its += 1
            Vm = np.array(Vs)
            h = Vm @ w
            w = w - Vm.T @ h
            h2 = Vm @ w
            w = w - Vm.T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            jd = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0 or its >= maxit:
                break
            Vs.append(w / hn)
        y = sla.solve_triangular(H[:jd, :jd], g[:jd])
        x = x + np.array(Zs[:jd]).T @ y
        r = b - apply_M(x)
        beta = np.linalg.norm(r)
        restarts += 1
        hist.append(beta / bnorm)


def solve(p, precond="fft", tol=None, m=None, maxit=200):
    """AaO solve of Eq. 2.2 by right-preconditioned FGMRES(m) with P_alpha (FP64)."""
    M = assemble_M(p)
    b = assemble_b(p)
    tol = p["tol"] if tol is None else tol
    m = p["m"] if m is None else m
    if precond == "fft":
        Pinv = lambda v: precond_fft(p, v)
    elif precond == "dense":
        Pinv = lambda v: precond_dense(p, v)
    else:
        Pinv = lambda v: v
    return fgmres(lambda x: M @ x, Pinv, b, tol, m, maxit)


# ----------------------------------------------------------------------------------------
# Black-Scholes closed form (the PDE check for 'bs'), textbook formula.
# ----------------------------------------------------------------------------------------


def bs_price(S, K, r, sigma, T, kind="put"):
    S = np.asarray(S, dtype=np.float64)
    with np.errstate(divide="ignore"):
        d1 = (np.log(S / K) + (r + 0.5 * sigma ** 2) * T) / (sigma * math.sqrt(T))
    d2 = d1 - sigma * math.sqrt(T)
    N = sps.ndtr
    if kind == "call":
        return S * N(d1) - K * math.exp(-r * T) * N(d2)
    return K * math.exp(-r * T) * N(-d2) - S * N(-d1)


def heston_char(u, T, v0, kappa, eta, sigma, rho):
    """E[exp(i u X_T)] for X_T = ln(S_T / S_0) - r T under the Heston dynamics (Heston 1993), in the
    form of Albrecher et al. (2007), "The little Heston trap", whose complex logarithm stays on its
    principal branch: d = sqrt((kappa - i rho sigma u)^2 + sigma^2 (i u + u^2)),
    g = (kappa - i rho sigma u - d) / (kappa - i rho sigma u + d),
    C = kappa eta / sigma^2 ((kappa - i rho sigma u - d) T - 2 ln((1 - g e^{-dT}) / (1 - g))),
    D = (kappa - i rho sigma u - d) / sigma^2 (1 - e^{-dT}) / (1 - g e^{-dT}), phi = exp(C + D v0)."""
    u = np.asarray(u, dtype=np.complex128)
    b = kappa - 1j * rho * sigma * u
    d = np.sqrt(b * b + sigma * sigma * (1j * u + u * u))
    g = (b - d) / (b + d)
    e = np.exp(-d * T)
    C = kappa * eta / sigma ** 2 * ((b - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))
    D = (b - d) / sigma ** 2 * (1.0 - e) / (1.0 - g * e)
    return np.exp(C + D * v0)


def heston_call(S0, v0, K, T, r, kappa, eta, sigma, rho):
    """European call under Heston by the single-integral Fourier formula of Lewis (2000):
    C = S0 - sqrt(S0 K) e^{-rT/2} / pi * int_0^inf Re[e^{i u k} phi(u - i/2)] / (u^2 + 1/4) du,
    k = ln(S0 / K) + r T, phi = heston_char (numerical quadrature)."""
    import scipy.integrate as si
    k = math.log(S0 / K) + r * T

    def integrand(u):
        return (np.exp(1j * u * k) * heston_char(u - 0.5j, T, v0, kappa, eta, sigma, rho)).real / (u * u + 0.25)

    val, _ = si.quad(integrand, 0.0, np.inf, limit=800, epsabs=1e-10, epsrel=1e-10)
    return S0 - math.sqrt(S0 * K) * math.exp(-0.5 * r * T) / math.pi * val


# ----------------------------------------------------------------------------------------
# Spectral quantities (Lemma 3.1, Theorem 3.1, Theorem 2.2, Lemma 4.1) on tiny grids.
# ----------------------------------------------------------------------------------------


def preconditioned_eigs(p, alpha=None):
    """Eigenvalues of P_alpha^{-1} M (dense)."""
    return np.linalg.eigvals(np.linalg.solve(dense_P(p, alpha), dense_M(p)))


def R_matrix(p):
    """R with P_alpha = M - alpha R (Sec. 4): the only non-zero block is Q2 = I + A~/2 in
    block position (1, Nt)."""
    nt, nx = int(p["nt"]), n_space(p)
    _, tau = time_grid(p)
    R = np.zeros((nt * nx, nt * nx))
    R[:nx, (nt - 1) * nx:] = np.eye(nx) + 0.5 * tau * _dense(mean_operator(p))
    return R
